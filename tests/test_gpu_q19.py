"""The D3Q19 lattice (Eq. 22-24) on the GPU vs the FP64 oracle, through the
C ABI (gpu).

Integer set-up products (active set, wall and reactive link classes) must
match bit for bit; floating-point results within the bounds of each storage
mode, as for D3Q7:
  fp32     C as double-float, 18 f32 deviations: the f32 rounding of the
           returned O(1) field;
  fp16dev  deviations as scaled f16 (11-bit significand);
  fp32pop  19 plain f32 populations: ulps of O(1) values per step.
Sizes span several 128-cell x blocks and 8-cell store sectors with ragged
tails.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1410_1914_gb300 import inputs
from tolerances import field_tol, step_sampled

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
STORAGES = ["fp32", "fp16dev", "fp32pop"]
C19 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
       (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
       (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
A19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _solver(shape, storage="fp32pop", **params):
    from paper_1410_1914_gb300 import Solver
    return Solver(shape, storage=storage, lattice="d3q19", **params)


def _oracle(ph, react=None, **params):
    return oracle.OracleLBM(ph, react=react, lattice=1, **params)


def _tol(steps, storage="fp32pop"):
    return {"fp32": 1e-7 + 1e-10 * steps, "fp16dev": 8e-5 + 1e-7 * steps,
            "fp32pop": 2e-6 + 1e-7 * steps}[storage]


CASES = {
    "pt_ragged": ("pt_cl_256", (13, 17, 291), 21, dict(k_ms=2e4)),
    "pt_deff": ("pt_cl_48", (19, 23, 37), 22, {}),
    "npmc": ("npmc_cl_400", (24, 20, 150), 23, dict(k_ms=5e3)),
    "thin": ("pt_cl_256", (3, 5, 40), 24, dict(k_ms=2e4)),
    "pt_physical_k": ("pt_cl_256", (13, 17, 291), 25, {}),   # k dt / dx ~1e-8 of cs^2
}


def _case(name):
    wl, shape, seed, extra = CASES[name]
    ph, react, params = inputs.make_workload(wl, shape=shape, seed=seed)
    return ph, react, dict(params, **extra)


def _walls_from_active(act):
    """Wall links from the active set: the end cell of the link (the mirror
    image of the end plane when it leaves the box in x) is not active."""
    nz, ny, nx = act.shape
    out = np.zeros(act.shape, np.uint32)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for i in range(1, 19):
        cx, cy, cz = C19[i]
        ex = x + cx
        ex = np.where((ex < 0) | (ex >= nx), x, ex)
        end = act[(z + cz) % nz, (y + cy) % ny, ex]
        out |= np.where(act & ~end, np.uint32(1 << (i - 1)), np.uint32(0))
    return out


@pytest.mark.parametrize("name", sorted(CASES))
def test_setup_bit_exact(cuda_lib, name):
    ph, react, params = _case(name)
    s = _solver(ph.shape, **params)
    s.set_structure(ph, react)
    su = s.setup()
    o = _oracle(ph, react, **params)
    act = o.active() > 0
    np.testing.assert_array_equal(su["active"], o.active())
    wall, rlinks = s.links()
    np.testing.assert_array_equal(rlinks, o.react())
    np.testing.assert_array_equal(wall, _walls_from_active(act))
    np.testing.assert_allclose(su["omega"][act], 1.0 / o.tau()[act], rtol=1e-6)
    info = s.info()
    assert info["n_active"] == int(act.sum())
    assert info["n_wall_links"] == int(sum(bin(int(v)).count("1") for v in wall[act]))
    assert info["n_react_links"] == int(sum(bin(int(v)).count("1") for v in rlinks[act]))
    assert info["dt_s"] == pytest.approx(o.dt, rel=1e-12)   # Eq. 24 with cs^2 = 1/3
    assert info["k_lu"] == pytest.approx(o.k_lu, rel=1e-12)
    s.close()


def test_all_pore_solid_rule_equals_the_full_mask(cuda_lib):
    ph, _, params = _case("npmc")
    full = inputs.reactive_faces(ph, 1.0, 0)
    a = _solver(ph.shape, react_rule=1, **params)
    a.set_structure(ph, None)
    b = _solver(ph.shape, **params)
    b.set_structure(ph, full)
    np.testing.assert_array_equal(a.links()[1], b.links()[1])
    assert a.links()[1].any()


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("steps", [1, 2, 10, 150])
def test_trajectory(cuda_lib, storage, name, steps):
    ph, react, params = _case(name)
    s = _solver(ph.shape, storage, **params)
    s.set_structure(ph, react)
    s.step(steps)
    o = _oracle(ph, react, **params)
    dmax = step_sampled(o, steps)
    tol = field_tol(storage, steps, dmax, q=19)
    err = float(np.abs(s.field() - o.concentration()).max())
    assert err <= tol, f"max|dC| {err:.3e} > {tol:.3e} (max|delta| {dmax:.3e}, err / (2^-11 max|delta|) = " \
        f"{err / max(2.0 ** -11 * dmax, 1e-300):.2f})"
    fg, fo = s.fluxes(), o.fluxes()
    nyz = ph.shape[0] * ph.shape[1]
    ftol = {"fp32": 1e-6, "fp16dev": 5e-4, "fp32pop": 2e-5}[storage]
    floor = {"fp32": 1e-9, "fp16dev": 2e-6, "fp32pop": 6e-8}[storage] * nyz + 1e-7
    assert fg["n_active"] == fo["n_active"]
    for k in ("J_in", "J_out"):
        assert abs(fg[k] - fo[k]) <= ftol * max(abs(fo["J_in"]), 1e-30) + floor
    assert abs(fg["R"] - fo["R"]) <= ftol * max(abs(fo["R"]), 1e-30) + min(floor, 1e-3 * abs(fo["R"]))
    assert fg["sum_C"] == pytest.approx(fo["sum_C"], rel=max(ftol, 1e-6))
    tg, pRg, pCg = s.reaction_rate()
    to, pRo, pCo = o.reaction_rate()
    assert tg == pytest.approx(to, rel=ftol, abs=1e-30)
    np.testing.assert_allclose(pCg, pCo, atol=tol)
    assert s.current_density() == pytest.approx(o.current_density(), rel=ftol, abs=1e-30)
    s.close()


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 3, 5), (2, 1, 33), (5, 9, 1), (4, 8, 32), (1, 16, 128),
                                   (2, 3, 129)])
def test_degenerate_boxes(cuda_lib, storage, shape):
    """Single cells, single rows and planes (a diagonal then wraps onto its
    own row), rows of exactly one block or one cell over."""
    rng = np.random.default_rng(sum(shape))
    ph = (rng.random(shape) < 0.2).astype(np.uint8)
    ph[..., 0] = 0
    react = rng.integers(0, 64, shape).astype(np.uint8)
    params = dict(dx_m=1e-8, D_bulk=1e-5, k_ms=40.0, c_in=1.0, c_out=0.25)
    s = _solver(shape, storage, **params)
    s.set_structure(ph, react)
    s.step(37)
    o = _oracle(ph, react, **params)
    o.step(37)
    np.testing.assert_allclose(s.field(), o.concentration(), rtol=0, atol=_tol(37, storage))


@pytest.mark.parametrize("storage", STORAGES)
def test_populations_layout_and_seed_spread(cuda_lib, storage):
    """Populations come back as [19][nz][ny][nx] in the order of Eq. 22 as
    listed in the header: after one step from a single seeded cell at tau = 1
    cell x + c_i holds a_i C0 in population i (the Eq. 23 weights)."""
    ph = np.zeros((7, 7, 40), np.uint8)
    s = _solver(ph.shape, storage, dx_m=1e-8, D_bulk=1e-5, tau_ref=1.0, bc_in=1, bc_out=1)
    s.set_structure(ph)
    C0 = np.zeros(ph.shape, np.float32)
    C0[3, 3, 20] = 1.0
    s.init(C0)
    s.step(1)
    g = s.populations()
    assert g.shape == (19,) + ph.shape
    # post-collision populations at tau = 1 are a_j C at each cell: cell
    # x + c_i received C = a_i, so its population j holds a_j a_i
    for i, (cx, cy, cz) in enumerate(C19):
        np.testing.assert_allclose(g[:, 3 + cz, 3 + cy, 20 + cx], A19 * A19[i], rtol=1e-6 if storage != "fp16dev" else 2e-3,
                                   atol=1e-12 if storage != "fp16dev" else 1e-6)
    np.testing.assert_allclose(g.sum(axis=0), s.field(), atol=1e-7)
    assert abs(s.field().sum() - 1.0) < 1e-6


@pytest.mark.parametrize("storage", STORAGES)
def test_custom_init_and_step_counter(cuda_lib, storage):
    ph, react, params = _case("pt_deff")
    rng = np.random.default_rng(0)
    C0 = rng.random(ph.shape).astype(np.float32)
    s = _solver(ph.shape, storage, **params)
    s.set_structure(ph, react)
    s.init(C0)
    s.step(65)  # one 64-step graph + one single step
    o = _oracle(ph, react, **params)
    o.init_field(C0.astype(np.float64))
    o.step(65)
    np.testing.assert_allclose(s.field(), o.concentration(), atol=_tol(65, storage) * 10)
    assert s.steps == 65


def test_lattice_and_batch_limits(cuda_lib):
    from paper_1410_1914_gb300 import Solver
    from paper_1410_1914_gb300.batch import Batch
    from paper_1410_1914_gb300._lib import ClError
    with pytest.raises(ClError):
        Solver((4, 4, 8), storage="fp32pop", lattice=2)
    ph, react, params = _case("thin")
    s = _solver(ph.shape, "fp32", **params)
    s.set_structure(ph, react)
    with pytest.raises(ClError):
        Batch([s])


@pytest.mark.parametrize("storage,rel", [("fp32", 1e-3), ("fp16dev", 5e-3)])
def test_converged_deff_small_workload_state(cuda_lib, storage, rel):
    """48^3 plain-method workload on D3Q19 with the (C, delta) state: the
    stopping rule fires and the GPU D_eff matches the converged FP64
    oracle (tests/golden/c1_deff_d3q19.json): 1e-3 relative for FP32, 5e-3
    for FP16 storage."""
    with open(os.path.join(HERE, "golden", "c1_deff_d3q19.json")) as fh:
        gold = json.load(fh)
    ph, react, params = inputs.make_workload("pt_cl_48")
    s = _solver(ph.shape, storage, check_every=200, tol_rel=1e-5, tol_flux=1e-4, max_steps=3_000_000, **params)
    s.set_structure(ph, react)
    info = s.solve()
    assert info["converged"] == 1, info
    d, ratio = s.effective_diffusivity()
    assert ratio == pytest.approx(gold["D_eff_over_Db"], rel=rel)
    assert d == pytest.approx(gold["D_eff_m2s"], rel=rel)


def test_converged_deff_small_workload(cuda_lib):
    """48^3 plain-method workload on D3Q19: D_eff after 300,000 steps (ten
    times what the FP64 oracle needs to a relative change of 1e-8 per 100
    steps) against the converged FP64 oracle (tests/golden/c1_deff_d3q19.json),
    1e-3 relative.  The 19 plain f32 populations stall at an FP32 rounding
    floor: the outlet flux is right to ~2e-4, but the inlet and outlet
    fluxes keep a ~6e-4 imbalance, so the flux-balance test of the stopping
    rule (1e-4) does not fire, as for the D3Q7 populations."""
    with open(os.path.join(HERE, "golden", "c1_deff_d3q19.json")) as fh:
        gold = json.load(fh)
    ph, react, params = inputs.make_workload("pt_cl_48")
    s = _solver(ph.shape, check_every=200, tol_rel=1e-5, tol_flux=1e-4, **params)
    s.set_structure(ph, react)
    info = s.solve_budget(300_000)
    assert info["steps"] == 300_000
    d, ratio = s.effective_diffusivity()
    assert ratio == pytest.approx(gold["D_eff_over_Db"], rel=1e-3)
    assert d == pytest.approx(gold["D_eff_m2s"], rel=1e-3)


def _stencil_deff_uniform(solid):
    """D_eff / D of the D3Q19 steady state at tau = 1 with uniform D on the
    open cells ~solid (all of them connected here), Dirichlet 1 | 0 in x,
    periodic y and z: the lattice's own 19-point system (every
    post-collision population is a_i C at tau = 1), assembled with numpy and
    solved by conjugate gradients.  Its equivalence with the scheme is
    pinned on the oracle (test_oracle_q19.py)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    nz, ny, nx = solid.shape
    op = ~solid
    N = solid.size
    ids = np.arange(N).reshape(solid.shape)
    rows, cols, vals = [], [], []
    diag = np.zeros(N)
    b = np.zeros(N)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    jout = []
    for i in range(1, 19):
        cx, cy, cz = C19[i]
        a = A19[i]
        ex = x + cx
        out = (ex < 0) | (ex >= nx)
        exm = np.where(out, x, ex)
        ey, ez = (y + cy) % ny, (z + cz) % nz
        end_open = op[ez, ey, exm]
        inner = op & ~out & end_open
        rows.append(ids[inner])
        cols.append(ids[ez, ey, exm][inner])
        vals.append(np.full(inner.sum(), -a))
        np.add.at(diag, ids[inner], a)
        bnd = op & out & end_open
        np.add.at(diag, ids[bnd], 2 * a)
        if cx < 0:
            np.add.at(b, ids[bnd], 2 * a * 1.0)  # C_in = 1 at x = 0
        else:
            jout.append((ids[bnd], 2 * a))
    diag[diag == 0] = 1.0
    A = sp.csr_matrix((np.concatenate(vals + [diag]), (np.concatenate(rows + [np.arange(N)]),
                                                       np.concatenate(cols + [np.arange(N)]))), shape=(N, N))
    C, info = spl.cg(A, b, rtol=1e-12, maxiter=200000, M=sp.diags(1 / diag))
    assert info == 0
    J = sum((w * C[ix]).sum() for ix, w in jout)  # 2 a (C - C_out), C_out = 0
    return float(J * nx / (ny * nz) / (1.0 / 6.0))  # D_lu = (tau - 1/2) / 3 at tau = 1


def test_sphere_in_cube_96(cuda_lib):
    """The validation geometry of Sec. 5.1, which the paper computed on this
    lattice (0.3317 at 200^3): at 96^3 the converged GPU D_eff (FP32 state)
    equals the lattice's own tau = 1 steady state to 5e-5 and lies within
    4 % of the printed value."""
    n = 96
    c = (np.arange(n) + 0.5) - n / 2
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    solid = (x * x + y * y + z * z) < (n / 2) ** 2
    ph = solid.astype(np.uint8)
    with _solver(ph.shape, "fp32", D_bulk=1e-5, knudsen=0, tau_ref=1.0, check_every=500, tol_rel=1e-7,
                 tol_flux=1e-6, max_steps=3_000_000) as s:
        s.set_structure(ph)
        info = s.solve()
        assert info["status"] == "CL_OK", info
        _, d_rel = s.effective_diffusivity()
    ref_stencil = _stencil_deff_uniform(solid)
    assert d_rel == pytest.approx(ref_stencil, rel=5e-5), (info, d_rel, ref_stencil)
    with open(os.path.join(HERE, "golden", "paper_values.json")) as fh:
        ref = json.load(fh)["sphere_in_cube_deff"]["value"]
    assert d_rel == pytest.approx(ref, rel=0.04)


@pytest.mark.parametrize("storage", STORAGES)
def test_protons_on_d3q19(cuda_lib, storage):
    """Proton conduction in the ionomer (Eq. 16) on the D3Q19 lattice: the
    ionomer active set and its link classes bit for bit, and the trajectory
    against the oracle."""
    ph = inputs.pt_cl((16, 20, 70), 31, 0.45, 0.1887)
    params = dict(dx_m=2e-9, D_bulk=2.9e-5, knudsen=1, D_ionomer=2.5, carrier=1, tau_ref=0.9, c_in=1.0, c_out=0.0)
    s = _solver(ph.shape, storage, **params)
    s.set_structure(ph)
    o = _oracle(ph, **params)
    act = o.active() > 0
    np.testing.assert_array_equal(s.setup()["active"], o.active())
    np.testing.assert_array_equal(s.links()[0], _walls_from_active(act))
    s.step(60)
    o.step(60)
    np.testing.assert_allclose(s.field(), o.concentration(), rtol=0, atol=_tol(60, storage))
    with pytest.raises(Exception):
        s.current_density()  # no sink for protons


@pytest.mark.parametrize("storage", STORAGES)
def test_wide_offsets(cuda_lib, storage, monkeypatch):
    """Boxes whose 19 planes exceed 2^32 elements (about 610^3 cells) take
    64-bit element offsets; CL_LBM_WIDE_INDEX=1 forces that path here, on a
    small box, against the oracle (and the D3Q7 population kernel with it)."""
    monkeypatch.setenv("CL_LBM_WIDE_INDEX", "1")
    ph, react, params = _case("pt_ragged")
    s = _solver(ph.shape, storage, **params)
    s.set_structure(ph, react)
    s.step(10)
    o = _oracle(ph, react, **params)
    o.step(10)
    np.testing.assert_allclose(s.field(), o.concentration(), rtol=0, atol=_tol(10, storage))
    from paper_1410_1914_gb300 import Solver
    s7 = Solver(ph.shape, storage="fp32pop", **params)
    s7.set_structure(ph, react)
    s7.step(10)
    o7 = oracle.OracleLBM(ph, react=react, **params)
    o7.step(10)
    np.testing.assert_allclose(s7.field(), o7.concentration(), rtol=0, atol=_tol(10, "fp32pop"))
