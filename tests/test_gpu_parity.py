"""CUDA path vs the FP64 oracle, through the C ABI (gpu).

Integer set-up products (connectivity, 13-direction lengths, link masks) must
match bit for bit; floating-point results within the bounds stated per
storage mode (tests/tolerances.py):
  fp32     C as double-float, deviations f32: the f32 rounding of the
           returned O(1) field (1e-7);
  fp16dev  deviations as scaled f16 (11-bit significand): 8 * 2^-11 of the
           largest deviation the oracle's populations show over the case's
           trajectory, so mild cases get a bound as tight as their
           deviations and strongly catalytic walls a looser one;
  fp32pop  7 plain f32 populations: ulps of O(1) values per step.
Sizes span several 64-cell x tiles and 8-row y tiles with ragged tails.
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


def _solver(shape, storage="fp32", **params):
    from paper_1410_1914_gb300 import Solver
    return Solver(shape, storage=storage, **params)


def _tol(storage, steps):
    return {"fp32": 1e-7 + 1e-10 * steps, "fp16dev": 8e-5 + 1e-7 * steps,
            "fp32pop": 2e-6 + 1e-7 * steps}[storage]


CASES = {
    # (workload recipe, shape (nz, ny, nx), seed, extra params)
    "pt_ragged": ("pt_cl_256", (13, 17, 291), 21, dict(k_ms=2e4)),
    "pt_deff": ("pt_cl_48", (19, 23, 37), 22, {}),
    "npmc": ("npmc_cl_400", (24, 20, 150), 23, dict(k_ms=5e3)),
    "thin": ("pt_cl_256", (3, 5, 40), 24, dict(k_ms=2e4)),
    # the workloads' own rate constants: at nm voxels k dt / dx is ~1e-8 (Pt, 1e-3 m/s) and
    # ~1e-10 (NPMC, 1e-5 m/s) of 2w, where 1 - r must be formed without cancellation
    "pt_physical_k": ("pt_cl_256", (13, 17, 291), 25, {}),
    "npmc_physical_k": ("npmc_cl_400", (24, 20, 150), 26, {}),
}


def _case(name):
    wl, shape, seed, extra = CASES[name]
    ph, react, params = inputs.make_workload(wl, shape=shape, seed=seed)
    params = dict(params, **extra)
    return ph, react, params


@pytest.mark.parametrize("name", sorted(CASES))
def test_setup_bit_exact(cuda_lib, name):
    ph, react, params = _case(name)
    s = _solver(ph.shape, **params)
    s.set_structure(ph, react)
    su = s.setup(chord=True)
    o = oracle.OracleLBM(ph, react=react, **params)
    np.testing.assert_array_equal(su["active"], o.active())
    np.testing.assert_array_equal(su["chord"], oracle.chord_counts(ph))
    np.testing.assert_array_equal((su["mask"] >> 6) & 0x3F, o.react())
    tau = o.tau()
    act = o.active() > 0
    np.testing.assert_allclose(su["omega"][act], 1.0 / tau[act], rtol=1e-6)
    assert np.all(su["omega"][~act] == 0)
    info = s.info()
    assert info["n_active"] == int(act.sum())
    assert info["D_max"] == pytest.approx(o.D_max, rel=1e-12)
    # the 13-direction pore lengths of Sec. 2.1.3 (walked line by line on the GPU)
    pore = (ph == 0) | (ph == 3)
    d_p = oracle.pore_diameter(ph, params["dx_m"])
    assert info["mean_pore_diameter_m"] == pytest.approx(d_p[pore].mean(), rel=1e-12)
    assert info["dt_s"] == pytest.approx(o.dt, rel=1e-12)
    assert info["k_lu"] == pytest.approx(o.k_lu, rel=1e-12)
    s.close()


def test_react_rule_all_pore_solid(cuda_lib):
    """The all-faces rule equals an explicit mask of every pore-solid face."""
    ph, _, params = _case("npmc")
    full = inputs.reactive_faces(ph, 1.0, 0)
    a = _solver(ph.shape, react_rule=1, **params)
    a.set_structure(ph, None)
    b = _solver(ph.shape, **params)
    b.set_structure(ph, full)
    np.testing.assert_array_equal(a.setup()["mask"], b.setup()["mask"])


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("steps", [1, 2, 10, 150])
def test_trajectory(cuda_lib, storage, name, steps):
    ph, react, params = _case(name)
    s = _solver(ph.shape, storage, **params)
    s.set_structure(ph, react)
    s.step(steps)
    o = oracle.OracleLBM(ph, react=react, **params)
    dmax = step_sampled(o, steps)
    C = s.field()
    ref = o.concentration()
    tol = field_tol(storage, steps, dmax)
    err = float(np.abs(C - ref).max())
    assert err <= tol, f"max|dC| {err:.3e} > {tol:.3e} (max|delta| {dmax:.3e}, err / (2^-11 max|delta|) = " \
        f"{err / max(2.0 ** -11 * dmax, 1e-300):.2f})"
    fg, fo = s.fluxes(), o.fluxes()
    scale = max(abs(fo["J_in"]), 1e-30)
    ftol = {"fp32": 1e-6, "fp16dev": 5e-4, "fp32pop": 2e-5}[storage]
    # absolute floor: one rounding of an O(0.1) stored value per boundary term
    nyz = ph.shape[0] * ph.shape[1]
    floor = {"fp32": 1e-9, "fp16dev": 2e-6, "fp32pop": 6e-8}[storage] * nyz + 1e-7
    assert fg["n_active"] == fo["n_active"]
    assert abs(fg["J_in"] - fo["J_in"]) <= ftol * scale + floor
    assert abs(fg["J_out"] - fo["J_out"]) <= ftol * scale + floor
    assert abs(fg["R"] - fo["R"]) <= ftol * max(abs(fo["R"]), 1e-30) + min(floor, 1e-3 * abs(fo["R"]))
    assert fg["sum_C"] == pytest.approx(fo["sum_C"], rel=max(ftol, 1e-6))
    tg, pRg, pCg = s.reaction_rate()
    to, pRo, pCo = o.reaction_rate()
    assert tg == pytest.approx(to, rel=ftol, abs=1e-30)
    np.testing.assert_allclose(pCg, pCo, atol=tol)
    assert s.current_density() == pytest.approx(o.current_density(), rel=ftol, abs=1e-30)
    s.close()


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 3, 5), (2, 1, 33), (5, 9, 1), (4, 8, 32), (1, 16, 64)])
def test_degenerate_boxes(cuda_lib, storage, shape):
    """Single cells, single rows/planes, tiles exactly full or one cell over."""
    rng = np.random.default_rng(sum(shape))
    ph = (rng.random(shape) < 0.2).astype(np.uint8)
    ph[..., 0] = 0
    react = rng.integers(0, 64, shape).astype(np.uint8)
    params = dict(dx_m=1e-8, D_bulk=1e-5, k_ms=40.0, c_in=1.0, c_out=0.25)
    s = _solver(shape, storage, **params)
    s.set_structure(ph, react)
    s.step(37)
    o = oracle.OracleLBM(ph, react=react, **params)
    dmax = step_sampled(o, 37)
    np.testing.assert_allclose(s.field(), o.concentration(), rtol=0, atol=field_tol(storage, 37, dmax))


def test_populations_layout(cuda_lib):
    """Post-collision populations, layout [7][nz][ny][nx]; their sum is C."""
    ph, react, params = _case("pt_ragged")
    for storage in STORAGES:
        s = _solver(ph.shape, storage, **params)
        s.set_structure(ph, react)
        s.step(3)
        g = s.populations()
        np.testing.assert_allclose(g.sum(axis=0), s.field(), rtol=0, atol=1e-6)
        assert s.steps == 3
        o = oracle.OracleLBM(ph, react=react, **params)
        o.step(3)
        # oracle populations are pre-collision; compare the moments instead
        np.testing.assert_allclose(g.sum(axis=0), o.populations().sum(axis=0), atol=_tol(storage, 3) + 1e-7)


@pytest.mark.parametrize("storage", STORAGES)
def test_custom_init_and_step_counter(cuda_lib, storage):
    ph, react, params = _case("pt_deff")
    rng = np.random.default_rng(0)
    C0 = rng.random(ph.shape).astype(np.float32)
    s = _solver(ph.shape, storage, **params)
    s.set_structure(ph, react)
    s.init(C0)
    s.step(65)  # one 64-step graph + one single step
    o = oracle.OracleLBM(ph, react=react, **params)
    o.init_field(C0.astype(np.float64))
    dmax = step_sampled(o, 65)
    # a random start: FP16 takes its per-case bound, the others ten times their O(1)-field bound
    tol = field_tol(storage, 65, dmax) if storage == "fp16dev" else _tol(storage, 65) * 10
    np.testing.assert_allclose(s.field(), o.concentration(), atol=tol)
    assert s.steps == 65


@pytest.mark.parametrize("storage,rel", [("fp32", 1e-3), ("fp16dev", 5e-3)])
def test_converged_deff_small_workload(cuda_lib, storage, rel):
    """48^3 plain-method workload: GPU solve vs the converged FP64 oracle
    D_eff (tests/golden/c1_deff.json): 1e-3 relative for FP32, 5e-3 for FP16
    storage."""
    with open(os.path.join(HERE, "golden", "c1_deff.json")) as fh:
        gold = json.load(fh)
    ph, react, params = inputs.make_workload("pt_cl_48")
    s = _solver(ph.shape, storage, check_every=200, tol_rel=1e-5, tol_flux=1e-4, max_steps=3_000_000, **params)
    s.set_structure(ph, react)
    info = s.solve()
    assert info["converged"] == 1, info
    d, ratio = s.effective_diffusivity()
    assert ratio == pytest.approx(gold["D_eff_over_Db"], rel=rel)
    assert d == pytest.approx(gold["D_eff_m2s"], rel=rel)


def _fv_deff_uniform(solid):
    """D_eff / D of the cell-centred finite-volume solution (uniform D on the
    conducting cells ~solid, half-cell Dirichlet faces 1 | 0 in x, periodic
    y and z), assembled with numpy and solved by conjugate gradients.  With
    tau = 1 this is the steady state of the D3Q7 scheme (pinned on the
    oracle in test_oracle_pins.py)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    nz, ny, nx = solid.shape
    Dl = (~solid).astype(float)
    N = solid.size
    ids = np.arange(N).reshape(solid.shape)
    rows, cols, vals = [], [], []
    diag = np.zeros(N)
    b = np.zeros(N)
    for ax, periodic in ((2, False), (1, True), (0, True)):
        nb, ia = np.roll(Dl, -1, axis=ax), np.roll(ids, -1, axis=ax)
        g = Dl * nb
        if not periodic:
            sl = [slice(None)] * 3
            sl[ax] = -1
            g[tuple(sl)] = 0.0
        m = g > 0
        rows += [ids[m], ia[m]]
        cols += [ia[m], ids[m]]
        vals += [-g[m], -g[m]]
        np.add.at(diag, ids[m], g[m])
        np.add.at(diag, ia[m], g[m])
    gi = 2 * Dl[:, :, 0]
    diag[ids[:, :, 0]] += gi
    b[ids[:, :, 0]] += gi
    diag[ids[:, :, -1]] += 2 * Dl[:, :, -1]
    diag[diag == 0] = 1.0
    A = sp.csr_matrix((np.concatenate(vals + [diag]), (np.concatenate(rows + [np.arange(N)]),
                                                       np.concatenate(cols + [np.arange(N)]))), shape=(N, N))
    C, info = spl.cg(A, b, rtol=1e-12, maxiter=200000, M=sp.diags(1 / diag))
    assert info == 0
    C = C.reshape(solid.shape)
    return float((2 * Dl[:, :, 0] * (1 - C[:, :, 0])).sum() * nx / (ny * nz))


def test_sphere_in_cube_96(cuda_lib):
    """The validation geometry of Sec. 5.1 (solid sphere, diameter = cube
    side) at 96^3 through the C ABI: the converged GPU D_eff equals the
    finite-volume value of the same voxels (the scheme's steady state at
    tau = 1) to 2e-5, and lies within 4 % of the printed 0.3317."""
    n = 96
    c = (np.arange(n) + 0.5) - n / 2
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    solid = (x * x + y * y + z * z) < (n / 2) ** 2
    ph = solid.astype(np.uint8)
    with _solver(ph.shape, storage="fp32", D_bulk=1e-5, knudsen=0, tau_ref=1.0, check_every=500,
                 tol_rel=1e-7, tol_flux=1e-6, max_steps=3_000_000) as s:
        s.set_structure(ph)
        info = s.solve()
        assert info["status"] == "CL_OK", info
        _, d_rel = s.effective_diffusivity()
    fv = _fv_deff_uniform(solid)
    assert d_rel == pytest.approx(fv, rel=2e-5)
    with open(os.path.join(HERE, "golden", "paper_values.json")) as fh:
        ref = json.load(fh)["sphere_in_cube_deff"]["value"]
    assert d_rel == pytest.approx(ref, rel=0.04)


# ------------------------------------------------ proton conduction (Eq. 16)
SIGMA = 2.5  # ionomer conductivity (any unit; results are normalised by it)


def _proton_case(shape=(16, 20, 70), seed=31):
    ph = inputs.pt_cl(shape, seed, 0.45, 0.1887)
    params = dict(dx_m=2e-9, D_bulk=2.9e-5, knudsen=1, D_ionomer=SIGMA, carrier=1, tau_ref=0.9,
                  c_in=1.0, c_out=0.0)
    return ph, params


@pytest.mark.parametrize("storage", ["fp32", "fp16dev"])
def test_protons_setup_and_trajectory(cuda_lib, storage):
    """Protons in the ionomer of a QSGS layer: the active set (ionomer
    6-connected to x = 0) is bit-exact, omega matches, and the field after
    150 steps matches the oracle within the storage tolerance."""
    ph, params = _proton_case()
    o = oracle.OracleLBM(ph, **params)
    with _solver(ph.shape, storage, **params) as s:
        s.set_structure(ph)
        su = s.setup()
        act = o.active() > 0
        np.testing.assert_array_equal(su["active"], o.active())
        assert not act[ph != 2].any()
        np.testing.assert_allclose(su["omega"][act], 1.0 / o.tau()[act], rtol=1e-6)
        s.step(150)
        dmax = step_sampled(o, 150)
        np.testing.assert_allclose(s.field(), o.concentration(), rtol=0, atol=field_tol(storage, 150, dmax))


def test_protons_effective_conductivity_against_finite_volume(cuda_lib):
    """Converged effective proton conductivity (Sec. 5.2) of a 40 x 40 x 64
    layer through the C ABI equals the finite-volume value on the same
    ionomer cells (tau = 1 everywhere: uniform conductivity) to 2e-5."""
    ph, params = _proton_case((40, 40, 64), 32)
    params = dict(params, tau_ref=1.0)
    act = oracle.active_mask(ph, protons=True).astype(bool)
    with _solver(ph.shape, "fp32", check_every=500, tol_rel=1e-7, tol_flux=1e-6, max_steps=4_000_000,
                 **params) as s:
        s.set_structure(ph)
        info = s.solve()
        assert info["status"] == "CL_OK", info
        d, ratio = s.effective_diffusivity()
    fv = _fv_deff_uniform(~act)
    assert ratio == pytest.approx(fv, rel=2e-5)
    assert d == pytest.approx(fv * SIGMA, rel=2e-5)
    assert 0 < ratio < (ph == 2).mean()  # below the ionomer volume fraction (tortuosity)


def test_protons_reject_sink_or_missing_conductivity(cuda_lib):
    from paper_1410_1914_gb300 import _lib as L
    with pytest.raises(L.ClError):
        _solver((4, 4, 8), "fp32", carrier=1, D_ionomer=0.0)
    with pytest.raises(L.ClError):
        _solver((4, 4, 8), "fp32", carrier=1, D_ionomer=1.0, k_ms=1.0)


def test_pore_lengths_by_thread_per_line(cuda_lib):
    """Lines longer than the warp kernels' masks (2048 cells) are walked one
    thread per line; CL_LBM_LINE_THREADS=1 forces that path, which must give
    the same set-up (a subprocess: the switch is read once per process)."""
    import subprocess
    import sys
    code = (
        "import json, numpy as np\n"
        "from paper_1410_1914_gb300 import Solver, inputs\n"
        "ph, react, params = inputs.make_workload('pt_cl_256', shape=(13, 17, 291), seed=21)\n"
        "s = Solver(ph.shape, **params); s.set_structure(ph, react); i = s.info()\n"
        "print(json.dumps([i['mean_pore_diameter_m'], i['D_max']]))\n")
    env = dict(os.environ, CL_LBM_LINE_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True,
                         cwd=os.path.dirname(HERE))
    mean_dp, dmax = json.loads(out.stdout.strip().splitlines()[-1])
    ph, react, params = inputs.make_workload("pt_cl_256", shape=(13, 17, 291), seed=21)
    pore = (ph == 0) | (ph == 3)
    assert mean_dp == pytest.approx(oracle.pore_diameter(ph, params["dx_m"])[pore].mean(), rel=1e-12)
    o = oracle.OracleLBM(ph, react=react, **params)
    assert dmax == pytest.approx(o.D_max, rel=1e-12)


@pytest.mark.parametrize("storage", ["fp32", "fp16dev"])
@pytest.mark.parametrize("lattice", [0, 1])
def test_ionomer_o2_trajectory(cuda_lib, storage, lattice):
    """O2 dissolved in the ionomer (Eq. 10-15, ionomer_o2 = 1): the ionomer
    joins the transport set with D = D_e RT/H, about 2e5 times below the
    bulk D here (relaxation near 1/2 in the ionomer); set-up and trajectory
    against the oracle."""
    ph, react, params = _case("pt_deff")
    params = dict(params, ionomer_o2=1, k_ms=5e3)
    s = _solver(ph.shape, storage, lattice=lattice, **params)
    s.set_structure(ph, react)
    o = oracle.OracleLBM(ph, react=react, lattice=lattice, **params)
    act = o.active() > 0
    np.testing.assert_array_equal(s.setup()["active"], o.active())
    assert (act & (ph == 2)).any()   # ionomer cells carry O2
    np.testing.assert_allclose(s.setup()["omega"][act], 1.0 / o.tau()[act], rtol=1e-6)
    s.step(60)
    dmax = step_sampled(o, 60)
    np.testing.assert_allclose(s.field(), o.concentration(), rtol=0,
                               atol=field_tol(storage, 60, dmax, q=19 if lattice else 7))
    s.close()
