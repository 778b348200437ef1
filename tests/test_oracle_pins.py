"""The FP64 oracle pinned to results fixed by mathematics, not by itself.

  * closed forms of the discrete scheme: homogeneous slab (D_eff = D), layers
    in series (cell-wise harmonic mean), layers in parallel (porosity-weighted
    mean), 1D diffusion into a first-order reactive wall;
  * a textbook special case: with one relaxation time tau = 1 the steady
    state of the D3Q7 scheme with half-way walls equals the cell-centred
    finite-volume solution of Eq. 6 (7-point stencil, half-cell Dirichlet
    faces, reactive faces as series resistances); checked on random porous
    boxes against scipy's sparse direct solver;
  * invariants: mass conservation in a closed box, the exact per-step balance
    sum C(t+1) - sum C(t) = J_in - J_out - R, mirror symmetries, tau_ref
    invariance of 1D steady states;
  * the validation geometry of Sec. 5.1 (a solid sphere filling a cube) in a
    band around its printed D_eff.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import oracle

DX = 1e-8
DB = 1e-5


def _solve(o, tol=1e-14, check=200, max_steps=5_000_000):
    n = o.solve(tol=tol, check_every=check, max_steps=max_steps)
    assert n > 0, "oracle did not reach the tolerance"
    return n


def test_homogeneous_slab():
    ph = np.zeros((4, 5, 24), np.uint8)
    o = oracle.OracleLBM(ph, dx_m=DX, D_bulk=DB, tau_ref=0.9)
    o.init_field(np.zeros(ph.shape))
    _solve(o)
    d, ratio, dlu = o.effective_diffusivity()
    assert ratio == pytest.approx(1.0, rel=1e-11)
    assert dlu == pytest.approx(0.25 * (0.9 - 0.5), rel=1e-11)  # D = cs^2 (tau - 1/2)
    # linear profile between the half-way faces
    C = o.concentration()[0, 0]
    x = (np.arange(24) + 0.5) / 24
    np.testing.assert_allclose(C, 1 - x, atol=1e-11)


def test_series_layers_harmonic_mean():
    rng = np.random.default_rng(3)
    nx = 15
    Dx = rng.uniform(0.2, 1.0, nx) * DB
    ph = np.zeros((3, 4, nx), np.uint8)
    D = np.broadcast_to(Dx, ph.shape).copy()
    o = oracle.OracleLBM(ph, D=D, dx_m=DX, D_bulk=DB)
    o.init_field(np.zeros(ph.shape))
    _solve(o)
    assert o.effective_diffusivity()[0] == pytest.approx(nx / np.sum(1.0 / Dx), rel=1e-11)


def test_parallel_layers_weighted_mean():
    rng = np.random.default_rng(4)
    ny, nx = 7, 10
    Dy = rng.uniform(0.2, 1.0, ny) * DB
    ph = np.zeros((3, ny, nx), np.uint8)
    ph[:, 2, :] = 1  # a solid layer counts with D = 0
    ph[:, 5, :] = 2  # impermeable ionomer layer
    D = np.broadcast_to(Dy[None, :, None], ph.shape).copy()
    o = oracle.OracleLBM(ph, D=D, dx_m=DX, D_bulk=DB)
    o.init_field(np.zeros(ph.shape))
    _solve(o)
    Dw = Dy.copy()
    Dw[[2, 5]] = 0.0
    assert o.effective_diffusivity()[0] == pytest.approx(Dw.mean(), rel=1e-11)


@pytest.mark.parametrize("tau_ref,k", [(0.8, 80.0), (1.3, 5.0)])
def test_reactive_wall_1d(tau_ref, k):
    """Fixed C0 at x = 0, first-order sink on the wall at x = L:
    c(x) = c0 (1 - k x / (D + k L)), rate per area k D c0 / (D + k L)."""
    nx = 40
    ph = np.zeros((2, 3, nx + 1), np.uint8)
    ph[:, :, -1] = 1
    react = np.zeros_like(ph)
    react[:, :, nx - 1] = 1  # face toward +x
    o = oracle.OracleLBM(ph, react=react, dx_m=DX, D_bulk=DB, k_ms=k, bc_out=1, tau_ref=tau_ref, c_in=0.7)
    _solve(o)
    L = nx * DX
    xi = (np.arange(nx) + 0.5) * DX
    C = o.concentration()[1, 2, :nx]
    np.testing.assert_allclose(C, 0.7 * (1 - k * xi / (DB + k * L)), rtol=0, atol=1e-11)
    R, prof_R, prof_C = o.reaction_rate()
    area = 2 * 3 * DX * DX
    assert R / area == pytest.approx(k * DB * 0.7 / (DB + k * L), rel=1e-10)
    assert prof_R[nx - 1] == pytest.approx(R, rel=1e-12) and np.all(prof_R[: nx - 1] == 0)
    f = o.fluxes()
    assert f["J_in"] == pytest.approx(f["R"], rel=1e-10)  # steady state: inflow = consumption
    # Eq. 25: i_d = 4 F (rate per area), here 4 F k D c0 / (D + k L)
    assert o.current_density() == pytest.approx(4 * 96485.33212 * k * DB * 0.7 / (DB + k * L), rel=1e-10)


# ---------------------------------------------------------------- FV pin
def _fv_solution(phase_active, D_lu, react_bits, k_lu, bc_in, bc_out, c_in, c_out):
    """Cell-centred finite volumes for div(D grad C) = 0 on the active cells:
    harmonic face conductances, half-cell Dirichlet faces, catalytic faces as a
    half-cell resistance in series with 1/k."""
    nz, ny, nx = phase_active.shape
    idx = lambda x, y, z: x + nx * (y + ny * z)
    N = nx * ny * nz
    A = sp.lil_matrix((N, N))
    b = np.zeros(N)
    dirs = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                c = idx(x, y, z)
                if not phase_active[z, y, x]:
                    A[c, c] = 1.0
                    continue
                Dc = D_lu[z, y, x]
                for d, (ex, ey, ez) in enumerate(dirs):
                    qx = x + ex
                    if qx < 0 or qx >= nx:
                        bc, cb = (bc_in, c_in) if qx < 0 else (bc_out, c_out)
                        if bc == 0:
                            A[c, c] += 2 * Dc
                            b[c] += 2 * Dc * cb
                        continue
                    qy, qz = (y + ey) % ny, (z + ez) % nz
                    if not phase_active[qz, qy, qx]:
                        if k_lu > 0 and (react_bits[z, y, x] >> d) & 1:
                            A[c, c] += 1.0 / (1.0 / (2 * Dc) + 1.0 / k_lu)
                        continue
                    g = 1.0 / (1.0 / (2 * Dc) + 1.0 / (2 * D_lu[qz, qy, qx]))
                    A[c, c] += g
                    A[c, idx(qx, qy, qz)] -= g
    return spl.spsolve(A.tocsr(), b).reshape(nz, ny, nx)


@pytest.mark.parametrize("seed,bc_out,k", [(1, 0, 0.0), (2, 1, 50.0), (3, 0, 20.0)])
def test_tau1_equals_finite_volume(seed, bc_out, k):
    rng = np.random.default_rng(seed)
    shape = (5, 6, 9)
    ph = (rng.random(shape) < 0.3).astype(np.uint8)
    ph[rng.random(shape) < 0.05] = 3  # micropores transport like pores
    react = rng.integers(0, 64, shape).astype(np.uint8)
    o = oracle.OracleLBM(ph, react=react, dx_m=DX, D_bulk=DB, k_ms=k, tau_ref=1.0, bc_out=bc_out,
                         c_in=1.0, c_out=0.2)
    _solve(o, tol=1e-15, check=500)
    act = o.active() > 0
    C = o.concentration()
    D_lu = np.where(act, 0.25 * (o.tau() - 0.5), 0.0)
    Cf = _fv_solution(act, D_lu, o.react(), o.k_lu, 0, bc_out, 1.0, 0.2)
    np.testing.assert_allclose(C[act], Cf[act], rtol=0, atol=1e-11)


# ------------------------------------------------------------ invariants
def test_closed_box_conserves_mass():
    rng = np.random.default_rng(5)
    ph = (rng.random((6, 7, 8)) < 0.35).astype(np.uint8)
    ph[:, :, 0] = 0  # keep an inlet plane so the set-up has active cells
    D = rng.uniform(0.3, 1.0, ph.shape) * DB
    o = oracle.OracleLBM(ph, D=D, dx_m=DX, D_bulk=DB, bc_in=1, bc_out=1)
    o.init_field(rng.random(ph.shape))
    m0 = o.fluxes()["sum_C"]
    o.step(300)
    assert o.fluxes()["sum_C"] == pytest.approx(m0, rel=1e-13)


@pytest.mark.parametrize("bc_out", [0, 1])
def test_per_step_balance(bc_out):
    rng = np.random.default_rng(6)
    ph = (rng.random((7, 6, 11)) < 0.3).astype(np.uint8)
    react = rng.integers(0, 64, ph.shape).astype(np.uint8)
    o = oracle.OracleLBM(ph, react=react, dx_m=DX, D_bulk=DB, k_ms=30.0, bc_out=bc_out, c_out=0.1,
                         knudsen=1, T_K=353.0)
    o.init_field(rng.random(ph.shape))
    for _ in range(20):
        f0 = o.fluxes()
        o.step(1)
        f1 = o.fluxes()
        assert f1["sum_C"] - f0["sum_C"] == pytest.approx(f0["J_in"] - f0["J_out"] - f0["R"], abs=1e-12)


def test_mirror_symmetries():
    rng = np.random.default_rng(7)
    ph = (rng.random((6, 7, 10)) < 0.3).astype(np.uint8)
    react = rng.integers(0, 64, ph.shape).astype(np.uint8)

    def run(p, r, **kw):
        o = oracle.OracleLBM(p, react=r, dx_m=DX, D_bulk=DB, k_ms=30.0, **kw)
        o.init_linear()
        o.step(250)
        return o

    base = run(ph, react)
    # y mirror: swap the +y/-y face bits (d = 3, 4 -> bits 2, 3)
    ry = react[:, ::-1, :].copy()
    ry = (ry & ~np.uint8(0b1100)) | ((ry & 0b0100) << 1) | ((ry & 0b1000) >> 1)
    my = run(ph[:, ::-1, :].copy(), ry)
    np.testing.assert_allclose(my.concentration(), base.concentration()[:, ::-1, :], atol=1e-13)
    # z mirror: swap +z/-z (bits 4, 5)
    rz = react[::-1].copy()
    rz = (rz & ~np.uint8(0b110000)) | ((rz & 0b010000) << 1) | ((rz & 0b100000) >> 1)
    mz = run(ph[::-1].copy(), rz)
    np.testing.assert_allclose(mz.concentration(), base.concentration()[::-1], atol=1e-13)
    # transposing y and z (cube in y-z) with the face bits exchanged
    sq = (rng.random((6, 6, 10)) < 0.3).astype(np.uint8)
    a = oracle.OracleLBM(sq, dx_m=DX, D_bulk=DB)
    a.step(200)
    b = oracle.OracleLBM(sq.transpose(1, 0, 2).copy(), dx_m=DX, D_bulk=DB)
    b.step(200)
    np.testing.assert_allclose(b.concentration(), a.concentration().transpose(1, 0, 2), atol=1e-13)


def test_x_mirror_swapped_boundaries_same_deff():
    rng = np.random.default_rng(8)
    ph = (rng.random((5, 6, 12)) < 0.25).astype(np.uint8)
    ph[:, :, 0] = 0
    ph[:, :, -1] = 0
    a = oracle.OracleLBM(ph, dx_m=DX, D_bulk=DB, c_in=1.0, c_out=0.0)
    _solve(a)
    b = oracle.OracleLBM(ph[:, :, ::-1].copy(), dx_m=DX, D_bulk=DB, c_in=1.0, c_out=0.0)
    _solve(b)
    assert a.effective_diffusivity()[0] == pytest.approx(b.effective_diffusivity()[0], rel=1e-10)


def test_tau_ref_invariance_1d():
    ph = np.zeros((2, 2, 16), np.uint8)
    rng = np.random.default_rng(9)
    D = np.broadcast_to(rng.uniform(0.3, 1, 16) * DB, ph.shape).copy()
    vals = []
    for tau in (0.6, 1.0, 1.7):
        o = oracle.OracleLBM(ph, D=D, dx_m=DX, D_bulk=DB, tau_ref=tau)
        o.init_field(np.zeros(ph.shape))
        _solve(o)
        vals.append(o.effective_diffusivity()[0])
    assert vals[0] == pytest.approx(vals[1], rel=1e-10) and vals[2] == pytest.approx(vals[1], rel=1e-10)


def test_no_path_is_an_error():
    ph = np.ones((3, 3, 5), np.uint8)
    with pytest.raises(ValueError):
        oracle.OracleLBM(ph, dx_m=DX, D_bulk=DB)


HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------- sphere in a cube
def _sphere_phase(n):
    c = (np.arange(n) + 0.5) - n / 2
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return ((x * x + y * y + z * z) < (n / 2) ** 2).astype(np.uint8)  # 1 = solid


def test_sphere_in_cube_matches_the_printed_validation_band():
    """Sec. 5.1 validates the solver on a cube holding a solid sphere whose
    diameter is the cube side and prints D_eff/D = 0.3317.  Voxel rule and
    lattice differ here (cell centres inside the sphere are solid; D3Q7), so
    the printed value is a band: the oracle at 32^3 must land within 4 %.
    The resolution error of this geometry is itself a few per cent at 32^3
    (0.321 at 32^3, 0.332 at 48^3, 0.338 at 96^3 by the finite-volume
    equivalent of the scheme)."""
    import json
    with open(os.path.join(HERE, "golden", "paper_values.json")) as fh:
        ref = json.load(fh)["sphere_in_cube_deff"]["value"]
    ph = _sphere_phase(32)
    o = oracle.OracleLBM(ph, D_bulk=1e-5, knudsen=0, tau_ref=1.0)
    o.solve(tol=1e-9, check_every=200, max_steps=400_000)
    d_eff, d_rel, _ = o.effective_diffusivity()
    assert d_rel == pytest.approx(ref, rel=0.04)
    # the porosity of the voxelised sphere is close to 1 - pi/6
    assert 1 - ph.mean() == pytest.approx(1 - np.pi / 6, abs=0.01)


# ------------------------------------------------ proton conduction (Eq. 16)
SIGMA = 3.0  # ionomer conductivity in any unit (the normalised results do not depend on it)


def test_protons_see_the_ionomer_and_o2_the_pores():
    """Parallel channels along x: ionomer fills 5 of 20 cross-section cells,
    pore 8, solid the rest.  Protons (Eq. 16, uniform conductivity, no
    source) give sigma_eff / sigma = 5/20 exactly; O2 in the same box gives
    D_eff / D_b = 8/20.  The carrier alone decides which phase conducts."""
    ph = np.ones((4, 5, 12), np.uint8)  # (nz, ny, nx)
    ph[0, 0:5, :] = 2                   # 5 ionomer lines
    ph[2, 0:5, :] = 0                   # 5 pore lines
    ph[3, 1:4, :] = 0                   # 3 more pore lines
    op = oracle.OracleLBM(ph, dx_m=DX, D_bulk=DB, D_ionomer=SIGMA, carrier=1, tau_ref=0.8)
    _solve(op)
    assert op.effective_diffusivity()[1] == pytest.approx(5 / 20, rel=1e-11)
    assert op.active().sum() == 5 * 12
    oo = oracle.OracleLBM(ph, dx_m=DX, D_bulk=DB, tau_ref=0.8)
    _solve(oo)
    assert oo.effective_diffusivity()[1] == pytest.approx(8 / 20, rel=1e-11)


def test_protons_ignore_ionomer_pockets_and_pore_links():
    """An ionomer pocket joined to the inlet only through pore cells is not
    on the proton path (the active set is ionomer 6-connected to x = 0)."""
    ph = np.ones((3, 3, 8), np.uint8)
    ph[1, 1, :] = 2          # one ionomer line through the box
    ph[0, 0, 0:3] = 0        # pore from the inlet ...
    ph[0, 0, 3:6] = 2        # ... to an ionomer pocket
    act = oracle.active_mask(ph, protons=True)
    assert act[1, 1].all() and not act[0, 0].any()
    o = oracle.OracleLBM(ph, dx_m=DX, D_bulk=DB, D_ionomer=SIGMA, carrier=1)
    _solve(o)
    assert o.effective_diffusivity()[1] == pytest.approx(1 / 9, rel=1e-11)


@pytest.mark.parametrize("seed", [4, 5])
def test_protons_tau1_equal_finite_volume(seed):
    """Random ionomer network: the proton steady state at tau = 1 equals
    the finite-volume solution on the ionomer cells connected to x = 0."""
    rng = np.random.default_rng(seed)
    shape = (5, 6, 9)
    ph = rng.choice([0, 1, 2, 3], size=shape, p=[0.3, 0.2, 0.45, 0.05]).astype(np.uint8)
    ph[:, :, 0] = 2  # an ionomer inlet plane
    o = oracle.OracleLBM(ph, dx_m=DX, D_bulk=DB, D_ionomer=SIGMA, carrier=1, tau_ref=1.0, c_in=1.0, c_out=0.0)
    _solve(o, tol=1e-15, check=500)
    act = o.active() > 0
    assert act.sum() == oracle.active_mask(ph, protons=True).sum()
    assert not act[ph != 2].any()
    D_lu = np.where(act, 0.25 * (o.tau() - 0.5), 0.0)
    Cf = _fv_solution(act, D_lu, np.zeros(shape, np.uint8), 0.0, 0, 0, 1.0, 0.0)
    np.testing.assert_allclose(o.concentration()[act], Cf[act], rtol=0, atol=1e-11)


def test_protons_need_a_conductivity_and_no_sink():
    ph = np.full((2, 2, 4), 2, np.uint8)
    with pytest.raises(ValueError):
        oracle.OracleLBM(ph, carrier=1)                 # D_ionomer = 0
    with pytest.raises(ValueError):
        oracle.OracleLBM(ph, carrier=1, D_ionomer=1.0, k_ms=1.0)
