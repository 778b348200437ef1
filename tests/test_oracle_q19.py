"""The FP64 oracle on the paper's D3Q19 lattice (Eq. 22-24), pinned to results
fixed by mathematics, not by itself.

  * Eq. 22-23 directly: one streaming step from a single seeded cell puts
    a_i C on x + c_i, which shows the velocity set (6 axis and 12 face
    diagonal neighbours, no corners) and the weights 1/3, 1/18, 1/36;
  * closed forms of the discrete scheme: homogeneous slab (D_eff = D, any
    tau), layers in series (cell-wise harmonic mean, any tau: an
    x-dependent problem reduces to a three-velocity chain), 1D diffusion
    into a first-order reactive wall (any tau), and x-invariant channels at
    tau = 1 (the profile is linear and every cross-section cell conducts in
    proportion to the weight of its open +x links);
  * a textbook special case: at tau = 1 the post-collision populations are
    a_i C, so the steady state solves the lattice's own 19-point linear
    system, assembled here link by link and solved by scipy;
  * invariants: mass conservation, the per-step balance, mirror symmetries;
  * the validation geometry of Sec. 5.1, which the paper computed on this
    lattice, in a band around its printed D_eff.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import oracle

DX = 1e-8
DB = 1e-5
Q19 = 1
HERE = os.path.dirname(os.path.abspath(__file__))

# Eq. 22 written out for the tests (0 rest, 6 axes, 12 face diagonals)
AXES = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
DIAG = [(1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
        (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
C19 = [(0, 0, 0)] + AXES + DIAG
A19 = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12


def _solve(o, tol=1e-14, check=200, max_steps=5_000_000):
    n = o.solve(tol=tol, check_every=check, max_steps=max_steps)
    assert n > 0, "oracle did not reach the tolerance"
    return n


def test_one_step_spreads_a_seed_over_the_d3q19_stencil():
    """tau = 1: the post-collision populations of a cell are a_i C, and one
    step carries each to x + c_i.  The receiving cells are exactly the 18
    face and edge neighbours (Eq. 22) and each gets a_i C (Eq. 23)."""
    ph = np.zeros((7, 7, 9), np.uint8)
    o = oracle.OracleLBM(ph, dx_m=DX, D_bulk=DB, tau_ref=1.0, lattice=Q19, bc_in=1, bc_out=1)
    C0 = np.zeros(ph.shape)
    C0[3, 3, 4] = 1.0
    o.init_field(C0)
    np.testing.assert_allclose(o.populations()[:, 3, 3, 4], A19, rtol=1e-15)
    o.step(1)
    C = o.concentration()
    expect = np.zeros(ph.shape)
    for (cx, cy, cz), a in zip(C19, A19):
        expect[3 + cz, 3 + cy, 4 + cx] = a
    np.testing.assert_allclose(C, expect, rtol=0, atol=1e-16)
    assert C.sum() == pytest.approx(1.0, rel=1e-15)


def test_homogeneous_slab():
    ph = np.zeros((4, 5, 24), np.uint8)
    o = oracle.OracleLBM(ph, dx_m=DX, D_bulk=DB, tau_ref=0.9, lattice=Q19)
    o.init_field(np.zeros(ph.shape))
    _solve(o)
    d, ratio, dlu = o.effective_diffusivity()
    assert ratio == pytest.approx(1.0, rel=1e-11)
    assert dlu == pytest.approx((0.9 - 0.5) / 3, rel=1e-11)  # Eq. 24: D = (tau - 1/2) / 3
    x = (np.arange(24) + 0.5) / 24
    np.testing.assert_allclose(o.concentration()[2, 3], 1 - x, atol=1e-11)


def test_series_layers_harmonic_mean():
    rng = np.random.default_rng(3)
    nx = 15
    Dx = rng.uniform(0.2, 1.0, nx) * DB
    ph = np.zeros((3, 4, nx), np.uint8)
    D = np.broadcast_to(Dx, ph.shape).copy()
    o = oracle.OracleLBM(ph, D=D, dx_m=DX, D_bulk=DB, lattice=Q19)
    o.init_field(np.zeros(ph.shape))
    _solve(o)
    assert o.effective_diffusivity()[0] == pytest.approx(nx / np.sum(1.0 / Dx), rel=1e-11)


@pytest.mark.parametrize("seed", [1, 2])
def test_channels_tau1_closed_form(seed):
    """x-invariant structure at tau = 1: C is the linear ramp in every open
    cell, and a cell of the cross-section carries the flux of the open +x
    links of its stencil.  A +x link is open when the cross-section cell it
    lands on (y + c_y, z + c_z) is open.  So D_eff / D = mean over the
    cross-section of (sum of a_i over open +x links) / (1/6).  A wall
    parallel to the flow takes one 1/36 diagonal from each cell next to
    it: the bounce-back wall of this lattice conducts less than the open
    fraction (by 1/6 per wall-adjacent cell and wall)."""
    rng = np.random.default_rng(seed)
    ny, nz, nx = 7, 6, 9
    sec = rng.random((nz, ny)) < 0.3
    sec[0, 0] = False
    ph = np.broadcast_to(sec[:, :, None], (nz, ny, nx)).astype(np.uint8)
    o = oracle.OracleLBM(ph, dx_m=DX, D_bulk=DB, tau_ref=1.0, lattice=Q19)
    _solve(o, tol=1e-15)
    act = o.active()[:, :, 0] > 0
    # every open line touches the inlet plane, so every open cell is active
    assert np.array_equal(act, ~sec)
    x = (np.arange(nx) + 0.5) / nx
    C = o.concentration()
    np.testing.assert_allclose(C[act], np.broadcast_to(1 - x, (act.sum(), nx)), atol=1e-12)
    cond = 0.0
    for z in range(nz):
        for y in range(ny):
            if not act[z, y]:
                continue
            for (cx, cy, cz), a in zip(C19, A19):
                if cx == 1 and act[(z + cz) % nz, (y + cy) % ny]:
                    cond += a
    assert o.effective_diffusivity()[1] == pytest.approx(cond / (1 / 6) / (ny * nz), rel=1e-11)


@pytest.mark.parametrize("tau_ref,k", [(0.8, 80.0), (1.3, 5.0)])
def test_reactive_wall_1d(tau_ref, k):
    """Fixed C0 at x = 0, first-order sink on the wall at x = L:
    c(x) = c0 (1 - k x / (D + k L)), rate per area k D c0 / (D + k L).  The
    axis link and the four diagonals that cross the catalytic face share
    the face's rate in proportion to their weights."""
    nx = 40
    ph = np.zeros((2, 3, nx + 1), np.uint8)
    ph[:, :, -1] = 1
    react = np.zeros_like(ph)
    react[:, :, nx - 1] = 1  # face toward +x
    o = oracle.OracleLBM(ph, react=react, dx_m=DX, D_bulk=DB, k_ms=k, bc_out=1, tau_ref=tau_ref, c_in=0.7,
                         lattice=Q19)
    _solve(o)
    L = nx * DX
    xi = (np.arange(nx) + 0.5) * DX
    C = o.concentration()[1, 2, :nx]
    np.testing.assert_allclose(C, 0.7 * (1 - k * xi / (DB + k * L)), rtol=0, atol=1e-11)
    R, prof_R, _ = o.reaction_rate()
    area = 2 * 3 * DX * DX
    assert R / area == pytest.approx(k * DB * 0.7 / (DB + k * L), rel=1e-10)
    assert prof_R[nx - 1] == pytest.approx(R, rel=1e-12) and np.all(prof_R[: nx - 1] == 0)
    # the five links that cross the +x face: +x and the diagonals with c_x = +1
    bits = o.react()[0, 0, nx - 1]
    links = {C19[i] for i in range(1, 19) if bits >> (i - 1) & 1}
    assert links == {c for c in C19 if c[0] == 1}


# --------------------------------------------------------- link rules
def _end_cell(x, y, z, c, shape):
    """End cell of the link toward x + c, with the mirror image of the end
    planes beyond x = 0 and x = L; also whether it left the box."""
    nz, ny, nx = shape
    qx = x + c[0]
    out = qx < 0 or qx >= nx
    return (x if out else qx), (y + c[1]) % ny, (z + c[2]) % nz, out


def _face_catalytic(ph, react, x, y, z, f):
    nz, ny, nx = ph.shape
    ex, ey, ez = AXES[f]
    qx = x + ex
    if qx < 0 or qx >= nx or not (react[z, y, x] >> f) & 1:
        return False
    return ph[(z + ez) % nz, (y + ey) % ny, qx] == 1


def _reactive_links(ph, react, act):
    """Link i reacts: its end cell is solid and it crosses a face of the
    cell that is marked and borders solid."""
    out = np.zeros(ph.shape, np.uint32)
    nz, ny, nx = ph.shape
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if not act[z, y, x]:
                    continue
                for i in range(1, 19):
                    c = C19[i]
                    ex, ey, ez, _ = _end_cell(x, y, z, c, ph.shape)
                    if ph[ez, ey, ex] != 1:
                        continue
                    faces = [f for f, (ax, ay, az) in enumerate(AXES)
                             if (ax and ax == c[0]) or (ay and ay == c[1]) or (az and az == c[2])]
                    if any(_face_catalytic(ph, react, x, y, z, f) for f in faces):
                        out[z, y, x] |= np.uint32(1 << (i - 1))
    return out


def test_reactive_link_rule_hand_cases():
    """A catalytic floor is crossed by five links; a solid edge that only
    touches the cell between two open faces is a plain wall; in a concave
    corner the diagonal into the corner reacts when either face it crosses
    is catalytic."""
    ph = np.zeros((3, 5, 6), np.uint8)  # (z, y, x)
    ph[:, 0, :] = 1                     # solid floor y = 0
    ph[:, 3, 3] = 1                     # a solid column at (x 3, y 3)
    ph[:, 1, 5] = 1                     # a solid block at (x 5, y 1) on the floor
    react = np.full(ph.shape, 0x3F, np.uint8)
    react[:, 1, 4] = 0x01               # cell (x 4, y 1): only its +x face is marked
    o = oracle.OracleLBM(ph, react=react, dx_m=DX, D_bulk=DB, k_ms=1.0, lattice=Q19)
    bits = o.react()
    got = lambda x, y: {C19[i] for i in range(1, 19) if bits[1, y, x] >> (i - 1) & 1}
    # on the floor: the five links with c_y = -1
    assert got(1, 1) == {c for c in C19 if c[1] == -1}
    # the column cell (3, 3) is reached from (2, 2) only by the (+1, +1)
    # diagonal, through the edge between two open faces: a plain wall
    assert got(2, 2) == set()
    # under the column: the links with c_y = +1 that end in the column
    assert got(3, 2) == {(0, 1, 0), (0, 1, 1), (0, 1, -1)}
    # corner of floor and block, only +x marked: the +x links and the
    # (+1, -1) diagonal into the corner; the floor links stay walls
    assert got(4, 1) == {(1, 0, 0), (1, 0, 1), (1, 0, -1), (1, -1, 0)}
    assert np.array_equal(bits, _reactive_links(ph, react, o.active() > 0))


# ------------------------------------------------ tau = 1 linear system
def _stencil_solution(ph, act, react_links, k_lu, bc_in, bc_out, c_in, c_out):
    """Steady state of the D3Q19 scheme at tau = 1 from its own linear
    system.  With tau = 1 every post-collision population is a_i C, so the
    population arriving along c_i is a_i C(x - c_i) over an open link,
    r a_i C(x) from a wall (r = 1 unless reactive), -a_i C(x) + 2 a_i C_b
    over a Dirichlet face and a_i C(x) over a zero-flux face; C(x) is their
    sum."""
    nz, ny, nx = ph.shape
    cs2 = 1 / 3
    r = (cs2 - k_lu) / (cs2 + k_lu)
    idx = lambda x, y, z: x + nx * (y + ny * z)
    N = ph.size
    A = sp.lil_matrix((N, N))
    b = np.zeros(N)
    opp = {c: C19.index((-c[0], -c[1], -c[2])) for c in C19}
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                row = idx(x, y, z)
                A[row, row] += 1.0
                if not act[z, y, x]:
                    continue
                A[row, row] -= A19[0]
                for i in range(1, 19):
                    a = A19[i]
                    j = opp[C19[i]]  # the link the population arrives through
                    ex, ey, ez, out = _end_cell(x, y, z, C19[j], ph.shape)
                    if out and act[ez, ey, ex]:
                        bc, cb = (bc_in, c_in) if x + C19[j][0] < 0 else (bc_out, c_out)
                        if bc == 0:
                            A[row, row] += a
                            b[row] += 2 * a * cb
                        else:
                            A[row, row] -= a
                    elif not act[ez, ey, ex]:
                        rr = r if (react_links[z, y, x] >> (j - 1)) & 1 else 1.0
                        A[row, row] -= rr * a
                    else:
                        A[row, idx(ex, ey, ez)] -= a
    return spl.spsolve(A.tocsr(), b).reshape(ph.shape)


@pytest.mark.parametrize("seed,bc_out,k", [(1, 0, 0.0), (2, 1, 50.0), (3, 0, 20.0)])
def test_tau1_equals_stencil_system(seed, bc_out, k):
    rng = np.random.default_rng(seed)
    shape = (5, 6, 9)
    ph = (rng.random(shape) < 0.3).astype(np.uint8)
    ph[rng.random(shape) < 0.05] = 3
    react = rng.integers(0, 64, shape).astype(np.uint8)
    o = oracle.OracleLBM(ph, react=react, dx_m=DX, D_bulk=DB, k_ms=k, tau_ref=1.0, bc_out=bc_out,
                         c_in=1.0, c_out=0.2, lattice=Q19)
    _solve(o, tol=1e-15, check=500)
    act = o.active() > 0
    links = _reactive_links(ph, react, act) if k > 0 else np.zeros(shape, np.uint32)
    if k > 0:
        np.testing.assert_array_equal(o.react(), links)
    Cs = _stencil_solution(ph, act, links, o.k_lu, 0, bc_out, 1.0, 0.2)
    np.testing.assert_allclose(o.concentration()[act], Cs[act], rtol=0, atol=1e-11)


# ------------------------------------------------------------ invariants
def test_closed_box_conserves_mass():
    rng = np.random.default_rng(5)
    ph = (rng.random((6, 7, 8)) < 0.35).astype(np.uint8)
    ph[:, :, 0] = 0
    D = rng.uniform(0.3, 1.0, ph.shape) * DB
    o = oracle.OracleLBM(ph, D=D, dx_m=DX, D_bulk=DB, bc_in=1, bc_out=1, lattice=Q19)
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
                         knudsen=1, T_K=353.0, lattice=Q19)
    o.init_field(rng.random(ph.shape))
    for _ in range(20):
        f0 = o.fluxes()
        o.step(1)
        f1 = o.fluxes()
        assert f1["sum_C"] - f0["sum_C"] == pytest.approx(f0["J_in"] - f0["J_out"] - f0["R"], abs=1e-12)


def _swap_bits(r, a, b):
    ba, bb = np.uint8(1 << a), np.uint8(1 << b)
    out = r & ~np.uint8(ba | bb)
    out |= np.where(r & ba, bb, 0).astype(np.uint8)
    out |= np.where(r & bb, ba, 0).astype(np.uint8)
    return out


def test_mirror_symmetries():
    """Mirroring the box in y or z (with the face bits mirrored), or
    exchanging y and z, mirrors the field: catches a wrong sign, index or
    opposite in the 19-velocity tables."""
    rng = np.random.default_rng(7)
    ph = (rng.random((6, 7, 10)) < 0.3).astype(np.uint8)
    react = rng.integers(0, 64, ph.shape).astype(np.uint8)

    def run(p, r, **kw):
        o = oracle.OracleLBM(p, react=r, dx_m=DX, D_bulk=DB, k_ms=30.0, lattice=Q19, **kw)
        o.init_linear()
        o.step(250)
        return o

    base = run(ph, react)
    my = run(ph[:, ::-1, :].copy(), _swap_bits(react[:, ::-1, :], 2, 3))
    np.testing.assert_allclose(my.concentration(), base.concentration()[:, ::-1, :], atol=1e-13)
    mz = run(ph[::-1].copy(), _swap_bits(react[::-1], 4, 5))
    np.testing.assert_allclose(mz.concentration(), base.concentration()[::-1], atol=1e-13)
    sq = (rng.random((6, 6, 10)) < 0.3).astype(np.uint8)
    rs = rng.integers(0, 64, sq.shape).astype(np.uint8)
    a = run(sq, rs)
    rt = rs.transpose(1, 0, 2).copy()
    rt = _swap_bits(_swap_bits(rt, 2, 4), 3, 5)
    b = run(sq.transpose(1, 0, 2).copy(), rt)
    np.testing.assert_allclose(b.concentration(), a.concentration().transpose(1, 0, 2), atol=1e-13)


def test_x_mirror_swapped_boundaries_same_deff():
    rng = np.random.default_rng(8)
    ph = (rng.random((5, 6, 12)) < 0.25).astype(np.uint8)
    ph[:, :, 0] = 0
    ph[:, :, -1] = 0
    a = oracle.OracleLBM(ph, dx_m=DX, D_bulk=DB, lattice=Q19)
    _solve(a)
    b = oracle.OracleLBM(ph[:, :, ::-1].copy(), dx_m=DX, D_bulk=DB, lattice=Q19)
    _solve(b)
    assert a.effective_diffusivity()[0] == pytest.approx(b.effective_diffusivity()[0], rel=1e-10)


def test_lattice_code_is_checked():
    with pytest.raises(ValueError):
        oracle.OracleLBM(np.zeros((2, 2, 3), np.uint8), lattice=2)


# ------------------------------------------------------- sphere in a cube
def test_sphere_in_cube_d3q19():
    """Sec. 5.1 computed D_eff/D = 0.3317 for a solid sphere filling a cube
    on this lattice at 200^3.  At 32^3 the oracle must land within 6 % of it
    (the bounce-back walls of D3Q19 conduct less than the open fraction, so
    the coarse grid sits below; 0.313 here against 0.321 on D3Q7) and
    within 4 % of the D3Q7 value of the same voxels."""
    with open(os.path.join(HERE, "golden", "paper_values.json")) as fh:
        ref = json.load(fh)["sphere_in_cube_deff"]["value"]
    n = 32
    c = (np.arange(n) + 0.5) - n / 2
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    ph = ((x * x + y * y + z * z) < (n / 2) ** 2).astype(np.uint8)
    vals = {}
    for lat in (0, 1):
        o = oracle.OracleLBM(ph, D_bulk=1e-5, knudsen=0, tau_ref=1.0, lattice=lat)
        o.solve(tol=1e-9, check_every=200, max_steps=400_000)
        vals[lat] = o.effective_diffusivity()[1]
    assert vals[1] == pytest.approx(ref, rel=0.06)
    assert vals[1] == pytest.approx(vals[0], rel=0.04)
