"""The fixed-point form of the steady state, on the FP64 oracle (no GPU).

The Krylov steady solve of the library rests on two facts about the scheme
of Eq. 21-24 with the boundaries of Sec. 3.5:
  * one step S on the stored populations is affine, and its linear part A
    is the same step with zero boundary concentrations:
    S(x) = A x + S(0);
  * the state the time march converges to is the solution of
    (I - A) x = S(0), so a Krylov method on that system reaches the same
    D_eff (Eq. 19) and reaction rate as the march, in far fewer
    applications of the step.
Both are checked here with the oracle's own step (scipy's BiCGSTAB as the
library routine), on both lattices and on a reactive case.
"""
import numpy as np
import pytest

import oracle
from paper_1410_1914_gb300 import inputs

SHAPE = (16, 18, 24)


def _oracle(lattice, **extra):
    ph, react, params = inputs.make_workload("pt_cl_48", shape=SHAPE, seed=51)
    params.update(extra)
    return oracle.OracleLBM(ph, react=react, lattice=lattice, **params), ph, react, params


def _apply(o, x):
    o.set_populations(x)
    o.step(1)
    return o.populations()


@pytest.mark.parametrize("lattice", [0, 1])
def test_step_is_affine_with_zero_boundary_linear_part(lattice):
    o, ph, react, params = _oracle(lattice)
    o0 = oracle.OracleLBM(ph, react=react, lattice=lattice, **dict(params, c_in=0.0, c_out=0.0))
    rng = np.random.default_rng(5)
    shape = (o.q,) + o.shape
    act = o.active().astype(bool)
    x = rng.uniform(0.0, 0.2, shape) * act
    y = rng.uniform(-0.1, 0.1, shape) * act
    b = _apply(o, np.zeros(shape))
    assert np.abs(b).max() > 0  # the Dirichlet terms
    Ax = _apply(o0, x)
    np.testing.assert_allclose(_apply(o, x) - b, Ax, rtol=0, atol=1e-15)
    # linear: A(2x + y) = 2 Ax + Ay
    np.testing.assert_allclose(_apply(o0, 2 * x + y), 2 * Ax + _apply(o0, y), rtol=0, atol=1e-15)
    # inactive cells stay zero
    assert np.all(Ax[:, ~act] == 0)


@pytest.mark.parametrize("lattice,extra,readout", [
    (0, {}, "deff"),
    (1, {}, "deff"),
    (0, dict(k_ms=2e4, bc_out=1), "R"),
])
def test_krylov_fixed_point_is_the_marched_steady_state(lattice, extra, readout):
    from scipy.sparse.linalg import LinearOperator, bicgstab

    march, ph, react, params = _oracle(lattice, **extra)
    steps = march.solve(tol=1e-11, check_every=100, max_steps=2_000_000)
    assert steps > 0
    o, _, _, _ = _oracle(lattice, **extra)
    o0 = oracle.OracleLBM(ph, react=react, lattice=lattice, **dict(params, c_in=0.0, c_out=0.0))
    shape = (o.q,) + o.shape
    n = int(np.prod(shape))
    b = _apply(o, np.zeros(shape)).ravel()
    count = [0]

    def mv(v):
        count[0] += 1
        return v - _apply(o0, v.reshape(shape)).ravel()

    o.init_linear()
    x0 = o.populations().ravel()
    x, info = bicgstab(LinearOperator((n, n), matvec=mv), b, x0=x0, rtol=1e-11, maxiter=5000)
    assert info == 0
    # the fixed point: one more step changes nothing
    o.set_populations(x.reshape(shape))
    assert np.linalg.norm(_apply(o, x.reshape(shape)).ravel() - x) <= 1e-9 * np.linalg.norm(x)
    o.set_populations(x.reshape(shape))
    if readout == "deff":
        assert o.effective_diffusivity()[1] == pytest.approx(march.effective_diffusivity()[1], rel=1e-8)
    else:
        assert o.fluxes()["R"] == pytest.approx(march.fluxes()["R"], rel=1e-8)
    assert count[0] * 10 < steps


C7 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
C19 = C7 + [(1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
            (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


def _link_laplacian(o, params):
    """L eps in numpy from the link classes: an open link moves w_i (eps_c -
    eps_end) out of a cell, a fixed-concentration boundary link 2 w_i eps_c,
    a catalytic wall link (1 - r) w_i eps_c, a bounce-back link nothing."""
    q = o.q
    c = C19 if q == 19 else C7
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12) if q == 19 else np.array([0.25] + [0.125] * 6)
    cs2 = 1 / 3 if q == 19 else 0.25
    r = (cs2 - o.k_lu) / (cs2 + o.k_lu)
    act = o.active().astype(bool)
    react = o.react()
    nz, ny, nx = o.shape

    def apply(eps):
        out = np.zeros(o.shape)
        for z, y, x in zip(*np.nonzero(act)):
            for i in range(1, q):
                cx, cy, cz = c[i]
                ex, ey, ez = x + cx, (y + cy) % ny, (z + cz) % nz
                leaves = not 0 <= ex < nx
                end = (ez, ey, x) if leaves else (ez, ey, ex)  # mirror end cell for a link that leaves in x
                if act[end] and not leaves:
                    out[z, y, x] += w[i] * (eps[z, y, x] - eps[end])
                elif act[end]:
                    bc = params["bc_in"] if cx < 0 else params["bc_out"]
                    out[z, y, x] += 2 * w[i] * eps[z, y, x] if bc == 0 else 0.0
                elif (react[z, y, x] >> (i - 1)) & 1:
                    out[z, y, x] += (1 - r) * w[i] * eps[z, y, x]
        return out
    return apply


@pytest.mark.parametrize("lattice", [0, 1])
def test_one_step_mass_response_is_the_link_laplacian(lattice):
    """The operator behind the diffusion preconditioner: from an
    equilibrium-shaped state w_i eps, one step with zero boundary values
    changes the cell sums by exactly -L eps."""
    ph, _, params = inputs.make_workload("pt_cl_256", shape=(6, 7, 12), seed=61)
    react = inputs.reactive_faces(ph, 0.5, 3)
    params = dict(params, k_ms=3e4, bc_out=0, c_in=0.0, c_out=0.0)
    o = oracle.OracleLBM(ph, react=react, lattice=lattice, **params)
    act = o.active().astype(bool)
    assert ((o.react() != 0) & act).any()
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12) if o.q == 19 else np.array([0.25] + [0.125] * 6)
    eps = np.random.default_rng(7).uniform(0.2, 1.0, o.shape) * act
    o.set_populations(w[:, None, None, None] * eps[None])
    o.step(1)
    dC = o.populations().sum(axis=0) - eps
    np.testing.assert_allclose(dC, -_link_laplacian(o, params)(eps), rtol=0, atol=1e-14)


def _laplacian_matrix(o, params):
    """The link Laplacian of _link_laplacian as a sparse matrix over the
    active cells (vectorised; periodic y, z; either lattice, the mirror end
    cell for links that leave through an x face)."""
    import scipy.sparse as sp
    q = o.q
    c = C19 if q == 19 else C7
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12) if q == 19 else np.array([0.25] + [0.125] * 6)
    cs2 = 1 / 3 if q == 19 else 0.25
    act = o.active().astype(bool)
    nz, ny, nx = o.shape
    r = (cs2 - o.k_lu) / (cs2 + o.k_lu)
    react = o.react()
    idx = -np.ones(o.shape, np.int64)
    idx[act] = np.arange(act.sum())
    zz, yy, xx = np.nonzero(act)
    me = idx[zz, yy, xx]
    rows, cols, vals = [], [], []
    for i in range(1, q):
        cx, cy, cz = c[i]
        ex, ey, ez = xx + cx, (yy + cy) % ny, (zz + cz) % nz
        leaves = (ex < 0) | (ex >= nx)
        end = idx[ez, ey, np.where(leaves, xx, ex)]
        open_ = ~leaves & (end >= 0)
        rows += [me[open_], me[open_]]
        cols += [me[open_], end[open_]]
        vals += [np.full(open_.sum(), w[i]), np.full(open_.sum(), -w[i])]
        bnd = leaves & (end >= 0)
        if (params["bc_in"] if cx < 0 else params["bc_out"]) == 0:
            rows.append(me[bnd]); cols.append(me[bnd]); vals.append(np.full(bnd.sum(), 2 * w[i]))
        sink = (end < 0) & (((react[zz, yy, xx] >> (i - 1)) & 1) == 1)
        rows.append(me[sink]); cols.append(me[sink]); vals.append(np.full(sink.sum(), (1 - r) * w[i]))
    n = int(act.sum())
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def test_diffusion_preconditioner_count_does_not_grow_with_the_box():
    """GMRES on (I - A) x = b, right-preconditioned by P v = v + w_i eps
    with L eps = sum_i v_i (exact inner solve), on Knudsen Pt layers: the
    step applications grow less than the edge from 16^3 to 32^3 (they
    level off near 100 beyond that), stay far below the unpreconditioned
    count, and the result is the march's fixed point."""
    from scipy.sparse.linalg import LinearOperator, bicgstab, gmres, splu

    w = np.array([0.25] + [0.125] * 6)
    counts = {}
    for edge in (16, 32):
        ph, react, params = inputs.make_workload("pt_cl_256", shape=(edge, edge, edge), reactive=False)
        o = oracle.OracleLBM(ph, react=react, **params)
        o0 = oracle.OracleLBM(ph, react=react, **dict(params, c_in=0.0, c_out=0.0))
        act = o.active().astype(bool)
        lu = splu(_laplacian_matrix(o, params))
        shape = (7,) + o.shape
        n = int(np.prod(shape))
        b = _apply(o, np.zeros(shape)).ravel()
        cnt = [0]

        def mv(v):
            cnt[0] += 1
            return v - _apply(o0, v.reshape(shape)).ravel()

        def prec(v):
            V = v.reshape(shape)
            eps = np.zeros(o.shape)
            eps[act] = lu.solve(V.sum(axis=0)[act])
            return (V + w[:, None, None, None] * eps[None]).ravel()

        o.init_linear()
        x0 = o.populations().ravel()
        r0 = b - mv(x0)
        cnt[0] = 0
        y, info = gmres(LinearOperator((n, n), matvec=lambda v: mv(prec(v))), r0, rtol=1e-10, restart=50,
                        maxiter=20)
        assert info == 0
        counts[edge] = cnt[0]
        x = x0 + prec(y)
        assert np.linalg.norm(_apply(o, x.reshape(shape)).ravel() - x) <= 1e-8 * np.linalg.norm(x)
        if edge == 16:
            cnt[0] = 0
            _, info = bicgstab(LinearOperator((n, n), matvec=mv), b, x0=x0, rtol=1e-10, maxiter=20000)
            unprec = cnt[0]
    print("D3Q7 step applications", counts, "unpreconditioned at 16^3", unprec)
    assert counts[32] < 2 * counts[16] and counts[32] <= 150, counts
    assert unprec >= 4 * counts[16], (unprec, counts)


@pytest.mark.parametrize("lattice", [0, 1])
def test_laplacian_matrix_matches_the_link_rules(lattice):
    """The vectorised matrix equals the cell-by-cell link rules (which are
    pinned on the oracle's step above) on a reactive layer."""
    ph, _, params = inputs.make_workload("pt_cl_256", shape=(6, 7, 12), seed=61)
    react = inputs.reactive_faces(ph, 0.5, 3)
    params = dict(params, k_ms=3e4, bc_out=0)
    o = oracle.OracleLBM(ph, react=react, lattice=lattice, **params)
    act = o.active().astype(bool)
    eps = np.random.default_rng(9).uniform(0.2, 1.0, o.shape) * act
    ref = _link_laplacian(o, params)(eps)[act]
    np.testing.assert_allclose(_laplacian_matrix(o, params) @ eps[act], ref, rtol=0, atol=1e-14)


def test_diffusion_preconditioner_on_the_paper_lattice():
    """The same preconditioner with the D3Q19 link Laplacian (weights 1/18,
    1/36, mirror end cells) on a Knudsen Pt layer: far fewer step
    applications than without it, and the march's fixed point."""
    from scipy.sparse.linalg import LinearOperator, bicgstab, gmres, splu

    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    ph, react, params = inputs.make_workload("pt_cl_256", shape=(16, 16, 16), reactive=False)
    o = oracle.OracleLBM(ph, react=react, lattice=1, **params)
    o0 = oracle.OracleLBM(ph, react=react, lattice=1, **dict(params, c_in=0.0, c_out=0.0))
    act = o.active().astype(bool)
    lu = splu(_laplacian_matrix(o, params))
    shape = (19,) + o.shape
    n = int(np.prod(shape))
    b = _apply(o, np.zeros(shape)).ravel()
    cnt = [0]

    def mv(v):
        cnt[0] += 1
        return v - _apply(o0, v.reshape(shape)).ravel()

    def prec(v):
        V = v.reshape(shape)
        eps = np.zeros(o.shape)
        eps[act] = lu.solve(V.sum(axis=0)[act])
        return (V + w[:, None, None, None] * eps[None]).ravel()

    o.init_linear()
    x0 = o.populations().ravel()
    r0 = b - mv(x0)
    cnt[0] = 0
    y, info = gmres(LinearOperator((n, n), matvec=lambda v: mv(prec(v))), r0, rtol=1e-10, restart=50, maxiter=20)
    assert info == 0
    pre = cnt[0]
    x = x0 + prec(y)
    assert np.linalg.norm(_apply(o, x.reshape(shape)).ravel() - x) <= 1e-8 * np.linalg.norm(x)
    cnt[0] = 0
    bicgstab(LinearOperator((n, n), matvec=mv), b, x0=x0, rtol=1e-10, maxiter=20000)
    print("D3Q19 step applications: preconditioned", pre, "unpreconditioned", cnt[0])
    assert cnt[0] >= 4 * pre, (cnt[0], pre)
