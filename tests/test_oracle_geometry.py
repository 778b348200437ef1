"""Set-up steps of the oracle (Sec. 2.1.3) against independent algorithms.

13-direction pore lengths: the oracle walks from every cell; here every
lattice line is decomposed once into maximal pore runs (cycles for the lines
without an x component).  Connectivity: the oracle's breadth-first search
against networkx connected components of the periodic 6-neighbour graph.
Plus hand-computed geometries.
"""
import itertools

import numpy as np
import pytest

import oracle

DIRS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1),
        (0, 1, -1), (1, 1, 1), (1, 1, -1), (1, -1, 1), (1, -1, -1)]


def runs_by_lines(phase):
    nz, ny, nx = phase.shape
    pore = np.isin(phase, [0, 3])
    out = np.zeros((nz, ny, nx, 13), np.int32)
    for d, (ex, ey, ez) in enumerate(DIRS):
        lines = []
        if ex:
            for y0 in range(ny):
                for z0 in range(nz):
                    lines.append(([(t, (y0 + ey * t) % ny, (z0 + ez * t) % nz) for t in range(nx)], False))
        else:
            seen = np.zeros((nz, ny, nx), bool)
            for z0, y0, x0 in itertools.product(range(nz), range(ny), range(nx)):
                if seen[z0, y0, x0]:
                    continue
                cyc, (x, y, z) = [], (x0, y0, z0)
                while not seen[z, y, x]:
                    seen[z, y, x] = True
                    cyc.append((x, y, z))
                    y, z = (y + ey) % ny, (z + ez) % nz
                lines.append((cyc, True))
        for cells, cyclic in lines:
            flags = [pore[z, y, x] for x, y, z in cells]
            n = len(cells)
            if cyclic and all(flags):
                for x, y, z in cells:
                    out[z, y, x, d] = n
                continue
            # rotate a cycle so that it starts just after a non-pore cell
            start = 0
            if cyclic:
                start = (flags.index(False) + 1) % n
            order = [(start + i) % n for i in range(n)]
            run = []
            for i in order + [None]:
                if i is not None and flags[i]:
                    run.append(i)
                    continue
                for j in run:
                    x, y, z = cells[j]
                    out[z, y, x, d] = len(run)
                run = []
    return out


@pytest.mark.parametrize("seed,shape,frac", [(0, (6, 7, 8), 0.35), (1, (5, 4, 9), 0.2), (2, (8, 8, 8), 0.5),
                                             (3, (3, 6, 4), 0.1)])
def test_chords_against_line_decomposition(seed, shape, frac):
    rng = np.random.default_rng(seed)
    ph = (rng.random(shape) < frac).astype(np.uint8)
    ph[rng.random(shape) < 0.1] = 3
    ph[rng.random(shape) < 0.05] = 2
    np.testing.assert_array_equal(oracle.chord_counts(ph), runs_by_lines(ph))


def test_chords_hand_computed_slab():
    """Pore slab: solid plane at z = 0, box 6 x 5 x 4 (x, y, z)."""
    ph = np.zeros((4, 5, 6), np.uint8)
    ph[0] = 1
    ch = oracle.chord_counts(ph)
    assert np.all(ch[0] == 0)
    c = ch[1:]
    assert np.all(c[..., 0] == 6)   # along x: the whole bounded line
    assert np.all(c[..., 1] == 5)   # along y: the periodic loop of 5
    assert np.all(c[..., 2] == 3)   # along z: the three pore planes
    assert np.all(c[..., 3] == 6) and np.all(c[..., 4] == 6)
    assert np.all(c[..., 7] == 3) and np.all(c[..., 8] == 3)  # y-z diagonals hit z = 0 every 4 steps
    # (1,0,1) through (x=2, z=1): (3,2), (4,3) pore, (5,0) solid; (1,0) solid -> 3
    assert ch[1, 0, 2, 5] == 3
    # (1,0,-1) through (x=2, z=1): (3,0) solid; (1,2), (0,3) pore -> 3
    assert ch[1, 0, 2, 6] == 3
    # d_p of a cell: mean of counts * |e| * dx
    dp = oracle.pore_diameter(ph, 1e-9)
    lens = np.array([1, 1, 1] + [np.sqrt(2)] * 6 + [np.sqrt(3)] * 4)
    assert dp[1, 0, 2] == pytest.approx(np.dot(ch[1, 0, 2], lens) * 1e-9 / 13, rel=1e-15)


def test_chords_square_channel():
    """A 3x3 pore channel along x through solid, box 10 x 7 x 7."""
    ph = np.ones((7, 7, 10), np.uint8)
    ph[2:5, 2:5, :] = 0
    ch = oracle.chord_counts(ph)
    assert np.all(ch[2:5, 2:5, :, 0] == 10)
    assert np.all(ch[2:5, 2:5, :, 1] == 3) and np.all(ch[2:5, 2:5, :, 2] == 3)
    # centre cell: both in-plane diagonals span the 3x3 section
    assert ch[3, 3, 5, 7] == 3 and ch[3, 3, 5, 8] == 3
    # corner cell (y=2, z=2): (0,1,1) diagonal spans 3, (0,1,-1) only itself
    assert ch[2, 2, 5, 7] == 3 and ch[2, 2, 5, 8] == 1


def test_fully_open_loops_are_capped_at_their_period():
    ph = np.zeros((4, 6, 3), np.uint8)  # nz=4, ny=6
    ch = oracle.chord_counts(ph)
    assert np.all(ch[..., 1] == 6) and np.all(ch[..., 2] == 4)
    assert np.all(ch[..., 7] == 12) and np.all(ch[..., 8] == 12)  # lcm(6, 4)
    assert np.all(ch[..., 0] == 3)


# -------------------------------------------------------------- connectivity
def _reachable_networkx(ph, ion):
    nx_ = pytest.importorskip("networkx")
    nz, ny, nx = ph.shape
    tr = np.isin(ph, [0, 3, 2] if ion else [0, 3])
    G = nx_.Graph()
    for z, y, x in zip(*np.nonzero(tr)):
        G.add_node((x, y, z))
        for ex, ey, ez in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            qx, qy, qz = x + ex, (y + ey) % ny, (z + ez) % nz
            if qx < nx and tr[qz, qy, qx]:
                G.add_edge((x, y, z), (qx, qy, qz))
    out = np.zeros(ph.shape, np.uint8)
    for comp in nx_.connected_components(G):
        if any(c[0] == 0 for c in comp):
            for x, y, z in comp:
                out[z, y, x] = 1
    return out


@pytest.mark.parametrize("seed,ion", [(0, False), (1, True), (2, False), (3, True)])
def test_active_mask_against_networkx(seed, ion):
    rng = np.random.default_rng(seed)
    ph = rng.choice([0, 1, 2, 3], size=(7, 8, 9), p=[0.4, 0.35, 0.15, 0.1]).astype(np.uint8)
    np.testing.assert_array_equal(oracle.active_mask(ph, ion), _reachable_networkx(ph, ion))


def test_active_mask_periodic_wrap():
    """A pocket reachable only through the y wrap-around is active."""
    ph = np.ones((3, 5, 6), np.uint8)
    ph[1, 0, 0:3] = 0      # inlet channel along x at y = 0
    ph[1, 4, 2:6] = 0      # reached from (x=2, y=0) across the y seam
    a = oracle.active_mask(ph)
    assert a[1, 4, 5] == 1 and a[1, 0, 0] == 1 and a.sum() == 7
    ph[1, 4, 2] = 1        # cut the seam crossing
    assert oracle.active_mask(ph)[1, 4, 5] == 0


# ------------------------------------------------- warm-start network oracle
def test_network_oracle_conv_matches_scipy_correlate():
    """oracle.unet.conv3d: x zero padded, y and z periodic, equals a sum of
    scipy.ndimage.correlate calls on numpy-padded inputs (wrap in z and y,
    zeros in x)."""
    import scipy.ndimage as ndi

    import oracle.unet as OU
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 5, 6, 7, 3))
    w = rng.standard_normal((27, 2, 3))
    b = rng.standard_normal(2)
    got = OU.conv3d(x, w, b)
    for o in range(2):
        ref = np.full(x.shape[1:4], b[o])
        for i in range(3):
            k = w[:, o, i].reshape(3, 3, 3)  # taps ordered (kz, ky, kx)
            xp = np.pad(x[0, ..., i], ((1, 1), (1, 1), (0, 0)), mode="wrap")
            xp = np.pad(xp, ((0, 0), (0, 0), (1, 1)), mode="constant")
            ref += ndi.correlate(xp, k, mode="constant", cval=0.0)[1:-1, 1:-1, 1:-1]
        np.testing.assert_allclose(got[0, ..., o], ref, atol=1e-12)


def test_network_oracle_pool_up_are_adjoint_scaled():
    """<pool(a), b> = <a, up(b)> / 8 (average pooling vs nearest upsampling)."""
    import oracle.unet as OU
    rng = np.random.default_rng(1)
    a = rng.standard_normal((1, 4, 6, 8, 3))
    bb = rng.standard_normal((1, 2, 3, 4, 3))
    assert np.sum(OU.pool(a) * bb) == pytest.approx(np.sum(a * OU.up(bb)) / 8, rel=1e-12)
