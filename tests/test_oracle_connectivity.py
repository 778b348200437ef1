"""The oracle's connected-phase labelling (Sec. 2.1.3) pinned against a graph
library and hand-built cases.

  * networkx connected components of the 26- (Fig. 4a) or 6-neighbour graph,
    with and without y/z wrap: same portions, same smallest-index labels;
  * "transport" portions (cells on both end planes x = 0 and x = L) and the
    surface faces counted independently with numpy;
  * corner contact (26 joins, 6 does not), a 2x2x2 block (24 faces), a line
    through the box (transport) against one that stops short (dead), a
    portion joined only through the y wrap.
"""
import itertools

import numpy as np
import pytest

import oracle


def _graph_components(ph, codes, neighbours, periodic):
    nx_ = pytest.importorskip("networkx")
    nz, ny, nx = ph.shape
    inset = np.isin(ph, list(codes))
    G = nx_.Graph()
    idx = lambda x, y, z: x + nx * (y + ny * z)
    offs = [o for o in itertools.product((-1, 0, 1), repeat=3)
            if any(o) and (neighbours == 26 or sum(map(abs, o)) == 1)]
    for z, y, x in zip(*np.nonzero(inset)):
        c = idx(x, y, z)
        G.add_node(c)
        for dz, dy, dx in offs:
            qx, qy, qz = x + dx, y + dy, z + dz
            if not 0 <= qx < nx:
                continue
            if periodic:
                qy, qz = qy % ny, qz % nz
            elif not (0 <= qy < ny and 0 <= qz < nz):
                continue
            if inset[qz, qy, qx]:
                G.add_edge(c, idx(qx, qy, qz))
    return list(nx_.connected_components(G)), inset


def _faces(inset, periodic):
    """Faces between a set cell and an in-box cell outside the set."""
    n = 0
    for ax in (0, 1, 2):
        for sh in (1, -1):
            nb = np.roll(inset, sh, axis=ax)
            ok = np.ones_like(inset)
            if ax == 2 or not periodic:  # x never wraps
                sl = [slice(None)] * 3
                sl[ax] = 0 if sh == 1 else -1
                ok[tuple(sl)] = False
            n += int((inset & ~nb & ok).sum())
    return n


@pytest.mark.parametrize("seed,codes,neighbours,periodic", [
    (0, (1,), 26, False), (1, (1,), 6, False), (2, (0, 3), 26, True), (3, (2,), 6, True),
    (4, (0,), 26, True), (5, (1, 2), 6, False)])
def test_against_graph_components(seed, codes, neighbours, periodic):
    rng = np.random.default_rng(seed)
    ph = rng.choice([0, 1, 2, 3], size=(6, 7, 9), p=[0.35, 0.35, 0.25, 0.05]).astype(np.uint8)
    labels, st = oracle.phase_connectivity(ph, codes, neighbours, periodic)
    comps, inset = _graph_components(ph, codes, neighbours, periodic)
    nz, ny, nx = ph.shape
    flat = labels.reshape(-1)
    assert np.all(flat[~inset.reshape(-1)] == -1)
    for comp in comps:
        lab = {int(flat[c]) for c in comp}
        assert lab == {min(comp)}
    assert st["n_portions"] == len(comps)
    assert st["n_cells"] == int(inset.sum())
    xs = lambda comp: {c % nx for c in comp}
    tr = [c for c in comps if {0, nx - 1} <= xs(c)]
    assert st["n_transport_portions"] == len(tr)
    assert st["n_transport_cells"] == sum(len(c) for c in tr)
    assert st["largest_portion"] == max((len(c) for c in comps), default=0)
    assert st["surface_faces"] == _faces(inset, periodic)
    tmask = np.zeros(ph.size, bool)
    for c in tr:
        tmask[list(c)] = True
    assert st["transport_surface_faces"] == _faces(tmask.reshape(ph.shape) & inset, periodic) - \
        _shared_faces(tmask.reshape(ph.shape), inset & ~tmask.reshape(ph.shape), periodic)


def _shared_faces(a, b, periodic):
    """Faces between a cell of a and a cell of b (counted from a)."""
    n = 0
    for ax in (0, 1, 2):
        for sh in (1, -1):
            nb = np.roll(b, sh, axis=ax)
            ok = np.ones_like(a)
            if ax == 2 or not periodic:
                sl = [slice(None)] * 3
                sl[ax] = 0 if sh == 1 else -1
                ok[tuple(sl)] = False
            n += int((a & nb & ok).sum())
    return n


def test_corner_contact_joins_only_with_26_neighbours():
    ph = np.zeros((4, 4, 4), np.uint8)
    ph[0, 0, 0] = 1
    ph[1, 1, 1] = 1
    assert oracle.phase_connectivity(ph, [1], 26)[1]["n_portions"] == 1
    assert oracle.phase_connectivity(ph, [1], 6)[1]["n_portions"] == 2


def test_block_surface_and_lines():
    ph = np.zeros((6, 6, 8), np.uint8)
    ph[2:4, 2:4, 3:5] = 1                  # a 2x2x2 block: 24 faces, dead
    ph[1, 4, :] = 2                        # an ionomer line through the box: transport
    ph[4, 1, 1:] = 2                       # a line that misses x = 0: dead
    _, s1 = oracle.phase_connectivity(ph, [1], 26)
    assert s1 == dict(n_cells=8, n_portions=1, n_transport_portions=0, n_transport_cells=0, surface_faces=24,
                      transport_surface_faces=0, largest_portion=8)
    _, s2 = oracle.phase_connectivity(ph, [2], 26)
    assert s2["n_portions"] == 2 and s2["n_transport_portions"] == 1 and s2["n_transport_cells"] == 8
    # the through-line has 8 cells x 4 side faces; the other 7 x 4 + its x = 0
    # end face (faces on the box's own x faces are not surface)
    assert s2["surface_faces"] == 8 * 4 + 7 * 4 + 1
    assert s2["transport_surface_faces"] == 8 * 4


def test_y_wrap_joins_a_portion():
    ph = np.zeros((3, 5, 6), np.uint8)
    ph[1, 0, 0:3] = 1
    ph[1, 4, 3:6] = 1                      # meets the first run only across y = 0 | y = 4
    _, closed = oracle.phase_connectivity(ph, [1], 26, periodic_yz=False)
    _, wrapped = oracle.phase_connectivity(ph, [1], 26, periodic_yz=True)
    assert closed["n_portions"] == 2 and closed["n_transport_portions"] == 0
    assert wrapped["n_portions"] == 1 and wrapped["n_transport_portions"] == 1
