"""Connected-phase labelling of Sec. 2.1.3 on the GPU vs the oracle's
breadth-first search, through the C ABI (gpu).  Labels (the smallest cell
index of each portion) and every count must match exactly."""
import numpy as np
import pytest

import oracle
from paper_1410_1914_gb300 import inputs

pytestmark = pytest.mark.gpu

PHASES = {"C/Pt": (1,), "void": (0, 3), "ionomer": (2,)}


def _gpu(ph, codes, nb, periodic, labels=True):
    from paper_1410_1914_gb300 import _lib as L
    lab = np.zeros(ph.shape, np.int32) if labels else None
    st = L.cl_phase_connectivity(ph, codes, nb, periodic, lab)
    return lab, st


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 3, 5), (2, 1, 33), (5, 9, 1), (7, 13, 29), (33, 40, 70)])
@pytest.mark.parametrize("nb,periodic", [(26, False), (26, True), (6, False), (6, True)])
def test_random_boxes(cuda_lib, shape, nb, periodic):
    rng = np.random.default_rng(sum(shape) + nb + periodic)
    ph = rng.choice([0, 1, 2, 3], size=shape, p=[0.4, 0.3, 0.25, 0.05]).astype(np.uint8)
    for codes in PHASES.values():
        lab, st = _gpu(ph, codes, nb, periodic)
        olab, ost = oracle.phase_connectivity(ph, codes, nb, periodic)
        np.testing.assert_array_equal(lab, olab)
        assert st == ost, (codes, st, ost)


@pytest.mark.parametrize("wl,shape,seed", [("pt_cl_256", (40, 48, 96), 3), ("npmc_cl_400", (48, 40, 64), 4)])
def test_workload_structures_all_phases(cuda_lib, wl, shape, seed):
    ph, _, _ = inputs.make_workload(wl, shape=shape, seed=seed)
    for codes in PHASES.values():
        for nb in (26, 6):
            lab, st = _gpu(ph, codes, nb, False)
            olab, ost = oracle.phase_connectivity(ph, codes, nb, False)
            np.testing.assert_array_equal(lab, olab)
            assert st == ost


def test_full_256_structure(cuda_lib):
    """The 256^3 Pt layer of the bench, the three phases of Sec. 2.1.3 with
    26 neighbours: every count equals the oracle's."""
    ph, _, _ = inputs.make_workload("pt_cl_256")
    for codes in PHASES.values():
        _, st = _gpu(ph, codes, 26, False, labels=False)
        _, ost = oracle.phase_connectivity(ph, codes, 26, False)
        assert st == ost
        assert st["n_transport_cells"] <= st["n_cells"]


def test_device_tensors(cuda_lib):
    import torch
    rng = np.random.default_rng(9)
    ph = rng.choice([0, 1, 2], size=(12, 14, 30), p=[0.5, 0.3, 0.2]).astype(np.uint8)
    tph = torch.from_numpy(ph).cuda()
    tlab = torch.empty(ph.shape, dtype=torch.int32, device="cuda")
    from paper_1410_1914_gb300 import _lib as L
    st = L.cl_phase_connectivity(tph, (0,), 26, True, tlab)
    olab, ost = oracle.phase_connectivity(ph, (0,), 26, True)
    np.testing.assert_array_equal(tlab.cpu().numpy(), olab)
    assert st == ost


def test_bad_arguments(cuda_lib):
    from paper_1410_1914_gb300 import _lib as L
    from paper_1410_1914_gb300._lib import ClError
    ph = np.zeros((2, 2, 2), np.uint8)
    with pytest.raises(ClError):
        L.cl_phase_connectivity(ph, (1,), 7)
    with pytest.raises(ClError):
        L.cl_phase_connectivity(ph, (), 26)
    bad = ph.copy()
    bad[1, 1, 1] = 5
    with pytest.raises(ClError):
        L.cl_phase_connectivity(bad, (1,), 26)
