"""Structure generation on the GPU (QSGS of Sec. 2.1.2, micropores of Sec.
5.3, reactive-face sampling) against the host generator: byte for byte."""
import numpy as np
import pytest

from paper_1410_1914_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,seed,pore,ion", [((13, 17, 29), 5, 0.45, 0.19), ((40, 48, 96), 6, 0.35, 0.22),
                                                  ((1, 3, 40), 7, 0.5, 0.2), ((64, 64, 64), 8, 0.65, 0.12)])
def test_pt_layer_matches_host(cuda_lib, shape, seed, pore, ion):
    from paper_1410_1914_gb300 import structures
    g = structures.pt_cl(shape, seed, pore, ion).cpu().numpy()
    h = inputs.pt_cl(shape, seed, pore, ion)
    np.testing.assert_array_equal(g, h)


def test_npmc_layer_matches_host(cuda_lib):
    from paper_1410_1914_gb300 import structures
    shape = (48, 40, 64)
    g = structures.npmc_cl(shape, 9, 0.45, inputs.EQ4_EPS045_IONOMER, 0.55).cpu().numpy()
    h = inputs.npmc_cl(shape, 9, 0.45, inputs.EQ4_EPS045_IONOMER, 0.55)
    np.testing.assert_array_equal(g, h)
    assert (g == 3).sum() == round(0.10 * g.size)


def test_full_256_workload_and_faces(cuda_lib):
    """The 256^3 Pt layer of the bench and its 5 % reactive faces."""
    import torch
    from paper_1410_1914_gb300 import structures
    w = inputs.WORKLOADS["pt_cl_256"]
    g = structures.pt_cl(w["shape"], w["seed"], w["pore"], w["ionomer"], w["c_d"])
    h = inputs.pt_cl(w["shape"], w["seed"], w["pore"], w["ionomer"], w["c_d"])
    np.testing.assert_array_equal(g.cpu().numpy(), h)
    hr = inputs.with_reservoir(h)
    gr = torch.from_numpy(hr).cuda()
    np.testing.assert_array_equal(structures.reactive_faces(gr, 0.05, w["seed"]).cpu().numpy(),
                                  inputs.reactive_faces(hr, 0.05, w["seed"]))
    np.testing.assert_array_equal(structures.reactive_faces(gr, 1.0, 3).cpu().numpy(),
                                  inputs.reactive_faces(hr, 1.0, 3))


def test_grow_edge_cases(cuda_lib):
    import torch
    from paper_1410_1914_gb300 import _lib as L
    ph = torch.zeros((4, 5, 6), dtype=torch.uint8, device="cuda")
    # no seeds and nothing grown: the sweeps find no candidate and stop at the bound
    assert L.cl_qsgs_grow(ph, 1, 1, 2, 50, 0.0, 0.5, 1, 1, max_sweeps=5) == 0
    assert int(ph.sum()) == 0
    # a target already reached changes nothing
    ph[0, 0, :] = 1
    assert L.cl_qsgs_grow(ph, 1, 1, 2, 3, 0.1, 0.5, 1, 1) == 6
    assert int((ph == 1).sum()) == 6
    # the whole box
    assert L.cl_qsgs_grow(ph, 1, 1, 2, ph.numel(), 0.05, 0.1, 2, 1) == ph.numel()
    assert bool((ph == 1).all())


def test_connectivity_of_a_gpu_structure(cuda_lib):
    """The three phases of a GPU-generated layer: the statistics equal the
    oracle's on the same bytes."""
    import oracle
    from paper_1410_1914_gb300 import structures
    g = structures.pt_cl((32, 40, 80), 11, 0.45, 0.19)
    stats = structures.connectivity(g)
    h = g.cpu().numpy()
    for name, codes in structures.PHASE_SETS.items():
        assert stats[name] == oracle.phase_connectivity(h, codes, 26, False)[1]
