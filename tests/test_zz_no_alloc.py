"""The allocation-free connectivity entry point (gpu).

Callers that cannot allocate device memory when they need the answer use
cl_active_mask_noalloc, whose scratch lives in a static device array.  This
checks it through the C ABI against the handle-based set-up (cl_lbm_get_setup's
active mask) on two calls in a row, bit for bit, since the mask is integer
work; the second call reuses the scratch the first one left behind.  The file
is collected last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

from paper_1410_1914_gb300 import inputs

pytestmark = pytest.mark.gpu


def _handle_active(ph, params):
    from paper_1410_1914_gb300 import Solver
    s = Solver(ph.shape, **params)
    s.set_structure(ph, None)
    act = s.setup()["active"]
    s.close()
    return act


def test_noalloc_matches_handle_api_on_two_calls(cuda_lib):
    import torch

    from paper_1410_1914_gb300 import _lib
    cases = [inputs.make_workload("pt_cl_48", shape=(40, 50, 61), seed=31, reactive=False),
             inputs.make_workload("npmc_cl_400", shape=(33, 17, 129), seed=32, reactive=False)]
    for ph, _, params in cases:
        ref = _handle_active(ph, params)
        dph = torch.from_numpy(ph).cuda()
        out = torch.full(ph.shape, 7, dtype=torch.uint8, device="cuda")
        _lib.cl_active_mask_noalloc(dph, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_array_equal(got, ref)
        assert got.sum() > 0


def test_noalloc_rejects_oversized_boxes(cuda_lib):
    import torch

    from paper_1410_1914_gb300 import _lib
    ph = torch.zeros((1, 1, 8), dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(ph)
    st = cuda_lib.cl_active_mask_noalloc(ctypes_ptr(ph), 2048, 2048, 2, 0, ctypes_ptr(out), None)
    assert st == _lib.CL_ERR_ARG


def ctypes_ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())
