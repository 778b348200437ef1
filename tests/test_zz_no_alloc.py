"""The allocation-free connectivity entry point (gpu).

Some callers cannot allocate device memory at the moment they need the
inlet-connected transport mask (a host application that owns every device
allocation, a pipeline that forbids allocation after start-up).  They call
cl_active_mask_noalloc, whose union-find scratch lives in a static device
array.  These tests call it through the C ABI and compare its mask bit for
bit (the mask is integer work) with the FP64 oracle's flood fill and with the
handle API's set-up, on two calls in a row, so that the second call runs on
the scratch the first one left behind.  The file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1410_1914_gb300 import inputs

pytestmark = pytest.mark.gpu


def _handle_active(ph, params):
    from paper_1410_1914_gb300 import Solver
    s = Solver(ph.shape, **params)
    s.set_structure(ph, None)
    act = s.setup()["active"]
    s.close()
    return act


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


CASES = [
    # (recipe, shape (nz, ny, nx), seed, ionomer counted as transport)
    ("pt_cl_48", (40, 50, 61), 31, False),
    ("npmc_cl_400", (33, 17, 129), 32, False),
    ("pt_cl_48", (24, 37, 70), 33, True),
]


@pytest.mark.parametrize("recipe,shape,seed,ionomer", CASES)
def test_noalloc_matches_oracle_on_two_calls(cuda_lib, recipe, shape, seed, ionomer):
    import torch

    from paper_1410_1914_gb300 import _lib
    ph, _, params = inputs.make_workload(recipe, shape=shape, seed=seed, reactive=False)
    ref = oracle.active_mask(ph, ionomer_transport=ionomer)
    if ionomer:
        params = dict(params, D_ionomer=1e-9)  # the handle API then counts ionomer as transport
    handle = _handle_active(ph, params)
    np.testing.assert_array_equal(handle, ref)
    dph = torch.from_numpy(ph).cuda()
    for call in range(2):
        out = torch.full(ph.shape, 7, dtype=torch.uint8, device="cuda")
        _lib.cl_active_mask_noalloc(dph, out, ionomer_transport=ionomer)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_array_equal(got, ref, err_msg=f"call {call}")
        assert got.sum() > 0


def test_noalloc_rejects_bad_input(cuda_lib):
    import torch

    from paper_1410_1914_gb300 import _lib
    # larger than the static scratch
    ph = torch.zeros((1, 1, 8), dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(ph)
    assert cuda_lib.cl_active_mask_noalloc(_ptr(ph), 2048, 2048, 2, 0, _ptr(out), None) == _lib.CL_ERR_ARG
    # a phase code outside 0..3, found by the validation kernel
    bad = torch.zeros((4, 5, 6), dtype=torch.uint8, device="cuda")
    bad[2, 3, 4] = 5
    out = torch.zeros_like(bad)
    assert cuda_lib.cl_active_mask_noalloc(_ptr(bad), 6, 5, 4, 0, _ptr(out), None) == _lib.CL_ERR_ARG
    # host memory is refused before any launch
    host = np.zeros((4, 5, 6), dtype=np.uint8)
    hp = host.ctypes.data_as(ctypes.c_void_p)
    assert cuda_lib.cl_active_mask_noalloc(hp, 6, 5, 4, 0, _ptr(out), None) == _lib.CL_ERR_ARG
    assert cuda_lib.cl_active_mask_noalloc(_ptr(bad), 6, 5, 4, 0, hp, None) == _lib.CL_ERR_ARG
    # a valid call still works after the refusals
    good = torch.zeros((4, 5, 6), dtype=torch.uint8, device="cuda")
    _lib.cl_active_mask_noalloc(good, out)
    assert int(out.sum()) == 4 * 5 * 6
