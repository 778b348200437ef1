"""Failure paths, injected on the host (gpu): no kernel is made to fault or
hang.

* an allocator callback that fails at its n-th call: cl_lbm_create returns
  CL_ERR_OOM, every block it did get is handed back, nothing is created;
* a non-finite value in the initial field (through the public cl_lbm_init):
  the solve stops with CL_ERR_DIVERGED at the first check;
* a step budget below what convergence needs: CL_ERR_NOT_CONVERGED with the
  interval's readouts.
"""
import ctypes

import numpy as np
import pytest

from paper_1410_1914_gb300 import inputs

pytestmark = pytest.mark.gpu


class FailingAllocator:
    """cudaMalloc-backed allocator that returns NULL at call `fail_at`."""

    def __init__(self, fail_at):
        import torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}

        def _alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            ptr = int(torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0)))
            self.live[ptr] = nbytes
            return ptr

        def _free(ptr, nbytes, stream, ctx):
            self.live.pop(int(ptr))
            torch.cuda.caching_allocator_delete(int(ptr))

        from paper_1410_1914_gb300 import _lib as L
        self.alloc = L.cl_alloc_fn(_alloc)
        self.free = L.cl_free_fn(_free)


@pytest.mark.parametrize("fail_at", [1, 2, 5, 12])
@pytest.mark.parametrize("storage", ["fp16dev", "fp32pop"])
def test_allocation_failure_is_reported_and_cleaned_up(cuda_lib, fail_at, storage):
    from paper_1410_1914_gb300 import _lib as L
    from paper_1410_1914_gb300.solver import _STORAGE
    fa = FailingAllocator(fail_at)
    p = L.cl_params_default(nx=40, ny=24, nz=16)
    p.storage = _STORAGE[storage]
    p.alloc, p.free = fa.alloc, fa.free
    h = ctypes.c_void_p()
    st = L.load().cl_lbm_create(ctypes.byref(h), ctypes.byref(p))
    assert st == L.CL_ERR_OOM
    assert h.value is None
    assert fa.calls == fail_at
    assert fa.live == {}


def test_nonfinite_initial_field_diverges(cuda_lib):
    from paper_1410_1914_gb300 import Solver
    from paper_1410_1914_gb300 import _lib as L
    ph, react, params = inputs.make_workload("pt_cl_256", shape=(12, 16, 40), reactive=False)
    with Solver(ph.shape, storage="fp32", check_every=10, **params) as s:
        s.set_structure(ph, react)
        act = s.setup()["active"].astype(bool)
        C0 = np.where(act, 0.5, 0.0).astype(np.float32)
        z, y, x = np.argwhere(act)[len(np.argwhere(act)) // 2]
        C0[z, y, x] = np.nan
        s.init(C0)
        with pytest.raises(L.ClError) as ei:
            s.solve_budget(40)
        assert ei.value.status == L.CL_ERR_DIVERGED
        assert "non-finite" in str(ei.value)
        assert s.steps == 10  # stopped at the first check


def test_step_budget_reports_not_converged(cuda_lib):
    from paper_1410_1914_gb300 import Solver
    ph, react, params = inputs.make_workload("pt_cl_256", shape=(12, 16, 40), reactive=False)
    with Solver(ph.shape, storage="fp16dev", check_every=20, **params) as s:
        s.set_structure(ph, react)
        d = s.solve_budget(60)
        assert d["status"] == "CL_ERR_NOT_CONVERGED"
        assert d["steps"] == 60
        assert d["J_in"] > 0 and np.isfinite(d["J_out"])
