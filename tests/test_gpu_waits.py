"""Bounded device-side waits that run out (gpu), made to do so on purpose.

The step kernel's plane loads are guarded by mbarrier waits, and in the
batched launch an item of step t waits until its member's step t - 1 is
done (a per-member count of finished items); each wait gives up
after a bound and raises an error bit that the host maps to CL_ERR_TIMEOUT.
The test hooks shorten the bound to a few hundred SM clock cycles and make
the awaited event one that never happens (a plane load the producer never
issues; one finished item more than the member has).  The call must return
CL_ERR_TIMEOUT, the kernel must not touch the state it would have written,
and the handle or batch must step normally again once the hook is reset --
no fault, no trap, no hang.
"""
import numpy as np
import pytest

from paper_1410_1914_gb300 import inputs

pytestmark = pytest.mark.gpu

SHORT = 400  # SM clock cycles


def _solver(storage, check_every=20):
    from paper_1410_1914_gb300 import Solver
    ph, react, params = inputs.make_workload("pt_cl_256", shape=(13, 17, 291), seed=21)
    s = Solver(ph.shape, storage=storage, check_every=check_every, **dict(params, k_ms=2e4))
    s.set_structure(ph, react)
    return s


@pytest.mark.parametrize("storage", ["fp32", "fp16dev"])
def test_step_kernel_wait_runs_out(cuda_lib, storage):
    from paper_1410_1914_gb300 import _lib as L
    s = _solver(storage)
    s.solve_budget(20)
    before = s.populations()
    assert L.load().cl_lbm_set_wait_test(s.h, SHORT, 1) == L.CL_OK
    with pytest.raises(L.ClError) as e:
        s.solve_budget(20)
    assert e.value.status == L.CL_ERR_TIMEOUT
    # the consumers gave up before their first plane: nothing was written
    np.testing.assert_array_equal(s.populations(), before)
    # back to normal: the same trajectory as a fresh handle, bit for bit
    assert L.load().cl_lbm_set_wait_test(s.h, 0, 0) == L.CL_OK
    s.init()
    s.step(50)
    ref = _solver(storage)
    ref.step(50)
    np.testing.assert_array_equal(s.populations(), ref.populations())
    info = s.solve_budget(20)
    assert info["status"] == "CL_ERR_NOT_CONVERGED"
    s.close()
    ref.close()


def test_wait_hook_arguments(cuda_lib):
    from paper_1410_1914_gb300 import _lib as L
    s = _solver("fp32")
    lib = L.load()
    assert lib.cl_lbm_set_wait_test(s.h, -1, 0) == L.CL_ERR_ARG
    assert lib.cl_lbm_set_wait_test(s.h, 0, 1) == L.CL_ERR_ARG  # never_arrive needs a limit
    assert lib.cl_lbm_set_wait_test(None, 100, 0) == L.CL_ERR_ARG
    # a short limit alone (the loads do arrive) must not change the arithmetic
    assert lib.cl_lbm_set_wait_test(s.h, 0, 0) == L.CL_OK
    s.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16dev"])
def test_batch_step_wait_runs_out(cuda_lib, storage):
    from paper_1410_1914_gb300 import _lib as L
    from paper_1410_1914_gb300.batch import Batch
    members = []
    for wl, shape, seed in (("pt_cl_256", (20, 30, 70), 41), ("npmc_cl_400", (33, 17, 45), 42)):
        from paper_1410_1914_gb300 import Solver
        ph, react, params = inputs.make_workload(wl, shape=shape, seed=seed)
        s = Solver(ph.shape, storage=storage, check_every=20, **params)
        s.set_structure(ph, react)
        members.append(s)
    b = Batch(members, z_chunk=8)
    b.step(2)
    lib = L.load()
    assert lib.cl_batch_set_wait_test(b.b, SHORT, 1) == L.CL_OK
    assert lib.cl_batch_step(b.b, 2) == L.CL_ERR_TIMEOUT
    assert lib.cl_batch_set_wait_test(b.b, 0, 0) == L.CL_OK
    # usable again: from a fresh start, batched steps equal each member stepped alone
    for s in members:
        s.init()
    b.step(36)
    for s, (wl, shape, seed) in zip(members, (("pt_cl_256", (20, 30, 70), 41), ("npmc_cl_400", (33, 17, 45), 42))):
        ph, react, params = inputs.make_workload(wl, shape=shape, seed=seed)
        from paper_1410_1914_gb300 import Solver
        ref = Solver(ph.shape, storage=storage, check_every=20, **params)
        ref.set_structure(ph, react)
        ref.step(36)
        np.testing.assert_array_equal(s.populations(), ref.populations())
        ref.close()
    b.close()
    for s in members:
        s.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16dev"])
def test_member_plane_wait_runs_out_inside_batch(cuda_lib, storage):
    """A member's own plane wait gives up inside the batched launch: its
    block raises the abort word, every other block leaves its queue or its
    step wait, and the step reports CL_ERR_TIMEOUT through the member's
    error word.  A member's wait settings reach the batch when the batch is
    created or configured."""
    from paper_1410_1914_gb300 import Solver
    from paper_1410_1914_gb300 import _lib as L
    from paper_1410_1914_gb300.batch import Batch
    spec = (("pt_cl_256", (20, 30, 70), 43), ("npmc_cl_400", (33, 17, 45), 44))

    def make():
        out = []
        for wl, shape, seed in spec:
            ph, react, params = inputs.make_workload(wl, shape=shape, seed=seed)
            s = Solver(ph.shape, storage=storage, check_every=20, **params)
            s.set_structure(ph, react)
            out.append(s)
        return out

    members = make()
    lib = L.load()
    assert lib.cl_lbm_set_wait_test(members[1].h, SHORT, 1) == L.CL_OK
    b = Batch(members, z_chunk=8)
    assert lib.cl_batch_step(b.b, 4) == L.CL_ERR_TIMEOUT
    assert lib.cl_lbm_set_wait_test(members[1].h, 0, 0) == L.CL_OK
    b.configure(8, 0, 0)  # the members' arguments again, without the hook
    for s in members:
        s.init()
    b.step(30)
    refs = make()
    for s, r in zip(members, refs):
        r.step(30)
        np.testing.assert_array_equal(s.populations(), r.populations())
        r.close()
    b.close()
    for s in members:
        s.close()
