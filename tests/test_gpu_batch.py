"""Batched persistent launch (gpu): bit-identical to stepping each structure
alone, per-structure convergence matching single solves, the autotuner."""
import numpy as np
import pytest

from paper_1410_1914_gb300 import inputs

pytestmark = pytest.mark.gpu

MEMBERS = [
    ("pt_cl_256", (20, 30, 70), 41, dict(k_ms=2e4)),
    ("npmc_cl_400", (33, 17, 45), 42, dict(k_ms=5e3)),
    ("pt_cl_48", (24, 24, 24), 43, {}),
    ("pt_cl_256", (12, 40, 130), 44, dict(k_ms=1e4)),
    ("npmc_cl_400", (9, 9, 9), 45, dict(k_ms=3e3)),
]


def _make(storage, check_every=20, **over):
    from paper_1410_1914_gb300 import Solver
    out = []
    for wl, shape, seed, extra in MEMBERS:
        ph, react, params = inputs.make_workload(wl, shape=shape, seed=seed)
        params = dict(params, **extra)
        params.update(over)
        s = Solver(ph.shape, storage=storage, check_every=check_every, **params)
        s.set_structure(ph, react)
        out.append((s, ph, react, params))
    return out


@pytest.mark.parametrize("storage", ["fp32", "fp16dev"])
@pytest.mark.parametrize("steps", [1, 36])
def test_batch_step_equals_single_steps(cuda_lib, storage, steps):
    from paper_1410_1914_gb300.batch import Batch
    alone = _make(storage)
    together = _make(storage)
    for s, *_ in alone:
        s.step(steps)
    b = Batch([s for s, *_ in together], z_chunk=8)
    b.step(steps)
    for (sa, *_), (sb, *_) in zip(alone, together):
        np.testing.assert_array_equal(sb.field(), sa.field())
        np.testing.assert_array_equal(sb.populations(), sa.populations())
        assert sb.steps == sa.steps == steps
    b.close()


def test_batch_matches_oracle_after_steps(cuda_lib):
    import oracle
    from paper_1410_1914_gb300.batch import Batch
    members = _make("fp32")
    b = Batch([s for s, *_ in members])
    b.step(40)
    for s, ph, react, params in members:
        o = oracle.OracleLBM(ph, react=react, **params)
        o.step(40)
        np.testing.assert_allclose(s.field(), o.concentration(), rtol=0, atol=1e-7)
    b.close()


def test_batch_solve_matches_single_solves(cuda_lib):
    from paper_1410_1914_gb300.batch import Batch
    kw = dict(tol_rel=1e-6, tol_flux=1e-5)
    alone = _make("fp32", check_every=100, **kw)
    together = _make("fp32", check_every=100, **kw)
    single = []
    for s, *_ in alone:
        info = s.solve()
        assert info["converged"] == 1, info
        single.append(s.reaction_rate()[0] if s.params.bc_out == 1 else s.effective_diffusivity()[0])
    b = Batch([s for s, *_ in together])
    status, infos, nconv = b.solve(2_000_000)
    assert status == "CL_OK" and nconv == len(MEMBERS), (status, infos)
    assert b.info()["n_items"] > 0
    for (s, *_), ref, info in zip(together, single, infos):
        assert info["converged"] == 1
        got = s.reaction_rate()[0] if s.params.bc_out == 1 else s.effective_diffusivity()[0]
        assert got == pytest.approx(ref, rel=1e-4)
    b.close()


def test_batch_autotune_and_cache(cuda_lib, tmp_path):
    from paper_1410_1914_gb300.batch import Batch
    members = _make("fp16dev", check_every=20)
    b = Batch([s for s, *_ in members])
    cache = str(tmp_path / "tune.json")
    zc, pf, tr, ms, cached = b.autotune(steps_per_trial=4, cache=cache)
    assert zc in (8, 16, 32, 64) and pf in (0, 2) and tr in (1, 2, 4) and ms > 0 and not cached
    zc2, pf2, tr2, ms2, cached2 = b.autotune(steps_per_trial=4, cache=cache)
    assert cached2 and (zc2, pf2, tr2) == (zc, pf, tr)
    steps = members[0][0].steps
    assert steps == 3 * 6 * 4  # every trial is a real step: 3 shapes x z chunks 8, 16, 32 x 2 prefetch
    b.step(2)
    b.close()


def test_batch_rejects_mixed_members(cuda_lib):
    from paper_1410_1914_gb300 import Solver
    from paper_1410_1914_gb300 import _lib as L
    from paper_1410_1914_gb300.batch import Batch
    ph, react, params = inputs.make_workload("pt_cl_48", shape=(8, 8, 8), seed=3)
    a = Solver(ph.shape, storage="fp32", **params)
    a.set_structure(ph, react)
    c = Solver(ph.shape, storage="fp16dev", **params)
    c.set_structure(ph, react)
    with pytest.raises(L.ClError):
        Batch([a, c])
    d = Solver(ph.shape, storage="fp32pop", **params)
    d.set_structure(ph, react)
    with pytest.raises(L.ClError):
        Batch([d])
