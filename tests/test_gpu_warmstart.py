"""Learned warm start: the committed network shortens the solve (gpu).

On held-out 96^3 cubes (seeds 5000-5002, never in training) the FP32-state
solve is run from the linear ramp to an extrapolated relative change below
1e-9 (its last D_eff is the reference) and again from the network's
prediction.  The warm start must leave the converged D_eff unchanged and
reach 1e-3 of it in fewer steps: at least 20 % fewer over the three cubes
(the trained weights give about 34 %).  The lattice Boltzmann steps still
compute the answer; the network only chooses where they start.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_warm_start_saves_steps(cuda_lib):
    from paper_1410_1914_gb300 import warmstart as W
    from paper_1410_1914_gb300.warmstart_train import evaluate
    net = W.load_pretrained()
    rows = evaluate(net, size=96, n=3, seed0=5000)
    ramp = sum(r["ramp"]["steps"] for r in rows)
    warm = sum(r["warm"]["steps"] for r in rows)
    for r in rows:
        # same fixed point: the warm run ends on the ramp run's D_eff
        assert r["warm"]["final_rel_err"] < 1e-4, r
    assert warm <= 0.8 * ramp, rows
