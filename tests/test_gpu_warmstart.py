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


def test_warm_start_on_d3q19(cuda_lib):
    """The network (trained on D3Q7 solutions) starts a D3Q19 solve too: on a
    64^3 D_eff set-up of the Pt recipe the FP32-state run from the warm
    start stops on the same D_eff as the run from the ramp (1e-4) and takes
    fewer steps."""
    from paper_1410_1914_gb300 import Solver, inputs
    from paper_1410_1914_gb300 import warmstart as W
    net = W.load_pretrained()
    ph, _, params = inputs.make_workload("pt_cl_256", shape=(64, 64, 64), seed=5003, reactive=False)
    out = {}
    for warm in (False, True):
        with Solver(ph.shape, storage="fp32", lattice="d3q19", check_every=200, tol_rel=1e-7, tol_flux=1e-5,
                    max_steps=3_000_000, **params) as s:
            s.set_structure(ph)
            if warm:
                W.warm_start(net, s)
            info = s.solve()
            assert info["converged"] == 1, info
            out[warm] = (info["steps"], s.effective_diffusivity()[1])
    assert out[True][1] == pytest.approx(out[False][1], rel=1e-4)
    assert out[True][0] < out[False][0], out
