"""Converged D_eff and reaction rate of 64^3 instances of the full-size
settings against the converged FP64 oracle (gpu).

The 256^3 Pt recipe (Knudsen D; D_eff set-up, and the reactive set-up with
5 % catalytic faces at k = 1e-3 m/s) and the 400^3 NPMC recipe at 1 nm
(micropores, every pore-solid face catalytic at k = 1e-5 m/s), each at 64^3
with its own seed.  The expected values (tests/golden/c2_deff_64.json, ...)
were written by
tests/golden/make_golden.py, which marches the FP64 oracle until the
tracked readout's remaining change is below 1e-10 of it.  The GPU solve
stops by its own rule; the bound is 1e-3 relative for the FP32 state and
5e-3 for FP16 storage.
"""
import json
import os

import pytest

from paper_1410_1914_gb300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


CONVERGED = [("c2_deff_64", "fp32", 1e-3), ("c2_deff_64", "fp16dev", 5e-3)]


@pytest.mark.parametrize("name,storage,rel", CONVERGED)
def test_converged_64_against_oracle(cuda_lib, name, storage, rel):
    """The stopping rule's answer on 64^3 instances of the full-size settings
    against the converged FP64 oracle: D_eff (Eq. 19) of the D_eff set-up,
    the reaction rate of the reactive ones."""
    from paper_1410_1914_gb300 import Solver
    with open(os.path.join(HERE, "golden", name + ".json")) as fh:
        gold = json.load(fh)
    assert gold["converged"]
    ph, react, params = inputs.make_workload(gold["workload"], shape=tuple(gold["shape"]), seed=gold["seed"],
                                             reactive=gold["reactive"])
    # FP16 storage balances the fluxes to about 2e-5 at best (rounding of the stored deviations)
    s = Solver(ph.shape, storage=storage, check_every=500, tol_rel=1e-6, tol_flux=1e-4 if storage == "fp16dev" else 2e-5,
               max_steps=3_000_000, **params)
    s.set_structure(ph, react)
    info = s.solve()
    assert info["converged"] == 1, info
    f = s.fluxes()
    assert f["n_active"] == gold["n_active"]
    if gold["reactive"]:
        R, _, _ = s.reaction_rate()
        assert R == pytest.approx(gold["R"], rel=rel)
        assert f["J_in"] == pytest.approx(gold["J_in"], rel=rel)
    else:
        d, ratio = s.effective_diffusivity()
        assert ratio == pytest.approx(gold["D_eff_over_Db"], rel=rel)
        assert d == pytest.approx(gold["D_eff_m2s"], rel=rel)
    s.close()
