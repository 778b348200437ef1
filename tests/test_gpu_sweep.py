"""The porosity sweep on the GPU (gpu): generated layers equal the host
generator's, each D_eff equals a direct solve of the same structure, the
readout grows with porosity, and the Eq. 28 exponent comes out finite."""
import math

import numpy as np
import pytest

from paper_1410_1914_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_small_sweep(cuda_lib):
    from paper_1410_1914_gb300 import Solver, sweep
    rows, fit = sweep.run(edge=32, eps_list=(0.4, 0.6), seed0=11, knudsen=1, storage="fp32", warm=False,
                          tol_rel=1e-6, check_every=200)
    assert [r["converged"] for r in rows] == [True, True]
    assert rows[1]["D_eff_over_Db"] > rows[0]["D_eff_over_Db"] > 0
    assert all(math.isfinite(a) for a in fit["alpha_per_point"])
    # the first point again, from the host generator and a direct solve
    eps = 0.4
    ph = inputs.pt_cl((32, 32, 32), 11, eps, sweep.IONOMER_SHARE * (1 - eps))
    assert float((ph == 0).mean()) == pytest.approx(rows[0]["eps"], abs=0)
    with Solver(ph.shape, storage="fp32", dx_m=5e-9, T_K=333.0, p_atm=1.0, M_kgmol=0.032, knudsen=1, bc_in=0,
                bc_out=0, c_in=1.0, c_out=0.0, tau_ref=1.0, check_every=200, tol_rel=1e-6, tol_flux=1e-4,
                max_steps=5_000_000) as s:
        s.set_structure(ph)
        s.solve()
        assert s.effective_diffusivity()[1] == pytest.approx(rows[0]["D_eff_over_Db"], rel=1e-12)
