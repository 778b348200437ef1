"""The steady state with the populations eliminated along lines
(cl_lbm_solve_steady_lines) against the FP64 oracle (gpu).

Both sides compute the fixed point of one step of the same scheme: the
oracle by a sparse direct solve of (I - A) x = S(0) on its populations
(oracle/steady.py), the GPU by flexible GMRES on C = F(C) with the
populations eliminated exactly.  The cases include O2 dissolved in the
ionomer at the physical contrast of Eq. 10-15 (ionomer_o2 = 1: relaxation
times within 1e-5 of 1/2), where the time march and the population-space
Krylov solves stall.  Both results are exact up to rounding: the solve's
own FP64 fluxes agree to 1e-6, the readouts of its f32 populations (and
the field) to 1e-5.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import steady
from paper_1410_1914_gb300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _gpu(ph, react, params, **kw):
    from paper_1410_1914_gb300 import Solver
    s = Solver(ph.shape, storage="fp32pop", **params)
    s.set_structure(ph, react)
    info = s.solve_steady_lines(**kw)
    return s, info


def test_bulk_layer_against_golden(cuda_lib):
    with open(os.path.join(HERE, "golden", "c1_deff.json")) as fh:
        gold = json.load(fh)
    ph, react, params = inputs.make_workload("pt_cl_48")
    s, info = _gpu(ph, react, params)
    print("\nbulk 48^3", info)
    assert info["status"] == "CL_OK"
    d, ratio = s.effective_diffusivity()
    assert ratio == pytest.approx(gold["D_eff_over_Db"], rel=1e-5)
    f = s.fluxes()
    assert abs(f["J_in"] - f["J_out"]) <= 1e-5 * f["J_in"]
    s.close()


CASES = [
    # (name, recipe, shape (nz, ny, nx), reactive, extra params)
    ("knudsen", "pt_cl_256", (24, 24, 24), False, {}),
    ("dissolved_o2", "pt_cl_256", (24, 24, 24), False, dict(ionomer_o2=1)),
    ("dissolved_o2_sites", "pt_cl_256", (24, 24, 24), True, dict(ionomer_o2=1, react_rule=2, k_ms=1e-3)),
    ("npmc_dissolved_o2", "npmc_cl_400", (21, 24, 30), True, dict(ionomer_o2=1, k_ms=1e-3)),
    ("dissolved_o2_33", "pt_cl_256", (33, 33, 32), False, dict(ionomer_o2=1)),
]


@pytest.mark.parametrize("name,recipe,shape,reactive,extra", CASES)
def test_against_exact_oracle_steady_state(cuda_lib, name, recipe, shape, reactive, extra):
    ph, react, params = inputs.make_workload(recipe, shape=shape, seed=7, reactive=reactive)
    params = dict(params, **extra)
    if params.get("react_rule") == 2:
        react = None
        from oracle.coupled import ionomer_solid_faces
        oreact = ionomer_solid_faces(ph)
    else:
        oreact = react
    oparams = {k: v for k, v in params.items() if k != "react_rule"}
    o = oracle.OracleLBM(ph, react=oreact, **oparams)
    steady.solve(o)
    s, info = _gpu(ph, react, params)
    print(f"\n{name} {shape}", info)
    assert info["status"] == "CL_OK"
    if extra.get("ionomer_o2"):
        assert ((s.setup()["active"] > 0) & (ph == 2)).any()   # the ionomer carries O2
    fg, fo = s.fluxes(), o.fluxes()
    assert fg["n_active"] == fo["n_active"]
    # the solve's own FP64 fluxes against the oracle's
    assert info["J_in"] == pytest.approx(fo["J_in"], rel=1e-6)
    assert info["J_out"] == pytest.approx(fo["J_out"], rel=1e-6, abs=1e-12)
    assert info["R"] == pytest.approx(fo["R"], rel=1e-6, abs=1e-15)
    if reactive:
        assert fo["R"] > 0
        # from the stored f32 populations: a small inflow is a difference of O(w C_in)
        # populations, so these carry their rounding (about 1e-8 per boundary cell)
        nyz = ph.shape[0] * ph.shape[1]
        assert abs(fg["R"] - fo["R"]) <= 1e-5 * fo["R"] + 2e-8 * nyz
    else:
        assert s.effective_diffusivity()[1] == pytest.approx(o.effective_diffusivity()[1], rel=1e-5)
    C, Co = s.field(), o.concentration()
    np.testing.assert_allclose(C, Co, rtol=0, atol=1e-5 * np.abs(Co).max())
    s.close()


def test_henry_series_slab_closed_form(cuda_lib):
    """A pore layer in series with an ionomer layer at the physical contrast:
    the steady flux is that of the two resistances with Henry's jump at the
    interface, (C_in - C_out) / (L_p / D_p + L_i H / (R T D_e)) (Eq. 10-15)."""
    from paper_1410_1914_gb300 import _lib as L
    nx, lp = 40, 25
    ph = np.zeros((3, 3, nx), np.uint8)
    ph[:, :, lp:] = 2
    T = 353.0
    params = dict(dx_m=2e-9, T_K=T, knudsen=0, D_bulk=2.5e-5, ionomer_o2=1, bc_in=0, bc_out=0, c_in=1.0,
                  c_out=0.0, k_ms=0.0)
    s, info = _gpu(ph, None, params)
    assert info["status"] == "CL_OK", info
    H = oracle.henry_constant(T)
    De = oracle.ionomer_o2_diffusivity(T)
    R = 8.314462618
    dx = params["dx_m"]
    flux = 1.0 / (lp * dx / 2.5e-5 + (nx - lp) * dx * H / (R * T * De))   # mol / (m^2 s) per unit C_in
    d, _ = s.effective_diffusivity()
    # Eq. 19: D_eff = flux L / (C_in - C_out)
    assert d == pytest.approx(flux * nx * dx, rel=1e-6)
    s.close()


def test_argument_and_storage_errors(cuda_lib):
    from paper_1410_1914_gb300 import Solver
    from paper_1410_1914_gb300 import _lib as L
    ph, react, params = inputs.make_workload("pt_cl_256", shape=(6, 6, 12), seed=3)
    s = Solver(ph.shape, storage="fp32", **params)
    s.set_structure(ph, react)
    with pytest.raises(L.ClError) as e:
        s.solve_steady_lines()
    assert e.value.status == L.CL_ERR_STATE
    s.close()
    s = Solver(ph.shape, storage="fp32pop", **params)
    s.set_structure(ph, react)
    for kw in (dict(tol=0.0), dict(max_iter=0), dict(restart=0), dict(cg_tol=1.0)):
        with pytest.raises(L.ClError) as e:
            s.solve_steady_lines(**kw)
        assert e.value.status == L.CL_ERR_ARG
    s.close()
