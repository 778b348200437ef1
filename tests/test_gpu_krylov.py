"""The Krylov steady solve (cl_lbm_solve_krylov) on the GPU against the FP64
oracle, through the C ABI (gpu).

The mixed-precision solve of the fixed-point equation of the step map (the
formulation is pinned on the oracle in test_oracle_fixed_point.py) must
land on the steady state of the time march: the converged 48^3 D_eff of
both lattices (tests/golden/, written by the oracle) within 1e-3, the
FP32 bound of the converged-D_eff tests, and the oracle's converged
reaction rate on a reactive layer with a zero-flux outlet.  Its residual is
taken in FP64, so the state it returns balances the fluxes far below the
stopping rule's 1e-4 although the plain f32 populations alone do not.
"""
import json
import os

import pytest

import oracle
from paper_1410_1914_gb300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _solver(shape, lattice="d3q7", storage="fp32pop", **params):
    from paper_1410_1914_gb300 import Solver
    return Solver(shape, storage=storage, lattice=lattice, **params)


@pytest.mark.parametrize("lattice,golden,max_steps", [("d3q7", "c1_deff.json", 2000),
                                                      ("d3q19", "c1_deff_d3q19.json", 0)])
def test_krylov_converged_deff_small_workload(cuda_lib, lattice, golden, max_steps):
    """D3Q7: read after up to 2000 steps of the time march (the stopping
    rule's certificate); D3Q19: the Krylov state as it is (max_steps 0)."""
    with open(os.path.join(HERE, "golden", golden)) as fh:
        gold = json.load(fh)
    ph, react, params = inputs.make_workload("pt_cl_48")
    s = _solver(ph.shape, lattice, check_every=200, tol_rel=1e-5, tol_flux=1e-4, max_steps=3_000_000, **params)
    s.set_structure(ph, react)
    info = s.solve_krylov(tol=1e-8, max_iter=3000, max_steps=0)
    print(lattice, info)
    assert 0 < info["iterations"] <= 2000
    assert info["steps"] == 0 and info["status"] == "CL_ERR_NOT_CONVERGED"
    f = s.fluxes()
    assert abs(f["J_in"] - f["J_out"]) < 1e-4 * f["J_in"]
    if max_steps:
        info = s.solve_budget(max_steps)
        print(lattice, "march from the Krylov state", info)
    d, ratio = s.effective_diffusivity()
    assert ratio == pytest.approx(gold["D_eff_over_Db"], rel=1e-3)
    assert d == pytest.approx(gold["D_eff_m2s"], rel=1e-3)
    s.close()


def test_krylov_reaction_rate_zero_flux_outlet(cuda_lib):
    """Reactive Pt layer (reservoir plane, fixed inlet, zero-flux outlet,
    strong first-order sink) through torch's caching allocator: R of the
    Krylov state against the oracle's converged R."""
    ph, react, params = inputs.make_workload("pt_cl_256", shape=(12, 14, 32), seed=41)
    params = dict(params, k_ms=2e4)
    o = oracle.OracleLBM(ph, react=react, **params)
    o.solve(tol=1e-10, check_every=100, max_steps=400_000)
    R_ref = o.fluxes()["R"]
    s = _solver(ph.shape, torch_alloc=True, check_every=200, tol_rel=1e-5, tol_flux=1e-4, max_steps=3_000_000,
                **params)
    s.set_structure(ph, react)
    info = s.solve_krylov(tol=1e-8, max_iter=3000, max_steps=0)
    print(info)
    assert 0 < info["iterations"] <= 2000
    f = s.fluxes()
    assert f["R"] == pytest.approx(R_ref, rel=1e-3)
    assert f["J_in"] == pytest.approx(R_ref, rel=1e-3)
    s.close()


def test_krylov_argument_errors(cuda_lib):
    from paper_1410_1914_gb300 import _lib as L
    ph, react, params = inputs.make_workload("pt_cl_48", shape=(8, 8, 16), seed=3)
    s = _solver(ph.shape, storage="fp32", **params)
    s.set_structure(ph, react)
    with pytest.raises(L.ClError) as ei:
        s.solve_krylov()
    assert ei.value.status == L.CL_ERR_STATE
    s.close()
    s = _solver(ph.shape, **params)
    s.set_structure(ph, react)
    for bad in (dict(tol=0.0), dict(tol=1e-5, max_iter=-1), dict(tol=1e-5, max_steps=-1)):
        with pytest.raises(L.ClError) as ei:
            s.solve_krylov(**bad)
        assert ei.value.status == L.CL_ERR_ARG
    # max_iter 0: no iteration, the state is unchanged
    before = s.field()
    info = s.solve_krylov(tol=1e-5, max_iter=0, max_steps=0)
    assert info["iterations"] == 0
    assert (s.field() == before).all()
    s.close()
