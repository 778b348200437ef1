"""The diffusion-preconditioned Krylov steady solve
(cl_lbm_solve_krylov_dsa) against the FP64 oracle, through the C ABI (gpu).

Cases: the bulk-D 48^3 layer against the golden converged D_eff (1e-3);
a Knudsen Pt layer, where the unpreconditioned solve stalls, against the
oracle's converged D_eff (1e-3) within a step-application budget that does
not grow with the box; a reactive layer's R against the oracle (1e-3);
the same on the paper's D3Q19 lattice (Eq. 22-24), against the golden
D3Q19 D_eff and the oracle's exact steady state (a sparse direct solve of
its own step, oracle/steady.py); the storages it refuses.
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


def test_dsa_bulk_deff_small_workload(cuda_lib):
    with open(os.path.join(HERE, "golden", "c1_deff.json")) as fh:
        gold = json.load(fh)
    ph, react, params = inputs.make_workload("pt_cl_48")
    s = _solver(ph.shape, check_every=200, tol_rel=1e-5, tol_flux=1e-4, **params)
    s.set_structure(ph, react)
    info = s.solve_krylov_dsa(tol=1e-8, max_iter=2000, max_steps=0)
    print(info)
    assert 0 < info["iterations"] <= 600
    assert s.effective_diffusivity()[1] == pytest.approx(gold["D_eff_over_Db"], rel=1e-3)
    s.close()


@pytest.mark.parametrize("edge", [24, 32])
def test_dsa_knudsen_layer(cuda_lib, edge):
    ph, react, params = inputs.make_workload("pt_cl_256", shape=(edge, edge, edge), reactive=False)
    o = oracle.OracleLBM(ph, react=react, **params)
    o.solve(tol=1e-10, check_every=200, max_steps=2_000_000)
    ref = o.effective_diffusivity()[1]
    s = _solver(ph.shape, check_every=200, tol_rel=1e-5, tol_flux=1e-4, **params)
    s.set_structure(ph, react)
    info = s.solve_krylov_dsa(tol=1e-8, max_iter=2000, max_steps=0)
    print(edge, info)
    assert 0 < info["iterations"] <= 600
    f = s.fluxes()
    assert abs(f["J_in"] - f["J_out"]) < 1e-4 * f["J_in"]
    assert s.effective_diffusivity()[1] == pytest.approx(ref, rel=1e-3)
    s.close()


def test_dsa_reaction_rate_zero_flux_outlet(cuda_lib):
    ph, react, params = inputs.make_workload("pt_cl_256", shape=(12, 14, 32), seed=41)
    params = dict(params, k_ms=2e4)
    o = oracle.OracleLBM(ph, react=react, **params)
    o.solve(tol=1e-10, check_every=100, max_steps=400_000)
    R_ref = o.fluxes()["R"]
    s = _solver(ph.shape, check_every=200, tol_rel=1e-5, tol_flux=1e-4, **params)
    s.set_structure(ph, react)
    info = s.solve_krylov_dsa(tol=1e-8, max_iter=2000, max_steps=0)
    print(info)
    assert s.fluxes()["R"] == pytest.approx(R_ref, rel=1e-3)
    s.close()


def test_dsa_refuses_the_state_storages(cuda_lib):
    from paper_1410_1914_gb300 import _lib as L
    ph, react, params = inputs.make_workload("pt_cl_48", shape=(8, 8, 16), seed=3)
    for kw in (dict(storage="fp16dev"), dict(storage="fp32"), dict(lattice="d3q19", storage="fp16dev")):
        s = _solver(ph.shape, **dict(params, **kw))
        s.set_structure(ph, react)
        with pytest.raises(L.ClError) as ei:
            s.solve_krylov_dsa()
        assert ei.value.status == L.CL_ERR_STATE
        s.close()


def test_dsa_d3q19_bulk_deff_small_workload(cuda_lib):
    with open(os.path.join(HERE, "golden", "c1_deff_d3q19.json")) as fh:
        gold = json.load(fh)
    ph, react, params = inputs.make_workload("pt_cl_48")
    s = _solver(ph.shape, "d3q19", check_every=200, tol_rel=1e-5, tol_flux=1e-4, **params)
    s.set_structure(ph, react)
    info = s.solve_krylov_dsa(tol=1e-8, max_iter=2000, max_steps=0)
    print("d3q19 bulk", info)
    assert 0 < info["iterations"] <= 600
    f = s.fluxes()
    assert abs(f["J_in"] - f["J_out"]) < 1e-4 * f["J_in"]
    assert s.effective_diffusivity()[1] == pytest.approx(gold["D_eff_over_Db"], rel=1e-3)
    s.close()


def _exact(ph, react, params):
    """The D3Q19 oracle set to the exact fixed point of its own step."""
    from oracle import steady
    o = oracle.OracleLBM(ph, react=react, lattice=1, **params)
    steady.solve(o)
    return o


def test_dsa_d3q19_knudsen_layer_against_exact_steady_state(cuda_lib):
    ph, react, params = inputs.make_workload("pt_cl_256", shape=(12, 12, 18), seed=51, reactive=False)
    o = _exact(ph, react, params)
    ref = o.effective_diffusivity()[1]
    assert ref > 0
    s = _solver(ph.shape, "d3q19", check_every=200, tol_rel=1e-5, tol_flux=1e-4, **params)
    s.set_structure(ph, react)
    info = s.solve_krylov_dsa(tol=1e-8, max_iter=2000, max_steps=0)
    print("d3q19 knudsen", info)
    assert 0 < info["iterations"] <= 600
    assert s.effective_diffusivity()[1] == pytest.approx(ref, rel=1e-3)
    s.close()


def test_dsa_d3q19_reaction_rate_against_exact_steady_state(cuda_lib):
    ph, react, params = inputs.make_workload("pt_cl_256", shape=(12, 12, 24), seed=52)
    params = dict(params, k_ms=2e4)
    o = _exact(ph, react, params)
    R_ref = o.fluxes()["R"]
    assert R_ref > 0
    s = _solver(ph.shape, "d3q19", check_every=200, tol_rel=1e-5, tol_flux=1e-4, **params)
    s.set_structure(ph, react)
    info = s.solve_krylov_dsa(tol=1e-8, max_iter=2000, max_steps=0)
    print("d3q19 reactive", info)
    assert s.fluxes()["R"] == pytest.approx(R_ref, rel=1e-3)
    s.close()
