"""The diffusion-preconditioned Krylov steady solve
(cl_lbm_solve_krylov_dsa) against the FP64 oracle, through the C ABI (gpu).

Cases: the bulk-D 48^3 layer against the golden converged D_eff (1e-3);
a Knudsen Pt layer, where the unpreconditioned solve stalls, against the
oracle's converged D_eff (1e-3) within a step-application budget that does
not grow with the box; a reactive layer's R against the oracle (1e-3);
the lattice and storage it refuses.
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


def test_dsa_refuses_other_lattice_and_storage(cuda_lib):
    from paper_1410_1914_gb300 import _lib as L
    ph, react, params = inputs.make_workload("pt_cl_48", shape=(8, 8, 16), seed=3)
    for kw in (dict(lattice="d3q19"), dict(storage="fp16dev")):
        s = _solver(ph.shape, **dict(params, **kw))
        s.set_structure(ph, react)
        with pytest.raises(L.ClError) as ei:
            s.solve_krylov_dsa()
        assert ei.value.status == L.CL_ERR_STATE
        s.close()
