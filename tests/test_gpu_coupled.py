"""Non-uniform kinetics, sources and the coupled O2 / proton steady state
(Sec. 3.3-3.4, Eq. 16-18) on the GPU against the FP64 oracle (gpu).

* Per-cell rate factors (Eq. 17b with a non-uniform potential) and per-cell
  sources (the a_i S term of Eq. 21) in the plain-population step kernel:
  a trajectory and the per-cell consumption readout, element by element.
* The coupled solve (cl_coupled_solve: Picard on the ionomer potential,
  steady states of both carriers in the library's kernels) against
  oracle/coupled.py (exact steady states by a sparse direct solve) on a
  small Pt layer: potential, O2 field, current from both sides.  With the
  population-space Krylov solve the ionomer's O2 diffusivity is given (that
  solve does not reach the ~1e5 contrast of Eq. 13); with the
  line-eliminated solve also at the physical contrast of Eq. 10-13.
"""
import numpy as np
import pytest

import oracle
from oracle import coupled as ocoupled
from paper_1410_1914_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_rate_scale_and_source_trajectory(cuda_lib):
    from paper_1410_1914_gb300 import Solver
    ph, react, params = inputs.make_workload("pt_cl_256", shape=(12, 15, 40), seed=61)
    params = dict(params, k_ms=2e4)
    rng = np.random.default_rng(5)
    ks = rng.uniform(0.0, 3.0, ph.shape)
    S = rng.uniform(-1e-4, 1e-4, ph.shape)
    s = Solver(ph.shape, storage="fp32pop", **params)
    s.set_structure(ph, react)
    s.set_rate_scale(ks)
    s.set_source(S)
    s.init()  # the stored post-collision state carries the source from the start
    o = oracle.OracleLBM(ph, react=react, **params)
    o.set_rate_scale(ks)
    o.set_source(S)
    s.step(40)
    o.step(40)
    np.testing.assert_allclose(s.field(), o.concentration(), rtol=0, atol=2e-6 + 1e-7 * 40)
    rg, ro = s.cell_reaction(), o.cell_reaction()
    assert ro.max() > 0
    np.testing.assert_allclose(rg, ro, rtol=1e-4, atol=1e-9)
    fg, fo = s.fluxes(), o.fluxes()
    assert fg["R"] == pytest.approx(fo["R"], rel=2e-5)
    # removing them restores the uniform step
    s.set_rate_scale(None)
    s.set_source(None)
    s.init()
    s.step(10)
    o2 = oracle.OracleLBM(ph, react=react, **params)
    o2.step(10)
    np.testing.assert_allclose(s.field(), o2.concentration(), rtol=0, atol=2e-6 + 1e-7 * 10)
    s.close()


def test_per_cell_arrays_need_plain_populations(cuda_lib):
    from paper_1410_1914_gb300 import Solver
    from paper_1410_1914_gb300 import _lib as L
    ph, react, params = inputs.make_workload("pt_cl_256", shape=(6, 6, 20), seed=62)
    s = Solver(ph.shape, storage="fp32", **params)
    s.set_structure(ph, react)
    with pytest.raises(L.ClError) as e:
        s.set_rate_scale(np.ones(ph.shape))
    assert e.value.status == L.CL_ERR_STATE
    s.close()


def _layer(seed=2):
    ph = inputs.with_reservoir(inputs.pt_cl((9, 9, 20), seed, 0.35, 0.35))
    params = dict(dx_m=5e-9, T_K=333.0, p_atm=1.0, M_kgmol=0.032, knudsen=1, bc_in=0, bc_out=1,
                  c_in=7.7, c_out=0.0, tau_ref=1.0)
    return ph, params


@pytest.mark.parametrize("sigma,ionomer_D,solver", [(1e-4, 2e-7, "krylov"), (1e4, 2e-7, "krylov"),
                                                    (1e-4, 2e-7, "lines"), (1e-4, None, "lines"),
                                                    (1e4, None, "lines")])
def test_coupled_against_oracle(cuda_lib, sigma, ionomer_D, solver):
    """ionomer_D None: O2 dissolved in the ionomer by Eq. 10-13 (the physical
    contrast), reached by the line-eliminated steady solve."""
    from paper_1410_1914_gb300 import coupled
    ph, params = _layer()
    ref = ocoupled.solve(ph, params, sigma=sigma, phi_m=0.6, k_ref=1e-2, ionomer_D=ionomer_D)
    got = coupled.solve(ph, params, sigma=sigma, phi_m=0.6, k_ref=1e-2, ionomer_D=ionomer_D, tol_phi=1e-7,
                        steady_solver=solver, krylov_max_iter=3000)
    assert ref["converged"] and got["converged"], got["status"]
    site = ref["site"]
    assert site.sum() > 0
    pa = ~np.isnan(ref["phi"])
    np.testing.assert_allclose(got["phi"][pa], ref["phi"][pa], rtol=0, atol=1e-6)
    assert np.all(got["phi"][~pa] == 0)
    np.testing.assert_allclose(got["C"], ref["C"], rtol=0, atol=1e-5 * params["c_in"])
    assert got["current_A_o2"] == pytest.approx(ref["current_A_o2"], rel=1e-5)
    if sigma > 1:
        # the membrane flux is then a difference of f32 populations of 0.6 V / 8 that
        # cancel to 1e-9 V: rounding, not a number to compare
        assert np.abs(got["phi"][pa] - 0.6).max() < 1e-6
    else:
        assert got["current_A_membrane"] == pytest.approx(ref["current_A_membrane"], rel=1e-4)
        # the membrane passes what the sites draw
        assert got["current_A_membrane"] == pytest.approx(got["current_A_o2"], rel=1e-4)
        assert got["phi"][pa].min() < 0.6 - 1e-4
    got["o2"].close()
    got["protons"].close()


def test_coupled_arguments(cuda_lib):
    from paper_1410_1914_gb300 import Solver
    from paper_1410_1914_gb300 import _lib as L
    ph, params = _layer()
    a = Solver(ph.shape, storage="fp32pop", react_rule=L.CL_REACT_IONOMER_SOLID, D_ionomer=2e-7, k_ms=1e-2,
               **params)
    a.set_structure(ph)
    b = Solver(ph.shape, storage="fp32", carrier=L.CL_CARRIER_PROTON, D_ionomer=1e-4, k_ms=0.0, knudsen=0,
               dx_m=5e-9, bc_in=0, bc_out=1, c_in=0.6, c_out=0.6)
    b.set_structure(np.ascontiguousarray(ph[:, :, ::-1]))
    cp = L.cl_coupled_params(alpha=0.61, phi_m=0.6, phi_ref=0.6, relax=0.5, tol_phi=1e-7, max_outer=5,
                             krylov_tol=1e-10, krylov_max_iter=100, steady_solver=0)
    lib = L.load()
    import ctypes
    info = L.cl_coupled_info()
    assert lib.cl_coupled_solve(a.h, b.h, ctypes.byref(cp), None, 0, ctypes.byref(info)) == L.CL_ERR_STATE
    assert lib.cl_coupled_solve(a.h, a.h, ctypes.byref(cp), None, 0, ctypes.byref(info)) == L.CL_ERR_ARG
    cp.relax = 0.0
    assert lib.cl_coupled_solve(a.h, a.h, ctypes.byref(cp), None, 0, ctypes.byref(info)) == L.CL_ERR_ARG
    cp.relax = 0.5
    cp.steady_solver = 2
    assert lib.cl_coupled_solve(a.h, a.h, ctypes.byref(cp), None, 0, ctypes.byref(info)) == L.CL_ERR_ARG
    a.close()
    b.close()
