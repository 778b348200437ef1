"""Parity at the full workload sizes, in the launch configuration the
benchmark times (gpu).

* The 256^3 Pt layer of the benchmark (Knudsen D, 5 % catalytic faces at
  k = 1e-3 m/s, reservoir plane, zero-flux outlet), FP32 and FP16 states and
  plain f32 populations: one 100-step check interval (the CUDA graph of 100
  fused steps the benchmark replays, the last with the FP64 reduction) from
  the ramp, against 100 FP64 oracle steps, element by element, with the
  fluxes, the reaction rate and its plane profile.
* The 400^3 NPMC layer at 1 nm (micropores, every pore-solid face
  catalytic at k = 1e-5 m/s), FP16 state: 50 steps, likewise.

Element tolerances: tests/tolerances.py (per case from the oracle's own
deviations for FP16 storage).
"""
import numpy as np
import pytest

import oracle
from paper_1410_1914_gb300 import inputs
from tolerances import field_tol, step_sampled

pytestmark = pytest.mark.gpu


def _interval_run(ph, react, params, storage, steps):
    """`steps` lattice steps as one check interval (the benchmark's graph)."""
    from paper_1410_1914_gb300 import Solver
    s = Solver(ph.shape, storage=storage, check_every=steps, **params)
    s.set_structure(ph, react)
    s.solve_budget(steps)
    assert s.steps == steps
    return s


def _compare(s, o, storage, steps, dmax, ph):
    C = s.field()
    ref = o.concentration()
    tol = field_tol(storage, steps, dmax)
    err = float(np.abs(C - ref).max())
    print(f"\n{storage} {ph.shape} {steps} steps: max|dC| {err:.3e} tol {tol:.3e} max|delta| {dmax:.3e} "
          f"err/(2^-11 max|delta|) {err / max(2.0 ** -11 * dmax, 1e-300):.2f}")
    assert err <= tol
    fg, fo = s.fluxes(), o.fluxes()
    assert fg["n_active"] == fo["n_active"]
    ftol = {"fp32": 1e-6, "fp16dev": 5e-4, "fp32pop": 2e-5}[storage]
    nyz = ph.shape[0] * ph.shape[1]
    floor = {"fp32": 1e-9, "fp16dev": 2e-6, "fp32pop": 6e-8}[storage] * nyz + 1e-7
    assert abs(fg["J_in"] - fo["J_in"]) <= ftol * abs(fo["J_in"]) + floor
    # the rate itself to the storage's relative bound: physical rates are ~1e-18 mol/s at
    # these voxel sizes, so no absolute slack (pytest.approx's default 1e-12 would pass anything)
    assert fo["R"] > 0
    assert fg["R"] == pytest.approx(fo["R"], rel=ftol, abs=0)
    assert fg["sum_C"] == pytest.approx(fo["sum_C"], rel=max(ftol, 1e-6))
    tg, pRg, pCg = s.reaction_rate()
    to, pRo, pCo = o.reaction_rate()
    assert to > 0
    assert tg == pytest.approx(to, rel=ftol, abs=0)
    np.testing.assert_allclose(pCg, pCo, atol=tol)


@pytest.fixture(scope="module")
def pt256():
    ph, react, params = inputs.make_workload("pt_cl_256")
    o = oracle.OracleLBM(ph, react=react, **params)
    dmax = step_sampled(o, 100)
    return ph, react, params, o, dmax


@pytest.mark.parametrize("storage", ["fp32", "fp16dev", "fp32pop"])
def test_pt_256_interval_against_oracle(cuda_lib, pt256, storage):
    ph, react, params, o, dmax = pt256
    s = _interval_run(ph, react, params, storage, 100)
    _compare(s, o, storage, 100, dmax, ph)
    s.close()


def test_npmc_400_against_oracle(cuda_lib):
    ph, react, params = inputs.make_workload("npmc_cl_400")
    assert ph.shape == (400, 400, 400)
    s = _interval_run(ph, react, params, "fp16dev", 50)
    o = oracle.OracleLBM(ph, react=react, **params)
    dmax = step_sampled(o, 50)
    _compare(s, o, "fp16dev", 50, dmax, ph)
    s.close()
