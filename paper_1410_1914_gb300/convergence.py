"""Time-to-converged D_eff: how long a solve takes until its Eq. 19 readout
stays within a relative tolerance of the converged value.

The solver is advanced one check interval at a time through
cl_lbm_solve_budget (K fused steps and the FP64 flux reduction, one CUDA
graph); after each interval the outlet flux gives D_eff.  The first interval
from which every later D_eff stays within `rel` of the reference is the
convergence point.  The clock covers the device work and the per-check host
synchronisation, which is what a caller of cl_lbm_solve pays.
"""
from __future__ import annotations

import time

import numpy as np


def deff_trace(solver, max_steps: int, check_every: int, stop_rel_change: float = 1e-7):
    """Run from the current state; return (steps, seconds, D_eff/D_b) per check.

    Stops after max_steps or once the extrapolated relative change of the
    outlet flux falls below stop_rel_change (the solver's own stopping rule
    with tol_rel = stop_rel_change)."""
    info = solver.info()
    nz, ny, nx = solver.shape
    p = solver.params
    scale = nx / ((p.c_in - p.c_out) * ny * nz) * p.dx_m * p.dx_m / info["dt_s"] / info["D_b"]
    steps, secs, vals = [], [], []
    q_prev = dq_prev = None
    t0 = time.perf_counter()
    n = 0
    while n + check_every <= max_steps:
        d = solver.solve_budget(check_every)
        n += check_every
        q = d["J_out"]
        steps.append(n)
        secs.append(time.perf_counter() - t0)
        vals.append(q * scale)
        if q_prev is not None and dq_prev is not None and dq_prev != 0:
            dq = q - q_prev
            rho = dq / dq_prev
            est = abs(dq) * rho / (1 - rho) if 0 < rho < 1 else (abs(dq) if rho <= 0 else np.inf)
            if abs(q) > 0 and est / abs(q) < stop_rel_change:
                break
            dq_prev = dq
        elif q_prev is not None:
            dq_prev = q - q_prev
        q_prev = q
    return np.array(steps), np.array(secs), np.array(vals)


def time_to_tolerance(steps, secs, vals, ref: float, rel: float = 1e-3):
    """(steps, seconds) at the first check after which |D - ref| <= rel*|ref|
    holds for every remaining check; (None, None) if never."""
    ok = np.abs(vals - ref) <= rel * abs(ref)
    if not ok[-1]:
        return None, None
    bad = np.nonzero(~ok)[0]
    i = 0 if bad.size == 0 else bad[-1] + 1
    return int(steps[i]), float(secs[i])
