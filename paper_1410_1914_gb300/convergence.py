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


def remaining_change(dq: float, dq_prev: float) -> float:
    """Remaining change of a readout from its last two increments: the
    geometric tail |dq| rho/(1 - rho) when they shrink with the same sign,
    unbounded when they do not shrink, and the larger increment when the
    sign flips (a turning point must not pass for convergence).  The same
    rule as the library's stopping test."""
    if dq == 0.0 and dq_prev == 0.0:
        return 0.0
    rho = dq / dq_prev if dq_prev != 0.0 else (np.inf if dq > 0 else -np.inf)
    if rho >= 1.0:
        return np.inf
    if rho > 0.0:
        return abs(dq) * rho / (1.0 - rho)
    return max(abs(dq), abs(dq_prev))


class StopRule:
    """Feed the tracked readout once per check; `update` returns True when
    the estimated remaining relative change has been below `tol` at two
    checks in a row (a single quiet check at a turning point does not stop).
    The library's stopping test applies the same rule."""

    def __init__(self, tol: float):
        self.tol = tol
        self.q = self.dq = None
        self.quiet = 0

    def update(self, q: float) -> bool:
        if self.q is not None:
            dq = q - self.q
            if self.dq is not None:
                est = remaining_change(dq, self.dq)
                self.quiet = self.quiet + 1 if (q != 0 and est / abs(q) < self.tol) else 0
            self.dq = dq
        self.q = q
        return self.quiet >= 2


def deff_trace(solver, max_steps: int, check_every: int, stop_rel_change: float = 1e-7):
    """Run from the current state; return (steps, seconds, D_eff/D_b) per check
    (sigma_eff / sigma for the proton carrier).

    Stops after max_steps or once the extrapolated relative change of the
    outlet flux has been below stop_rel_change at two checks in a row (the
    solver's own stopping rule with tol_rel = stop_rel_change, without its
    flux-balance test)."""
    info = solver.info()
    nz, ny, nx = solver.shape
    p = solver.params
    # D_eff / D_b for O2; sigma_eff / sigma (the ionomer's own) for protons
    ref = p.D_ionomer if getattr(p, "carrier", 0) == 1 else info["D_b"]
    scale = nx / ((p.c_in - p.c_out) * ny * nz) * p.dx_m * p.dx_m / info["dt_s"] / ref
    steps, secs, vals = [], [], []
    rule = StopRule(stop_rel_change)
    t0 = time.perf_counter()
    n = 0
    while n + check_every <= max_steps:
        d = solver.solve_budget(check_every)
        n += check_every
        q = d["J_out"]
        steps.append(n)
        secs.append(time.perf_counter() - t0)
        vals.append(q * scale)
        if rule.update(q):
            break
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
