"""Parity tolerances of the GPU storage modes, per case.

The (C, delta) state stores the post-collision deviations delta_i = g*_i -
w_i C; with FP16 storage each is an f16 (11-bit significand) of delta
scaled by a power of two, so one store rounds it by at most 2^-12 |delta|
(plus 2^-38 in the subnormal range).  One step adds to C the six incoming
deviations of the neighbours (or of the cell itself at a wall) and
subtracts the cell's own six: twelve rounded values, at most
6 * 2^-11 * max|delta| when every rounding has the same sign.  Later steps
spread that error by diffusion and add their own; in three dimensions the
sum over past steps of the heat kernel at a point converges, so the error
stays a small multiple of one step's.  The bound is therefore
FP16_FACTOR * 2^-11 * max|delta| of the case, with max|delta| measured on
the FP64 oracle's own populations over the trajectory (its pre-collision
deviations bound the post-collision ones: delta* = (1 - omega) delta with
omega in [1, 2)), plus the f32 rounding of the returned field.

On the paper's D3Q19 lattice a step adds 18 incoming and subtracts 18 own
deviations, three times as many rounded values, and the factor is three
times larger (FP16_FACTOR_Q19).

FP32 state: deviations in f32 (2^-24 relative) and C as a double-float, so
the returned f32 field is off by its own rounding (1e-7 for C <= 1).

Plain f32 populations: each of seven O(1) populations is rounded every
step, and nothing compensates: ulps of O(1) values per step.
"""
import numpy as np

FP16_FACTOR = 8.0
FP16_FACTOR_Q19 = 24.0
OUT_ROUND = 1e-7  # f32 rounding of a returned C <= 1
W_D3Q7 = 0.125


def max_deviation(o) -> float:
    """max over active cells and i = 1..q-1 of |g_i - w_i C| of the oracle's
    current (pre-collision) populations; D3Q7 weights for q = 7, the
    lattice's own for q = 19."""
    g = o.populations()
    C = g.sum(axis=0)
    if o.q == 7:
        w = [W_D3Q7] * 6
    else:
        w = [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12
    act = o.active() > 0
    m = 0.0
    for i in range(1, o.q):
        d = np.abs(g[i] - w[i - 1] * C)
        if act.any():
            m = max(m, float(d[act].max()))
    return m


def step_sampled(o, steps: int, samples=(1, 2, 10)) -> float:
    """Step the oracle `steps` times; return max|delta| seen at the sample
    steps (those below `steps`) and at the end."""
    done = 0
    dmax = 0.0
    for s in sorted(set(v for v in samples if 0 < v < steps)) + [steps]:
        if s > done:
            o.step(s - done)
            done = s
            dmax = max(dmax, max_deviation(o))
    return dmax


def field_tol(storage: str, steps: int, dmax: float, q: int = 7) -> float:
    """Bound on max |C_gpu - C_oracle| after `steps` steps on a lattice of
    q velocities."""
    if storage == "fp32":
        return OUT_ROUND + 1e-10 * steps
    if storage == "fp16dev":
        return (FP16_FACTOR if q == 7 else FP16_FACTOR_Q19) * 2.0 ** -11 * dmax + OUT_ROUND
    if storage == "fp32pop":
        return 2e-6 + 1e-7 * steps
    raise ValueError(storage)
