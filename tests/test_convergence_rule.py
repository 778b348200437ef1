"""The stopping rule's estimate of the remaining change (host logic, CPU)."""
import numpy as np
import pytest

from paper_1410_1914_gb300.convergence import StopRule, remaining_change, time_to_tolerance


def test_geometric_tail_is_exact_for_a_geometric_sequence():
    # q_n = 1 - 0.5 * 0.9^n: increments shrink by 0.9, remaining change 0.5 * 0.9^n
    q = [1 - 0.5 * 0.9 ** n for n in range(6)]
    dq, dq_prev = q[5] - q[4], q[4] - q[3]
    assert remaining_change(dq, dq_prev) == pytest.approx(0.5 * 0.9 ** 5, rel=1e-12)


def test_sign_flip_takes_the_larger_increment():
    assert remaining_change(-1e-12, 3e-4) == 3e-4
    assert remaining_change(2e-5, -3e-4) == 3e-4


def test_a_turning_point_does_not_stop_the_rule():
    """An overshoot such as a warm start gives: the readout rises, stalls for
    one check at the top, then relaxes back.  One quiet check at the top is
    not enough; the relaxation afterwards is followed to its end."""
    top = [1.0 + 3e-3 * (1 - 0.5 ** n) for n in range(12)]
    q = top + [top[-1]] + [1.0 + 3e-3 * 0.7 ** n for n in range(1, 80)]
    rule = StopRule(1e-8)
    stop_at = next((i for i, v in enumerate(q) if rule.update(v)), None)
    assert stop_at is not None and stop_at > len(top) + 20
    # the remaining change at the stop is what the rule estimated: within 10x of 1e-8
    assert abs(q[stop_at] - 1.0) < 1e-7


def test_growing_increments_and_stagnation():
    assert remaining_change(2e-3, 1e-3) == np.inf
    assert remaining_change(1e-3, 1e-3) == np.inf
    assert remaining_change(0.0, 0.0) == 0.0
    assert remaining_change(1e-6, 0.0) == np.inf
    assert remaining_change(-1e-6, 0.0) == 1e-6


def test_time_to_tolerance_takes_the_last_entry_into_the_band():
    steps = np.array([100, 200, 300, 400, 500])
    vals = np.array([1.5, 1.0005, 1.01, 1.0004, 1.0001])
    assert time_to_tolerance(steps, steps * 0.1, vals, 1.0, 1e-3) == (400, 40.0)
    assert time_to_tolerance(steps, steps * 0.1, vals[:3], 1.0, 1e-3) == (None, None)
