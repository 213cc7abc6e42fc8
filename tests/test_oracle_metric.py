"""Pins of the oracle's error metric: every parity check goes through it.

``oracle.frobenius`` (the C routine ``oracle_frobenius``), ``oracle.rel_error``
and ``oracle.max_elem_error`` decide whether a GPU result passes, so each is
checked here against values worked out by hand or fixed by mathematics (not by
re-typing its formula):

* Pythagorean quadruples: ||(3, 4, 12)|| = 13, ||(2, 3, 6)|| = 7, and a 2 x 2
  matrix ((1, 2), (2, 4)) of norm 5;
* ||ones(n)|| = sqrt(n) and ||c a|| = |c| ||a|| (homogeneity), ||-a|| = ||a||;
* rel_error((1, 2, 2), (0, 2, 2)) = 1 / sqrt(8), rel_error((1, 1), (3, 4)) = sqrt(13) / 5;
* the zero-reference branch returns the absolute norm of the difference;
* a uniform relative perturbation ref (1 + e) has relative error exactly e;
* max_elem_error: one wrong entry off by +d or -d against max |ref| = m gives d / m.

tests/test_oracle_mutations.py plants mistakes in copies of these routines and
checks that these pins catch them.
"""
import math

import numpy as np
import pytest

import oracle


def metric_pins_hold(frobenius, rel_error, max_elem_error=None) -> bool:
    """True when the given implementations satisfy every pin (used on mutated copies too)."""
    def close(a, b, tol=1e-14):
        return abs(a - b) <= tol * max(1.0, abs(b))

    checks = [
        close(frobenius(np.array([3.0, 4.0, 12.0])), 13.0),
        close(frobenius(np.array([2.0, -3.0, 6.0])), 7.0),
        close(frobenius(np.array([[1.0, 2.0], [2.0, 4.0]])), 5.0),
        close(frobenius(np.ones(1000)), math.sqrt(1000.0)),
        close(frobenius(np.zeros(7)), 0.0),
        close(frobenius(np.array([-5.0])), 5.0),
        close(frobenius(-3.0 * np.array([3.0, 4.0, 12.0])), 39.0),
        close(rel_error(np.array([1.0, 2.0, 2.0]), np.array([0.0, 2.0, 2.0])), 1.0 / math.sqrt(8.0)),
        close(rel_error(np.array([1.0, 1.0]), np.array([3.0, 4.0])), math.sqrt(13.0) / 5.0),
        close(rel_error(np.array([3.0, 4.0]), np.zeros(2)), 5.0),          # zero reference: absolute
        close(rel_error(np.array([2.0, 3.0]), np.array([2.0, 3.0])), 0.0),
    ]
    rng = np.random.default_rng(5)
    ref = rng.standard_normal((17, 9))
    checks.append(close(rel_error(ref * (1.0 + 1e-3), ref), 1e-3, tol=1e-9))
    checks.append(close(rel_error(ref * (1.0 - 2.5e-6), ref), 2.5e-6, tol=1e-6))
    # symmetric in the sign of the difference, but not in its arguments
    checks.append(close(rel_error(ref + 0.01 * ref[::-1], ref), rel_error(ref - 0.01 * ref[::-1], ref)))
    checks.append(not close(rel_error(2.0 * ref, ref), rel_error(ref, 2.0 * ref)))
    if max_elem_error is not None:
        m = np.array([[1.0, -8.0], [2.0, 0.5]])
        g = m.copy()
        g[1, 1] += 0.2
        checks.append(close(max_elem_error(g, m), 0.2 / 8.0))
        checks.append(close(max_elem_error(np.array([0.0, 0.3]), np.zeros(2)), 0.3))   # absolute
        g2 = m.copy()
        g2[0, 0] -= 0.3                       # the largest deviation is negative
        checks.append(close(max_elem_error(g2, m), 0.3 / 8.0))
        checks.append(close(max_elem_error(m, m), 0.0))
        checks.append(close(max_elem_error(-m, m), 2.0))
    return all(checks)


def test_metric_pins_hold_for_the_oracle():
    assert metric_pins_hold(oracle.frobenius, oracle.rel_error, oracle.max_elem_error)


@pytest.mark.parametrize("a", [[3.0, 4.0, 12.0], [[1.0, 2.0], [2.0, 4.0]], [1e-300, 1e-300]])
def test_frobenius_matches_math_hypot(a):
    flat = np.ravel(a)
    want = math.hypot(*flat)
    assert abs(oracle.frobenius(np.array(a)) - want) <= 1e-15 * max(want, 1e-300)


def test_frobenius_long_double_sum_beats_naive_rounding():
    # 1 + 2^-30 summed 2^20 times: the FP64 norm squared is 2^20 (1 + 2^-29 + 2^-60); a
    # long-double accumulation keeps it to within one FP64 rounding of the true norm
    n = 1 << 20
    a = np.full(n, 1.0 + 2.0 ** -30)
    want = math.sqrt(n) * (1.0 + 2.0 ** -30)
    assert abs(oracle.frobenius(a) - want) <= 2.0 ** -52 * want


def test_rel_error_refuses_mismatched_shapes():
    with pytest.raises(ValueError):
        oracle.rel_error(np.zeros((3, 1)), np.zeros(3))
    with pytest.raises(ValueError):
        oracle.max_elem_error(np.zeros((3, 1)), np.zeros(3))


def test_max_elem_error_of_empty_arrays_is_zero():
    assert oracle.max_elem_error(np.zeros((0, 4)), np.zeros((0, 4))) == 0.0
