"""Pins of the threshold formulas against the paper's printed Table II and
Eq. 15 values, and against a numerical root of the defining inequality."""

import math
import os

import pytest

from oracle import thresholds as th

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_thresholds.txt")


def golden_rows():
    rows = {"table": {}, "reduction": {}, "measured": {}}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "reduction":
                rows["reduction"][int(parts[1])] = (float(parts[2]), int(parts[3]))
            elif parts[0] == "measured":
                rows["measured"][int(parts[1])] = (float(parts[2]), float(parts[3]))
            else:
                rows["table"][int(parts[0])] = (float(parts[1]), float(parts[2]))
    return rows


@pytest.mark.parametrize("n", [2, 3, 4])
def test_table2_slope_delta(n):
    slope, delta = golden_rows()["table"][n]
    s, d = th.slope_delta(n)
    assert abs(s - slope) < 1e-12 and abs(d - delta) < 1e-12


@pytest.mark.parametrize("n", [2, 3, 4])
def test_eq15_reduction_as_printed(n):
    value, decimals = golden_rows()["reduction"][n]
    assert round(th.nonuniform_reduction(n), decimals) == value


def root_of_eq12(q, n, depth_factor):
    """Largest real c_total with N_sub(c) * depth_factor < 2^{q(1-1/n)}, where
    N_sub is 2 * 2^c for n = 2 and (n-2) 2^{2c/(n-1)} for n >= 3 (the interior
    approximation of Sec. IV.B.1).  depth_factor = D_seg/D (1/n uniform, 1
    worst case).  Solved by bisection on the log of the inequality."""
    def f(c):
        if n == 2:
            nsub = 2.0 * 2.0 ** c
        else:
            nsub = (n - 2) * 2.0 ** (2.0 * c / (n - 1))
        return math.log2(nsub * depth_factor) - q * (1.0 - 1.0 / n)
    lo, hi = -100.0, 500.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0:
            lo = mid
        else:
            hi = mid
    return lo


@pytest.mark.parametrize("q", [12, 18, 24, 30])
@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_closed_forms_are_roots_of_eq12(q, n):
    assert abs(th.threshold(q, n) - root_of_eq12(q, n, 1.0 / n)) < 1e-9
    # Eq. 15: the worst-case depth factor moves the root by the reduction
    worst = root_of_eq12(q, n, 1.0)
    assert abs((th.threshold(q, n) - worst) - th.nonuniform_reduction(n)) < 1e-9


@pytest.mark.parametrize("q,c,expect", [(20, 9, True), (20, 10, False), (21, 10, True)])
def test_n2_condition_exact(q, c, expect):
    # Eq. 12 with the exact N_sub = 2 * 2^c equals Eq. 13: c < q/2
    assert th.speedup_condition(q, 2, th.n_sub_equal(2, c)) == expect
    assert (c < th.threshold_n2(q)) == expect


def test_relative_speedup_sign():
    assert th.relative_speedup(1.0, 2.0) == -0.5
    assert th.relative_speedup(3.0, 2.0) == 0.5
