"""Cost-model thresholds of the threshold analysis (Sec. IV).

All functions take Schmidt rank k = 2 (CZ/CX cutting), equal partitioning into
n segments of q/n qubits and c cuts per boundary (c_total = c (n - 1)).
"""

from __future__ import annotations

import math


def n_sub_equal(n: int, c: int, k: int = 2) -> int:
    """N_sub = sum_i k^{c_i}: the two edge segments see c cuts, the n-2 interior
    segments see 2c (Algorithm 1 complexity note)."""
    if n == 1:
        return 1
    return 2 * k ** c + (n - 2) * k ** (2 * c)


def speedup_condition(q: float, n: int, n_sub: float) -> bool:
    """Eq. 12: N_sub / n < 2^{q (1 - 1/n)} (T_sub < T_orig, depth-free)."""
    return n_sub / n < 2.0 ** (q * (1.0 - 1.0 / n))


def threshold_n2(q: float) -> float:
    """Eq. 13: c_total < q / 2 for n = 2."""
    return q / 2.0


def threshold_nge3(q: float, n: int) -> float:
    """Eq. 14: c_total < q (n-1)^2 / (2n) + (n-1) log2(n / (n-2)) / 2, n >= 3,
    obtained with N_sub ~ (n-2) 2^{2 c_total / (n-1)}."""
    if n < 3:
        raise ValueError("Eq. 14 needs n >= 3")
    return q * (n - 1) ** 2 / (2.0 * n) + (n - 1) * math.log2(n / (n - 2.0)) / 2.0


def threshold(q: float, n: int) -> float:
    return threshold_n2(q) if n == 2 else threshold_nge3(q, n)


def slope_delta(n: int):
    """Table II: c_total < slope * q + delta."""
    if n == 2:
        return 0.5, 0.0
    return (n - 1) ** 2 / (2.0 * n), (n - 1) * math.log2(n / (n - 2.0)) / 2.0


def nonuniform_reduction(n: int) -> float:
    """Eq. 15: the c_total threshold drops by this many cuts when D_seg = D
    instead of D/n (1 for n = 2, (n-1) log2(n) / 2 for n >= 3)."""
    if n == 2:
        return 1.0
    return (n - 1) * math.log2(n) / 2.0


def relative_speedup(t_cut: float, t_orig: float) -> float:
    """Delta = (T_cut - T_orig) / T_orig; negative means cutting is faster."""
    return (t_cut - t_orig) / t_orig
