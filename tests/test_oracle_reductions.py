"""Pins of the oracle's verification quantities (oracle/reductions.py): the
FP64 numbers the paper's exact-reconstruction claim (Sec. III) is checked
with -- max |a - b|, max |b|, <a|b>, the squared norms and the fidelity
|<a|b>|^2 / (|a|^2 |b|^2) -- against closed forms and a brute-force
element-by-element sum."""

import math

import numpy as np
import pytest

from oracle import reductions as rd


def brute(a, b):
    # <a|b> = sum_k conj(a_k) b_k, summed exactly-rounded with math.fsum
    re = math.fsum((x.conjugate() * y).real for x, y in zip(a, b))
    im = math.fsum((x.conjugate() * y).imag for x, y in zip(a, b))
    na = math.fsum(abs(x) ** 2 for x in a)
    nb = math.fsum(abs(y) ** 2 for y in b)
    return complex(re, im), na, nb


def test_closed_forms_on_two_amplitudes():
    s = 1 / math.sqrt(2)
    a = np.array([s, 1j * s])
    b = np.array([1.0, 0.0])
    r = rd.compare(a, b)
    # <a|b> = conj(a_0) b_0 = 1/sqrt 2; fidelity 1/2; |a - b| at index 0 is 1 - 1/sqrt 2
    assert abs(r["inner_re"] - s) < 1e-16 and r["inner_im"] == 0.0
    assert abs(r["fidelity"] - 0.5) < 1e-15
    assert abs(r["max_abs_diff"] - s) < 1e-16  # index 1: |i/sqrt 2 - 0|
    assert r["max_abs_b"] == 1.0
    assert abs(r["norm2_a"] - 1.0) < 1e-15 and r["norm2_b"] == 1.0
    # the first argument is the conjugated one: <b|a> = conj(<a|b>)
    a2 = np.array([1j, 0.0])
    r2 = rd.compare(a2, b)
    assert r2["inner_re"] == 0.0 and r2["inner_im"] == -1.0


def test_global_phase_seen_by_max_diff_not_by_fidelity():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    th = 0.37
    b = np.exp(1j * th) * a
    r = rd.compare(a, b)
    assert abs(r["fidelity"] - 1.0) < 1e-14
    assert abs(r["max_abs_diff"] - abs(1 - np.exp(1j * th)) * np.max(np.abs(a))) < 1e-13
    # <a|b> = e^{i th} |a|^2
    n2 = r["norm2_a"]
    assert abs(complex(r["inner_re"], r["inner_im"]) - np.exp(1j * th) * n2) < 1e-12 * n2


def test_orthogonal_and_identical():
    a = np.array([1.0, 0.0, 0.0, 0.0], dtype=complex)
    b = np.array([0.0, 0.0, 1j, 0.0])
    r = rd.compare(a, b)
    assert r["fidelity"] == 0.0 and r["inner_re"] == 0.0 and r["inner_im"] == 0.0
    assert r["max_abs_diff"] == 1.0
    r = rd.compare(b, b)
    assert r["fidelity"] == 1.0 and r["max_abs_diff"] == 0.0


def test_scale_invariance_of_fidelity():
    rng = np.random.default_rng(2)
    a = rng.standard_normal(32) + 1j * rng.standard_normal(32)
    b = a + 0.1 * (rng.standard_normal(32) + 1j * rng.standard_normal(32))
    f = rd.compare(a, b)["fidelity"]
    assert abs(rd.compare(3.0 * a, 0.5j * b)["fidelity"] - f) < 1e-14
    assert 0.0 < f < 1.0  # Cauchy-Schwarz, strict for non-parallel vectors


@pytest.mark.parametrize("n,seed", [(1, 0), (7, 1), (1000, 2)])
def test_matches_brute_force_sums(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    r = rd.compare(a, b)
    inner, na, nb = brute(a, b)
    tol = 1e-14 * math.sqrt(na * nb)
    assert abs(r["inner_re"] - inner.real) <= tol and abs(r["inner_im"] - inner.imag) <= tol
    assert abs(r["norm2_a"] - na) <= 1e-14 * na and abs(r["norm2_b"] - nb) <= 1e-14 * nb
    assert abs(r["fidelity"] - abs(inner) ** 2 / (na * nb)) <= 1e-13
    # (numpy's complex modulus and Python's may differ in the last bit)
    md = max(abs(x - y) for x, y in zip(a, b))
    assert abs(r["max_abs_diff"] - md) <= 4e-16 * md
    mb = max(abs(y) for y in b)
    assert abs(r["max_abs_b"] - mb) <= 4e-16 * mb


def test_empty_and_mismatched():
    r = rd.compare(np.zeros(0, complex), np.zeros(0, complex))
    assert r["max_abs_diff"] == 0.0 and r["fidelity"] == 0.0
    with pytest.raises(ValueError):
        rd.compare(np.zeros(2), np.zeros(3))


def deviation(compare) -> float:
    """Largest error of a compare function's fields against the brute-force
    sums over a few random pairs (one with unequal norms)."""
    rng = np.random.default_rng(9)
    worst = 0.0
    for n, sa, sb in [(5, 1.0, 1.0), (40, 0.3, 2.0)]:
        a = sa * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
        b = sb * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
        r = compare(a, b)
        inner, na, nb = brute(a, b)
        ref = {"inner_re": inner.real, "inner_im": inner.imag, "norm2_a": na, "norm2_b": nb,
               "fidelity": abs(inner) ** 2 / (na * nb),
               "max_abs_diff": max(abs(x - y) for x, y in zip(a, b)),
               "max_abs_b": max(abs(y) for y in b)}
        worst = max(worst, max(abs(r[k] - v) / max(abs(v), 1e-300) for k, v in ref.items()))
    return worst


def test_deviation_of_the_oracle_is_rounding():
    assert deviation(rd.compare) < 1e-13


@pytest.mark.parametrize("mistake", ["no conjugate", "fidelity not squared", "max of a",
                                     "norms swapped"])
def test_planted_mistakes_are_caught(mistake):
    def bad(a, b):
        r = dict(rd.compare(a, b))
        if mistake == "no conjugate":
            inner = np.dot(a, b)
            r["inner_re"], r["inner_im"] = float(inner.real), float(inner.imag)
            r["fidelity"] = float(abs(inner) ** 2 / (r["norm2_a"] * r["norm2_b"]))
        elif mistake == "fidelity not squared":
            r["fidelity"] = math.sqrt(r["fidelity"])
        elif mistake == "max of a":
            r["max_abs_b"] = float(np.max(np.abs(a)))
        else:
            r["norm2_a"], r["norm2_b"] = r["norm2_b"], r["norm2_a"]
        return r

    assert deviation(bad) > 1e-3
