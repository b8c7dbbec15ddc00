"""Planted mistakes in the oracle (on the CPU) must be caught by the pins.

Each case monkeypatches one plausible error into the oracle -- a wrong sign, a
swapped term, a transposed operand, a wrong bit position, a dropped term -- and
asserts that at least one pin now reports a large error.
"""

import numpy as np
import pytest

import workload as w
from oracle import cutting as ct
from oracle import statevector as sv
import pins

GATES = w.brickwork_cut(10, 6, 3, [4, 6], 3)
STAIR = w.staircase(8, 2)


def caught(*errs):
    return max(errs) > 1e-6


def test_wrong_eq2_coefficient_sign(monkeypatch):
    orig = ct.local_terms

    def bad(kind, decomp, gate=None):
        coef, a, b = orig(kind, decomp, gate)
        return (coef[0], -coef[1]), a, b

    monkeypatch.setattr(ct, "local_terms", bad)
    assert caught(pins.pin_decomposition("CZ", "s_sdg"),
                  pins.pin_cut_equals_uncut(10, GATES, [4, 6], "s_sdg"))


def test_projector_terms_swapped_on_one_side(monkeypatch):
    orig = ct.local_terms

    def bad(kind, decomp, gate=None):
        coef, a, b = orig(kind, decomp, gate)
        return coef, a, (b[1], b[0])

    monkeypatch.setattr(ct, "local_terms", bad)
    assert caught(pins.pin_cut_equals_uncut(10, GATES, [4, 6], "projector"))


def test_cx_target_without_hadamards(monkeypatch):
    orig = ct.local_terms

    def bad(kind, decomp, gate=None):
        return orig("CZ", decomp)

    monkeypatch.setattr(ct, "local_terms", bad)
    assert caught(pins.pin_cut_equals_uncut(8, STAIR, [4, 4], "projector"),
                  pins.pin_cut_equals_uncut(8, STAIR, [4, 4], "s_sdg"))


def test_transposed_u3(monkeypatch):
    orig = sv.u3
    monkeypatch.setattr(sv, "u3", lambda t, p, l: orig(t, p, l).T.copy())
    assert caught(pins.pin_u3_euler())


def test_wrong_target_axis(monkeypatch):
    orig = sv.apply_1q
    monkeypatch.setattr(sv, "apply_1q", lambda psi, u, j, q: orig(psi, u, q - 1 - j, q))
    assert caught(pins.pin_bruteforce(5, w.random_circuit(5, 30, 1)))


def test_swapped_two_qubit_basis(monkeypatch):
    orig = sv.apply_2q
    monkeypatch.setattr(sv, "apply_2q", lambda psi, u, a, b, q: orig(psi, u, b, a, q))
    assert caught(pins.pin_bruteforce(4, [w.Gate("H", 0), w.Gate("CX", 0, 2)]))


def test_kron_order_reversed(monkeypatch):
    def bad_merge(pre, states):
        alpha = ct.alphas(pre)
        psi = np.zeros(1 << pre.q, dtype=np.complex128)
        for m, rs in enumerate(pre.merge_table):
            phi = states[0][rs[0]]
            for i in range(1, len(rs)):
                phi = np.kron(phi, states[i][rs[i]])
            psi += alpha[m] * phi
        return psi

    monkeypatch.setattr(ct, "merge", bad_merge)
    assert caught(pins.pin_cut_equals_uncut(10, GATES, [4, 6], "projector"))


def test_dropped_merge_term(monkeypatch):
    orig = ct.alphas

    def bad(pre):
        a = orig(pre).copy()
        a[-1] = 0
        return a

    monkeypatch.setattr(ct, "alphas", bad)
    assert caught(pins.pin_cut_equals_uncut(10, GATES, [4, 6], "s_sdg"))


def test_variant_bits_reversed_in_one_segment(monkeypatch):
    orig = ct.preprocess

    def bad(*a, **k):
        pre = orig(*a, **k)
        c1 = len(pre.seg_cuts[1])
        pre.merge_table = [
            (r0, int(format(r1, f"0{c1}b")[::-1], 2) if c1 else r1)
            for r0, r1 in pre.merge_table
        ]
        return pre

    monkeypatch.setattr(ct, "preprocess", bad)
    assert caught(pins.pin_cut_equals_uncut(10, GATES, [4, 6], "projector"))


def test_sampled_amplitudes_with_segment_bits_from_the_wrong_offset(monkeypatch):
    # the per-amplitude form of Algorithm 3 (used at sizes where the full
    # merge cannot be formed) must take each segment's bits from its own
    # offset; reading segment i at the offset of segment n-1-i is caught by
    # the comparison with the full merge
    q, segs = 12, [5, 7]
    gates = w.brickwork_cut(q, 6, 5, segs, 3)
    psi, pre, states = ct.cut_simulate(q, gates, segs, "projector")
    xs = np.array(w.sample_indices(q, 300, 17))
    good = ct.amplitudes(pre, states, xs)
    assert np.max(np.abs(good - psi[xs])) < 1e-15
    pre.seg_starts = list(reversed(pre.seg_starts))
    bad = ct.amplitudes(pre, states, xs)
    assert caught(float(np.max(np.abs(bad - psi[xs]))))


@pytest.mark.parametrize("mistake", ["no realignment", "dropped smallest term"])
def test_schmidt_terms_mistakes(monkeypatch, mistake):
    # the operator-Schmidt terms of a rank-4 cut (Eq. 1, k = 4): an SVD of the
    # matrix itself instead of its realignment, or a dropped term, no longer
    # rebuilds the gate, and the cut simulation no longer equals the uncut one
    orig = ct.schmidt_terms

    def bad(u, rtol=1e-12):
        if mistake == "no realignment":
            w_, sig, vh = np.linalg.svd(u)
            return (tuple(complex(x) for x in sig), tuple(w_[:, l].reshape(2, 2) for l in range(4)),
                    tuple(vh[l, :].reshape(2, 2) for l in range(4)))
        coef, a, b = orig(u, rtol)
        return coef[:-1], a[:-1], b[:-1]

    monkeypatch.setattr(ct, "schmidt_terms", bad)
    g = w.Gate("CAN", 0, 1, 0.3, 1.1, 2.9)
    coef, a, b = ct.local_terms("CAN", "projector", g)
    u = sum(c * np.kron(x, y) for c, x, y in zip(coef, a, b))
    q, segs = 8, [4, 4]
    gates = w.brickwork_cut(q, 4, 7, segs, 1, boundary_kind="CAN")
    assert caught(float(np.max(np.abs(u - sv.gate_matrix(g)))),
                  pins.pin_cut_equals_uncut(q, gates, segs, "projector"))
