"""Pins of the oracle's Algorithms 1-3 (decomposition identities, Schmidt
ranks, exact reconstruction, closed-form cut states, counts)."""

import math

import numpy as np
import pytest

import workload as w
from oracle import cutting as ct
from oracle import statevector as sv
import pins

DECOMPS = ["projector", "s_sdg"]


@pytest.mark.parametrize("kind", ["CZ", "CX"])
@pytest.mark.parametrize("decomp", DECOMPS)
def test_two_term_decomposition_identity(kind, decomp):
    assert pins.pin_decomposition(kind, decomp) < 1e-15


def test_eq2_coefficients():
    # Eq. 2: CZ = [S(x)S + i S^dag(x)S^dag] / (1 + i)
    coef, first, second = ct.local_terms("CZ", "s_sdg")
    assert abs(coef[0] - (1 - 1j) / 2) < 1e-16
    assert abs(coef[1] - (1 + 1j) / 2) < 1e-16
    assert np.allclose(first[0], np.diag([1, 1j])) and np.allclose(first[1], np.diag([1, -1j]))


def test_cx_is_hadamard_conjugated_cz():
    ih = np.kron(sv.I2, sv.H)
    assert np.max(np.abs(ih @ sv.CZ @ ih - sv.CX)) < 1e-15


def test_schmidt_ranks():
    # Sec. II.A.2: k = 2 for controlled unitaries, k = 4 for SWAP
    swap = np.eye(4)[[0, 2, 1, 3]].astype(complex)
    assert pins.schmidt_rank(sv.CZ) == 2
    assert pins.schmidt_rank(sv.CX) == 2
    assert pins.schmidt_rank(swap) == 4
    assert pins.schmidt_rank(np.kron(sv.H, sv.T)) == 1


@pytest.mark.parametrize("decomp", DECOMPS)
@pytest.mark.parametrize("q,depth,seed,segs", [
    (12, 4, 0, [6, 6]),
    (10, 6, 1, [5, 5]),
    (11, 5, 2, [6, 5]),
    (12, 6, 3, [4, 4, 4]),
    (13, 4, 4, [5, 4, 4]),
])
def test_cut_equals_uncut_brickwork(decomp, q, depth, seed, segs):
    assert pins.pin_cut_equals_uncut(q, w.brickwork(q, depth, seed), segs, decomp) < 1e-13


@pytest.mark.parametrize("decomp", DECOMPS)
@pytest.mark.parametrize("q,c,segs", [(12, 5, [6, 6]), (12, 3, [4, 4, 4]), (14, 8, [7, 7])])
def test_cut_equals_uncut_swept_cuts(decomp, q, c, segs):
    gates = w.brickwork_cut(q, 8, 11, segs, c)
    pre = ct.preprocess(q, gates, segs, decomp)
    assert pre.c_total == c * (len(segs) - 1)
    assert pins.pin_cut_equals_uncut(q, gates, segs, decomp) < 1e-13


@pytest.mark.parametrize("decomp", DECOMPS)
@pytest.mark.parametrize("segs", [[4, 4], [3, 5], [2, 3, 3]])
def test_cut_equals_uncut_staircase_cx(decomp, segs):
    gates = w.staircase(8, 3)
    assert pins.pin_cut_equals_uncut(8, gates, segs, decomp) < 1e-13


@pytest.mark.parametrize("decomp", DECOMPS)
@pytest.mark.parametrize("seed", range(4))
def test_cut_equals_uncut_random_positions(decomp, seed):
    # far-apart two-qubit gates: cuts between non-adjacent segments too
    gates = w.random_circuit(9, 70, seed)
    assert pins.pin_cut_equals_uncut(9, gates, [3, 3, 3], decomp) < 1e-12


@pytest.mark.parametrize("decomp", DECOMPS)
def test_ghz_cut_closed_form(decomp):
    q = 8
    psi, pre, _ = ct.cut_simulate(q, w.ghz(q), [4, 4], decomp)
    assert pre.c_total == 1 and pre.cuts[0].kind == "CX"
    ref = np.zeros(1 << q, complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - ref)) < 1e-15


@pytest.mark.parametrize("decomp", DECOMPS)
def test_graph_state_cut_closed_form(decomp):
    q = 8
    edges = [(0, 1), (3, 4), (2, 5), (1, 7), (4, 6), (0, 4)]
    psi, pre, _ = ct.cut_simulate(q, w.graph_state(q, edges), [4, 4], decomp)
    assert pre.c_total == 4
    for x in range(1 << q):
        s = sum(((x >> a) & 1) * ((x >> b) & 1) for a, b in edges)
        assert abs(psi[x] - (-1) ** s / math.sqrt(1 << q)) < 1e-15


def test_no_cut_is_kronecker_of_segments():
    q, segs = 10, [4, 6]
    gates = w.brickwork_cut(q, 5, 3, segs, 0)
    psi, pre, states = ct.cut_simulate(q, gates, segs)
    assert pre.c_total == 0 and pre.n_sub == 2
    a = sv.simulate(4, [g for g in gates if max(g.q0, g.q1) < 4])
    b = sv.simulate(6, [g._replace(q0=g.q0 - 4, q1=(g.q1 - 4 if g.q1 >= 0 else -1))
                        for g in gates if g.q0 >= 4])
    assert np.max(np.abs(psi - np.kron(b, a))) < 1e-15


def test_projector_variant_sum():
    gates = w.brickwork_cut(10, 6, 9, [5, 5], 4)
    assert pins.pin_projector_variant_sum(10, gates, [5, 5]) < 1e-13


@pytest.mark.parametrize("n,c", [(2, 1), (2, 4), (3, 2), (4, 1)])
def test_subcircuit_counts(n, c):
    from oracle import thresholds as th
    q = 4 * n
    segs = w.equal_partition(q, n)
    pre = ct.preprocess(q, w.brickwork_cut(q, 6, 0, segs, c), segs)
    assert pre.c_total == c * (n - 1)
    # edges see c cuts, interior segments 2c; N_sub = sum_i 2^{c_i}
    assert [len(x) for x in pre.seg_cuts] == [c] + [2 * c] * (n - 2) + [c]
    assert pre.n_sub == th.n_sub_equal(n, c)
    if n == 2:
        assert pre.n_sub == 2 * 2 ** c


def test_merge_table_is_bit_slicing():
    segs = [4, 4, 4]
    pre = ct.preprocess(12, w.brickwork_cut(12, 6, 0, segs, 2), segs)
    for m, rs in enumerate(pre.merge_table):
        for i, r in enumerate(rs):
            for t, j in enumerate(pre.seg_cuts[i]):
                assert ((r >> t) & 1) == ((m >> j) & 1)


@pytest.mark.parametrize("decomp", DECOMPS)
def test_sampled_amplitudes_match_full_merge(decomp):
    q, segs = 12, [6, 6]
    gates = w.brickwork_cut(q, 6, 5, segs, 3)
    psi, pre, states = ct.cut_simulate(q, gates, segs, decomp)
    xs = w.sample_indices(q, 300, 17)
    amp = ct.amplitudes(pre, states, xs)
    assert np.max(np.abs(amp - psi[np.array(xs)])) < 1e-15


def test_uncuttable_gate_rejected():
    with pytest.raises(ValueError):
        ct.local_terms("FOO", "projector")
    with pytest.raises(ValueError):
        ct.local_terms("SWAP", "projector")  # a rank-4 cut needs its gate
    with pytest.raises(ValueError):
        ct.preprocess(4, [w.Gate("H", 0)], [2, 1])


# ----------------------------------------------------------- rank-4 cuts
def test_canonical_gate_closed_forms():
    # CAN(tx, ty, tz) = exp(-i (tx XX + ty YY + tz ZZ) / 2): special angles
    # reduce to SWAP (up to the phase e^{i pi/4}), ISWAP and textbook forms
    h = math.pi / 2
    assert np.max(np.abs(sv.can(-h, -h, -h) - np.exp(1j * math.pi / 4) * sv.SWAP)) < 1e-15
    assert np.max(np.abs(sv.can(-h, -h, 0.0) - sv.ISWAP)) < 1e-15
    th = 0.731
    zz = np.diag(np.exp(-0.5j * th * np.array([1, -1, -1, 1])))
    assert np.max(np.abs(sv.can(0.0, 0.0, th) - zz)) < 1e-15
    xx = math.cos(th / 2) * np.eye(4) - 1j * math.sin(th / 2) * np.kron(sv.X, sv.X)
    assert np.max(np.abs(sv.can(th, 0.0, 0.0) - xx)) < 1e-15
    # SWAP exchanges the two qubits' basis states
    for a in range(2):
        for b in range(2):
            e = np.zeros(4)
            e[2 * a + b] = 1
            assert np.array_equal(sv.SWAP @ e, np.eye(4)[2 * b + a])


@pytest.mark.parametrize("gate,rank", [
    (w.Gate("SWAP", 0, 1), 4), (w.Gate("ISWAP", 0, 1), 4),
    (w.Gate("CAN", 0, 1, 0.3, 1.1, 2.9), 4), (w.Gate("CAN", 0, 1, 0.0, 0.0, 0.8), 2),
    (w.Gate("CAN", 0, 1, 1.4, 0.0, 0.0), 2)])
def test_operator_schmidt_terms_rebuild_the_gate(gate, rank):
    coef, first, second = ct.local_terms(gate.kind, "projector", gate)
    assert len(coef) == rank == pins.schmidt_rank(sv.gate_matrix(gate))
    u = sum(c * np.kron(a, b) for c, a, b in zip(coef, first, second))
    assert np.max(np.abs(u - sv.gate_matrix(gate))) < 1e-14


@pytest.mark.parametrize("kind", ["SWAP", "ISWAP", "CAN"])
@pytest.mark.parametrize("segs,c", [([5, 5], 2), ([4, 3, 3], [1, 2]), ([3, 4, 3], 1)])
def test_cut_equals_uncut_rank4_boundaries(kind, segs, c):
    q = sum(segs)
    gates = w.brickwork_cut(q, 6, 7, segs, c, boundary_kind=kind)
    pre = ct.preprocess(q, gates, segs)
    cpb = [c] * (len(segs) - 1) if isinstance(c, int) else c
    assert pre.c_total == sum(cpb) and all(k == 4 for k in pre.ranks)
    # every segment has prod_{adjacent cuts} k_j variants
    assert pre.n_sub == sum(4 ** len(x) for x in pre.seg_cuts)
    assert pins.pin_cut_equals_uncut(q, gates, segs, "projector") < 1e-13


@pytest.mark.parametrize("seed", [101, 105, 112])
def test_cut_equals_uncut_mixed_ranks_random_positions(seed):
    kinds = ("U3", "H", "T", "CZ", "CX", "SWAP", "CAN")
    gates = w.random_circuit(9, 18, seed, kinds)
    pre = ct.preprocess(9, gates, [3, 3, 3], "s_sdg")
    assert pre.n_terms <= 4096, pre.ranks  # keeps the literal merge small
    assert pins.pin_bruteforce(9, gates) < 1e-13
    assert pins.pin_cut_equals_uncut(9, gates, [3, 3, 3], "s_sdg") < 1e-12


def test_mixed_radix_merge_table():
    segs = [4, 4, 4]
    gates = w.brickwork_cut(12, 6, 2, segs, [1, 1], boundary_kind="SWAP")
    gates = gates + [w.Gate("CZ", 3, 4)]  # one rank-2 cut after the rank-4 ones
    pre = ct.preprocess(12, gates, segs)
    assert pre.ranks == [4, 4, 2] and pre.n_terms == 32
    for m, rs in enumerate(pre.merge_table):
        d = [m % 4, (m // 4) % 4, m // 16]
        for i, r in enumerate(rs):
            radix = [pre.ranks[j] for j in pre.seg_cuts[i]]
            assert [ct.digit(r, radix, t) for t in range(len(radix))] == \
                [d[j] for j in pre.seg_cuts[i]]
