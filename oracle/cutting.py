"""Gate cutting with exact full-state reconstruction, written out literally.

Follows the paper's three phases (Eq. 3, Appendix B):

* ``preprocess``            -- Algorithm 1: find the two-qubit gates that
                               straddle a partition boundary, split each
                               segment's gate list into fragments at those
                               gates, and for every bit string b in {0,1}^{c_i}
                               build the subcircuit S_i^(b) by appending the
                               b_j-th local term of cut j between fragments;
                               build the merge index table M.
* ``simulate_subcircuits``  -- Algorithm 2: simulate every S_i^(r) from |0>.
* ``merge``                 -- Algorithm 3: Psi = sum_m alpha_m
                               psi_1^(r_1) (x) ... (x) psi_n^(r_n).
* ``amplitudes``            -- the Algorithm 3 sum evaluated at chosen indices
                               only (same terms, same alpha_m), for q where the
                               2^q vector is too large to build on the host.

Schmidt-rank-4 gates (SWAP, ISWAP, CAN; Eq. 1 with k = 4) are cut with the
operator-Schmidt decomposition itself, U = sum_l s_l A_l (x) B_l, computed as
the singular value decomposition of U realigned so that its rows index the
first qubit's (out, in) pair and its columns the second's (the textbook
construction); term l puts s_l A_l on the first qubit and B_l on the second.
A cut with k_j terms contributes a base-k_j digit to the variant and merge
indices (mixed radix; for k = 2 this is the bit slicing below).

Cut decompositions (Schmidt rank k = 2, Eq. 1):

* ``"s_sdg"``      -- Eq. 2: CZ = [S (x) S + i S^dag (x) S^dag] / (1+i).
                      Term b=0 puts S on both cut qubits with coefficient
                      1/(1+i); term b=1 puts S^dag on both with coefficient
                      i/(1+i).
* ``"projector"``  -- CZ = |0><0| (x) I + |1><1| (x) Z (coefficients 1, 1):
                      term b puts the projector |b><b| on the first qubit of
                      the gate and Z^b on the second.

A CX straddling a boundary is first rewritten as CX = (I (x) H) CZ (I (x) H)
(Sec. II.A.2, Algorithm 1 preamble), so its target side receives H A_b H in
place of A_b: H S H / H S^dag H for Eq. 2 (Algorithm 1 appends "HSH") and
H Z^b H = X^b for the projector split.

Readings of the paper where it is silent (also listed in the design notes):

* the same bit b_j selects the term on both sides of cut j;
* segment i's variant index is r = sum_t b_{j_t} 2^t over its adjacent cuts
  j_0 < j_1 < ... in circuit order, so M is bit slicing of the global index m;
* Algorithm 3 sums over all 2^{c_total} global combinations m (this equals the
  printed 2^{c_max} for n <= 3 on a line partition);
* segments are contiguous qubit ranges, segment 0 holding the lowest qubits, so
  Psi = psi_{n-1} (x) ... (x) psi_0 in numpy's kron order.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

from . import statevector as sv


@dataclass
class CutInfo:
    index: int          # j, in circuit order
    kind: str           # "CZ" or "CX"
    qubits: Tuple[int, int]
    segments: Tuple[int, int]


@dataclass
class Preprocessed:
    q: int
    seg_sizes: List[int]
    seg_starts: List[int]
    cuts: List[CutInfo]
    coefs: List[Tuple[complex, ...]]       # per cut j: coefficient of each term
    seg_cuts: List[List[int]]              # per segment: adjacent cut indices, circuit order
    fragments: List[List[List[sv.Op]]]     # per segment: F_i^(0..c_i) (local qubit indices)
    subcircuits: List[List[List[sv.Op]]]   # per segment: S_i^(r), r = 0..prod k - 1
    merge_table: List[Tuple[int, ...]] = field(default_factory=list)  # M[m] = (r_1..r_n)

    @property
    def c_total(self) -> int:
        return len(self.cuts)

    @property
    def ranks(self) -> List[int]:
        return [len(c) for c in self.coefs]

    @property
    def n_terms(self) -> int:
        return len(self.merge_table)

    @property
    def n_sub(self) -> int:
        return sum(len(s) for s in self.subcircuits)


def schmidt_terms(u: np.ndarray, rtol: float = 1e-12):
    """Operator-Schmidt decomposition (Eq. 1) of a 4x4 matrix in the basis
    |x_a x_b>: U = sum_l s_l kron(A_l, B_l).  Realign U into
    R[(out_a, in_a), (out_b, in_b)] and take its SVD R = W diag(s) V^H; then
    A_l = W[:, l] and B_l = V^H[l, :], each reshaped to 2x2.  Terms with
    s_l <= rtol * s_0 are dropped, so len(result) is the Schmidt rank k."""
    r = u.reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)
    w, sig, vh = np.linalg.svd(r)
    keep = [l for l in range(4) if sig[l] > rtol * sig[0]]
    coef = tuple(complex(sig[l]) for l in keep)
    first = tuple(w[:, l].reshape(2, 2) for l in keep)
    second = tuple(vh[l, :].reshape(2, 2) for l in keep)
    return coef, first, second


def local_terms(kind: str, decomp: str, gate=None):
    """Per term: (coefficient, operator on the gate's first qubit, operator on
    its second qubit).  CZ and CX use the chosen rank-2 split; SWAP, ISWAP
    and CAN the operator-Schmidt decomposition of their matrix."""
    if kind in ("SWAP", "ISWAP", "CAN"):
        if gate is None or gate.kind != kind:
            raise ValueError(f"a {kind} cut needs its gate")
        return schmidt_terms(sv.gate_matrix(gate))
    if decomp == "s_sdg":
        coef = (1.0 / (1.0 + 1.0j), 1.0j / (1.0 + 1.0j))
        first = (sv.S, sv.SDG)
        second = (sv.S, sv.SDG)
    elif decomp == "projector":
        coef = (1.0 + 0j, 1.0 + 0j)
        first = (sv.P0, sv.P1)
        second = (sv.I2, sv.Z)
    else:
        raise ValueError(f"unknown decomposition {decomp!r}")
    if kind == "CX":
        second = tuple(sv.H @ a @ sv.H for a in second)
    elif kind != "CZ":
        raise ValueError(f"cannot cut a {kind} gate with a rank-2 decomposition")
    return coef, first, second


def digit(r: int, radix: Sequence[int], t: int) -> int:
    """Digit t of r in the mixed radix `radix` (digit 0 least significant)."""
    for k in radix[:t]:
        r //= k
    return r % radix[t]


def compose(digits: Sequence[int], radix: Sequence[int]) -> int:
    """Inverse of digit(): sum_t digits[t] * prod(radix[:t])."""
    r, w = 0, 1
    for d, k in zip(digits, radix):
        r += d * w
        w *= k
    return r


def segment_map(q: int, seg_sizes: Sequence[int]):
    if sum(seg_sizes) != q or any(s < 1 for s in seg_sizes):
        raise ValueError("segment sizes must be positive and sum to q")
    starts, seg_of = [], []
    acc = 0
    for i, s in enumerate(seg_sizes):
        starts.append(acc)
        seg_of.extend([i] * s)
        acc += s
    return starts, seg_of


def preprocess(q: int, gates: Sequence, seg_sizes: Sequence[int],
               decomp: str = "projector") -> Preprocessed:
    """Algorithm 1."""
    sv.check_circuit(q, gates)
    starts, seg_of = segment_map(q, seg_sizes)
    n = len(seg_sizes)

    # Scan C and identify the gates that straddle partition boundaries; every
    # other gate goes, with local qubit indices, into its segment's item list.
    cuts: List[CutInfo] = []
    cut_gates = []
    items: List[list] = [[] for _ in range(n)]
    for g in gates:
        m, qs = sv.gate_op(g)
        segs = tuple(seg_of[x] for x in qs)
        if len(qs) == 2 and segs[0] != segs[1]:
            j = len(cuts)
            cuts.append(CutInfo(j, g.kind, (qs[0], qs[1]), (segs[0], segs[1])))
            cut_gates.append(g)
            items[segs[0]].append(("cut", j, 0, qs[0] - starts[segs[0]]))
            items[segs[1]].append(("cut", j, 1, qs[1] - starts[segs[1]]))
        else:
            s = segs[0]
            items[s].append(("gate", (m, tuple(x - starts[s] for x in qs))))

    coefs, firsts, seconds = [], [], []
    for c, g in zip(cuts, cut_gates):
        co, fi, se = local_terms(c.kind, decomp, g)
        coefs.append(co)
        firsts.append(fi)
        seconds.append(se)
    ranks = [len(co) for co in coefs]

    seg_cuts: List[List[int]] = []
    fragments: List[List[List[sv.Op]]] = []
    subcircuits: List[List[List[sv.Op]]] = []
    for i in range(n):
        # Split at each boundary gate into fragments F_i^(0..c_i).
        frags: List[List[sv.Op]] = [[]]
        markers = []  # (cut j, side, local qubit) in order
        for it in items[i]:
            if it[0] == "gate":
                frags[-1].append(it[1])
            else:
                markers.append(it[1:])
                frags.append([])
        seg_cuts.append([mk[0] for mk in markers])
        fragments.append(frags)
        radix = [ranks[mk[0]] for mk in markers]
        subs = []
        for r in range(int(np.prod(radix, dtype=np.int64)) if radix else 1):
            ops = list(frags[0])
            for t, (j, side, lq) in enumerate(markers):
                b = digit(r, radix, t)
                op_mat = firsts[j][b] if side == 0 else seconds[j][b]
                ops.append((op_mat, (lq,)))
                ops.extend(frags[t + 1])
            subs.append(ops)
        subcircuits.append(subs)

    # Merge index table: global combination m (one base-k_j digit per cut)
    # -> per-segment indices (the digits of the segment's adjacent cuts).
    table = []
    n_terms = int(np.prod(ranks, dtype=np.int64)) if ranks else 1
    for m in range(n_terms):
        table.append(tuple(
            compose([digit(m, ranks, j) for j in seg_cuts[i]], [ranks[j] for j in seg_cuts[i]])
            for i in range(n)
        ))
    return Preprocessed(q, list(seg_sizes), starts, cuts, coefs, seg_cuts,
                        fragments, subcircuits, table)


def simulate_subcircuits(pre: Preprocessed) -> List[List[np.ndarray]]:
    """Algorithm 2: |psi_i^(r)> = StateVectorSimulate(S_i^(r))."""
    return [[sv.simulate_ops(pre.seg_sizes[i], ops) for ops in pre.subcircuits[i]]
            for i in range(len(pre.seg_sizes))]


def alphas(pre: Preprocessed) -> np.ndarray:
    """alpha_m = prod_j coef_j[m_j] for every global combination m."""
    ranks = pre.ranks
    out = np.ones(pre.n_terms, dtype=np.complex128)
    for m in range(pre.n_terms):
        for j in range(pre.c_total):
            out[m] *= pre.coefs[j][digit(m, ranks, j)]
    return out


def merge(pre: Preprocessed, states: List[List[np.ndarray]]) -> np.ndarray:
    """Algorithm 3: one accumulator Psi and one temporary phi_m."""
    alpha = alphas(pre)
    psi = np.zeros(1 << pre.q, dtype=np.complex128)
    for m, rs in enumerate(pre.merge_table):
        phi = states[0][rs[0]]
        for i in range(1, len(rs)):
            phi = np.kron(states[i][rs[i]], phi)  # segment i holds the higher bits
        psi += alpha[m] * phi
    return psi


def cut_simulate(q: int, gates: Sequence, seg_sizes: Sequence[int],
                 decomp: str = "projector"):
    """T_pre + T_sub + T_merge of Eq. 3; returns (Psi, preprocessed, states)."""
    pre = preprocess(q, gates, seg_sizes, decomp)
    states = simulate_subcircuits(pre)
    return merge(pre, states), pre, states


def amplitudes(pre: Preprocessed, states: List[List[np.ndarray]],
               xs: Sequence[int]) -> np.ndarray:
    """Psi[x] = sum_m alpha_m prod_i psi_i^(r_i(m))[x restricted to G_i]."""
    xs = np.asarray(xs, dtype=np.int64)
    alpha = alphas(pre)
    out = np.zeros(len(xs), dtype=np.complex128)
    locs = [(xs >> pre.seg_starts[i]) & ((1 << pre.seg_sizes[i]) - 1)
            for i in range(len(pre.seg_sizes))]
    for m, rs in enumerate(pre.merge_table):
        term = np.full(len(xs), alpha[m], dtype=np.complex128)
        for i, r in enumerate(rs):
            term = term * states[i][r][locs[i]]
        out += term
    return out
