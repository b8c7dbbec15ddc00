"""Circuit families used as synthetic inputs.

Families
--------
* ``brickwork``      -- random U3 + CZ brickwork on a 1D line: every layer puts
                        U3(theta, phi, lambda) on every qubit (angles i.i.d.
                        uniform in [0, 2*pi)) and then CZ(i, i+1) on the pairs
                        whose lower qubit has the layer's parity.  The layer
                        structure (alternating one-qubit and two-qubit layers)
                        is the repeated-block layout of the paper's circuit
                        family (Sec. V.A.2, Fig. 1).
* ``brickwork_cut``  -- the same generator with an exact number of
                        boundary-crossing CZs per partition boundary (the knob
                        used to sweep c_total).
* ``staircase``      -- the paper's own H/T/CX family (Fig. 1): a Hadamard
                        layer, then blocks of a CX ladder dressed with T gates;
                        a block repeated b times crosses each n=2 boundary b
                        times (Sec. V.A.2).
* ``ghz``, ``graph_state``, ``random_circuit`` -- small structured and random
                        circuits for closed-form and gate-position tests.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) so that every consumer draws the
identical stream from the same seed.  Draw order for the brickwork: layer,
then qubit, then (theta, phi, lambda); a double is ``(u64 >> 11) * 2**-53``.
"""

from __future__ import annotations

import math
from typing import List, NamedTuple, Optional, Sequence, Union

MASK64 = (1 << 64) - 1

ONE_QUBIT_KINDS = ("U3", "H", "X", "Z", "S", "SDG", "T", "TDG")
TWO_QUBIT_KINDS = ("CZ", "CX")
GATE_KINDS = ONE_QUBIT_KINDS + TWO_QUBIT_KINDS
# Schmidt-rank-4 gates (Eq. 1 with k = 4); CAN carries its three angles in
# (theta, phi, lam).
RANK4_KINDS = ("SWAP", "ISWAP", "CAN")
ALL_TWO_QUBIT_KINDS = TWO_QUBIT_KINDS + RANK4_KINDS


class Gate(NamedTuple):
    """One gate of a circuit.

    ``q1`` is -1 for one-qubit gates.  For CX, ``q0`` is the control and
    ``q1`` the target.  ``theta, phi, lam`` are only meaningful for U3 and,
    as the angles (t_x, t_y, t_z), for CAN.
    """

    kind: str
    q0: int
    q1: int = -1
    theta: float = 0.0
    phi: float = 0.0
    lam: float = 0.0


class SplitMix64:
    """Counter-based 64-bit generator (SplitMix64, Steele et al. 2014)."""

    GOLDEN = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + self.GOLDEN) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def next_double(self) -> float:
        """Uniform double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (2.0 ** -53)

    def next_angle(self) -> float:
        """Uniform angle in [0, 2*pi)."""
        return 2.0 * math.pi * self.next_double()


def equal_partition(q: int, n: int) -> List[int]:
    """Split q qubits into n contiguous segments whose sizes differ by at most
    one, larger segments first (e.g. 26 -> 9/9/8)."""
    if n < 1 or n > q:
        raise ValueError(f"cannot split {q} qubits into {n} segments")
    base, extra = divmod(q, n)
    return [base + (1 if i < extra else 0) for i in range(n)]


def cut_layers(depth: int, c: int) -> List[int]:
    """Layers that carry a boundary-crossing CZ when a boundary must be crossed
    exactly ``c`` times in ``depth`` layers: l_i = floor((2i+1) * D / (2c)),
    i = 0..c-1, i.e. evenly spread and centred in their D/c-layer windows."""
    if c < 0 or c > depth:
        raise ValueError(f"c={c} boundary crossings need 0 <= c <= depth={depth}")
    return [((2 * i + 1) * depth) // (2 * c) for i in range(c)]


def _u3_layer(rng: SplitMix64, q: int) -> List[Gate]:
    out = []
    for j in range(q):
        theta = rng.next_angle()
        phi = rng.next_angle()
        lam = rng.next_angle()
        out.append(Gate("U3", j, -1, theta, phi, lam))
    return out


def brickwork(q: int, depth: int, seed: int) -> List[Gate]:
    """Plain brickwork: layer l = U3 on qubits 0..q-1, then CZ(i, i+1) for every
    i with i % 2 == l % 2 and i + 1 < q."""
    rng = SplitMix64(seed)
    gates: List[Gate] = []
    for layer in range(depth):
        gates.extend(_u3_layer(rng, q))
        for i in range(layer % 2, q - 1, 2):
            gates.append(Gate("CZ", i, i + 1))
    return gates


def brickwork_cut(
    q: int,
    depth: int,
    seed: int,
    seg_sizes: Sequence[int],
    cuts_per_boundary: Union[int, Sequence[int]],
    boundary_kind: str = "CZ",
) -> List[Gate]:
    """Brickwork whose boundary-crossing CZs are chosen to give an exact cut
    count.  ``boundary_kind`` replaces every boundary gate by "SWAP",
    "ISWAP" or "CAN" (a canonical gate whose three angles come, in order,
    from a second SplitMix64 stream seeded with seed ^ 0x5EED, uniform in
    [0, 2*pi)); the brickwork's own angle stream is unchanged.

    Boundary b sits between qubits (p-1, p), p = sum(seg_sizes[:b+1]).  All
    natural CZs on boundary pairs are removed; boundary b instead gets a CZ in
    each layer of ``cut_layers(depth, c_b)``.  A boundary CZ placed in a layer of
    the other parity overlaps its neighbours' CZs in that layer; CZ gates are
    diagonal and commute, so the circuit stays well defined.  The angle stream
    does not depend on the cut choice.
    """
    if sum(seg_sizes) != q or any(s < 1 for s in seg_sizes):
        raise ValueError("segment sizes must be positive and sum to q")
    n_b = len(seg_sizes) - 1
    if isinstance(cuts_per_boundary, int):
        cpb = [cuts_per_boundary] * n_b
    else:
        cpb = list(cuts_per_boundary)
    if len(cpb) != n_b:
        raise ValueError("need one cut count per boundary")
    bpos = []
    acc = 0
    for s in seg_sizes[:-1]:
        acc += s
        bpos.append(acc)
    layer_sets = [set(cut_layers(depth, c)) for c in cpb]
    boundary_lower = {p - 1: b for b, p in enumerate(bpos)}
    if boundary_kind not in ("CZ",) + RANK4_KINDS:
        raise ValueError(f"unsupported boundary gate {boundary_kind!r}")
    rng = SplitMix64(seed)
    rng_can = SplitMix64(seed ^ 0x5EED)
    gates: List[Gate] = []
    for layer in range(depth):
        gates.extend(_u3_layer(rng, q))
        for i in range(0, q - 1):
            if i in boundary_lower:
                if layer in layer_sets[boundary_lower[i]]:
                    if boundary_kind == "CAN":
                        t, p, l = rng_can.next_angle(), rng_can.next_angle(), rng_can.next_angle()
                        gates.append(Gate("CAN", i, i + 1, t, p, l))
                    else:
                        gates.append(Gate(boundary_kind, i, i + 1))
            elif i % 2 == layer % 2:
                gates.append(Gate("CZ", i, i + 1))
    return gates


def split_cuts(c_total: int, n: int) -> List[int]:
    """Spread c_total cuts over the n-1 boundaries, earlier boundaries first."""
    if n < 2:
        if c_total:
            raise ValueError("a single segment has no boundary to cut")
        return []
    base, extra = divmod(c_total, n - 1)
    return [base + (1 if b < extra else 0) for b in range(n - 1)]


class BatchItem(NamedTuple):
    gates: List[Gate]
    q: int
    depth: int
    seg_sizes: List[int]
    cuts_per_boundary: List[int]
    seed: int


def uneven_sizes(rng: SplitMix64, q: int, n: int, min_size: int = 4) -> List[int]:
    """n contiguous segment sizes, each >= min_size, summing to q: every
    segment starts at min_size and each remaining qubit goes to a segment
    drawn uniformly."""
    if n * min_size > q:
        raise ValueError("q too small for n segments of min_size")
    sizes = [min_size] * n
    for _ in range(q - n * min_size):
        sizes[rng.next_u64() % n] += 1
    return sizes


def uneven_batch(
    n_circ: int,
    seed: int,
    q_range: Sequence[int] = (16, 26),
    depths: Sequence[int] = (8, 16, 32),
    n_choices: Sequence[int] = (2, 3),
    c_range: Sequence[int] = (2, 6),
) -> List[BatchItem]:
    """Independent random brickwork circuits for a batch: q uniform in
    q_range (inclusive), depth from depths, n from n_choices, unequal
    contiguous segments (uneven_sizes), c_total uniform in c_range spread
    over the boundaries (split_cuts).  Circuit i uses brickwork seed
    seed * 1000003 + i."""
    rng = SplitMix64(seed)
    out: List[BatchItem] = []
    for i in range(n_circ):
        q = q_range[0] + int(rng.next_u64() % (q_range[1] - q_range[0] + 1))
        depth = depths[rng.next_u64() % len(depths)]
        n = n_choices[rng.next_u64() % len(n_choices)]
        c = c_range[0] + int(rng.next_u64() % (c_range[1] - c_range[0] + 1))
        sizes = uneven_sizes(rng, q, n)
        cpb = split_cuts(c, n)
        s = seed * 1000003 + i
        out.append(BatchItem(brickwork_cut(q, depth, s, sizes, cpb), q, depth, sizes, cpb, s))
    return out


def staircase(q: int, blocks: int) -> List[Gate]:
    """The paper's H/T/CX family (Fig. 1).

    Block: T on qubits 0 and 1, then for j = 0..q-2 a CX(j -> j+1) followed by
    T on each of j, j+1, j+2 that exists.  The first block is preceded by H on
    every qubit; repeated blocks omit it (Sec. V.A.2).
    """
    gates: List[Gate] = [Gate("H", j) for j in range(q)]
    for _ in range(blocks):
        for j in (0, 1):
            if j < q:
                gates.append(Gate("T", j))
        for j in range(q - 1):
            gates.append(Gate("CX", j, j + 1))
            for t in (j, j + 1, j + 2):
                if t < q:
                    gates.append(Gate("T", t))
    return gates


def staircase_depth(q: int, blocks: int, p: int) -> List[Gate]:
    """The depth-augmented staircase of the paper's depth sweep (Sec. V.C,
    supplementary Fig. 8): after the H layer, 10^p single-qubit layers on
    qubit 0, alternating T and X (T first); then the staircase blocks; then
    10^p more such layers on qubit q-1.  q and the cut count are unchanged."""
    n_layers = 10 ** p
    base = staircase(q, blocks)
    pad_top = [Gate("T" if i % 2 == 0 else "X", 0) for i in range(n_layers)]
    pad_bot = [Gate("T" if i % 2 == 0 else "X", q - 1) for i in range(n_layers)]
    return base[:q] + pad_top + base[q:] + pad_bot


def ghz(q: int) -> List[Gate]:
    """H on qubit 0, then the CX chain 0->1->...->q-1."""
    return [Gate("H", 0)] + [Gate("CX", j, j + 1) for j in range(q - 1)]


def graph_state(q: int, edges: Sequence[Sequence[int]]) -> List[Gate]:
    """H on every qubit, then CZ on every edge (in the order given)."""
    return [Gate("H", j) for j in range(q)] + [Gate("CZ", a, b) for a, b in edges]


def random_circuit(
    q: int,
    n_gates: int,
    seed: int,
    kinds: Optional[Sequence[str]] = None,
) -> List[Gate]:
    """Gates of random kind on random qubits (two-qubit gates on random,
    possibly far-apart, pairs).  Used to exercise every gate position."""
    rng = SplitMix64(seed)
    kinds = tuple(kinds) if kinds is not None else GATE_KINDS
    gates: List[Gate] = []
    for _ in range(n_gates):
        kind = kinds[rng.next_u64() % len(kinds)]
        if kind in ALL_TWO_QUBIT_KINDS and q >= 2:
            a = rng.next_u64() % q
            b = rng.next_u64() % (q - 1)
            if b >= a:
                b += 1
            if kind == "CAN":
                t, p, l = rng.next_angle(), rng.next_angle(), rng.next_angle()
                gates.append(Gate(kind, int(a), int(b), t, p, l))
            else:
                gates.append(Gate(kind, int(a), int(b)))
        elif kind in ALL_TWO_QUBIT_KINDS:
            continue
        elif kind == "U3":
            t, p, l = rng.next_angle(), rng.next_angle(), rng.next_angle()
            gates.append(Gate("U3", int(rng.next_u64() % q), -1, t, p, l))
        else:
            gates.append(Gate(kind, int(rng.next_u64() % q)))
    return gates


def sample_indices(q: int, count: int, seed: int) -> List[int]:
    """``count`` amplitude indices drawn uniformly from [0, 2**q): the top q bits
    of successive SplitMix64 outputs."""
    rng = SplitMix64(seed)
    if q == 0:
        return [0] * count
    return [rng.next_u64() >> (64 - q) for _ in range(count)]
