"""The host side of cutting pinned on the CPU: every segment's compiled
program (cc_plan_program_image, Algorithm 1), run by the numpy interpreter of
the device program (Algorithm 2), summed over all global cut combinations
with each segment's variant taken by its cut bits (Algorithm 3 written out),
equals the FP64 oracle's uncut state.  This covers the cut items and their
coefficients for both rank-2 splits, CX cuts, rank-4 (SWAP/ISWAP/CAN) cuts by
Pauli products, chains of three segments, small tiles and both rotation
engine settings.  The plan's merge stages and index tables, applied as the
chained merge the merge kernels run, give the same state.  No GPU is used."""

import numpy as np
import pytest

import workload as w
from oracle import statevector as sv
from paper_2603_01443_gb300 import api
from program_interp import parse, run


def parse_stages(tail, c_i):
    """The merge stages (seg, qa, qb, K, Z, aidx_off, bidx_off) and the index
    table that follow a segment's cut ids in its image."""
    i = 2 + c_i
    n_st = int(tail[i])
    stages = [tuple(int(v) for v in tail[i + 1 + 7 * j:i + 8 + 7 * j]) for j in range(n_st)]
    i += 1 + 7 * n_st
    n_tab = int(tail[i])
    tab = np.asarray(tail[i + 1:i + 1 + n_tab], dtype=np.int64)
    assert len(tab) == n_tab and i + 1 + n_tab == len(tail)
    return stages, tab


def chained_merge(vecs, stages, tab):
    """Algorithm 3 as the plan stages it: stage s absorbs segment s into the
    product of the segments before it, U_s[z][x_s 2^qa + x] = sum_k
    U_{s-1}[aidx(z, k)][x] seg_s[bidx(z, k)][x_s], U_0 the variants of
    segment 0; the result is U_{n-1}[0]."""
    u = vecs[0]
    for seg, qa, qb, K, Z, ao, bo in stages:
        assert u.shape[1] == 1 << qa and vecs[seg].shape[1] == 1 << qb
        nxt = np.zeros((Z, 1 << (qa + qb)), dtype=complex)
        for z in range(Z):
            for k in range(K):
                a = u[tab[ao + z * K + k]]
                b = vecs[seg][tab[bo + z * K + k]]
                nxt[z] += np.kron(b, a)
        u = nxt
    assert u.shape[0] == 1
    return u[0]


def cut_state(gates, q, segs, decomp, prec, tile_bits):
    """The exhaustive sum over all global cut combinations, checked against
    the plan's chained merge of the same segment states."""
    vecs, ids, n_bits, staged = [], [], None, None
    for i, qi in enumerate(segs):
        words, reals = api.plan_program_image(gates, q, segs, i, decomp, prec, tile_bits)
        prog, tail = parse(words, reals, trailing=True)
        n_bits, c_i = tail[0], tail[1]
        ids.append(tail[2:2 + c_i])
        st = parse_stages(tail, c_i)
        if staged is None:
            staged = st
        else:  # every segment's image carries the same plan-wide stages
            assert st[0] == staged[0] and np.array_equal(st[1], staged[1])
        assert prog.nq == qi + c_i and prog.n_state == qi
        vecs.append(run(prog).reshape(1 << c_i, 1 << qi))  # variant r at rows, x_i at columns
    assert n_bits <= 10, "too many cut bits for the exhaustive term sum"
    psi = 0
    for m in range(1 << n_bits):
        phi = None
        for i in range(len(segs)):
            r = sum(((m >> b) & 1) << t for t, b in enumerate(ids[i]))
            phi = vecs[i][r] if phi is None else np.kron(vecs[i][r], phi)
        psi = psi + phi
    if len(segs) >= 2:
        chain = chained_merge(vecs, *staged)
        assert rel(chain, psi) <= 1e-13
    return psi


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("rot", ["1", "0"])
@pytest.mark.parametrize("decomp", ["projector", "s_sdg"])
@pytest.mark.parametrize("prec,tile_bits", [("c64", 5), ("c128", 4), ("c64", 0)])
def test_brickwork_cut_two_segments(host_lib, monkeypatch, rot, decomp, prec, tile_bits):
    monkeypatch.setenv("CUTSIM_ROT", rot)
    q, segs = 10, [5, 5]
    gates = w.brickwork_cut(q, 8, 11, segs, 3)
    got = cut_state(gates, q, segs, decomp, prec, tile_bits)
    assert rel(got, sv.simulate(q, gates)) <= 1e-12


@pytest.mark.parametrize("decomp", ["projector", "s_sdg"])
@pytest.mark.parametrize("segs", [[3, 3, 3], [4, 3, 2]])
def test_staircase_cx_cuts_three_segments(host_lib, decomp, segs):
    q = sum(segs)
    gates = w.staircase(q, 2)
    got = cut_state(gates, q, segs, decomp, "c64", 0)
    assert rel(got, sv.simulate(q, gates)) <= 1e-12


@pytest.mark.parametrize("kind", ["SWAP", "ISWAP", "CAN"])
@pytest.mark.parametrize("segs", [[4, 4], [3, 3, 3]])
def test_rank4_cuts(host_lib, kind, segs):
    q = sum(segs)
    gates = w.brickwork_cut(q, 6, 13, segs, 2, boundary_kind=kind)
    got = cut_state(gates, q, segs, "projector", "c64", 5)
    assert rel(got, sv.simulate(q, gates)) <= 1e-12


@pytest.mark.parametrize("rot", ["1", "0"])
@pytest.mark.parametrize("n_gates,seed", [(16, 1), (16, 4), (16, 6), (20, 4)])
def test_random_circuit_two_segments(host_lib, monkeypatch, rot, n_gates, seed):
    # random gate kinds and positions, rank-2 and rank-4 cuts anywhere across
    # the boundary (these seeds give 6 to 9 cut bits, so the term sum stays small)
    monkeypatch.setenv("CUTSIM_ROT", rot)
    q, segs = 8, [4, 4]
    gates = w.random_circuit(q, n_gates, seed,
                             kinds=["U3", "H", "T", "S", "CZ", "CX", "SWAP", "CAN"])
    got = cut_state(gates, q, segs, "projector", "c64", 5)
    assert rel(got, sv.simulate(q, gates)) <= 1e-12


@pytest.mark.parametrize("segs", [[3, 3, 3], [2, 3, 2, 2], [4, 5]])
def test_merge_stage_shapes(host_lib, segs):
    # stage s absorbs segment s: qa is the width of the segments before it,
    # K counts the combinations of the cut bits on boundary (s-1, s), Z those
    # on (s, s+1); the next stage sums over this stage's Z, the last has
    # Z = 1, every index stays inside the rows it indexes, and the two
    # boundaries' bits together are all the plan's bits
    q = sum(segs)
    gates = w.staircase(q, 2)
    tails = []
    for i in range(len(segs)):
        words, reals = api.plan_program_image(gates, q, segs, i, "projector", "c64", 0)
        tails.append(parse(words, reals, trailing=True)[1])
    n_bits = int(tails[0][0])
    c = [int(tl[1]) for tl in tails]
    stages, tab = parse_stages(tails[0], c[0])
    assert [st[0] for st in stages] == list(range(1, len(segs)))
    log_k = 0
    rows = 1 << c[0]
    for j, (seg, qa, qb, K, Z, ao, bo) in enumerate(stages):
        assert qa == sum(segs[:seg]) and qb == segs[seg]
        assert K == (stages[j - 1][4] if j else K) and K >= 2
        assert (Z == 1) == (j == len(stages) - 1)
        a = tab[ao:ao + Z * K]
        b = tab[bo:bo + Z * K]
        assert a.min() >= 0 and a.max() < rows
        assert b.min() >= 0 and b.max() < (1 << c[seg])
        assert len(set(zip(a.tolist(), b.tolist()))) == Z * K  # no term twice
        log_k += K.bit_length() - 1
        rows = Z
    assert log_k == n_bits


@pytest.mark.parametrize("which", ["aidx", "bidx"])
def test_chained_merge_rejects_wrong_tables(host_lib, which):
    # the staged merge check depends on every table entry: exchanging two
    # entries of one stage's row or segment indices moves the merged state
    segs, q = [3, 3, 3], 9
    gates = w.staircase(q, 2)
    vecs, staged = [], None
    for i, qi in enumerate(segs):
        words, reals = api.plan_program_image(gates, q, segs, i, "projector", "c64", 0)
        prog, tail = parse(words, reals, trailing=True)
        staged = parse_stages(tail, tail[1])
        vecs.append(run(prog).reshape(1 << tail[1], 1 << qi))
    stages, tab = staged
    good = chained_merge(vecs, stages, tab)
    assert rel(good, sv.simulate(q, gates)) <= 1e-12
    for seg, qa, qb, K, Z, ao, bo in stages:
        off = ao if which == "aidx" else bo
        bad = tab.copy()
        j = next(j for j in range(1, Z * K) if bad[off + j] != bad[off])
        bad[off], bad[off + j] = bad[off + j], bad[off]
        assert rel(chained_merge(vecs, stages, bad), good) > 1e-3, (seg, which)


@pytest.mark.parametrize("gates", [
    [],                                                    # no gates, no cuts
    [w.Gate("H", 0), w.Gate("H", 5), w.Gate("CZ", 2, 3)],  # one cut, boundary (1, 2) uncut
    [w.Gate("H", 7), w.Gate("CX", 7, 4), w.Gate("T", 4)],  # one CX cut on boundary (1, 2) only
])
def test_degenerate_cut_plans(host_lib, gates):
    # boundaries without cuts give stages with K = 1 or Z = 1; the staged and
    # the exhaustive merges both still give the uncut state
    q, segs = 8, [3, 3, 2]
    got = cut_state(gates, q, segs, "projector", "c64", 5)
    assert rel(got, sv.simulate(q, gates)) <= 1e-12


@pytest.mark.parametrize("segs,c", [([17, 17], 6), ([12, 11, 11], [3, 4])])
def test_largest_segment_programs_are_well_formed(host_lib, segs, c):
    # q = 34 plans: each segment's program over its qubits and variant bits
    # has the structure the kernels rely on, and its tables match the stages
    from test_program_host import validate

    q = sum(segs)
    gates = w.brickwork_cut(q, 8, 3, segs, c)
    for i, qi in enumerate(segs):
        words, reals = api.plan_program_image(gates, q, segs, i, "projector", "c64", 0)
        prog, tail = parse(words, reals, trailing=True)
        c_i = int(tail[1])
        assert prog.nq == qi + c_i and prog.n_state == qi
        validate(prog)
        stages, tab = parse_stages(tail, c_i)
        assert len(stages) == len(segs) - 1
        # each stage has Z K row indices and Z K segment indices
        assert sum(2 * K * Z for _, _, _, K, Z, _, _ in stages) == len(tab)
