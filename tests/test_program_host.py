"""The host program compiler pinned on the CPU: the gate program the pass
kernels would execute (cc_program_image), run by a plain numpy interpreter of
the device program's definition (tests/program_interp.py), equals the FP64
oracle's state vector.  Small tiles force many passes and stages and narrow
register widths; both rotation-engine settings and both precisions' layouts
are covered.  No GPU is used."""

import copy

import numpy as np
import pytest

import workload as w
from oracle import statevector as sv
from paper_2603_01443_gb300 import api, capi
from program_interp import (OP_DENSE, OP_ROT, OP_ROTC, OP_ROTS, TERM_PBLOCK, TERM_SIGN, parse,
                            run)

ALL_KINDS = ["U3", "H", "X", "Z", "S", "SDG", "T", "TDG", "CZ", "CX", "SWAP", "ISWAP", "CAN"]


def interp(gates, q, prec, tile_bits):
    words, reals = api.program_image(gates, q, prec, tile_bits)
    return parse(words, reals)


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("rot", ["1", "0"])
@pytest.mark.parametrize("prec,tile_bits", [("c64", 5), ("c64", 7), ("c64", 14), ("c128", 4),
                                            ("c128", 6), ("c128", 13)])
@pytest.mark.parametrize("q,n_gates,seed", [(6, 120, 1), (9, 200, 2), (10, 160, 3)])
def test_program_matches_oracle(host_lib, monkeypatch, rot, prec, tile_bits, q, n_gates,
                                seed):
    monkeypatch.setenv("CUTSIM_ROT", rot)
    gates = w.random_circuit(q, n_gates, seed, kinds=ALL_KINDS)
    prog = interp(gates, q, prec, tile_bits)
    if tile_bits < q:
        assert len(prog.passes) > 1
    got = run(prog)
    ref = sv.simulate(q, gates)
    assert rel(got, ref) <= 1e-12


@pytest.mark.parametrize("rot", ["1", "0"])
@pytest.mark.parametrize("prec,reg_bits,tile_bits", [("c64", 2, 7), ("c64", 3, 9), ("c64", 4, 13),
                                                     ("c128", 2, 6), ("c128", 3, 10)])
def test_fewer_register_bits(host_lib, monkeypatch, rot, prec, reg_bits, tile_bits):
    # CUTSIM_REG_BITS narrows every stage's register set (the kernels'
    # thread count per tile grows to match): more stages, each over fewer
    # bits, and phase blocks over fewer factors; the program still computes
    # the circuit
    monkeypatch.setenv("CUTSIM_ROT", rot)
    monkeypatch.setenv("CUTSIM_REG_BITS", str(reg_bits))
    q = 10
    gates = w.random_circuit(q, 180, 5, kinds=ALL_KINDS)
    prog = interp(gates, q, prec, tile_bits)
    assert all(P.rbits <= reg_bits for P in prog.passes)
    assert rel(run(prog), sv.simulate(q, gates)) <= 1e-12


@pytest.mark.parametrize("rot", ["1", "0"])
def test_brickwork_program_and_rotation_ops(host_lib, monkeypatch, rot):
    # a brickwork's fused one-qubit matrices become tangent-form rotations
    # (OP_ROT / OP_ROTC, and OP_ROTS for the rotations a stage flushes
    # together) with the engine on and complex 2x2 ops with it off
    monkeypatch.setenv("CUTSIM_ROT", rot)
    q = 11
    gates = w.brickwork(q, 12, 5)
    prog = interp(gates, q, "c64", 6)
    types = {op[0] for op in prog.ops}
    if rot == "1":
        assert types <= {1, 2, 3, 4} and types & {2, 3}
        wide = interp(gates, q, "c64", 11)  # five register bits per stage
        assert OP_ROTS in {op[0] for op in wide.ops}
        assert rel(run(wide), sv.simulate(q, gates)) <= 1e-12
        assert any(op[4] for op in prog.ops)  # phase blocks
    else:
        assert types <= {0, 1}
    assert rel(run(prog), sv.simulate(q, gates)) <= 1e-12


def test_deep_single_pass_program(host_lib):
    # one tile holds every qubit: one pass of thousands of rotations, whose
    # deferred scalar factors are folded in before the amplitudes grow large
    q = 8
    gates = w.brickwork(q, 400, 6)
    prog = interp(gates, q, "c64", 0)
    assert len(prog.passes) == 1
    got = run(prog)
    assert np.all(np.isfinite(got))
    assert rel(got, sv.simulate(q, gates)) <= 1e-11


def test_program_image_arguments(host_lib):
    gates = w.brickwork(6, 2, 0)
    arr = capi.GateArray(gates)
    L = capi.lib()
    from ctypes import byref, c_int64
    nw, nr = c_int64(0), c_int64(0)
    assert L.cc_program_image(arr.data, arr.n, 6, capi.PRECISION["c64"], 0, None, byref(nw),
                              None, byref(nr)) == 0
    assert nw.value > 9 and nr.value > 0
    small = np.zeros(4, dtype=np.int64)
    reals = np.zeros(nr.value)
    from ctypes import POINTER, c_double
    st = L.cc_program_image(arr.data, arr.n, 6, capi.PRECISION["c64"], 0,
                            small.ctypes.data_as(POINTER(c_int64)), byref(c_int64(4)),
                            reals.ctypes.data_as(POINTER(c_double)), byref(nr))
    assert capi.STATUS[st] == "CC_EBUFSIZE"
    with pytest.raises(capi.CutsimError):
        api.program_image(gates, 6, "c64", 4)  # not above the 4 contiguous low bits
    with pytest.raises(capi.CutsimError):
        api.program_image(gates, 6, "c128", 14)  # complex128 tiles hold at most 2^13


@pytest.mark.parametrize("prec,tile_bits", [("c64", 5), ("c128", 4), ("c128", 13)])
def test_phase_block_entries(host_lib, prec, tile_bits):
    # a phase block's 32 entries are K prod_i h_i^(bit i of j) over the
    # register bits times the signs of the CZ-type factors between two
    # register bits folded into it: (-1)^Q(j) with Q a quadratic form over
    # GF(2) (Q(j) = sum over folded pairs of j_a j_b).  So with
    # h_i = T[2^i] / T[0], T[j] / (T[0] prod h_i^(j_i)) is +-1 and its sign
    # bit is the sum of the pair terms Q(2^a + 2^b) over the set bits of j;
    # every entry is a unit complex number up to the common K.  The complex128
    # kernel skips slot 0 where the flag (bit 0) is clear, which needs T[0] = 1
    # exactly
    q = 10
    gates = w.random_circuit(q, 200, 9, kinds=ALL_KINDS)
    prog = interp(gates, q, prec, tile_bits)
    blocks = folded = 0
    for op in prog.ops:
        n_sign, n_phase = op[3], op[4]
        if not n_phase:
            continue
        kind, flags, _, tab = prog.terms[op[2] + n_sign]
        assert kind == 2  # TERM_PBLOCK
        blk = prog.tabs[4 * tab:4 * tab + 32]
        blocks += 1
        if not flags & 1:
            assert blk[0] == 1
        k = abs(blk[0])
        assert np.allclose(np.abs(blk), k, rtol=1e-12)
        h = [blk[1 << i] / blk[0] for i in range(5)]

        def sign(j):
            f = blk[0]
            for i in range(5):
                if (j >> i) & 1:
                    f = f * h[i]
            r = blk[j] / f
            assert abs(abs(r.real) - 1) <= 1e-12 and abs(r.imag) <= 1e-12
            return 1 if r.real < 0 else 0

        pair = {(a, b): sign((1 << a) | (1 << b)) for a in range(5) for b in range(a + 1, 5)}
        folded += any(pair.values())
        for j in range(32):
            bits = [i for i in range(5) if (j >> i) & 1]
            want = 0
            for x in range(len(bits)):
                for y in range(x + 1, len(bits)):
                    want ^= pair[(bits[x], bits[y])]
            assert sign(j) == want
    assert blocks > 0
    if max(P.rbits for P in prog.passes) >= 2:  # pairs of register bits exist
        assert folded > 0


def _mutations(prog):
    """One copy of the program per mutation, each changing one field the
    interpreter reads: a rotation's tangent, a dense matrix entry, a sign
    term's second bit, an adjacent-sign mask, a phase-block entry, two tile
    bits of a pass.  Each takes the last such field in the program, where the
    state is spread over every basis state (early in the first pass many
    amplitudes are still zero, and a changed factor on them changes
    nothing)."""
    out = {}

    def ops_of(pred):
        return [o for o, op in enumerate(prog.ops) if pred(op)]

    rot = ops_of(lambda op: op[0] in (OP_ROT, OP_ROTC) and abs(prog.mats[4 * op[6]].real) > 0.1)
    if rot:
        m = copy.deepcopy(prog)
        m.mats[4 * m.ops[rot[-1]][6]] *= -1
        out["rotation tangent"] = m
    dense = ops_of(lambda op: op[0] == OP_DENSE)
    if dense:
        m = copy.deepcopy(prog)
        m.mats[4 * m.ops[dense[-1]][6] + 1] *= 1j
        out["dense entry"] = m
    sign = [k for k, t in enumerate(prog.terms) if t[0] == TERM_SIGN and t[1] != t[2]]
    if sign:
        m = copy.deepcopy(prog)
        kind, p0, p1, tab = m.terms[sign[-1]]
        m.terms[sign[-1]] = (kind, p0, (p1 + 1) % m.nq if (p1 + 1) % m.nq != p0 else (p1 + 2) % m.nq, tab)
        out["sign term bit"] = m
    adj = ops_of(lambda op: op[7] != 0)
    if adj:
        m = copy.deepcopy(prog)
        op = list(m.ops[adj[-1]])
        op[7] &= op[7] - 1  # drop its lowest adjacent pair
        m.ops[adj[-1]] = tuple(op)
        out["adjacent sign mask"] = m
    blk = [t for t in prog.terms if t[0] == TERM_PBLOCK]
    if blk:
        m = copy.deepcopy(prog)
        m.tabs[4 * blk[-1][3]] *= np.exp(0.3j)  # the entry of the slot with no register bit set
        out["phase block entry"] = m
    packed = ops_of(lambda op: op[0] == OP_ROTS)
    if packed:
        # the lowest register bit of the last packed op: its tangent (real
        # slot i of the op's matrix) negated, and its form flipped
        o = packed[-1]
        i = ((prog.ops[o][1] & 0xFF) & -(prog.ops[o][1] & 0xFF)).bit_length() - 1
        m = copy.deepcopy(prog)
        k = 4 * m.ops[o][6] + i // 2
        z = m.mats[k]
        m.mats[k] = complex(-z.real, z.imag) if i % 2 == 0 else complex(z.real, -z.imag)
        out["packed rotation tangent"] = m
        m = copy.deepcopy(prog)
        op = list(m.ops[o])
        op[1] ^= 1 << (8 + i)
        m.ops[o] = tuple(op)
        out["packed rotation form"] = m
    multi = [i for i, P in enumerate(prog.passes) if P.k >= 6]
    if multi:
        m = copy.deepcopy(prog)
        P = m.passes[multi[-1]]
        P.tile_bit = list(P.tile_bit)
        P.tile_bit[P.k - 1], P.tile_bit[P.k - 2] = P.tile_bit[P.k - 2], P.tile_bit[P.k - 1]
        out["tile bit order"] = m
    return out


@pytest.mark.parametrize("rot", ["1", "0"])
def test_interpreter_rejects_mutated_programs(host_lib, monkeypatch, rot):
    # the host compiler's pins are only as strong as the interpreter: a
    # program with any one field changed must miss the oracle's state
    monkeypatch.setenv("CUTSIM_ROT", rot)
    q = 9
    gates = w.random_circuit(q, 160, 7, kinds=ALL_KINDS)
    ref = sv.simulate(q, gates)
    prog = interp(gates, q, "c64", 6)
    assert rel(run(prog), ref) <= 1e-12
    muts = _mutations(prog)
    expect = {"rotation tangent", "sign term bit", "phase block entry", "tile bit order"} \
        if rot == "1" else {"dense entry", "sign term bit", "tile bit order"}
    assert expect <= set(muts), sorted(muts)
    for name, m in muts.items():
        assert rel(run(m), ref) > 1e-3, name


def test_interpreter_rejects_mutated_packed_rotations(host_lib):
    # stages of five register bits flush several rotations as one packed op
    # (OP_ROTS): a changed tangent or rotation form in it must miss the oracle
    q = 10
    gates = w.brickwork(q, 8, 3)
    ref = sv.simulate(q, gates)
    prog = interp(gates, q, "c64", 10)
    assert rel(run(prog), ref) <= 1e-12
    muts = _mutations(prog)
    assert {"packed rotation tangent", "packed rotation form"} <= set(muts), sorted(muts)
    for name in ("packed rotation tangent", "packed rotation form"):
        assert rel(run(muts[name]), ref) > 1e-3, name


@pytest.mark.parametrize("prec,tile_bits", [("c64", 5), ("c128", 4), ("c64", 14)])
@pytest.mark.parametrize("gates", [[], [w.Gate("Z", 3)], [w.Gate("CZ", 0, 7)], [w.Gate("H", 7)]])
def test_degenerate_circuits(host_lib, prec, tile_bits, gates):
    # no gates, one diagonal gate (which leaves |0...0> unchanged), one gate on
    # the highest qubit: the program still starts from |0...0> and ends
    # with every pending factor applied
    q = 8
    prog = interp(gates, q, prec, tile_bits)
    assert len(prog.passes) >= 1
    assert rel(run(prog), sv.simulate(q, gates)) <= 1e-15


def validate(prog):
    """Structural checks of a program, the ones the kernels rely on: each pass
    orders all nq bits (tile bits, then the rest) with its low tile bits
    contiguous; stages partition the ops in order; register bits name
    distinct tile positions; every op's terms lie in its own range with the
    kinds of their section (signs, then one phase block and its per-bit
    phases, then tables); matrices and tables exist; bits lie below nq."""
    from program_interp import OP_DIAG, TERM_PFIX, TERM_TABLE

    n_mat, n_tab = len(prog.mats) // 4, len(prog.tabs) // 4
    next_stage, next_op = 0, 0
    for pi, P in enumerate(prog.passes):
        assert P.init_zero == (1 if pi == 0 else 0)
        order = list(P.tile_bit[:P.k]) + list(P.rest_bit[:P.n_rest])
        assert sorted(order) == list(range(prog.nq)) and P.k + P.n_rest == prog.nq
        assert P.stage_begin == next_stage and P.stage_end > P.stage_begin
        next_stage = P.stage_end
        for si in range(P.stage_begin, P.stage_end):
            op_begin, op_end, rb = prog.stages[si]
            assert op_begin == next_op and op_end >= op_begin
            next_op = op_end
            regs = list(rb[:P.rbits])
            assert len(set(regs)) == P.rbits and all(0 <= r < P.k for r in regs)
            for o in range(op_begin, op_end):
                typ, t, tb0, n_sign, n_phase, n_table, mat, sign_adj = prog.ops[o]
                assert 0 <= tb0 and tb0 + n_sign + n_phase + n_table <= len(prog.terms)
                assert sign_adj >> max(prog.nq - 1, 0) == 0
                if typ == OP_DIAG:
                    assert mat == -1
                elif typ == OP_ROTS:  # register-bit mask, OP_ROTC mask within it
                    bits, cot = t & 0xFF, t >> 8
                    assert 0 < bits < (1 << P.rbits) and cot & ~bits == 0
                    assert bin(bits).count("1") >= 2 and 0 <= mat < n_mat
                else:
                    assert 0 <= t < P.rbits and 0 <= mat < n_mat
                sec = ([TERM_SIGN] * n_sign + ([TERM_PBLOCK] if n_phase else [])
                       + [TERM_PFIX] * max(n_phase - 1, 0) + [TERM_TABLE] * n_table)
                for k, kind in zip(range(tb0, tb0 + len(sec)), sec):
                    tk, p0, p1, tab = prog.terms[k]
                    assert tk == kind
                    assert 0 <= p0 < prog.nq and 0 <= p1 < prog.nq
                    if kind == TERM_PBLOCK:
                        assert 0 <= tab and tab + 8 <= n_tab
                    elif kind != TERM_SIGN:
                        assert 0 <= tab < n_tab
    assert next_stage == len(prog.stages) and next_op == len(prog.ops)


@pytest.mark.parametrize("rot", ["1", "0"])
def test_programs_are_well_formed(host_lib, monkeypatch, rot):
    monkeypatch.setenv("CUTSIM_ROT", rot)
    for prec, tb in [("c64", 5), ("c64", 13), ("c128", 4), ("c128", 12)]:
        for q, n_gates, seed in [(6, 120, 1), (10, 300, 2)]:
            validate(interp(w.random_circuit(q, n_gates, seed, kinds=ALL_KINDS), q, prec, tb))


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_largest_programs_are_well_formed(host_lib, prec):
    # q = 34, the library's largest vector: too large to interpret here, so
    # the program is checked for the structure the kernels rely on
    q = 34
    gates = w.brickwork(q, 3, 5) + [w.Gate("SWAP", 0, 33), w.Gate("CX", 33, 1)]
    prog = interp(gates, q, prec, 0)
    validate(prog)
    assert len(prog.passes) >= 3
