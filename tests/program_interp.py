"""Host-side interpreter of the gate programs the pass kernels execute (test
infrastructure).

It reads the image `cc_program_image` returns and applies it to a complex128
state vector with numpy, following the device program's definition: passes in
order; in a pass, every amplitude's virtual index v puts its tile bits first
and the other bits above them; in each stage, every op first multiplies each
amplitude by its diagonal factors (adjacent-bit signs, sign terms, the phase
block's factor of the amplitude's register slot and its TERM_PFIX factors,
table terms)
and then applies its 2x2 matrix or rotation to the pairs differing in one
register bit (a packed rotation op: one rotation on each register bit of its
mask).  It shares nothing with the CUDA path beyond that image, so a
match with the oracle pins the host compiler (pass and stage planning,
deferred diagonals, the Euler split and phase blocks) without a GPU.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

OP_DENSE, OP_DIAG, OP_ROT, OP_ROTC, OP_ROTS = 0, 1, 2, 3, 4
TERM_SIGN, TERM_TABLE, TERM_PBLOCK, TERM_PFIX = 0, 1, 2, 3


@dataclass
class Pass:
    nq: int
    k: int
    init_zero: int
    stage_begin: int
    stage_end: int
    rbits: int
    n_rest: int
    tile_bit: List[int]
    rest_bit: List[int]


@dataclass
class Program:
    nq: int
    n_state: int
    passes: List[Pass]
    stages: List[tuple]  # (op_begin, op_end, rb[8])
    ops: List[tuple]     # (type, t, term_begin, n_sign, n_phase, n_table, mat, sign_adj)
    terms: List[tuple]   # (kind, p0, p1, tab)
    mats: np.ndarray     # complex, 4 per matrix
    tabs: np.ndarray     # complex, 4 per table


def parse(words: np.ndarray, reals: np.ndarray, trailing: bool = False):
    """The program of an image; with trailing=True also the words after it
    (a segment image's cut bits)."""
    w = [int(x) for x in words]
    assert w[0] == 1, "image version"
    nq, n_state, n_pass, n_stage, n_op, n_term, n_mat, n_tab = w[1:9]
    i = 9
    passes = []
    for _ in range(n_pass):
        f = w[i:i + 10]
        tile = w[i + 10:i + 26]
        rest = w[i + 26:i + 74]
        passes.append(Pass(nq=f[0], k=f[1], init_zero=f[3], stage_begin=f[4], stage_end=f[5],
                           rbits=f[6], n_rest=f[7], tile_bit=tile, rest_bit=rest))
        i += 74
    stages = []
    for _ in range(n_stage):
        stages.append((w[i], w[i + 1], w[i + 2:i + 10]))
        i += 10
    ops = []
    for _ in range(n_op):
        ops.append(tuple(w[i:i + 8]))
        i += 8
    terms = []
    for _ in range(n_term):
        terms.append(tuple(w[i:i + 4]))
        i += 4
    assert trailing or i == len(w)
    z = reals[0::2] + 1j * reals[1::2]
    prog = Program(nq, n_state, passes, stages, ops, terms, z[:n_mat], z[n_mat:n_mat + n_tab])
    return (prog, w[i:]) if trailing else prog


def _bit(v: np.ndarray, p: int) -> np.ndarray:
    return (v >> p) & 1


def run(prog: Program) -> np.ndarray:
    N = 1 << prog.nq
    x = np.arange(N, dtype=np.int64)
    psi = np.zeros(N, dtype=np.complex128)
    psi[(x & ((1 << prog.n_state) - 1)) == 0] = 1.0  # |0...0> of every variant
    for P in prog.passes:
        v = np.zeros(N, dtype=np.int64)
        for t in range(P.k):
            v |= _bit(x, P.tile_bit[t]) << t
        for r in range(P.n_rest):
            v |= _bit(x, P.rest_bit[r]) << (P.k + r)
        for si in range(P.stage_begin, P.stage_end):
            op_begin, op_end, rb = prog.stages[si]
            rb = rb[:P.rbits]
            for o in range(op_begin, op_end):
                typ, t, tb0, n_sign, n_phase, n_table, mat, sign_adj = prog.ops[o]
                f = np.ones(N, dtype=np.complex128)
                if sign_adj:
                    s = np.zeros(N, dtype=np.int64)
                    a = v & (v >> 1) & sign_adj
                    for p in range(64):
                        if (sign_adj >> p) & 1:
                            s ^= _bit(a, p)
                    f[s == 1] *= -1
                for k in range(tb0, tb0 + n_sign):
                    _, p0, p1, _ = prog.terms[k]
                    f[(_bit(v, p0) & _bit(v, p1)) == 1] *= -1
                if n_phase:
                    _, _, _, tab = prog.terms[tb0 + n_sign]
                    blk = prog.tabs[4 * tab:4 * tab + 32]
                    slot = np.zeros(N, dtype=np.int64)
                    for i2 in range(P.rbits):
                        slot |= _bit(v, rb[i2]) << i2
                    f *= blk[slot]
                    for k in range(tb0 + n_sign + 1, tb0 + n_sign + n_phase):
                        kind, p0, _, tab2 = prog.terms[k]
                        assert kind == TERM_PFIX
                        f[_bit(v, p0) == 1] *= prog.tabs[4 * tab2]
                for k in range(tb0 + n_sign + n_phase, tb0 + n_sign + n_phase + n_table):
                    kind, p0, p1, tab = prog.terms[k]
                    assert kind == TERM_TABLE
                    f *= prog.tabs[4 * tab + _bit(v, p0) + 2 * _bit(v, p1)]
                psi *= f
                if typ == OP_DIAG:
                    continue
                if typ == OP_ROTS:
                    # rotations on the register bits of t's low byte (distinct
                    # bits: any order), the OP_ROTC form where bit i of t >> 8
                    # is set, tangent of register bit i in real slot i
                    reals_of = np.stack([prog.mats[4 * mat:4 * mat + 4].real,
                                         prog.mats[4 * mat:4 * mat + 4].imag], axis=1).ravel()
                    for i in range(P.rbits):
                        if not (t >> i) & 1:
                            continue
                        vb = P.tile_bit[rb[i]]
                        i0 = x[_bit(x, vb) == 0]
                        i1 = i0 | (1 << vb)
                        a0, a1 = psi[i0].copy(), psi[i1].copy()
                        tt = reals_of[i]
                        if (t >> (8 + i)) & 1:
                            psi[i0] = tt * a0 - a1
                            psi[i1] = a0 + tt * a1
                        else:
                            psi[i0] = a0 - tt * a1
                            psi[i1] = a1 + tt * a0
                    continue
                vb = P.tile_bit[rb[t]]
                i0 = x[_bit(x, vb) == 0]
                i1 = i0 | (1 << vb)
                a0, a1 = psi[i0].copy(), psi[i1].copy()
                m = prog.mats[4 * mat:4 * mat + 4]
                if typ == OP_DENSE:
                    psi[i0] = m[0] * a0 + m[1] * a1
                    psi[i1] = m[2] * a0 + m[3] * a1
                elif typ == OP_ROT:
                    tt = m[0].real
                    psi[i0] = a0 - tt * a1
                    psi[i1] = a1 + tt * a0
                elif typ == OP_ROTC:
                    tt = m[0].real
                    psi[i0] = tt * a0 - a1
                    psi[i1] = a0 + tt * a1
                else:
                    raise AssertionError(f"unknown op type {typ}")
    return psi
