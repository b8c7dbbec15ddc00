"""Checks that pin the oracle to facts outside itself.

Each function returns an error magnitude (0 when the oracle is right) so that
the planted-mistake tests can call the same checks against a deliberately
broken oracle and see them fail.
"""

from __future__ import annotations

import cmath
import math

import numpy as np

from oracle import cutting as ct
from oracle import statevector as sv


# ------------------------------------------------------------ gate algebra
def rz(a):
    return np.array([[cmath.exp(-0.5j * a), 0], [0, cmath.exp(0.5j * a)]])


def ry(t):
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def pin_u3_euler(n=50, seed=1):
    """U3(t, p, l) = e^{i(p+l)/2} Rz(p) Ry(t) Rz(l): the ZYZ Euler form."""
    rng = np.random.default_rng(seed)
    err = 0.0
    for _ in range(n):
        t, p, l = rng.uniform(0, 2 * math.pi, 3)
        ref = cmath.exp(0.5j * (p + l)) * rz(p) @ ry(t) @ rz(l)
        err = max(err, float(np.max(np.abs(sv.u3(t, p, l) - ref))))
    return err


def full_unitary(q, op):
    """2^q x 2^q matrix of one op, built entry by entry from basis states."""
    m, qs = op
    dim = 1 << q
    u = np.zeros((dim, dim), dtype=np.complex128)
    for x in range(dim):
        if len(qs) == 1:
            j = qs[0]
            b = (x >> j) & 1
            for a in (0, 1):
                y = (x & ~(1 << j)) | (a << j)
                u[y, x] += m[a, b]
        else:
            j0, j1 = qs
            col = 2 * ((x >> j0) & 1) + ((x >> j1) & 1)
            for a0 in (0, 1):
                for a1 in (0, 1):
                    y = (x & ~(1 << j0) & ~(1 << j1)) | (a0 << j0) | (a1 << j1)
                    u[y, x] += m[2 * a0 + a1, col]
    return u


def pin_bruteforce(q, gates):
    """Gate-by-gate simulation vs the product of full 2^q x 2^q matrices."""
    dim = 1 << q
    utot = np.eye(dim, dtype=np.complex128)
    for g in gates:
        utot = full_unitary(q, sv.gate_op(g)) @ utot
    return float(np.max(np.abs(sv.simulate(q, gates) - utot[:, 0])))


def pin_basis_tracking(q, gates):
    """Circuits made of H on every qubit first, then only CX/CZ/X/Z/S/SDG/T/TDG:
    after the H layer every basis state |x> is carried to one basis state
    with a phase, so the exact output follows from integer tracking."""
    n_h = 0
    while n_h < len(gates) and gates[n_h].kind == "H":
        n_h += 1
    assert sorted(g.q0 for g in gates[:n_h]) == list(range(q))
    phase_of = {"Z": math.pi, "S": math.pi / 2, "SDG": -math.pi / 2,
                "T": math.pi / 4, "TDG": -math.pi / 4}
    out = np.zeros(1 << q, dtype=np.complex128)
    for x0 in range(1 << q):
        x, ph = x0, 0.0
        for g in gates[n_h:]:
            if g.kind == "CX":
                x ^= ((x >> g.q0) & 1) << g.q1
            elif g.kind == "CZ":
                if (x >> g.q0) & 1 and (x >> g.q1) & 1:
                    ph += math.pi
            elif g.kind == "X":
                x ^= 1 << g.q0
            elif g.kind in phase_of:
                if (x >> g.q0) & 1:
                    ph += phase_of[g.kind]
            else:
                raise ValueError(g.kind)
        out[x] += cmath.exp(1j * ph) / math.sqrt(1 << q)
    return out


# ------------------------------------------------------------ cutting
def pin_decomposition(kind, decomp):
    """sum_b coef_b A_b (x) B_b equals the gate's matrix (Eq. 1 / Eq. 2)."""
    coef, first, second = ct.local_terms(kind, decomp)
    total = sum(coef[b] * np.kron(first[b], second[b]) for b in (0, 1))
    return float(np.max(np.abs(total - sv.FIXED_2Q[kind])))


def schmidt_rank(u4, tol=1e-12):
    """Operator-Schmidt rank of a 4x4 two-qubit operator: the rank of
    R[(a_out a_in), (b_out b_in)] = U[(a_out b_out), (a_in b_in)]."""
    t = u4.reshape(2, 2, 2, 2)  # a_out, b_out, a_in, b_in
    r = t.transpose(0, 2, 1, 3).reshape(4, 4)
    s = np.linalg.svd(r, compute_uv=False)
    return int(np.sum(s > tol * s[0]))


def pin_cut_equals_uncut(q, gates, seg_sizes, decomp):
    """Relative max |Psi_cut - Psi_uncut| (Sec. III: exact up to rounding)."""
    ref = sv.simulate(q, gates)
    psi, _, _ = ct.cut_simulate(q, gates, seg_sizes, decomp)
    return float(np.max(np.abs(psi - ref)) / np.max(np.abs(ref)))


def pin_projector_variant_sum(q, gates, seg_sizes):
    """Projector split: |0><0| + |1><1| = I, so for a segment that carries only
    projector sides, the sum of all its variants equals the segment simulated
    with the cut operators left out (linearity, one bit at a time)."""
    pre = ct.preprocess(q, gates, seg_sizes, "projector")
    states = ct.simulate_subcircuits(pre)
    err = 0.0
    for i in range(len(seg_sizes)):
        sides = [0 if pre.cuts[j].segments[0] == i else 1 for j in pre.seg_cuts[i]]
        if not sides or any(s != 0 for s in sides):
            continue
        plain = [op for frag in pre.fragments[i] for op in frag]
        ref = sv.simulate_ops(seg_sizes[i], plain)
        total = sum(states[i])
        err = max(err, float(np.max(np.abs(total - ref))))
    return err
