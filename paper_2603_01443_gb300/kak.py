"""Two-qubit gates of any kind as one-qubit gates around a canonical gate.

Every two-qubit unitary U (Schmidt rank 4 in general, Eq. 1) factors as

    U = e^{i g} (A1 (x) B1) CAN(tx, ty, tz) (A0 (x) B0)

with one-qubit unitaries A, B and CAN(tx, ty, tz) = exp(-i (tx XX + ty YY +
tz ZZ) / 2) (the Cartan / KAK decomposition; Khaneja and Glaser 2001, Kraus
and Cirac 2001).  ``kak_gates`` returns that factorisation as gates the
engine takes (U3, CAN, and a phase on the first qubit), so a general gate can
be cut -- CAN is a rank-4 cut -- and simulated like any other.

Host arithmetic only (numpy); the engine never sees the 4x4 matrix.
Convention: a 4x4 matrix on (q0, q1) acts on the basis |x_q0 x_q1>, index
2 x_q0 + x_q1.
"""

from __future__ import annotations

import cmath
import math
from typing import List, NamedTuple

import numpy as np

# Magic (Bell) basis: in it, SU(2) (x) SU(2) is the real orthogonal group SO(4)
# and CAN is diagonal.
_M = np.array([[1, 0, 0, 1j], [0, 1j, 1, 0], [0, 1j, -1, 0], [1, 0, 0, -1j]],
              dtype=np.complex128) / math.sqrt(2.0)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


class Gate(NamedTuple):
    kind: str
    q0: int
    q1: int = -1
    theta: float = 0.0
    phi: float = 0.0
    lam: float = 0.0


def can_matrix(tx: float, ty: float, tz: float) -> np.ndarray:
    """exp(-i (tx XX + ty YY + tz ZZ) / 2), as a product of commuting factors."""
    out = np.eye(4, dtype=np.complex128)
    for t, p in ((tx, _X), (ty, _Y), (tz, _Z)):
        pp = np.kron(p, p)
        out = out @ (math.cos(t / 2) * np.eye(4) - 1j * math.sin(t / 2) * pp)
    return out


def _u3(theta: float, phi: float, lam: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -cmath.exp(1j * lam) * s],
                     [cmath.exp(1j * phi) * s, cmath.exp(1j * (phi + lam)) * c]])


def u3_params(u: np.ndarray):
    """(theta, phi, lam, g) with u = e^{i g} U3(theta, phi, lam) for a 2x2
    unitary u, U3 as in the engine: [[c, -e^{i lam} s], [e^{i phi} s,
    e^{i(phi+lam)} c]].  theta from atan2 of the entry magnitudes; phi + lam
    from u11 conj(u00) and phi - lam from u10 conj(-u01) (each weighted by
    the magnitude it multiplies, so a tiny pair only decides tiny entries);
    halving leaves phi, lam ambiguous by pi together, which flips the sign of
    both off-diagonal entries: the candidate that matches u is kept."""
    u = np.asarray(u, dtype=np.complex128)
    c_abs = 0.5 * (abs(u[0, 0]) + abs(u[1, 1]))
    s_abs = 0.5 * (abs(u[0, 1]) + abs(u[1, 0]))
    theta = 2.0 * math.atan2(s_abs, c_abs)
    sigma = cmath.phase(u[1, 1] * np.conj(u[0, 0])) if c_abs > 0.0 else 0.0
    delta = cmath.phase(u[1, 0] * np.conj(-u[0, 1])) if s_abs > 0.0 else 0.0
    best = None
    for shift in (0.0, math.pi):
        phi = 0.5 * (sigma + delta) + shift
        lam = 0.5 * (sigma - delta) + shift
        base = _u3(theta, phi, lam)
        # global phase from the larger entry
        i, j = (0, 0) if c_abs >= s_abs else (0, 1)
        g = cmath.phase(u[i, j] / base[i, j])
        err = float(np.max(np.abs(cmath.exp(1j * g) * base - u)))
        if best is None or err < best[0]:
            best = (err, theta, phi, lam, g)
    return best[1], best[2], best[3], best[4]


def _split_local(k: np.ndarray):
    """A (x) B from a 4x4 matrix known to be a tensor product (rank-1 in the
    realigned form): A, B with kron(A, B) = k."""
    r = k.reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)
    w, s, vh = np.linalg.svd(r)
    a = (w[:, 0] * math.sqrt(s[0])).reshape(2, 2)
    b = (vh[0, :] * math.sqrt(s[0])).reshape(2, 2)
    # give both factors determinant magnitude 1 (they are unitary up to scale)
    scale = math.sqrt(abs(np.linalg.det(a)))
    return a / scale, b * scale


def kak(u: np.ndarray, seed: int = 0):
    """(A0, B0, (tx, ty, tz), A1, B1, g) with
    u = e^{i g} kron(A1, B1) CAN(tx, ty, tz) kron(A0, B0)."""
    u = np.asarray(u, dtype=np.complex128)
    if u.shape != (4, 4) or not np.allclose(u.conj().T @ u, np.eye(4), atol=1e-10):
        raise ValueError("need a 4x4 unitary")
    det = np.linalg.det(u)
    g0 = cmath.phase(det) / 4.0
    up = u * cmath.exp(-1j * g0)  # det 1
    ub = _M.conj().T @ up @ _M
    m2 = ub.T @ ub  # symmetric unitary: m2 = P diag(e^{2 i d}) P^T, P in SO(4)
    rng = np.random.default_rng(seed)
    for _ in range(16):  # a generic real combination separates the eigenspaces
        a, b = rng.standard_normal(2)
        _, p = np.linalg.eigh(a * m2.real + b * m2.imag)
        d = np.diag(p.T @ m2 @ p)
        if np.allclose(p.T @ m2 @ p, np.diag(d), atol=1e-9):
            break
    else:
        raise RuntimeError("simultaneous diagonalisation failed")
    if np.linalg.det(p) < 0:
        p[:, 0] = -p[:, 0]
    half = np.angle(d) / 2.0
    k1 = ub @ p @ np.diag(np.exp(-1j * half))  # real orthogonal up to sign choices
    if np.linalg.det(k1).real < 0:  # move a pi into one eigenphase
        half[0] += math.pi
        k1 = ub @ p @ np.diag(np.exp(-1j * half))
    k2 = p.T
    # back to the computational basis
    a1b1 = _M @ k1 @ _M.conj().T
    a0b0 = _M @ k2 @ _M.conj().T
    # middle factor: M diag(e^{i half}) M^dag = e^{i g1} CAN(tx, ty, tz)
    mid = _M @ np.diag(np.exp(1j * half)) @ _M.conj().T
    # eigenphases of XX, YY, ZZ on the magic basis columns
    signs = np.array([[np.vdot(_M[:, j], np.kron(p_, p_) @ _M[:, j]).real for p_ in (_X, _Y, _Z)]
                      for j in range(4)])
    # half_j = g1 - (tx sx_j + ty sy_j + tz sz_j) / 2: least squares (exact)
    a_mat = np.column_stack([np.ones(4), -0.5 * signs])
    sol, *_ = np.linalg.lstsq(a_mat, half, rcond=None)
    g1, tx, ty, tz = sol
    if not np.allclose(mid, cmath.exp(1j * g1) * can_matrix(tx, ty, tz), atol=1e-9):
        raise RuntimeError("canonical parameters do not reproduce the middle factor")
    A1, B1 = _split_local(a1b1)
    A0, B0 = _split_local(a0b0)
    lhs = np.kron(A1, B1) @ can_matrix(tx, ty, tz) @ np.kron(A0, B0)
    # the remaining global phase (each split is exact up to a scalar)
    k = np.argmax(np.abs(lhs))
    g = cmath.phase(u.reshape(-1)[k] / lhs.reshape(-1)[k])
    return A0, B0, (float(tx), float(ty), float(tz)), A1, B1, g


def kak_gates(u: np.ndarray, q0: int, q1: int) -> List[Gate]:
    """Gates whose product is exactly u on (q0, q1), global phase included:
    U3 on each qubit, CAN, U3 on each qubit, and the phase as two U3 phase
    gates around X on q0 (P X P X = e^{i g} I for P = diag(1, e^{i g}))."""
    A0, B0, (tx, ty, tz), A1, B1, g = kak(u)
    out: List[Gate] = []
    phase = g
    for m, q in ((A0, q0), (B0, q1)):
        th, ph, la, gg = u3_params(m)
        phase += gg
        out.append(Gate("U3", q, -1, th, ph, la))
    out.append(Gate("CAN", q0, q1, tx, ty, tz))
    for m, q in ((A1, q0), (B1, q1)):
        th, ph, la, gg = u3_params(m)
        phase += gg
        out.append(Gate("U3", q, -1, th, ph, la))
    phase = math.remainder(phase, 2 * math.pi)
    if abs(phase) > 1e-15:
        out += [Gate("U3", q0, -1, 0.0, 0.0, phase), Gate("X", q0),
                Gate("U3", q0, -1, 0.0, 0.0, phase), Gate("X", q0)]
    return out
