"""Gate-by-gate FP64 state-vector simulation (the uncut reference).

Conventions (the paper fixes none of them; these are the readings used
throughout):

* amplitude index x = sum_j x_j 2^j: qubit j is bit j (little-endian);
* every circuit starts in |0...0>;
* U3(theta, phi, lambda) = [[cos(theta/2), -e^{i lambda} sin(theta/2)],
                            [e^{i phi} sin(theta/2), e^{i(phi+lambda)} cos(theta/2)]]
  (the OpenQASM 2 gate);
* S = diag(1, i) as in Eq. 2, T = diag(1, e^{i pi/4}), S^dagger and T^dagger
  their inverses, H, X, Z the textbook matrices;
* a two-qubit matrix acting on (qubit a, qubit b) is written in the basis
  |x_a x_b>, i.e. row/column index 2*x_a + x_b, so kron(A, B) puts A on qubit a.
  CZ = diag(1, 1, 1, -1); CX(control a, target b) flips x_b when x_a = 1;
  SWAP exchanges x_a and x_b; ISWAP does so with a factor i on |01>, |10>;
  CAN(tx, ty, tz) = exp(-i (tx XX + ty YY + tz ZZ) / 2).

The simulator applies the matrices one at a time to a complex128 vector of
length 2^q by reshaping it so that the target qubit is its own tensor axis.
"""

from __future__ import annotations

import cmath
import math
from typing import Iterable, List, Sequence, Tuple

import numpy as np

# ---------------------------------------------------------------- matrices
I2 = np.eye(2, dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)
SDG = np.array([[1, 0], [0, -1j]], dtype=np.complex128)
T = np.array([[1, 0], [0, cmath.exp(1j * math.pi / 4)]], dtype=np.complex128)
TDG = np.array([[1, 0], [0, cmath.exp(-1j * math.pi / 4)]], dtype=np.complex128)
P0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)  # |0><0|
P1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)  # |1><1|
CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
CX = np.array(
    [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128
)

SWAP = np.array(
    [[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128
)
ISWAP = np.array(
    [[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]], dtype=np.complex128
)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)

FIXED_1Q = {"H": H, "X": X, "Z": Z, "S": S, "SDG": SDG, "T": T, "TDG": TDG}
FIXED_2Q = {"CZ": CZ, "CX": CX, "SWAP": SWAP, "ISWAP": ISWAP}
TWO_QUBIT = ("CZ", "CX", "SWAP", "ISWAP", "CAN")


def can(tx: float, ty: float, tz: float) -> np.ndarray:
    """Canonical two-qubit gate exp(-i (tx XX + ty YY + tz ZZ) / 2), by a
    library matrix exponential of the Hermitian generator."""
    from scipy.linalg import expm

    gen = tx * np.kron(X, X) + ty * np.kron(Y, Y) + tz * np.kron(Z, Z)
    return expm(-0.5j * gen)


def u3(theta: float, phi: float, lam: float) -> np.ndarray:
    c = math.cos(theta / 2.0)
    s = math.sin(theta / 2.0)
    return np.array(
        [
            [c, -cmath.exp(1j * lam) * s],
            [cmath.exp(1j * phi) * s, cmath.exp(1j * (phi + lam)) * c],
        ],
        dtype=np.complex128,
    )


def gate_matrix(gate) -> np.ndarray:
    """2x2 or 4x4 complex128 matrix of a ``workload.Gate``."""
    if gate.kind == "U3":
        return u3(gate.theta, gate.phi, gate.lam)
    if gate.kind in FIXED_1Q:
        return FIXED_1Q[gate.kind]
    if gate.kind in FIXED_2Q:
        return FIXED_2Q[gate.kind]
    if gate.kind == "CAN":
        return can(gate.theta, gate.phi, gate.lam)
    raise ValueError(f"unknown gate kind {gate.kind!r}")


# An "op" is (matrix, qubits): a 2x2 matrix with one qubit or a 4x4 matrix with
# two qubits (a, b) in the basis |x_a x_b>.
Op = Tuple[np.ndarray, Tuple[int, ...]]


def gate_op(gate) -> Op:
    m = gate_matrix(gate)
    if m.shape == (2, 2):
        return m, (gate.q0,)
    return m, (gate.q0, gate.q1)


def zero_state(q: int) -> np.ndarray:
    psi = np.zeros(1 << q, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply_1q(psi: np.ndarray, u: np.ndarray, j: int, q: int) -> np.ndarray:
    """new[x] = sum_b u[x_j, b] psi[x with bit j set to b]."""
    view = psi.reshape(1 << (q - 1 - j), 2, 1 << j)
    return np.einsum("ab,xbz->xaz", u, view).reshape(-1)


def apply_2q(psi: np.ndarray, u: np.ndarray, a: int, b: int, q: int) -> np.ndarray:
    """Apply a 4x4 matrix on qubits (a, b), basis index 2*x_a + x_b."""
    tens = psi.reshape((2,) * q)  # axis k holds bit q-1-k
    ax_a, ax_b = q - 1 - a, q - 1 - b
    u4 = u.reshape(2, 2, 2, 2)  # [out_a, out_b, in_a, in_b]
    out = np.tensordot(u4, tens, axes=([2, 3], [ax_a, ax_b]))
    out = np.moveaxis(out, [0, 1], [ax_a, ax_b])
    return np.ascontiguousarray(out).reshape(-1)


def apply_op(psi: np.ndarray, op: Op, q: int) -> np.ndarray:
    m, qs = op
    if len(qs) == 1:
        return apply_1q(psi, m, qs[0], q)
    return apply_2q(psi, m, qs[0], qs[1], q)


def simulate_ops(q: int, ops: Iterable[Op], psi: np.ndarray = None) -> np.ndarray:
    """Apply ops in order to |0...0> (or to ``psi``)."""
    state = zero_state(q) if psi is None else np.array(psi, dtype=np.complex128)
    for op in ops:
        state = apply_op(state, op, q)
    return state


def simulate(q: int, gates: Sequence) -> np.ndarray:
    """Uncut simulation C|0...0> of a gate list (the T_orig baseline)."""
    return simulate_ops(q, (gate_op(g) for g in gates))


def check_circuit(q: int, gates: Sequence) -> None:
    for g in gates:
        qs = (g.q0,) if g.kind not in TWO_QUBIT else (g.q0, g.q1)
        for x in qs:
            if not 0 <= x < q:
                raise ValueError(f"qubit {x} out of range for q={q}")
        if len(qs) == 2 and qs[0] == qs[1]:
            raise ValueError("two-qubit gate on a single qubit")


def ops_of(gates: Sequence) -> List[Op]:
    return [gate_op(g) for g in gates]
