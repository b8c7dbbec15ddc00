"""Two-qubit gates of any kind as one-qubit gates around a canonical gate.

A general two-qubit unitary is a Schmidt-rank-4 gate (Eq. 1).  The library's
cc_kak_gates factors it as U = e^{i g} (A1 (x) B1) CAN(tx, ty, tz) (A0 (x) B0)
(the Cartan / KAK decomposition) and returns that product as gates the engine
takes: U3 on each qubit, CAN, U3 on each qubit, and the global phase as two
U3 phase gates around X on the first qubit.  This module only marshals the
4x4 matrix in and the gates out; the arithmetic is the library's host code.
Convention: a 4x4 matrix on (q0, q1) acts on |x_q0 x_q1>, index 2 x_q0 + x_q1.
"""

from __future__ import annotations

from ctypes import POINTER, byref, c_double, c_int32
from typing import List, NamedTuple

import numpy as np

from . import capi

_KIND_NAME = {v: k for k, v in capi.GATE_KIND.items()}
MAX_GATES = 9  # CC_KAK_MAX_GATES in include/cutsim.h


class Gate(NamedTuple):
    kind: str
    q0: int
    q1: int = -1
    theta: float = 0.0
    phi: float = 0.0
    lam: float = 0.0


def kak_gates(u, q0: int, q1: int) -> List[Gate]:
    """Gates whose product is exactly u on (q0, q1), global phase included."""
    m = np.ascontiguousarray(np.asarray(u, dtype=np.complex128))
    if m.shape != (4, 4):
        raise ValueError("need a 4x4 matrix")
    flat = np.ascontiguousarray(m.view(np.float64).reshape(-1))  # row-major, re/im interleaved
    out = (capi.CGate * MAX_GATES)()
    n = c_int32(0)
    capi.check(capi.lib().cc_kak_gates(flat.ctypes.data_as(POINTER(c_double)), q0, q1, out,
                                       byref(n)), "cc_kak_gates")
    gates = []
    for g in out[:n.value]:
        name = _KIND_NAME[g.kind]
        gates.append(Gate(name, g.q0, g.q1 if name in capi.TWO_QUBIT else -1, g.theta, g.phi,
                          g.lam))
    return gates
