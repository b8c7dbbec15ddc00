"""The two-qubit KAK factorisation (host helper): every gate list it returns
multiplies back, with the oracle's own gate matrices, to the input unitary
exactly (global phase included)."""

import math

import numpy as np
import pytest
from scipy.stats import unitary_group

from oracle import statevector as sv
from paper_2603_01443_gb300 import kak


def product(gates):
    u = np.eye(4, dtype=complex)
    for g in gates:
        m = sv.gate_matrix(g)
        if g.q1 >= 0:
            assert (g.q0, g.q1) == (0, 1)
            full = m
        elif g.q0 == 0:
            full = np.kron(m, np.eye(2))
        else:
            full = np.kron(np.eye(2), m)
        u = full @ u
    return u


SPECIAL = {
    "identity": np.eye(4), "cz": sv.CZ, "cx": sv.CX, "swap": sv.SWAP, "iswap": sv.ISWAP,
    "local": np.kron(sv.u3(0.3, 1.0, 2.0), sv.u3(2.2, -0.4, 0.9)),
    "can": sv.can(0.4, 1.3, -0.7),
    "sqrt_swap": sv.can(-math.pi / 4, -math.pi / 4, -math.pi / 4),
    "cx_reversed": np.kron(sv.H, sv.H) @ sv.CX @ np.kron(sv.H, sv.H),
}


@pytest.mark.parametrize("name", sorted(SPECIAL))
def test_special_gates(name):
    u = np.asarray(SPECIAL[name], dtype=complex)
    gates = kak.kak_gates(u, 0, 1)
    assert np.max(np.abs(product(gates) - u)) < 1e-10


@pytest.mark.parametrize("seed", range(20))
def test_random_unitaries(seed):
    u = unitary_group.rvs(4, random_state=seed)
    gates = kak.kak_gates(u, 0, 1)
    assert sum(1 for g in gates if g.kind == "CAN") == 1
    assert np.max(np.abs(product(gates) - u)) < 1e-10


def test_u3_params_roundtrip():
    rng = np.random.default_rng(1)
    for _ in range(50):
        u = unitary_group.rvs(2, random_state=rng)
        th, ph, la, g = kak.u3_params(u)
        assert np.allclose(np.exp(1j * g) * sv.u3(th, ph, la), u, atol=1e-12)


def test_rejects_non_unitary():
    with pytest.raises(ValueError):
        kak.kak(np.ones((4, 4)))
