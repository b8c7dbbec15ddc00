"""The two-qubit KAK factorisation (cc_kak_gates, host code behind the C
ABI): every gate list it returns multiplies back, with the oracle's own gate
matrices, to the input unitary exactly (global phase included)."""

import math

import numpy as np
import pytest
from scipy.stats import unitary_group

from oracle import statevector as sv
from paper_2603_01443_gb300 import capi, kak


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
    "phased_local": np.exp(0.7j) * np.kron(sv.H, sv.u3(1.1, 0.2, -2.4)),
}


@pytest.mark.parametrize("name", sorted(SPECIAL))
def test_special_gates(host_lib, name):
    u = np.asarray(SPECIAL[name], dtype=complex)
    gates = kak.kak_gates(u, 0, 1)
    assert len(gates) <= kak.MAX_GATES
    assert np.max(np.abs(product(gates) - u)) < 1e-10


@pytest.mark.parametrize("seed", range(40))
def test_random_unitaries(host_lib, seed):
    u = unitary_group.rvs(4, random_state=seed)
    gates = kak.kak_gates(u, 0, 1)
    assert sum(1 for g in gates if g.kind == "CAN") == 1
    assert [g.kind for g in gates[:5]] == ["U3", "U3", "CAN", "U3", "U3"]
    assert np.max(np.abs(product(gates) - u)) < 1e-10


def test_canonical_parameters_of_a_can_gate(host_lib):
    # CAN itself: the factorisation's middle gate reproduces it with local
    # factors that are identities up to phases and Pauli frame changes
    u = sv.can(0.4, 1.3, -0.7)
    gates = kak.kak_gates(u, 0, 1)
    can = [g for g in gates if g.kind == "CAN"][0]
    # CAN parameters are fixed up to sign and the Weyl-chamber symmetries:
    # the sorted magnitudes of the three angles modulo pi agree
    got = sorted(abs(math.remainder(x, math.pi)) for x in (can.theta, can.phi, can.lam))
    want = sorted(abs(math.remainder(x, math.pi)) for x in (0.4, 1.3, -0.7))
    assert np.allclose(got, want, atol=1e-9)


def test_rejects_bad_input(host_lib):
    with pytest.raises(capi.CutsimError):
        kak.kak_gates(np.ones((4, 4)), 0, 1)  # not unitary
    with pytest.raises(capi.CutsimError):
        kak.kak_gates(np.eye(4), 3, 3)  # one qubit twice
    with pytest.raises(capi.CutsimError):
        kak.kak_gates(np.full((4, 4), np.nan), 0, 1)
    with pytest.raises(ValueError):
        kak.kak_gates(np.eye(2), 0, 1)
