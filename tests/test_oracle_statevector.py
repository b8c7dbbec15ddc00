"""Pins of the uncut FP64 simulator (gate definitions, bit order, brute force,
norm)."""

import cmath
import math

import numpy as np
import pytest

import workload as w
from oracle import statevector as sv
import pins


def close(a, b, tol=1e-14):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) <= tol


def test_u3_matches_zyz_euler_form():
    assert pins.pin_u3_euler() < 1e-14


def test_fixed_gates_are_u3_special_cases():
    # H = U3(pi/2, 0, pi), X = U3(pi, 0, pi), phase gates = U3(0, 0, lambda)
    assert close(sv.H, sv.u3(math.pi / 2, 0.0, math.pi), 1e-15)
    assert close(sv.X, sv.u3(math.pi, 0.0, math.pi), 1e-15)
    assert close(sv.S, sv.u3(0.0, 0.0, math.pi / 2), 1e-15)
    assert close(sv.T, sv.u3(0.0, 0.0, math.pi / 4), 1e-15)
    assert close(sv.Z, sv.u3(0.0, 0.0, math.pi), 1e-15)
    assert close(sv.SDG, sv.u3(0.0, 0.0, -math.pi / 2), 1e-15)
    assert close(sv.TDG, sv.u3(0.0, 0.0, -math.pi / 4), 1e-15)


def test_phase_gate_algebra():
    assert close(sv.T @ sv.T, sv.S)
    assert close(sv.S @ sv.S, sv.Z)
    assert close(sv.S @ sv.SDG, sv.I2)
    assert close(sv.T @ sv.TDG, sv.I2)
    assert close(sv.H @ sv.Z @ sv.H, sv.X)
    assert close(sv.H @ sv.H, sv.I2)


@pytest.mark.parametrize("seed", range(5))
def test_u3_unitary(seed):
    rng = np.random.default_rng(seed)
    u = sv.u3(*rng.uniform(0, 2 * math.pi, 3))
    assert close(u.conj().T @ u, sv.I2)


def test_bit_order_little_endian():
    q = 5
    for j in range(q):
        psi = sv.simulate(q, [w.Gate("X", j)])
        assert np.argmax(np.abs(psi)) == (1 << j)


def test_cx_control_and_target():
    # X on qubit 0 then CX(0 -> 3) gives |x0=1, x3=1> = index 9
    psi = sv.simulate(4, [w.Gate("X", 0), w.Gate("CX", 0, 3)])
    assert np.argmax(np.abs(psi)) == 9
    # control in |0>: CX does nothing
    psi = sv.simulate(4, [w.Gate("X", 3), w.Gate("CX", 0, 3)])
    assert np.argmax(np.abs(psi)) == 8
    # reversed roles
    psi = sv.simulate(4, [w.Gate("X", 3), w.Gate("CX", 3, 1)])
    assert np.argmax(np.abs(psi)) == 10


def test_cz_sign():
    psi = sv.simulate(3, [w.Gate("H", 0), w.Gate("H", 2), w.Gate("CZ", 2, 0)])
    ref = np.zeros(8, complex)
    for x in (0, 1, 4, 5):
        ref[x] = 0.5
    ref[5] = -0.5
    assert close(psi, ref, 1e-15)


@pytest.mark.parametrize("q,n_gates,seed", [(3, 40, 0), (5, 60, 1), (6, 80, 2), (7, 60, 3)])
def test_bruteforce_unitary_product(q, n_gates, seed):
    gates = w.random_circuit(q, n_gates, seed)
    assert pins.pin_bruteforce(q, gates) < 1e-13


@pytest.mark.parametrize("q,depth,seed", [(4, 3, 0), (6, 4, 5)])
def test_bruteforce_brickwork(q, depth, seed):
    assert pins.pin_bruteforce(q, w.brickwork(q, depth, seed)) < 1e-13


@pytest.mark.parametrize("q,depth,seed", [(10, 8, 0), (14, 6, 1)])
def test_norm_preserved(q, depth, seed):
    psi = sv.simulate(q, w.brickwork(q, depth, seed))
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-13


def test_product_state_closed_form():
    q = 8
    layer = w.brickwork(q, 1, 7)[:q]  # the U3 layer alone
    psi = sv.simulate(q, layer)
    cols = [sv.u3(g.theta, g.phi, g.lam)[:, 0] for g in layer]
    for x in range(1 << q):
        ref = 1.0 + 0j
        for j in range(q):
            ref *= cols[j][(x >> j) & 1]
        assert abs(psi[x] - ref) < 1e-15


def test_ghz_closed_form():
    q = 9
    psi = sv.simulate(q, w.ghz(q))
    ref = np.zeros(1 << q, complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert close(psi, ref, 1e-15)


def test_staircase_by_basis_tracking():
    q = 8
    gates = w.staircase(q, 2)
    assert close(sv.simulate(q, gates), pins.pin_basis_tracking(q, gates), 1e-14)


def test_graph_state_closed_form():
    q = 7
    edges = [(0, 1), (1, 2), (2, 6), (3, 5), (0, 6), (4, 5)]
    psi = sv.simulate(q, w.graph_state(q, edges))
    for x in range(1 << q):
        s = sum(((x >> a) & 1) * ((x >> b) & 1) for a, b in edges)
        assert abs(psi[x] - (-1) ** s / math.sqrt(1 << q)) < 1e-15


def test_bad_qubit_rejected():
    with pytest.raises(ValueError):
        sv.check_circuit(3, [w.Gate("H", 3)])
    with pytest.raises(ValueError):
        sv.check_circuit(3, [w.Gate("CZ", 1, 1)])
