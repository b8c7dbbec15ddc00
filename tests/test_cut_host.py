"""The host side of cutting pinned on the CPU: every segment's compiled
program (cc_plan_program_image, Algorithm 1), run by the numpy interpreter of
the device program (Algorithm 2), summed over all global cut combinations
with each segment's variant taken by its cut bits (Algorithm 3 written out),
equals the FP64 oracle's uncut state.  This covers the cut items and their
coefficients for both rank-2 splits, CX cuts, rank-4 (SWAP/ISWAP/CAN) cuts by
Pauli products, chains of three segments, small tiles and both rotation
engine settings.  No GPU is used."""

import numpy as np
import pytest

import workload as w
from oracle import statevector as sv
from paper_2603_01443_gb300 import api
from program_interp import parse, run


def cut_state(gates, q, segs, decomp, prec, tile_bits):
    vecs, ids, n_bits = [], [], None
    for i, qi in enumerate(segs):
        words, reals = api.plan_program_image(gates, q, segs, i, decomp, prec, tile_bits)
        prog, tail = parse(words, reals, trailing=True)
        n_bits, c_i = tail[0], tail[1]
        ids.append(tail[2:2 + c_i])
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
