"""Schmidt-rank-4 gates (SWAP, ISWAP, CAN; Eq. 1 with k = 4) on the GPU:
cut at partition boundaries (two variant bits per cut, Pauli-product terms)
and simulated inside segments and in the uncut program (basis changes
around diagonal ZZ phases), against the FP64 oracle."""

import numpy as np
import pytest
import torch

import workload as w
from oracle import statevector as sv
from paper_2603_01443_gb300 import api, capi
from gpu_util import FID_TOL, TOL, assert_parity, fidelity, gpu_cut, gpu_uncut, rel_err

pytestmark = pytest.mark.gpu

PRECS = ["c64", "c128"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", ["SWAP", "ISWAP", "CAN"])
@pytest.mark.parametrize("segs,c", [([6, 6], 2), ([5, 7], 3), ([4, 4, 4], [1, 2])])
def test_rank4_boundary_cuts(cuda_lib, prec, kind, segs, c):
    q = sum(segs)
    gates = w.brickwork_cut(q, 8, 5, segs, c, boundary_kind=kind)
    psi, _, plan = gpu_cut(gates, q, segs, "projector", prec)
    n_cuts = sum([c] * (len(segs) - 1) if isinstance(c, int) else c)
    assert plan.info["c_total"] == n_cuts and plan.info["cut_bits"] == 2 * n_cuts
    assert all(plan.cut(j)["kind"] == capi.GATE_KIND[kind] for j in range(n_cuts))
    assert_parity(psi.cpu().numpy(), sv.simulate(q, gates), prec, kind)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_rank4_gates_uncut_and_inside_segments(cuda_lib, prec, seed):
    kinds = ("U3", "H", "T", "CZ", "CX", "SWAP", "ISWAP", "CAN")
    q = 10
    # complex64 rounding grows with the number of fused operations (a rank-4
    # gate expands into up to 3 ZZ phases and 4 basis changes per qubit): 40
    # random gates keep the per-amplitude operation count near that of the
    # depth-16 brickwork the 2e-6 tolerance is stated for
    gates = w.random_circuit(q, 40 if prec == "c64" else 60, 300 + seed, kinds)
    ref = sv.simulate(q, gates)
    psi_u, _ = gpu_uncut(gates, q, prec)
    assert_parity(psi_u.cpu().numpy(), ref, prec, "uncut rank-4")
    # one segment holds every gate: the rank-4 gates run inside it
    psi_1, _, _ = gpu_cut(gates, q, [q], "projector", prec)
    assert_parity(psi_1.cpu().numpy(), ref, prec, "one segment")


@pytest.mark.parametrize("prec", PRECS)
def test_rank4_cuts_at_random_positions(cuda_lib, prec):
    kinds = ("U3", "H", "T", "CZ", "CX", "SWAP", "ISWAP", "CAN")
    for seed in (7, 8, 9):
        q = 9
        gates = w.random_circuit(q, 24, seed, kinds)
        psi, _, plan = gpu_cut(gates, q, [4, 5], "s_sdg", prec)
        assert_parity(psi.cpu().numpy(), sv.simulate(q, gates), prec, f"seed {seed}")


def test_pure_zz_canonical_cut_takes_one_bit(cuda_lib):
    q, segs = 10, [5, 5]
    gates = w.brickwork(q, 4, 1) + [w.Gate("CAN", 4, 5, 0.0, 0.0, 0.9),
                                    w.Gate("CAN", 3, 6, 1.3, 0.0, 0.0),
                                    w.Gate("SWAP", 2, 7)] + w.brickwork(q, 2, 2)
    psi, _, plan = gpu_cut(gates, q, segs, "projector", "c128")
    # the brickwork's own boundary CZs, then a Z-only, an X-only and a full rank-4 cut
    n_cz = sum(1 for g in gates if g.kind == "CZ" and g.q0 < 5 <= g.q1)
    assert plan.info["cut_bits"] == n_cz + 1 + 1 + 2
    assert_parity(psi.cpu().numpy(), sv.simulate(q, gates), "c128", "mixed widths")


def test_rank4_batch_and_scale(cuda_lib):
    # a batch of rank-4-cut circuits, and one q = 22 circuit against the uncut GPU state
    items = [w.BatchItem(w.brickwork_cut(q, 8, 40 + q, s, c, boundary_kind=k), q, 8, s, [c], 0)
             for q, s, c, k in ((12, [6, 6], 2, "SWAP"), (13, [6, 7], 1, "CAN"),
                                (11, [5, 6], 2, "ISWAP"))]
    b = api.Batch([(it.gates, it.q, it.seg_sizes) for it in items])
    seg, psi, ws = b.alloc_buffers()
    b.run(seg, psi, ws)
    capi.check(capi.lib().cc_sync(torch.cuda.current_stream().cuda_stream), "cc_sync")
    for i, it in enumerate(items):
        assert rel_err(b.psi_view(psi, i).cpu().numpy(), sv.simulate(it.q, it.gates)) <= TOL["c64"]
    q, segs = 22, [11, 11]
    gates = w.brickwork_cut(q, 12, 3, segs, 3, boundary_kind="CAN")
    psi, _, plan = gpu_cut(gates, q, segs, "projector", "c64", "auto")
    psi_u, _ = gpu_uncut(gates, q, "c64")
    st = api.compare(psi, psi_u, "c64")
    assert st["max_abs_diff"] <= 4e-6 * st["max_abs_b"], st
    assert 1 - st["fidelity"] <= FID_TOL


@pytest.mark.parametrize("prec", PRECS)
def test_general_two_qubit_gates_via_kak(cuda_lib, prec):
    # random 4x4 unitaries, written as U3 / CAN / U3 by the KAK helper, cut
    # where they cross the boundary; the oracle applies the 4x4 matrices themselves
    from scipy.stats import unitary_group

    from paper_2603_01443_gb300 import kak

    q, segs = 10, [5, 5]
    rng = np.random.default_rng(11)
    ops, gates = [], []
    for layer in range(6):
        for j in range(q):
            g = w.Gate("U3", j, -1, *rng.uniform(0, 2 * np.pi, 3))
            gates.append(g)
            ops.append(sv.gate_op(g))
        for a in range(layer % 2, q - 1, 2):
            u = unitary_group.rvs(4, random_state=int(rng.integers(1 << 30)))
            gates += [w.Gate(*x) for x in kak.kak_gates(u, a, a + 1)]
            ops.append((u, (a, a + 1)))
    ref = sv.simulate_ops(q, ops)
    psi, _, plan = gpu_cut(gates, q, segs, "projector", prec)
    assert plan.info["c_total"] == 3  # the layers whose pairs straddle qubits 4-5
    assert_parity(psi.cpu().numpy(), ref, prec, "kak")
