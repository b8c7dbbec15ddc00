"""Edge cases of the CUDA path against the FP64 oracle: the largest segment
count, one-qubit segments carrying many cuts, tiny registers, K = 1 chains,
single-circuit and deep-chain batches."""

import numpy as np
import pytest
import torch

import workload as w
from oracle import statevector as sv
from paper_2603_01443_gb300 import api, capi
from gpu_util import TOL, assert_parity, gpu_cut, gpu_uncut, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_eight_segments_chain(cuda_lib, prec):
    segs = [2, 3, 2, 2, 3, 2, 2, 2]  # CC_MAX_SEGMENTS
    q = sum(segs)
    gates = w.brickwork_cut(q, 8, 4, segs, 1)
    psi, _, plan = gpu_cut(gates, q, segs, "s_sdg", prec)
    assert plan.info["n_seg"] == 8 and plan.info["c_total"] == 7
    assert_parity(psi.cpu().numpy(), sv.simulate(q, gates), prec, "n=8")


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_one_qubit_segments_with_many_cuts(cuda_lib, prec):
    # a 1-qubit middle segment adjacent to 7 cuts: a 2^8-amplitude program
    segs = [4, 1, 4]
    q = sum(segs)
    gates = w.brickwork_cut(q, 10, 6, segs, [3, 4])
    psi, _, plan = gpu_cut(gates, q, segs, "projector", prec)
    assert plan.info["seg_cuts"] == [3, 7, 4]
    assert_parity(psi.cpu().numpy(), sv.simulate(q, gates), prec, "1-qubit segment")


@pytest.mark.parametrize("q", [1, 2, 3, 5])
def test_tiny_uncut_and_cut(cuda_lib, q):
    gates = w.brickwork(q, 3, q)
    ref = sv.simulate(q, gates)
    psi_u, _ = gpu_uncut(gates, q, "c128")
    assert_parity(psi_u.cpu().numpy(), ref, "c128", f"uncut q={q}")
    if q >= 2:
        segs = w.equal_partition(q, 2)
        psi, _, _ = gpu_cut(gates, q, segs, "s_sdg", "c128")
        assert_parity(psi.cpu().numpy(), ref, "c128", f"cut q={q}")


def test_no_cut_chains(cuda_lib):
    # c_total = 0 with three segments: every stage has K = 1
    segs = [4, 5, 4]
    gates = w.brickwork_cut(13, 6, 8, segs, 0)
    psi, _, plan = gpu_cut(gates, 13, segs, "projector", "c64")
    assert plan.info["c_total"] == 0 and plan.info["n_sub"] == 3
    assert_parity(psi.cpu().numpy(), sv.simulate(13, gates), "c64", "K=1 chain")


def test_batch_of_one_and_deep_chains(cuda_lib):
    for circuits in (
        [(w.brickwork_cut(12, 6, 1, [6, 6], 2), 12, [6, 6])],
        [(w.brickwork_cut(14, 8, s, [4, 3, 4, 3], 1), 14, [4, 3, 4, 3]) for s in range(3)]
        + [(w.brickwork_cut(12, 8, 9, [3, 3, 3, 3], [1, 2, 1]), 12, [3, 3, 3, 3])],
    ):
        b = api.Batch(circuits, "s_sdg", "c128")
        seg, psi, ws = b.alloc_buffers()
        b.run(seg, psi, ws)
        capi.check(capi.lib().cc_sync(torch.cuda.current_stream().cuda_stream), "cc_sync")
        for i, (g, q, _) in enumerate(circuits):
            assert rel_err(b.psi_view(psi, i).cpu().numpy(), sv.simulate(q, g)) <= TOL["c128"]
