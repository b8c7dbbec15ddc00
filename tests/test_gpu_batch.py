"""Batched cut simulation of many independent circuits (one persistent
gate-pass launch, one merge launch per chain level, optional CUDA graph)
against the FP64 oracle and against the one-circuit path."""

import numpy as np
import pytest
import torch

import workload as w
from oracle import statevector as sv
from paper_2603_01443_gb300 import api, capi
from gpu_util import FID_TOL, TOL, fidelity, gpu_cut, rel_err

pytestmark = pytest.mark.gpu


def make_batch(items, decomp="projector", prec="c64", tile_bits=0, rows=0):
    return api.Batch([(it.gates, it.q, it.seg_sizes) for it in items], decomp, prec, tile_bits, rows)


def sync():
    capi.check(capi.lib().cc_sync(torch.cuda.current_stream().cuda_stream), "cc_sync")


@pytest.mark.parametrize("prec,decomp,tile_bits,rows", [
    ("c64", "projector", 0, 32), ("c64", "s_sdg", 10, 16), ("c64", "projector", 6, 32),
    ("c128", "projector", 0, 0), ("c128", "s_sdg", 9, 0)])
def test_batch_vs_oracle(cuda_lib, prec, decomp, tile_bits, rows):
    # small tiles force several passes per segment (dependency waits) and
    # tiny segments give jobs narrower than the block
    items = w.uneven_batch(10, seed=3 + tile_bits, q_range=(12, 16), depths=(4, 8),
                           c_range=(0, 4))
    b = make_batch(items, decomp, prec, tile_bits, rows)
    seg, psi, ws = b.alloc_buffers()
    stamps = b.alloc_stamps()
    b.run(seg, psi, ws, stamps)
    sync()
    for i, it in enumerate(items):
        got = b.psi_view(psi, i).cpu().numpy()
        ref = sv.simulate(it.q, it.gates)
        assert rel_err(got, ref) <= TOL[prec], (i, it.q, it.seg_sizes, rel_err(got, ref))
        assert 1 - fidelity(got, ref) <= FID_TOL
    st = stamps.cpu().numpy().view(np.uint64)
    assert st[0] > 0 and np.all(st[1:] >= st[0])


@pytest.mark.parametrize("batch_tc,form", [("1", "auto"), ("0", "fma")])
def test_batch_equals_one_circuit_path_bitwise(cuda_lib, monkeypatch, batch_tc, form):
    # same programs, same tile arithmetic: the batched result is bit-identical
    # (final stages with K >= 8 on the tensor cores, as AUTO does, by default)
    monkeypatch.setenv("CUTSIM_BATCH_TC", batch_tc)
    items = w.uneven_batch(8, seed=11, q_range=(14, 20), depths=(8, 16), c_range=(1, 5))
    b = make_batch(items)
    seg, psi, ws = b.alloc_buffers()
    stamps = b.alloc_stamps()
    b.run(seg, psi, ws, stamps)
    sync()
    for i, it in enumerate(items):
        one, _, _ = gpu_cut(it.gates, it.q, it.seg_sizes, "projector", "c64", form)
        assert torch.equal(b.psi_view(psi, i), one), i
    st = stamps.cpu().numpy().view(np.uint64)
    assert st[0] > 0 and np.all(st[1:] >= st[0])


def test_batch_graph_replay(cuda_lib):
    items = w.uneven_batch(16, seed=7, q_range=(14, 20), depths=(8,), c_range=(2, 5))
    b = make_batch(items)
    seg, psi, ws = b.alloc_buffers()
    b.run(seg, psi, ws)
    sync()
    ref = psi.clone()
    psi.zero_()
    seg.zero_()
    s = torch.cuda.Stream()
    stamps = b.alloc_stamps()
    torch.cuda.synchronize()
    b.capture(seg, psi, ws, stamps, stream=s)
    assert torch.count_nonzero(psi) == 0  # capture runs nothing
    b.launch(stream=s)
    b.launch(stream=s)
    s.synchronize()
    sync()
    assert torch.equal(psi, ref)
    st = stamps.cpu().numpy().view(np.uint64)
    assert st[0] > 0 and np.all(st[1:] >= st[0])


def test_batch_autotune_keeps_results(cuda_lib):
    items = w.uneven_batch(12, seed=5, q_range=(16, 20), depths=(8, 16), c_range=(2, 6))
    b = make_batch(items)
    seg, psi, ws = b.alloc_buffers()
    table = b.autotune(seg, psi, ws)
    assert len(table) == 2 * (14 - 10 + 1)
    best = min(table, key=lambda r: r["ms"])
    assert b.info["tile_bits"] == best["tile_bits"] and b.info["merge_rows"] == best["merge_rows"]
    b.run(seg, psi, ws)
    sync()
    for i in (0, 5, 11):
        it = items[i]
        assert rel_err(b.psi_view(psi, i).cpu().numpy(), sv.simulate(it.q, it.gates)) <= TOL["c64"]


def test_batch_rejects_small_buffers(cuda_lib):
    items = w.uneven_batch(3, seed=2, q_range=(12, 14), depths=(4,), c_range=(2, 3))
    b = make_batch(items)
    seg, psi, ws = b.alloc_buffers()
    with pytest.raises(capi.CutsimError) as e:
        b.run(seg, psi[:-32], ws)
    assert e.value.status == 5
    with pytest.raises(capi.CutsimError) as e:
        b.launch()
    assert e.value.status == 1


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_persistent_segment_launch_equals_per_pass(cuda_lib, monkeypatch, prec):
    # cc_simulate_segments runs every segment pass in one persistent launch by
    # default; one launch per pass must give the same bits
    for segs, c, depth in (([9, 10], 4, 8), ([6, 7, 7], [2, 3], 12), ([15, 5], 3, 6)):
        q = sum(segs)
        gates = w.brickwork_cut(q, depth, 17, segs, c)
        monkeypatch.delenv("CUTSIM_SEG_LAUNCH", raising=False)
        psi_a, seg_a, _ = gpu_cut(gates, q, segs, "s_sdg", prec, "fma")
        monkeypatch.setenv("CUTSIM_SEG_LAUNCH", "passes")
        psi_b, seg_b, _ = gpu_cut(gates, q, segs, "s_sdg", prec, "fma")
        sync()
        assert torch.equal(seg_a, seg_b)
        assert torch.equal(psi_a, psi_b)
        assert rel_err(psi_a.cpu().numpy(), sv.simulate(q, gates)) <= TOL[prec]
