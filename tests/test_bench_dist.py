"""The replica (N > 1) path of bench.py on CPU: two gloo ranks report the
slowest rank's timings, and the reference arm runs on rank 0 only."""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank], world, "cpu")
        out[rank] = got
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == [2.0, 10.0] and out[1] == [2.0, 10.0]


def test_single_process_is_identity():
    assert bench.max_over_ranks([3, 4.5], 1) == [3.0, 4.5]


def test_reference_arm_non_zero_rank_does_no_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "run_oracle_timing", lambda *a, **k: called.append(1))
    assert bench.reference_arm(bench.parse_args(["--impl", "reference"])) == 0
    assert not called and capsys.readouterr().out == ""


def test_oracle_timing_on_small_workload():
    # the pooled CPU oracle timing: Algorithm 2 in full over spawned workers,
    # slab estimates at S and 2S, and the oracle's sampled amplitudes
    import numpy as np

    import workload as w
    from oracle import cutting as ct

    a = bench.parse_args(["--q", "12", "--depth", "4", "--ctotal", "2"])
    d = bench.run_oracle_timing(a, [8, 16], sample_seed=2024)
    assert "error" not in d, d
    assert d["n_sub"] == 8 and d["cores"] >= 1
    assert [e["slabs"] for e in d["merge_estimates"]] == [8, 16]
    for e in d["merge_estimates"]:  # the median of three timed passes
        assert len(e["passes_s"]) == 3 and e["seconds"] == sorted(e["passes_s"])[1]
    rec = bench.cpu_record(d, a)
    assert rec["cores"] == d["cores"] and rec["kind"] == "oracle" and rec["value"] > 0
    assert set(rec["convergence"]) == {"slabs", "t_merge_s", "ratio"}
    segs = w.equal_partition(12, 2)
    gates = w.brickwork_cut(12, 4, 0, segs, [2])
    pre = ct.preprocess(12, gates, segs, "projector")
    ref = ct.amplitudes(pre, ct.simulate_subcircuits(pre), w.sample_indices(12, 4096, 2024))
    got = np.array([complex(re, im) for re, im in d["sample_amplitudes"]])
    assert np.array_equal(got, ref)
