"""Parity at the full benchmark sizes, through the same calls bench.py times.

The 2^26 .. 2^30 output is checked (1) on 4096 seeded amplitudes, each
computed on the CPU by the oracle's per-amplitude form of the Algorithm 3 sum
from its own FP64 subcircuit states, relative to max |psi| over the whole
vector (FP64 device reduction), and (2) for the benchmark workload, against
the GPU's own uncut simulation over the full vector, plus the norms.
"""

import numpy as np
import pytest
import torch

import workload as w
from oracle import cutting as ct
from paper_2603_01443_gb300 import api, capi
from gpu_util import FID_TOL, TOL

pytestmark = pytest.mark.gpu

FORM_TOL = {"fma": None, "auto": None, "tf32x3": TOL["c64"], "bf16x3": TOL["bf16x3"]}


def sampled_check(gates, q, segs, decomp, prec, form):
    plan = api.CutPlan(gates, q, segs, decomp, prec)
    seg = plan.alloc_seg_buf()
    psi = plan.alloc_psi()
    ws = plan.alloc_workspace()
    plan.simulate_segments(seg)
    plan.merge(seg, psi, ws, form)
    capi.check(capi.lib().cc_sync(torch.cuda.current_stream().cuda_stream), "cc_sync")
    xs = w.sample_indices(q, 4096, 2024)
    got = api.gather(psi, xs, prec)
    pre = ct.preprocess(q, gates, segs, decomp)
    states = ct.simulate_subcircuits(pre)
    ref = ct.amplitudes(pre, states, xs)
    stats = api.compare(psi, psi, prec)
    scale = stats["max_abs_b"]
    err = float(np.max(np.abs(got.astype(np.complex128) - ref))) / scale
    tol = FORM_TOL[form] or TOL[prec]
    assert err <= tol, f"sampled max|dpsi|/max|psi| = {err:.3e} > {tol:.1e}"
    assert abs(stats["norm2_a"] - 1.0) < 1e-4
    return psi, plan


def test_q30_n2_c6_bench_workload_sampled_and_vs_uncut(cuda_lib):
    q, depth, segs, c = 30, 16, [15, 15], 6
    gates = w.brickwork_cut(q, depth, 0, segs, c)
    psi, plan = sampled_check(gates, q, segs, "projector", "c64", "auto")
    assert plan.info["c_total"] == 6 and plan.info["n_sub"] == 128
    up = api.UncutPlan(gates, q, "c64")
    psi_u = up.alloc_psi()
    up.simulate(psi_u)
    st = api.compare(psi, psi_u, "c64")
    assert st["max_abs_diff"] <= TOL["c64"] * st["max_abs_b"], st
    assert 1 - st["fidelity"] <= FID_TOL, st
    assert abs(st["norm2_b"] - 1.0) < 1e-4


@pytest.mark.parametrize("q,n,c,decomp,prec,form", [
    (30, 2, 6, "projector", "c64", "bf16x3"),
    (30, 2, 2, "s_sdg", "c64", "auto"),
    (28, 2, 8, "s_sdg", "c64", "auto"),
    (28, 2, 7, "projector", "c64", "auto"),
    (28, 3, 6, "s_sdg", "c64", "auto"),
    (30, 3, 8, "projector", "c64", "auto"),
    (26, 2, 4, "projector", "c64", "fma"),
    (26, 2, 8, "projector", "c128", "fma"),
    (26, 3, 4, "s_sdg", "c128", "auto"),
    (30, 2, 8, "projector", "c64", "tf32x3"),   # K = 256: grouped 3xTF32
    (28, 2, 6, "projector", "c128", "auto"),    # complex128 at the larger sizes
    (28, 3, 4, "s_sdg", "c128", "auto"),
    (30, 2, 6, "projector", "c128", "auto"),    # 16 GiB complex128 output
    (32, 2, 4, "projector", "c64", "auto"),     # 32 GiB output, the largest case here
])
def test_sampled_parity_at_scale(cuda_lib, q, n, c, decomp, prec, form):
    segs = w.equal_partition(q, n)
    gates = w.brickwork_cut(q, 16, q + c, segs, w.split_cuts(c, n))
    sampled_check(gates, q, segs, decomp, prec, form)
