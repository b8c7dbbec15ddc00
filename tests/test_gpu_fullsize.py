"""Parity at the full benchmark sizes, through the same calls bench.py times.

The 2^28 / 2^30 output is checked (1) on 4096 seeded amplitudes, each
computed on the CPU by the oracle's per-amplitude form of the Algorithm 3 sum
from its own FP64 subcircuit states, and (2) against the GPU's own uncut
simulation over the full vector with the FP64 device reductions, plus the
norm (unitarity) of both.
"""

import numpy as np
import pytest
import torch

import workload as w
from oracle import cutting as ct
from paper_2603_01443_gb300 import api
from gpu_util import FID_TOL, TOL

pytestmark = pytest.mark.gpu


def sampled_check(gates, q, segs, decomp, prec, form, tol):
    plan = api.CutPlan(gates, q, segs, decomp, prec)
    seg = plan.alloc_seg_buf()
    psi = plan.alloc_psi()
    ws = plan.alloc_workspace()
    plan.simulate_segments(seg)
    plan.merge(seg, psi, ws, form)
    torch.cuda.synchronize()
    xs = w.sample_indices(q, 4096, 2024)
    got = api.gather(psi, xs, prec)
    pre = ct.preprocess(q, gates, segs, decomp)
    states = ct.simulate_subcircuits(pre)
    ref = ct.amplitudes(pre, states, xs)
    # tolerance relative to max |psi| over the whole vector (device reduction)
    stats = api.compare(psi, psi, prec)
    scale = stats["max_abs_b"]
    err = float(np.max(np.abs(got.astype(np.complex128) - ref))) / scale
    assert err <= tol, f"sampled max|dpsi|/max|psi| = {err:.3e}"
    assert abs(stats["norm2_a"] - 1.0) < 1e-4
    return psi, plan, err


def test_q30_n2_c6_sampled_and_vs_uncut(cuda_lib):
    q, depth, segs, c = 30, 16, [15, 15], 6
    gates = w.brickwork_cut(q, depth, 0, segs, c)
    psi, plan, err = sampled_check(gates, q, segs, "projector", "c64", "fma", TOL["c64"])
    assert plan.info["c_total"] == 6 and plan.info["n_sub"] == 128
    up = api.UncutPlan(gates, q, "c64")
    psi_u = up.alloc_psi()
    up.simulate(psi_u)
    st = api.compare(psi, psi_u, "c64")
    assert st["max_abs_diff"] <= TOL["c64"] * st["max_abs_b"], st
    assert 1 - st["fidelity"] <= FID_TOL, st
    assert abs(st["norm2_b"] - 1.0) < 1e-4


def test_q28_n3_chained_sampled(cuda_lib):
    q, depth, segs = 28, 16, w.equal_partition(28, 3)
    gates = w.brickwork_cut(q, depth, 1, segs, 3)
    sampled_check(gates, q, segs, "s_sdg", "c64", "fma", TOL["c64"])


def test_q26_n2_c8_complex128_sampled(cuda_lib):
    q, segs = 26, [13, 13]
    gates = w.brickwork_cut(q, 16, 2, segs, 8)
    sampled_check(gates, q, segs, "projector", "c128", "fma", TOL["c128"])
