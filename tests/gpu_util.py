"""Shared helpers for the GPU parity tests (all calls go through the C ABI)."""

import numpy as np
import torch

from oracle import reductions as rd
from paper_2603_01443_gb300 import api

# Tolerances on max |d psi| / max |psi| and on 1 - fidelity.
TOL = {"c64": 2e-6, "c128": 1e-12, "bf16x3": 5e-5}
FID_TOL = 1e-6


def rel_err(got, ref):
    """max |got - ref| / max |ref|, from the oracle's verification quantities."""
    r = rd.compare(np.asarray(got), np.asarray(ref))
    return r["max_abs_diff"] / r["max_abs_b"]


def fidelity(a, b):
    """|<a|b>|^2 / (|a|^2 |b|^2), from the oracle's verification quantities."""
    return rd.compare(np.asarray(a), np.asarray(b))["fidelity"]


def gpu_cut(gates, q, segs, decomp="projector", prec="c64", form="fma"):
    plan = api.CutPlan(gates, q, segs, decomp, prec)
    seg = plan.alloc_seg_buf()
    psi = plan.alloc_psi()
    ws = plan.alloc_workspace()
    plan.simulate_segments(seg)
    plan.merge(seg, psi, ws, form)
    torch.cuda.synchronize()
    return psi, seg, plan


def gpu_uncut(gates, q, prec="c64"):
    up = api.UncutPlan(gates, q, prec)
    psi = up.alloc_psi()
    up.simulate(psi)
    torch.cuda.synchronize()
    return psi, up


def assert_parity(got, ref, prec, what=""):
    err = rel_err(got, ref)
    fid = fidelity(got, ref)
    assert err <= TOL[prec], f"{what}: max|dpsi|/max|psi| = {err:.3e} > {TOL[prec]:.1e}"
    assert 1 - fid <= FID_TOL, f"{what}: fidelity {fid:.12f}"
    return err, fid
