"""The tcgen05 tensor-core merge forms (3xTF32 and split-BF16) against the FP64
oracle and against the CUDA-core form, on factors spanning one to many
128 x 256 output tiles and K from 1 to 1024 merge terms."""

import numpy as np
import pytest
import torch

import workload as w
from oracle import statevector as sv
from paper_2603_01443_gb300 import api, capi
from gpu_util import FID_TOL, TOL, fidelity, rel_err

pytestmark = pytest.mark.gpu

FORM_TOL = {"tf32x3": TOL["c64"], "bf16x3": TOL["bf16x3"], "f16x3": TOL["c64"]}


def run(gates, q, segs, form, decomp="projector"):
    plan = api.CutPlan(gates, q, segs, decomp, "c64")
    seg = plan.alloc_seg_buf()
    psi = plan.alloc_psi()
    ws = plan.alloc_workspace()
    plan.simulate_segments(seg)
    plan.merge(seg, psi, ws, form)
    capi.check(capi.lib().cc_sync(torch.cuda.current_stream().cuda_stream), "cc_sync")
    return psi, plan


CASES = [([7, 7], 0), ([7, 7], 3), ([8, 9], 5), ([9, 8], 6), ([10, 10], 4), ([8, 8], 6)]


DEEP = [([8, 8], 7), ([8, 8], 8), ([8, 8], 10), ([8, 8], 12), ([9, 10], 9)]


@pytest.mark.parametrize("form,segs,c", [("tf32x3",) + x for x in CASES + DEEP] +
                         [("bf16x3",) + x for x in CASES + DEEP] +
                         [("f16x3",) + x for x in CASES + DEEP])
def test_tc_merge_vs_oracle(cuda_lib, form, segs, c):
    q = sum(segs)
    gates = w.brickwork_cut(q, 12, 21 + c, segs, c)
    psi, plan = run(gates, q, segs, form, "s_sdg" if c % 2 else "projector")
    ref = sv.simulate(q, gates)
    got = psi.cpu().numpy()
    err = rel_err(got, ref)
    assert err <= FORM_TOL[form], f"{form} K={1 << c}: {err:.3e}"
    assert 1 - fidelity(got, ref) <= FID_TOL


@pytest.mark.parametrize("form", ["tf32x3", "bf16x3", "f16x3"])
def test_tc_merge_matches_fma_at_scale(cuda_lib, form):
    q, segs, c = 26, [13, 13], 6
    gates = w.brickwork_cut(q, 16, 3, segs, c)
    psi_tc, plan = run(gates, q, segs, form)
    psi_fma, _ = run(gates, q, segs, "fma")
    st = api.compare(psi_tc, psi_fma, "c64")
    assert st["max_abs_diff"] <= FORM_TOL[form] * st["max_abs_b"], st
    assert 1 - st["fidelity"] <= FID_TOL


def test_tc_merge_rejects_small_workspace(cuda_lib):
    gates = w.brickwork_cut(16, 8, 0, [8, 8], 4)
    plan = api.CutPlan(gates, 16, [8, 8], "projector", "c64")
    seg = plan.alloc_seg_buf()
    psi = plan.alloc_psi()
    plan.simulate_segments(seg)
    ws = plan.alloc_workspace()
    with pytest.raises(capi.CutsimError) as e:
        plan.merge(seg, psi, ws[:16], "tf32x3")
    assert e.value.status == 5


def test_tf32x3_deep_merge_matches_fma_at_scale(cuda_lib):
    # K = 256: four 64-term groups, the later ones added by tensor reduce-add stores
    q, segs, c = 24, [12, 12], 8
    gates = w.brickwork_cut(q, 12, 2, segs, c)
    psi_tc, _ = run(gates, q, segs, "tf32x3")
    psi_fma, _ = run(gates, q, segs, "fma")
    st = api.compare(psi_tc, psi_fma, "c64")
    assert st["max_abs_diff"] <= TOL["c64"] * st["max_abs_b"], st
    assert 1 - st["fidelity"] <= FID_TOL
    psi_auto, _ = run(gates, q, segs, "auto")
    psi_f16, _ = run(gates, q, segs, "f16x3")
    assert torch.equal(psi_auto, psi_f16)  # AUTO picks 3xFP16 at K = 256
    # 3xFP16 at K = 256: two 128-term groups
    st = api.compare(psi_f16, psi_fma, "c64")
    assert st["max_abs_diff"] <= TOL["c64"] * st["max_abs_b"], st


def test_f16x3_long_merge_in_64_term_groups(cuda_lib):
    # K = 1024: 3xFP16 accumulates 64 terms per group (sixteen groups, the
    # later ones added by tensor reduce-add stores) and stays within the
    # complex64 tolerance of the FMA merge
    q, segs, c = 24, [12, 12], 10
    gates = w.brickwork_cut(q, 12, 4, segs, c)
    psi_f16, _ = run(gates, q, segs, "f16x3")
    psi_fma, _ = run(gates, q, segs, "fma")
    st = api.compare(psi_f16, psi_fma, "c64")
    assert st["max_abs_diff"] <= TOL["c64"] * st["max_abs_b"], st
    assert 1 - st["fidelity"] <= FID_TOL


@pytest.mark.parametrize("form", ["tf32x3", "bf16x3", "f16x3", "auto"])
def test_tc_last_stage_of_chained_merge(cuda_lib, form):
    # n = 3: the last stage (2^q output, K = 2^4 terms) runs on tensor cores
    segs = [6, 7, 7]
    gates = w.brickwork_cut(20, 10, 13, segs, [2, 4])
    psi, plan = run(gates, 20, segs, form, "s_sdg")
    ref = sv.simulate(20, gates)
    tol = FORM_TOL.get(form, TOL["c64"])
    assert rel_err(psi.cpu().numpy(), ref) <= tol
    assert 1 - fidelity(psi.cpu().numpy(), ref) <= FID_TOL


@pytest.mark.parametrize("stationary", ["0", "1"])
@pytest.mark.parametrize("form", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("segs,c", [([8, 9], 5), ([10, 10], 6), ([9, 9], 4)])
def test_tc_forms_stationary_and_streaming(cuda_lib, monkeypatch, stationary, form, segs, c):
    # the streaming kernel (default) and the row-operand-stationary kernel
    # (opt-in where R fits) must agree with the oracle alike
    monkeypatch.setenv("CUTSIM_TC_STATIONARY", stationary)
    q = sum(segs)
    gates = w.brickwork_cut(q, 12, 31 + c, segs, c)
    psi, _ = run(gates, q, segs, form)
    ref = sv.simulate(q, gates)
    assert rel_err(psi.cpu().numpy(), ref) <= FORM_TOL[form]


@pytest.mark.parametrize("form", ["tf32x3", "bf16x3", "f16x3"])
@pytest.mark.parametrize("segs,c", [([7, 8], 4), ([9, 10], 6), ([10, 9], 8), ([8, 11], 5),
                                    ([9, 9], 10)])
def test_tc_kblock_forms(cuda_lib, monkeypatch, form, segs, c):
    # the streaming kernel with K in blocks of 128, 64 or 32 bytes (2, 4 or 8
    # stages of the same 192 KB) against the oracle; every block width issues
    # the same products in the same order per tile, so the bits agree
    q = sum(segs)
    gates = w.brickwork_cut(q, 12, 41 + c, segs, c)
    ref = sv.simulate(q, gates)
    first = None
    for kblock in ("128", "64", "32"):
        monkeypatch.setenv("CUTSIM_TC_KBLOCK", kblock)
        psi, _ = run(gates, q, segs, form)
        assert rel_err(psi.cpu().numpy(), ref) <= FORM_TOL[form], kblock
        if first is None:
            first = psi
        else:
            assert torch.equal(psi, first), kblock


def test_f16x3_scales_keep_tiny_rows_accurate(cuda_lib):
    # the fp16 form scales each operand row by a power of two: factors whose
    # amplitudes span many orders of magnitude (a basis-state-like segment
    # next to spread ones) keep the complex64 tolerance
    q, segs = 18, [9, 9]
    gates = [w.Gate("X", 2), w.Gate("H", 8), w.Gate("CZ", 8, 9)]
    gates += w.brickwork(18, 3, 77)
    gates += [w.Gate("CZ", 8, 9), w.Gate("H", 9), w.Gate("T", 9), w.Gate("CZ", 8, 9)]
    psi, _ = run(gates, q, segs, "f16x3")
    ref = sv.simulate(q, gates)
    assert rel_err(psi.cpu().numpy(), ref) <= TOL["c64"]
