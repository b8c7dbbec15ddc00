"""The two complex128 gate-pass arithmetics against the FP64 oracle: the
default double-float engine (each real an unevaluated sum of two FP32 numbers,
error-free TwoSum / TwoProduct transformations on the FP32 pipes) and native
FP64 (CUTSIM_C128_GATES=fp64).  Both must meet the complex128 tolerance on
single-pass and multi-pass programs (the double-float passes keep (h, l)
pairs in HBM between passes and write complex128 in the last one), on cut
plans, on amplitudes spanning far more than FP32's exponent range, and on
deep circuits; the switch must really change the engine.  The uncut passes'
two launch forms (program in the kernel parameter, or in global memory)
must agree bit for bit."""

import numpy as np
import pytest
import torch

import workload as w
from oracle import statevector as sv
from gpu_util import TOL, assert_parity, gpu_cut, gpu_uncut, rel_err

pytestmark = pytest.mark.gpu

ARITH = ["dfl", "fp64"]


@pytest.mark.parametrize("arith", ARITH)
@pytest.mark.parametrize("q,depth", [(6, 4), (12, 10), (16, 12), (20, 8)])
def test_uncut_engines_vs_oracle(cuda_lib, monkeypatch, arith, q, depth):
    # q <= 13 is one pass (init and last at once); q = 16, 20 run several
    # passes through the intermediate layout
    monkeypatch.setenv("CUTSIM_C128_GATES", arith)
    gates = w.brickwork(q, depth, 31 + q)
    psi, up = gpu_uncut(gates, q, "c128")
    assert_parity(psi.cpu().numpy(), sv.simulate(q, gates), "c128", f"uncut {arith} q={q}")


@pytest.mark.parametrize("arith", ARITH)
@pytest.mark.parametrize("segs,c", [([7, 7], 2), ([9, 9], 5), ([6, 7, 7], [2, 2])])
def test_cut_engines_vs_oracle(cuda_lib, monkeypatch, arith, segs, c):
    monkeypatch.setenv("CUTSIM_C128_GATES", arith)
    q = sum(segs)
    gates = w.brickwork_cut(q, 10, 8 + q, segs, c)
    psi, _, _ = gpu_cut(gates, q, segs, "s_sdg", "c128", "fma")
    assert_parity(psi.cpu().numpy(), sv.simulate(q, gates), "c128", f"cut {arith}")


def test_switch_changes_the_engine(cuda_lib, monkeypatch):
    # the two arithmetics round differently (about 2^-48 against 2^-53 per
    # operation), so their vectors differ in the last bits but agree far
    # inside the complex128 tolerance
    q = 18
    gates = w.brickwork(q, 12, 5)
    monkeypatch.setenv("CUTSIM_C128_GATES", "dfl")
    a, _ = gpu_uncut(gates, q, "c128")
    monkeypatch.setenv("CUTSIM_C128_GATES", "fp64")
    b, _ = gpu_uncut(gates, q, "c128")
    assert not torch.equal(a, b)
    assert rel_err(a.cpu().numpy(), b.cpu().numpy()) <= 1e-13


@pytest.mark.parametrize("arith", ARITH)
def test_amplitudes_below_fp32_range(cuda_lib, monkeypatch, arith):
    # RY(1e-15) on six qubits: the amplitude of |1...1> is ~(5e-16)^6 ~ 1e-92,
    # far below FP32's smallest normal; the double-float pairs flush such
    # amplitudes towards zero, which the absolute tolerance allows, and nothing
    # becomes inf or nan
    monkeypatch.setenv("CUTSIM_C128_GATES", arith)
    q = 14
    gates = [w.Gate("U3", i, -1, 1e-15, 0.0, 0.0) for i in range(6)]
    gates += [w.Gate("H", i) for i in range(6, q)]
    gates += [w.Gate("CZ", i, i + 1) for i in range(q - 1)]
    psi, _ = gpu_uncut(gates, q, "c128")
    got = psi.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert_parity(got, sv.simulate(q, gates), "c128", f"tiny amplitudes {arith}")


def test_deep_multi_pass_double_float(cuda_lib, monkeypatch):
    # depth 200 over 16 qubits (several passes, ~3200 rotations per
    # amplitude): double-float rounding grows like sqrt(G) 2^-48, ~2e-13
    monkeypatch.setenv("CUTSIM_C128_GATES", "dfl")
    q = 16
    gates = w.brickwork(q, 200, 12)
    psi, up = gpu_uncut(gates, q, "c128")
    assert up.info["n_passes"] > 1
    assert_parity(psi.cpu().numpy(), sv.simulate(q, gates), "c128", "deep dfl")


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_parameter_and_global_pass_launches_agree(cuda_lib, monkeypatch, prec):
    # an uncut pass reads its program from its kernel parameter when it fits
    # (the default) or from global memory; the arithmetic is the same, so
    # the vectors are bit-identical
    q = 20
    gates = w.brickwork(q, 14, 21)
    monkeypatch.setenv("CUTSIM_PARAM_PASSES", "1")
    a, _ = gpu_uncut(gates, q, prec)
    monkeypatch.setenv("CUTSIM_PARAM_PASSES", "0")
    b, _ = gpu_uncut(gates, q, prec)
    assert torch.equal(a, b)
    assert_parity(a.cpu().numpy(), sv.simulate(q, gates), prec, "parameter launch")
