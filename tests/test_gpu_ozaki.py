"""The complex128 tensor-core merge (Ozaki scheme: bf16 slices, exact
fixed-point level sums, one FP64 rounding) against the FP64 oracle at the
complex128 tolerance, for K from 1 to 4096 merge terms (one to 64 groups of
64 terms), factors spanning one to many 128 x 128 output tiles, both rank-2
decompositions, rank-4 cuts, the last stage of a three-segment chain, and
segment vectors with zero rows and columns."""

import numpy as np
import pytest
import torch

import workload as w
from oracle import cutting as ct
from oracle import statevector as sv
from gpu_util import TOL, assert_parity, gpu_cut

pytestmark = pytest.mark.gpu


CASES = [([7, 7], 0), ([7, 7], 1), ([7, 8], 3), ([8, 9], 5), ([9, 8], 6), ([10, 10], 6),
         ([8, 8], 7), ([9, 9], 8), ([8, 8], 10), ([8, 8], 12)]


@pytest.mark.parametrize("segs,c", CASES)
def test_ozaki_merge_vs_oracle(cuda_lib, segs, c):
    q = sum(segs)
    gates = w.brickwork_cut(q, 12, 70 + c, segs, c)
    psi, _, plan = gpu_cut(gates, q, segs, "s_sdg" if c % 2 else "projector", "c128", "ozaki")
    ref = sv.simulate(q, gates)
    assert_parity(psi.cpu().numpy(), ref, "c128", f"ozaki K={1 << c}")


@pytest.mark.parametrize("segs,c", [([8, 9], 5), ([9, 9], 8)])
def test_ozaki_matches_fma_and_auto(cuda_lib, segs, c):
    # AUTO runs the Ozaki form for complex128 (bit-identical to asking for
    # it); the native FP64 FMA form agrees within the complex128 tolerance
    q = sum(segs)
    gates = w.brickwork_cut(q, 16, 5 + c, segs, c)
    psi_oz, _, _ = gpu_cut(gates, q, segs, "projector", "c128", "ozaki")
    psi_auto, _, _ = gpu_cut(gates, q, segs, "projector", "c128", "auto")
    psi_fma, _, _ = gpu_cut(gates, q, segs, "projector", "c128", "fma")
    assert torch.equal(psi_oz, psi_auto)
    a, b = psi_oz.cpu().numpy(), psi_fma.cpu().numpy()
    assert np.max(np.abs(a - b)) <= TOL["c128"] * np.max(np.abs(b))


def test_ozaki_last_stage_of_chain(cuda_lib):
    segs = [7, 7, 8]
    gates = w.brickwork_cut(22, 10, 17, segs, [3, 4])
    psi, _, _ = gpu_cut(gates, 22, segs, "s_sdg", "c128", "ozaki")
    ref, _, _ = ct.cut_simulate(22, gates, segs, "s_sdg")
    assert_parity(psi.cpu().numpy(), ref, "c128", "ozaki n=3")


def test_ozaki_rank4_cuts(cuda_lib):
    # SWAP and CAN gates across the boundary: two variant bits per cut
    rng = np.random.default_rng(3)
    q, segs = 16, [8, 8]
    gates = list(w.brickwork(q, 4, 9))
    gates.append(w.Gate("SWAP", 7, 8))
    gates += w.brickwork(q, 2, 10)
    gates.append(w.Gate("CAN", 8, 7, *rng.uniform(0, 2 * np.pi, 3)))
    gates += w.brickwork(q, 2, 11)
    psi, _, plan = gpu_cut(gates, q, segs, "projector", "c128", "ozaki")
    ref = sv.simulate(q, gates)
    assert_parity(psi.cpu().numpy(), ref, "c128", "ozaki rank-4")


def test_ozaki_zero_rows_and_columns(cuda_lib):
    # basis-state-like segments: most amplitudes exactly zero, so whole rows
    # of both operands are zero (the split's zero-row exponent) next to rows
    # with a single nonzero entry
    q, segs = 16, [8, 8]
    gates = [w.Gate("X", 1), w.Gate("H", 7), w.Gate("CZ", 7, 8), w.Gate("H", 8),
             w.Gate("X", 12), w.Gate("CX", 6, 9), w.Gate("T", 9)]
    psi, _, _ = gpu_cut(gates, q, segs, "projector", "c128", "ozaki")
    ref = sv.simulate(q, gates)
    assert_parity(psi.cpu().numpy(), ref, "c128", "ozaki zero rows")


@pytest.mark.parametrize("cfg", ["0", "1", "2", "3"])
@pytest.mark.parametrize("segs,c", [([8, 9], 5), ([9, 8], 8)])
def test_ozaki_kernel_configurations(cuda_lib, monkeypatch, cfg, segs, c):
    # every kernel configuration (tile width, accumulator count and sets,
    # epilogue width, FP64 conversion) against the oracle; the default picks
    # by K
    monkeypatch.setenv("CUTSIM_OZ_CFG", cfg)
    q = sum(segs)
    gates = w.brickwork_cut(q, 12, 90 + c, segs, c)
    psi, _, _ = gpu_cut(gates, q, segs, "projector", "c128", "ozaki")
    ref = sv.simulate(q, gates)
    assert_parity(psi.cpu().numpy(), ref, "c128", f"ozaki cfg {cfg}")
