"""GPU parity: every stage of the CUDA path against the FP64 oracle on the same
seeded circuits, element by element (max |d psi| / max |psi| within 1e-12 in
complex128 and 2e-6 in complex64, fidelity within 1e-6 of 1)."""

import math

import numpy as np
import pytest
import torch

import workload as w
from oracle import cutting as ct
from oracle import statevector as sv
from oracle import reductions as rd
from paper_2603_01443_gb300 import api, capi
from gpu_util import FID_TOL, TOL, assert_parity, fidelity, gpu_cut, gpu_uncut, rel_err

pytestmark = pytest.mark.gpu

PRECS = ["c64", "c128"]
DECOMPS = ["projector", "s_sdg"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("decomp", DECOMPS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_small_brickwork_cut_and_uncut(cuda_lib, prec, decomp, seed):
    # q = 12, depth 4, two 6-qubit segments, the natural c_total = 2
    q, segs = 12, [6, 6]
    gates = w.brickwork(q, 4, seed)
    ref = sv.simulate(q, gates)
    psi, _, plan = gpu_cut(gates, q, segs, decomp, prec)
    assert plan.info["c_total"] == 2 and plan.info["n_sub"] == 8
    assert_parity(psi.cpu().numpy(), ref, prec, "cut")
    oracle_merge, _, _ = ct.cut_simulate(q, gates, segs, decomp)
    assert rel_err(psi.cpu().numpy(), oracle_merge) <= TOL[prec]
    u, _ = gpu_uncut(gates, q, prec)
    assert_parity(u.cpu().numpy(), ref, prec, "uncut")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("decomp", DECOMPS)
@pytest.mark.parametrize("q,segs,c", [(12, [6, 6], 3), (14, [5, 9], 4), (13, [4, 4, 5], 2)])
def test_segment_variants_match_oracle_subcircuits(cuda_lib, prec, decomp, q, segs, c):
    gates = w.brickwork_cut(q, 6, 7, segs, c)
    pre = ct.preprocess(q, gates, segs, decomp)
    states = ct.simulate_subcircuits(pre)
    _, seg, plan = gpu_cut(gates, q, segs, decomp, prec)
    for i in range(len(segs)):
        got = plan.segment_view(seg, i).cpu().numpy()
        assert got.shape == (len(states[i]), 1 << segs[i])
        for r, ref in enumerate(states[i]):
            # the library folds cut j's coefficient into the first-qubit side
            fac = 1.0 + 0j
            for t, j in enumerate(pre.seg_cuts[i]):
                if pre.cuts[j].segments[0] == i:
                    fac *= pre.coefs[j][(r >> t) & 1]
            want = fac * ref
            err = np.max(np.abs(got[r] - want))
            assert err <= TOL[prec] * max(np.max(np.abs(want)), 1e-300) or err < 1e-14, (i, r, err)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("q,n_gates,seed", [(5, 80, 0), (11, 300, 1), (15, 400, 2), (17, 300, 3)])
def test_uncut_random_gate_positions(cuda_lib, prec, q, n_gates, seed):
    # every gate kind, two-qubit gates on far-apart pairs, high and low qubits;
    # q > 14 (c64) / > 13 (c128) runs several HBM passes
    gates = w.random_circuit(q, n_gates, seed)
    u, up = gpu_uncut(gates, q, prec)
    if q >= 15:
        assert up.info["n_passes"] > 1
    assert_parity(u.cpu().numpy(), sv.simulate(q, gates), prec, "uncut")


@pytest.mark.parametrize("prec", PRECS)
def test_uncut_brickwork_multipass(cuda_lib, prec):
    q = 20
    gates = w.brickwork(q, 8, 3)
    u, up = gpu_uncut(gates, q, prec)
    assert up.info["n_passes"] > 1
    assert_parity(u.cpu().numpy(), sv.simulate(q, gates), prec, "uncut")


@pytest.mark.parametrize("prec,segs", [("c64", [15, 5]), ("c64", [5, 15]), ("c128", [14, 6])])
def test_segments_larger_than_one_tile(cuda_lib, prec, segs):
    # segment vectors beyond shared memory run as multi-pass programs
    q = sum(segs)
    gates = w.brickwork_cut(q, 6, 4, segs, 3)
    psi, _, plan = gpu_cut(gates, q, segs, "projector", prec)
    assert max(plan.info["seg_passes"]) > 1
    assert_parity(psi.cpu().numpy(), sv.simulate(q, gates), prec, "cut")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("segs", [[8, 8], [7, 9], [3, 13], [12, 4]])
@pytest.mark.parametrize("c", [0, 1, 5, 12])
def test_merge_term_counts(cuda_lib, prec, segs, c):
    # K = 2^c from 1 to 4096 merge terms, tiled and flat kernels, uneven factors
    q = sum(segs)
    gates = w.brickwork_cut(q, 16, 5, segs, c)
    psi, _, plan = gpu_cut(gates, q, segs, "s_sdg" if c % 2 else "projector", prec)
    assert plan.info["c_total"] == c
    assert_parity(psi.cpu().numpy(), sv.simulate(q, gates), prec, f"K={1 << c}")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("decomp", DECOMPS)
@pytest.mark.parametrize("segs,cpb", [([6, 6, 6], 2), ([7, 6, 5], [3, 1]), ([4, 4, 4, 4], 1)])
def test_chained_merge_three_or_more_segments(cuda_lib, prec, decomp, segs, cpb):
    q = sum(segs)
    gates = w.brickwork_cut(q, 8, 9, segs, cpb)
    psi, _, plan = gpu_cut(gates, q, segs, decomp, prec)
    assert_parity(psi.cpu().numpy(), sv.simulate(q, gates), prec, "chained")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("segs", [[4, 4, 4], [6, 6], [3, 9]])
def test_staircase_cx_cuts(cuda_lib, prec, segs):
    gates = w.staircase(12, 3)
    psi, _, plan = gpu_cut(gates, 12, segs, "s_sdg", prec)
    assert all(plan.cut(j)["kind"] == capi.GATE_KIND["CX"] for j in range(plan.info["c_total"]))
    assert_parity(psi.cpu().numpy(), sv.simulate(12, gates), prec, "staircase")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("p", [0, 2, 3])
def test_depth_augmented_staircase(cuda_lib, prec, p):
    # 10^p T/X layers on the edge qubits (the paper's depth sweep family)
    q = 10
    gates = w.staircase_depth(q, 4, p)
    for segs in ([5, 5], [4, 3, 3]):
        psi, _, plan = gpu_cut(gates, q, segs, "projector", prec)
        assert plan.info["c_total"] == 4 * (len(segs) - 1)
        assert_parity(psi.cpu().numpy(), sv.simulate(q, gates), prec, f"depth p={p}")
    psi_u, _ = gpu_uncut(gates, q, prec)
    assert_parity(psi_u.cpu().numpy(), sv.simulate(q, gates), prec, "uncut depth")


def test_ghz_closed_form(cuda_lib):
    q = 16
    psi, _, _ = gpu_cut(w.ghz(q), q, [8, 8], "projector", "c128")
    ref = np.zeros(1 << q, complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert rel_err(psi.cpu().numpy(), ref) <= TOL["c128"]


def test_single_segment_and_no_gates(cuda_lib):
    gates = w.brickwork(9, 3, 1)
    psi, _, plan = gpu_cut(gates, 9, [9], "projector", "c128")
    assert plan.info["c_total"] == 0
    assert_parity(psi.cpu().numpy(), sv.simulate(9, gates), "c128")
    psi, _, _ = gpu_cut([], 6, [3, 3], "projector", "c64")
    ref = np.zeros(64, complex)
    ref[0] = 1
    assert np.array_equal(psi.cpu().numpy(), ref.astype(np.complex64))


def check_compare(got, ref, mtol):
    """The device's verification quantities against the FP64 oracle's: the
    maxima within mtol (relative), the inner product and norms within 1e-11."""
    for k in ("max_abs_diff", "max_abs_b"):
        assert abs(got[k] - ref[k]) <= mtol * ref[k], k
    inner = abs(complex(ref["inner_re"], ref["inner_im"]))
    for k in ("inner_re", "inner_im"):
        assert abs(got[k] - ref[k]) <= 1e-11 * inner, k
    for k in ("norm2_a", "norm2_b"):
        assert abs(got[k] - ref[k]) <= 1e-11 * ref[k], k


@pytest.mark.parametrize("prec", PRECS)
def test_compare_and_gather(cuda_lib, prec):
    rng = np.random.default_rng(3)
    n = (1 << 20) + 37
    a = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(api.NUMPY_DTYPE[prec])
    b = a + (1e-3 * rng.standard_normal(n)).astype(api.NUMPY_DTYPE[prec])
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    got = api.compare(ta, tb, prec)
    # complex64: the maxima are taken in FP32 (2^-24 relative on the squares),
    # the sums in exact products + double-float runs + FP64, as accurate as FP64
    check_compare(got, rd.compare(a, b), 1e-12 if prec == "c128" else 1e-7)
    # a nearly equal pair: 1 - fidelity resolved far below the complex64 rounding level
    c = (a + (1e-6 * rng.standard_normal(n)).astype(a.dtype)).astype(a.dtype)
    tc = torch.from_numpy(c).cuda()
    f = api.compare(ta, tc, prec)["fidelity"]
    f_ref = rd.compare(a, c)["fidelity"]
    assert abs(f - f_ref) <= 1e-13, (f, f_ref)
    idx = w.sample_indices(20, 4096, 5) + [n - 1, 0]
    assert np.array_equal(api.gather(ta, idx, prec), a[np.array(idx)])
    with pytest.raises(capi.CutsimError):
        api.gather(ta, [n], prec)


@pytest.mark.parametrize("n", [1, 2, 3, 15, 4097, 2 * 608 * 256 * 8 + 3, 5 * 608 * 256 * 64 + 1])
def test_compare_lengths(cuda_lib, n):
    # complex64 compare reads two amplitudes per load, four loads in flight,
    # runs of 64 per thread: lengths below one load, odd tails, and lengths
    # that end inside a run or a grid stride
    rng = np.random.default_rng(n)
    a = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    b = (a + 1e-3 * rng.standard_normal(n)).astype(np.complex64)
    got = api.compare(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), "c64")
    check_compare(got, rd.compare(a, b), 1e-7)


def test_error_paths_on_device(cuda_lib):
    gates = w.brickwork(10, 3, 0)
    plan = api.CutPlan(gates, 10, [5, 5], "projector", "c128")
    seg = plan.alloc_seg_buf()
    psi = plan.alloc_psi()
    with pytest.raises(capi.CutsimError) as e:
        plan.simulate_segments(seg[:-1])
    assert e.value.status == 5
    plan.simulate_segments(seg)
    with pytest.raises(capi.CutsimError) as e:
        plan.merge(seg, psi[:-1])
    assert e.value.status == 5
    with pytest.raises(capi.CutsimError) as e:
        plan.merge(seg, psi, None, "bf16x3")
    assert e.value.status == 1
    up = api.UncutPlan(gates, 10, "c64")
    with pytest.raises(capi.CutsimError) as e:
        up.simulate(up.alloc_psi()[:100])
    assert e.value.status == 5


def test_expired_wait_is_reported_and_cleared(cuda_lib):
    # the error path of every bounded device wait, without any fault: a wait
    # on a word nothing writes gives up, cc_sync reports CC_ETIMEOUT once,
    # and the context stays usable
    stream = torch.cuda.current_stream().cuda_stream
    capi.check(cuda_lib.cc_sync(stream), "cc_sync")
    capi.check(cuda_lib.cc_check_wait_expiry(2000, stream), "cc_check_wait_expiry")
    assert cuda_lib.cc_sync(stream) == 7  # CC_ETIMEOUT
    assert b"bounded device wait" in cuda_lib.cc_last_error()
    assert cuda_lib.cc_sync(stream) == 0  # cleared
    psi, _, _ = gpu_cut(w.brickwork(10, 4, 3), 10, [5, 5], "projector", "c128")
    assert_parity(psi.cpu().numpy(), sv.simulate(10, w.brickwork(10, 4, 3)), "c128", "after")
    assert cuda_lib.cc_check_wait_expiry(0, stream) == 2  # CC_ERANGE


@pytest.mark.parametrize("n", [1, 7, (1 << 20) + 5])
def test_copy_to_host(cuda_lib, n):
    src = torch.randn(n, dtype=torch.complex64, device="cuda")
    pinned = torch.empty(n, dtype=torch.complex64, pin_memory=True)
    api.copy_to_host(src, pinned)
    torch.cuda.synchronize()
    assert torch.equal(pinned, src.cpu())
    plain = torch.zeros(n, dtype=torch.complex64)  # pageable: the copy-engine path
    api.copy_to_host(src, plain)
    torch.cuda.synchronize()
    assert torch.equal(plain, src.cpu())


@pytest.mark.parametrize("rot", ["1", "0"])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", ["brickwork", "random", "staircase_t", "rank4"])
def test_rotation_engine_on_and_off(cuda_lib, monkeypatch, rot, prec, kind):
    # Each fused one-qubit matrix as a tangent-form rotation between one-bit
    # phases collected into phase blocks (CUTSIM_ROT=1, the default), or as a
    # complex 2x2 with every phase a table term (CUTSIM_ROT=0): both equal the
    # oracle, on circuits whose fused matrices include diagonal, anti-diagonal
    # and general ones, in the uncut simulation and in the segments of a cut.
    monkeypatch.setenv("CUTSIM_ROT", rot)
    if kind == "brickwork":
        q, segs = 16, [8, 8]
        gates = w.brickwork_cut(q, 10, 5, segs, 3)
    elif kind == "random":
        q, segs = 14, [7, 7]
        gates = w.random_circuit(q, 160, 7)
    elif kind == "staircase_t":
        q, segs = 12, [6, 6]
        gates = w.staircase_depth(q, 3, 2)
    else:
        q, segs = 12, [6, 6]
        gates = w.brickwork_cut(q, 6, 9, segs, 2, boundary_kind="CAN")
    ref = sv.simulate(q, gates)
    u, _ = gpu_uncut(gates, q, prec)
    assert_parity(u.cpu().numpy(), ref, prec, "uncut")
    psi, _, _ = gpu_cut(gates, q, segs, "projector", prec)
    assert_parity(psi.cpu().numpy(), ref, prec, "cut")


@pytest.mark.parametrize("prec", PRECS)
def test_deep_single_pass(cuda_lib, prec):
    # 12 qubits fit one tile, so a depth-1000 brickwork is one pass of ~12000
    # rotations: the scalar factors the rotation engine defers (each
    # rotation's cos or sin) are folded in early enough that the amplitudes,
    # which carry their inverse, stay finite and accurate
    q = 12
    gates = w.brickwork(q, 1000, 4)
    ref = sv.simulate(q, gates)
    u, _ = gpu_uncut(gates, q, prec)
    got = u.cpu().numpy()
    assert np.all(np.isfinite(got))
    # rounding grows like sqrt(G) 2^-24 per amplitude over G ~ 12000 gate
    # applications (~7e-6 in complex64); an overflow would give inf or nan
    tol = 1e-4 if prec == "c64" else 1e-12
    assert rel_err(got, ref) <= tol
    assert 1 - fidelity(got, ref) <= FID_TOL


@pytest.mark.parametrize("segs", [[9, 5], [10, 8], [12, 3], [9, 9]])
@pytest.mark.parametrize("c", [0, 1, 2, 3])
def test_few_term_wide_merge(cuda_lib, monkeypatch, segs, c):
    # complex64 merges of K <= 8 terms with a lower factor of >= 2^9
    # amplitudes run as a direct store stream over 8 x 512 output tiles;
    # CUTSIM_MERGE_WIDE=0 selects the shared-memory tile form, which sums the
    # same terms in the same order
    q = sum(segs)
    gates = w.brickwork_cut(q, 8, 71 + c, segs, c)
    ref = sv.simulate(q, gates)
    monkeypatch.setenv("CUTSIM_MERGE_WIDE", "1")
    psi, _, _ = gpu_cut(gates, q, segs, "projector", "c64", "fma")
    assert_parity(psi.cpu().numpy(), ref, "c64", "wide merge")
    monkeypatch.setenv("CUTSIM_MERGE_WIDE", "0")
    psi_t, _, _ = gpu_cut(gates, q, segs, "projector", "c64", "fma")
    assert torch.equal(psi, psi_t)
