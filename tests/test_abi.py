"""The C-ABI library: it builds, loads, exports every function include/cutsim.h
declares, its struct layouts match the binding, and host-side validation
rejects bad arguments before any device work (no GPU needed)."""

import ctypes
import os
import subprocess
import tempfile
from ctypes import byref, c_double, c_int32, c_int64, c_void_p

import pytest

from paper_2603_01443_gb300 import api, capi

import workload as w


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(capi.LIB_PATH):
        from paper_2603_01443_gb300 import build

        build.build()
    return capi.lib()


def test_header_declares_the_boundary():
    names = capi.header_functions()
    for fn in ("cc_plan_create", "cc_simulate_segments", "cc_merge", "cc_simulate_uncut",
               "cc_uncut_create", "cc_compare", "cc_gather", "cc_last_error"):
        assert fn in names


def test_every_declared_symbol_is_exported(L):
    names = capi.header_functions()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding declares every one of them
    assert sorted(capi._SIGNATURES) == names


def test_struct_layout_matches_c(L):
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "cutsim.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(cc_gate), offsetof(cc_gate, theta),
             sizeof(cc_plan_info_t), offsetof(cc_plan_info_t, seg_offset),
             offsetof(cc_plan_info_t, n_sub), offsetof(cc_plan_info_t, workspace_bytes),
             offsetof(cc_plan_info_t, seg_passes));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.dirname(capi.HEADER), c, "-o", exe])
        vals = [int(x) for x in subprocess.check_output([exe]).split()]
    CI = capi.CPlanInfo
    assert vals == [ctypes.sizeof(capi.CGate), capi.CGate.theta.offset, ctypes.sizeof(CI),
                    CI.seg_offset.offset, CI.n_sub.offset, CI.workspace_bytes.offset,
                    CI.seg_passes.offset]
    assert vals[0] == 40


def test_version_and_last_error(L):
    assert b"sm_103a" in L.cc_version()
    assert isinstance(L.cc_last_error(), bytes)


def _create(L, gates, q, segs, decomp=0, prec=0):
    arr = capi.gate_array(gates)
    sizes = (c_int32 * len(segs))(*segs)
    h = c_void_p()
    st = L.cc_plan_create(arr, len(gates), q, sizes, len(segs), decomp, prec, byref(h))
    return st, h


def test_plan_rejects_bad_arguments(L):
    g = w.brickwork(8, 2, 0)
    assert _create(L, g, 8, [4, 3])[0] == 1          # sizes do not sum to q
    assert _create(L, g, 8, [4, 4, 0])[0] == 1       # empty segment
    assert _create(L, g, 35, [35])[0] == 2           # q too large
    assert _create(L, g, 8, [1] * 8 + [0])[0] == 2   # more than 8 segments
    assert _create(L, g, 8, [4, 4], decomp=7)[0] == 1
    assert _create(L, g, 8, [4, 4], prec=5)[0] == 1
    bad = g + [w.Gate("H", 8)]
    assert _create(L, bad, 8, [4, 4])[0] == 1        # qubit out of range
    assert b"out of range" in L.cc_last_error()
    bad = g + [w.Gate("CZ", 3, 3)]
    assert _create(L, bad, 8, [4, 4])[0] == 1        # two-qubit gate on one qubit
    sizes = (c_int32 * 2)(4, 4)
    assert L.cc_plan_create(capi.gate_array(g), len(g), 8, sizes, 2, 0, 0, None) == 1


def test_plan_rejects_too_many_cuts(L):
    g = w.brickwork_cut(16, 32, 0, [8, 8], 25)
    assert _create(L, g, 16, [8, 8])[0] == 2
    assert b"24" in L.cc_last_error()


def test_plan_rejects_non_adjacent_cut_for_chained_merge(L):
    g = [w.Gate("H", 0), w.Gate("CZ", 0, 8)]
    assert _create(L, g, 9, [3, 3, 3])[0] == 3
    assert b"non-adjacent" in L.cc_last_error()


def test_valid_plan_needs_a_device(L):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    st, _ = _create(L, w.brickwork(8, 2, 0), 8, [4, 4])
    assert st in (6, 8)  # no device / not sm_103


def test_entry_points_reject_null(L):
    assert L.cc_simulate_segments(None, None, 0, None) == 1
    assert L.cc_merge(None, None, 0, None, 0, None, 0, 0, None) == 1
    assert L.cc_simulate_uncut(None, None, 0, None) == 1
    out = (c_double * 6)()
    assert L.cc_compare(None, None, 4, 0, out, None) == 1
    idx = (c_int64 * 1)(5)
    assert L.cc_gather(c_void_p(16), 4, 0, idx, 1, c_void_p(16), None) == 2  # index >= n_amp
    assert L.cc_gather(c_void_p(16), 4, 3, idx, 1, c_void_p(16), None) == 1  # bad precision
    assert L.cc_plan_info(None, None) == 1
    assert L.cc_uncut_info(None, None, None, None) == 1
    L.cc_plan_destroy(None)
    L.cc_uncut_destroy(None)


def _batch_args(items):
    arrs = [capi.gate_array(it.gates) for it in items]
    n = sum(len(it.gates) for it in items)
    gates = (capi.CGate * max(n, 1))()
    goff = (c_int64 * (len(items) + 1))()
    at = 0
    for i, (it, a) in enumerate(zip(items, arrs)):
        goff[i] = at
        for j in range(len(it.gates)):
            gates[at + j] = a[j]
        at += len(it.gates)
    goff[len(items)] = at
    qs = (c_int32 * len(items))(*[it.q for it in items])
    sizes = [s for it in items for s in it.seg_sizes]
    seg_sizes = (c_int32 * len(sizes))(*sizes)
    soff = (c_int32 * (len(items) + 1))()
    at = 0
    for i, it in enumerate(items):
        soff[i] = at
        at += len(it.seg_sizes)
    soff[len(items)] = at
    return gates, goff, qs, seg_sizes, soff


@pytest.mark.parametrize("case", ["no_circuits", "one_segment", "bad_rows", "bad_tile",
                                  "bad_gate", "bad_offsets"])
def test_batch_host_validation(L, case):
    items = w.uneven_batch(3, seed=1, q_range=(12, 14), depths=(4,), c_range=(1, 2))
    gates, goff, qs, seg_sizes, soff = _batch_args(items)
    n, tile, rows = len(items), 0, 0
    if case == "no_circuits":
        n = 0
    elif case == "one_segment":  # circuit 0 as a single segment
        sizes = [items[0].q] + items[1].seg_sizes + items[2].seg_sizes
        seg_sizes = (c_int32 * len(sizes))(*sizes)
        n1, n2 = len(items[1].seg_sizes), len(items[2].seg_sizes)
        soff = (c_int32 * 4)(0, 1, 1 + n1, 1 + n1 + n2)
    elif case == "bad_rows":
        rows = 8
    elif case == "bad_tile":
        tile = 3
    elif case == "bad_gate":
        gates[goff[1] + 2].q0 = 99  # a qubit outside circuit 1
    elif case == "bad_offsets":
        goff[2] = goff[1] - 1
    h = c_void_p()
    st = L.cc_batch_create(gates, goff, n, qs, seg_sizes, soff, 0, 0, tile, rows, byref(h))
    want = {"no_circuits": 2, "one_segment": 1, "bad_rows": 1, "bad_tile": 2, "bad_gate": 1,
            "bad_offsets": 1}[case]
    assert st == want, (case, st, L.cc_last_error())
    assert not h.value
    if case == "bad_gate":
        assert b"circuit 1" in L.cc_last_error()


def test_cut_bits_limit_is_checked_on_the_host(L):
    # 13 SWAP cuts need 26 cut bits > CC_MAX_CUTS (24): rejected before any device work
    gates = [w.Gate("SWAP", 3, 4) for _ in range(13)]
    arr = capi.gate_array(gates)
    segs = (c_int32 * 2)(4, 4)
    h = c_void_p()
    st = L.cc_plan_create(arr, len(gates), 8, segs, 2, 0, 0, byref(h))
    assert st == 2 and b"cut bits" in L.cc_last_error()
    # twelve fit the limit exactly; the plan then fails only for want of a device
    st = L.cc_plan_create(arr, 12, 8, segs, 2, 0, 0, byref(h))
    assert st != 2
    if h.value:
        L.cc_plan_destroy(h)


def test_plan_image_rejects_bad_segment_arguments(L):
    # host-only checks, no device: a segment index outside the plan, and a
    # segment whose qubits plus variant bits exceed the 34-bit vector limit
    g = w.brickwork_cut(8, 4, 0, [4, 4], 2)
    for seg in (-1, 2):
        with pytest.raises(capi.CutsimError, match="segment index out of range"):
            api.plan_program_image(g, 8, [4, 4], seg)
    g = [w.Gate("H", 32), w.Gate("CZ", 32, 33), w.Gate("CZ", 32, 33), w.Gate("CZ", 32, 33)]
    with pytest.raises(capi.CutsimError, match="needs 2"):
        api.plan_program_image(g, 34, [33, 1], 0)


def test_last_error_is_per_thread(L):
    # each thread sees the message of its own last failed call
    import threading

    g = w.brickwork(8, 2, 0)
    msgs = {}
    ready = threading.Barrier(2)

    def fail_with(name, args):
        ready.wait()
        for _ in range(200):
            with pytest.raises(capi.CutsimError):
                api.plan_program_image(*args)
            msgs.setdefault(name, set()).add(L.cc_last_error())

    t1 = threading.Thread(target=fail_with, args=("seg", (g, 8, [4, 4], 5)))
    t2 = threading.Thread(target=fail_with, args=("sum", (g, 8, [4, 3], 0)))
    t1.start(); t2.start(); t1.join(); t2.join()
    assert msgs["seg"] == {b"segment index out of range"}
    assert msgs["sum"] == {b"segment sizes do not sum to q"}


def test_plans_leave_no_compile_threads(L):
    # segments after the first compile on threads that start before the gate
    # items are built; a plan that fails before its programs are compiled (a
    # cut between non-adjacent segments of an 8-segment chain) releases and
    # joins them, as does one that compiles: the process's thread count is
    # the same afterwards
    if not os.path.isdir("/proc/self/task"):
        pytest.skip("needs /proc/self/task")
    bad = [w.Gate("H", 0), w.Gate("CZ", 0, 8)]
    good = w.brickwork_cut(16, 6, 3, [2] * 8, [1] * 7)
    before = len(os.listdir("/proc/self/task"))
    for _ in range(50):
        assert _create(L, bad, 16, [2] * 8)[0] == 3
    for seg in range(8):
        words, _ = api.plan_program_image(good, 16, [2] * 8, seg)
        assert len(words) > 0
    assert len(os.listdir("/proc/self/task")) == before


def test_segment_programs_do_not_depend_on_thread_timing(L):
    # segments compile on concurrent threads: repeated plans of the same
    # circuit give byte-identical images for every segment
    segs = [4, 5, 4, 5]
    g = w.brickwork_cut(18, 10, 11, segs, [2, 3, 2])
    first = [api.plan_program_image(g, 18, segs, s) for s in range(4)]
    for _ in range(10):
        for s in range(4):
            words, reals = api.plan_program_image(g, 18, segs, s)
            assert words.tobytes() == first[s][0].tobytes()
            assert reals.tobytes() == first[s][1].tobytes()
