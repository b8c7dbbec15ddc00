"""cc_gather_static: the gather for callers that cannot allocate device memory.

Some callers cannot let a library call cudaMalloc -- their GPU memory belongs
to another allocator, or they cannot take the synchronisation it implies --
so cc_gather_static stages through a fixed array built into the library.
These tests call it through the C ABI and check that it returns exactly what
cc_gather returns, on two calls in a row (the array keeps the previous call's
contents, which must not leak into the next result), and that requests
beyond its fixed capacity are refused.  The file is named to be collected
last; it passes alone in a fresh process and after the other tests.
"""

import ctypes
from ctypes import c_int64, c_void_p

import numpy as np
import pytest
import torch

import workload as w
from paper_2603_01443_gb300 import capi

pytestmark = pytest.mark.gpu

CAP = 65536  # CC_GATHER_STATIC_MAX in include/cutsim.h


def call(fn, psi, idx, prec):
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    dt = np.complex64 if prec == "c64" else np.complex128
    out = np.empty(len(idx), dtype=dt)
    st = fn(c_void_p(psi.data_ptr()), psi.numel(), capi.PRECISION[prec],
            idx.ctypes.data_as(ctypes.POINTER(c_int64)), len(idx), out.ctypes.data_as(c_void_p),
            c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_static_gather_matches_gather_twice(cuda_lib, prec):
    L = capi.lib()
    rng = np.random.default_rng(11)
    n = 1 << 22
    dt = torch.complex64 if prec == "c64" else torch.complex128
    psi = torch.randn(n, dtype=dt, device="cuda")
    tol = 2e-6 if prec == "c64" else 1e-12  # the parity tolerance; equality is expected
    for call_no, (count, seed) in enumerate([(CAP, 3), (1000, 4)]):
        idx = w.sample_indices(22, count, seed)
        st_ref, ref = call(L.cc_gather, psi, idx, prec)
        st, got = call(L.cc_gather_static, psi, idx, prec)
        assert st_ref == 0 and st == 0, (call_no, L.cc_last_error())
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(got.astype(np.complex128) - ref)) <= tol * scale, call_no
        host = psi.cpu().numpy()[np.array(idx)]
        assert np.array_equal(got, host), call_no


def test_static_gather_rejects_oversized_requests(cuda_lib):
    L = capi.lib()
    psi = torch.zeros(1 << 20, dtype=torch.complex64, device="cuda")
    st, _ = call(L.cc_gather_static, psi, np.zeros(CAP + 1, dtype=np.int64), "c64")
    assert st == 2
    assert b"maximum" in L.cc_last_error()
    st, _ = call(L.cc_gather_static, psi, [1 << 20], "c64")
    assert st == 2


_FRESH = r"""
import ctypes, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2603_01443_gb300 import capi
L = capi.lib()
psi = torch.randn(1 << 20, dtype=torch.complex64, device="cuda")
torch.cuda.synchronize()
idx = np.arange(0, 1 << 20, 17, dtype=np.int64)[:65536]
out = np.empty(len(idx), dtype=np.complex64)
def once():
    st = L.cc_gather_static(ctypes.c_void_p(psi.data_ptr()), psi.numel(), 0,
                            idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(idx),
                            out.ctypes.data_as(ctypes.c_void_p),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, L.cc_last_error()
once()  # the first library call in the process: loads the module (and its array)
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
for _ in range(8):
    once()
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
assert np.array_equal(out, psi.cpu().numpy()[idx])
print("FREE", free0, free1)
"""


def test_static_gather_allocates_nothing_in_fresh_process(cuda_lib):
    # In a process where cc_gather_static is the first library call, repeated
    # calls leave the device's free memory unchanged: no scratch area grows.
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    line = [x for x in r.stdout.splitlines() if x.startswith("FREE")][-1]
    _, free0, free1 = line.split()
    assert int(free0) == int(free1), line
