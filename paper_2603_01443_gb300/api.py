"""Python face of the C ABI: plans, device buffers (torch) and streams.

Nothing here computes: every step of the path is a call into
``libcutsim.so``.  Torch only allocates device memory and provides the stream
handle passed to each call.
"""

from __future__ import annotations

import ctypes
from ctypes import POINTER, byref, c_double, c_int32, c_int64, c_void_p
from typing import Optional, Sequence

import numpy as np
import torch

from . import capi

TORCH_DTYPE = {"c64": torch.complex64, "c128": torch.complex128}
NUMPY_DTYPE = {"c64": np.complex64, "c128": np.complex128}
AMP_BYTES = {"c64": 8, "c128": 16}


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _nbytes(t: Optional[torch.Tensor]) -> int:
    return 0 if t is None else t.numel() * t.element_size()


class CutPlan:
    """Preprocessing (Algorithm 1) of one circuit and partition.

    ``gates`` is a sequence of gates (kind, q0, q1, theta, phi, lam) or a
    ``capi.GateArray`` packed once beforehand."""

    def __init__(self, gates: Sequence, q: int, seg_sizes: Sequence[int],
                 decomp: str = "projector", precision: str = "c64"):
        L = capi.lib()
        self.q = q
        self.precision = precision
        self.decomp = decomp
        arr = gates if isinstance(gates, capi.GateArray) else capi.GateArray(gates)
        sizes = (c_int32 * len(seg_sizes))(*seg_sizes)
        h = c_void_p()
        capi.check(L.cc_plan_create(arr.data, arr.n, q, sizes, len(seg_sizes),
                                    capi.DECOMP[decomp], capi.PRECISION[precision], byref(h)),
                   "cc_plan_create")
        self._h = h
        info = capi.CPlanInfo()
        capi.check(L.cc_plan_info(self._h, byref(info)), "cc_plan_info")
        n = info.n_seg
        self.info = {
            "q": info.q, "n_seg": n, "c_total": info.c_total,
            "seg_qubits": list(info.seg_qubits[:n]), "seg_start": list(info.seg_start[:n]),
            "seg_cuts": list(info.seg_cuts[:n]), "seg_passes": list(info.seg_passes[:n]),
            "seg_ops": list(info.seg_ops[:n]), "seg_offset": list(info.seg_offset[:n]),
            "n_sub": info.n_sub, "seg_buf_bytes": info.seg_buf_bytes,
            "psi_bytes": info.psi_bytes, "workspace_bytes": info.workspace_bytes,
            "table_bytes": info.table_bytes, "cut_bits": info.cut_bits,
        }

    def close(self):
        if getattr(self, "_h", None):
            capi.lib().cc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cut(self, j: int):
        vals = [c_int32() for _ in range(5)]
        capi.check(capi.lib().cc_plan_cut(self._h, j, *[byref(v) for v in vals]), "cc_plan_cut")
        q0, q1, kind, s0, s1 = (v.value for v in vals)
        return {"q0": q0, "q1": q1, "kind": kind, "seg0": s0, "seg1": s1}

    # buffers ------------------------------------------------------------
    def _alloc(self, nbytes: int, device) -> torch.Tensor:
        n = max(1, nbytes // AMP_BYTES[self.precision])
        return torch.empty(n, dtype=TORCH_DTYPE[self.precision], device=device)

    def alloc_seg_buf(self, device="cuda"):
        return self._alloc(self.info["seg_buf_bytes"], device)

    def alloc_psi(self, device="cuda"):
        return self._alloc(self.info["psi_bytes"], device)

    def alloc_workspace(self, device="cuda"):
        if self.info["workspace_bytes"] == 0:
            return None
        return self._alloc(self.info["workspace_bytes"], device)

    def segment_view(self, seg_buf: torch.Tensor, i: int) -> torch.Tensor:
        """Segment i's variants as a [2^{c_i}, 2^{q_i}] view of seg_buf."""
        off = self.info["seg_offset"][i]
        nv, na = 1 << self.info["seg_cuts"][i], 1 << self.info["seg_qubits"][i]
        return seg_buf[off:off + nv * na].view(nv, na)

    # stages -------------------------------------------------------------
    def simulate_segments(self, seg_buf: torch.Tensor, stream=None) -> None:
        capi.check(capi.lib().cc_simulate_segments(self._h, _ptr(seg_buf), _nbytes(seg_buf),
                                                   _stream(stream)), "cc_simulate_segments")

    def merge(self, seg_buf: torch.Tensor, psi: torch.Tensor, workspace=None, form="auto",
              stream=None) -> None:
        capi.check(capi.lib().cc_merge(self._h, _ptr(seg_buf), _nbytes(seg_buf), _ptr(psi),
                                       _nbytes(psi), _ptr(workspace), _nbytes(workspace),
                                       capi.MERGE_FORM[form], _stream(stream)), "cc_merge")


def program_image(gates: Sequence, q: int, precision: str = "c64", tile_bits: int = 0):
    """The uncut gate program of a circuit as (int64 words, float64 reals), as
    cc_program_image lays it out; host work, no device needed."""
    L = capi.lib()
    arr = gates if isinstance(gates, capi.GateArray) else capi.GateArray(gates)
    nw, nr = c_int64(0), c_int64(0)
    capi.check(L.cc_program_image(arr.data, arr.n, q, capi.PRECISION[precision], tile_bits,
                                  None, byref(nw), None, byref(nr)), "cc_program_image")
    words = np.zeros(max(nw.value, 1), dtype=np.int64)
    reals = np.zeros(max(nr.value, 1), dtype=np.float64)
    capi.check(L.cc_program_image(arr.data, arr.n, q, capi.PRECISION[precision], tile_bits,
                                  words.ctypes.data_as(POINTER(c_int64)), byref(nw),
                                  reals.ctypes.data_as(POINTER(c_double)), byref(nr)),
               "cc_program_image")
    return words[:nw.value], reals[:nr.value]


def plan_program_image(gates: Sequence, q: int, seg_sizes: Sequence[int], seg: int,
                       decomp: str = "projector", precision: str = "c64", tile_bits: int = 0):
    """Segment `seg`'s gate program of the plan for these arguments, as
    (int64 words, float64 reals) laid out by cc_plan_program_image; host work,
    no device needed."""
    L = capi.lib()
    arr = gates if isinstance(gates, capi.GateArray) else capi.GateArray(gates)
    sizes = (c_int32 * len(seg_sizes))(*seg_sizes)
    args = (arr.data, arr.n, q, sizes, len(seg_sizes), capi.DECOMP[decomp],
            capi.PRECISION[precision], tile_bits, seg)
    nw, nr = c_int64(0), c_int64(0)
    capi.check(L.cc_plan_program_image(*args, None, byref(nw), None, byref(nr)),
               "cc_plan_program_image")
    words = np.zeros(max(nw.value, 1), dtype=np.int64)
    reals = np.zeros(max(nr.value, 1), dtype=np.float64)
    capi.check(L.cc_plan_program_image(*args, words.ctypes.data_as(POINTER(c_int64)), byref(nw),
                                       reals.ctypes.data_as(POINTER(c_double)), byref(nr)),
               "cc_plan_program_image")
    return words[:nw.value], reals[:nr.value]


class UncutPlan:
    """Pass plan of the uncut simulation (T_orig)."""

    def __init__(self, gates: Sequence, q: int, precision: str = "c64"):
        L = capi.lib()
        self.q = q
        self.precision = precision
        arr = gates if isinstance(gates, capi.GateArray) else capi.GateArray(gates)
        h = c_void_p()
        capi.check(L.cc_uncut_create(arr.data, arr.n, q, capi.PRECISION[precision], byref(h)),
                   "cc_uncut_create")
        self._h = h
        npass, nops, tb = c_int32(), c_int32(), c_int32()
        capi.check(L.cc_uncut_info(self._h, byref(npass), byref(nops), byref(tb)), "cc_uncut_info")
        self.info = {"n_passes": npass.value, "n_ops": nops.value, "tile_bits": tb.value}

    def close(self):
        if getattr(self, "_h", None):
            capi.lib().cc_uncut_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alloc_psi(self, device="cuda"):
        return torch.empty(1 << self.q, dtype=TORCH_DTYPE[self.precision], device=device)

    def simulate(self, psi: torch.Tensor, stream=None) -> None:
        capi.check(capi.lib().cc_simulate_uncut(self._h, _ptr(psi), _nbytes(psi), _stream(stream)),
                   "cc_simulate_uncut")


def compare(a: torch.Tensor, b: torch.Tensor, precision: str, stream=None) -> dict:
    """FP64 device reductions between two state vectors (synchronizes)."""
    if a.numel() != b.numel():
        raise ValueError("size mismatch")
    out = (c_double * 6)()
    capi.check(capi.lib().cc_compare(_ptr(a), _ptr(b), a.numel(), capi.PRECISION[precision], out,
                                     _stream(stream)), "cc_compare")
    re, im, na, nb = out[2], out[3], out[4], out[5]
    return {
        "max_abs_diff": out[0], "max_abs_b": out[1], "inner_re": re, "inner_im": im,
        "norm2_a": na, "norm2_b": nb,
        "fidelity": (re * re + im * im) / (na * nb) if na > 0 and nb > 0 else 0.0,
    }


def copy_to_host(src: torch.Tensor, host: torch.Tensor, stream=None) -> None:
    """src (device) -> host (a pinned CPU tensor of the same size), asynchronous."""
    if host.is_cuda or not host.is_contiguous() or _nbytes(host) < _nbytes(src):
        raise ValueError("host must be a contiguous CPU tensor at least as large as src")
    capi.check(capi.lib().cc_copy_to_host(_ptr(src), host.data_ptr(), _nbytes(src),
                                          _stream(stream)), "cc_copy_to_host")


def gather(psi: torch.Tensor, idx: Sequence[int], precision: str, stream=None) -> np.ndarray:
    """psi[idx] copied to the host (synchronizes)."""
    idx_arr = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    out = np.empty(len(idx_arr), dtype=NUMPY_DTYPE[precision])
    capi.check(capi.lib().cc_gather(
        _ptr(psi), psi.numel(), capi.PRECISION[precision],
        idx_arr.ctypes.data_as(ctypes.POINTER(c_int64)), len(idx_arr),
        out.ctypes.data_as(c_void_p), _stream(stream)), "cc_gather")
    return out


def cut_simulate(gates, q, seg_sizes, decomp="projector", precision="c64", form="auto",
                 stream=None):
    """Preprocess, simulate segments and merge; returns (psi on the device, plan)."""
    plan = CutPlan(gates, q, seg_sizes, decomp, precision)
    seg = plan.alloc_seg_buf()
    psi = plan.alloc_psi()
    ws = plan.alloc_workspace()
    plan.simulate_segments(seg, stream)
    plan.merge(seg, psi, ws, form, stream)
    return psi, plan


class Batch:
    """Many independent circuits cut, simulated and merged together.

    ``circuits`` is a sequence of ``(gates, q, seg_sizes)``; gates may be a
    sequence of gates or a ``capi.GateArray``.  All segment passes of all
    circuits run in one persistent launch, then one merge launch per chain
    level; ``capture`` records that sequence into a CUDA graph."""

    def __init__(self, circuits, decomp: str = "projector", precision: str = "c64",
                 tile_bits: int = 0, merge_rows: int = 0):
        L = capi.lib()
        self.precision = precision
        arrays = [g if isinstance(g, capi.GateArray) else capi.GateArray(g) for g, _, _ in circuits]
        n_g = sum(a.n for a in arrays)
        gates = (capi.CGate * max(n_g, 1))()
        goff = (c_int64 * (len(circuits) + 1))()
        at = 0
        for i, a in enumerate(arrays):
            goff[i] = at
            ctypes.memmove(ctypes.byref(gates, at * ctypes.sizeof(capi.CGate)), a.data,
                           a.n * ctypes.sizeof(capi.CGate))
            at += a.n
        goff[len(circuits)] = at
        qs = (c_int32 * len(circuits))(*[q for _, q, _ in circuits])
        sizes = [s for _, _, segs in circuits for s in segs]
        seg_sizes = (c_int32 * max(len(sizes), 1))(*sizes)
        soff = (c_int32 * (len(circuits) + 1))()
        at = 0
        for i, (_, _, segs) in enumerate(circuits):
            soff[i] = at
            at += len(segs)
        soff[len(circuits)] = at
        h = c_void_p()
        capi.check(L.cc_batch_create(gates, goff, len(circuits), qs, seg_sizes, soff,
                                     capi.DECOMP[decomp], capi.PRECISION[precision], tile_bits,
                                     merge_rows, byref(h)), "cc_batch_create")
        self._h = h
        self.n_circ = len(circuits)
        self._refresh_info()
        self.circuits = []
        for i in range(self.n_circ):
            off, q, c, ns = c_int64(), c_int32(), c_int32(), c_int64()
            capi.check(L.cc_batch_circuit(self._h, i, byref(off), byref(q), byref(c), byref(ns)),
                       "cc_batch_circuit")
            self.circuits.append({"psi_offset": off.value, "q": q.value, "c_total": c.value,
                                  "n_sub": ns.value})

    def _refresh_info(self):
        info = capi.CBatchInfo()
        capi.check(capi.lib().cc_batch_info(self._h, byref(info)), "cc_batch_info")
        self.info = {f: getattr(info, f) for f, _ in capi.CBatchInfo._fields_}

    def close(self):
        if getattr(self, "_h", None):
            capi.lib().cc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _alloc(self, nbytes: int, device) -> torch.Tensor:
        n = max(1, nbytes // AMP_BYTES[self.precision])
        return torch.empty(n, dtype=TORCH_DTYPE[self.precision], device=device)

    def alloc_buffers(self, device="cuda"):
        """(seg_buf, psi, workspace) sized for the batch; workspace may be None."""
        ws = self.info["workspace_bytes"]
        return (self._alloc(self.info["seg_buf_bytes"], device),
                self._alloc(self.info["psi_bytes"], device),
                self._alloc(ws, device) if ws else None)

    def alloc_stamps(self, device="cuda") -> torch.Tensor:
        return torch.zeros(self.n_circ + 1, dtype=torch.int64, device=device)

    def psi_view(self, psi: torch.Tensor, i: int) -> torch.Tensor:
        c = self.circuits[i]
        return psi[c["psi_offset"]:c["psi_offset"] + (1 << c["q"])]

    def _args(self, seg, psi, ws, stamps):
        return (_ptr(seg), _nbytes(seg), _ptr(psi), _nbytes(psi), _ptr(ws), _nbytes(ws),
                _ptr(stamps))

    def run(self, seg, psi, ws=None, stamps=None, stream=None) -> None:
        capi.check(capi.lib().cc_batch_run(self._h, *self._args(seg, psi, ws, stamps),
                                           _stream(stream)), "cc_batch_run")

    def capture(self, seg, psi, ws=None, stamps=None, stream=None) -> None:
        capi.check(capi.lib().cc_batch_capture(self._h, *self._args(seg, psi, ws, stamps),
                                               _stream(stream)), "cc_batch_capture")

    def launch(self, stream=None) -> None:
        capi.check(capi.lib().cc_batch_launch(self._h, _stream(stream)), "cc_batch_launch")

    def autotune(self, seg, psi, ws=None, stream=None):
        """Time every (tile bits, merge rows) candidate, keep the fastest; returns the table."""
        n_max = 16
        tb, rows = (c_int32 * n_max)(), (c_int32 * n_max)()
        ms = (ctypes.c_float * n_max)()
        n = c_int32()
        capi.check(capi.lib().cc_batch_autotune(
            self._h, _ptr(seg), _nbytes(seg), _ptr(psi), _nbytes(psi), _ptr(ws), _nbytes(ws),
            _stream(stream), n_max, byref(n), tb, rows, ms), "cc_batch_autotune")
        self._refresh_info()
        return [{"tile_bits": tb[i], "merge_rows": rows[i], "ms": ms[i]} for i in range(n.value)]
