"""ctypes binding of ``libcutsim.so`` -- argument marshalling only.

Every function of ``include/cutsim.h`` is declared here with the same name.
The library must have been built (``python -m paper_2603_01443_gb300.build``
or ``__graft_entry__.build()``); loading fails loudly otherwise, and there is
no fallback of any kind.
"""

from __future__ import annotations

import ctypes
import os
import threading
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_uint64, c_void_p

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libcutsim.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "cutsim.h")

CC_MAX_SEGMENTS = 8

STATUS = {
    0: "CC_OK", 1: "CC_EINVAL", 2: "CC_ERANGE", 3: "CC_EUNSUPPORTED", 4: "CC_ENOMEM",
    5: "CC_EBUFSIZE", 6: "CC_ECUDA", 7: "CC_ETIMEOUT", 8: "CC_EDEVICE",
}
PRECISION = {"c64": 0, "c128": 1}
DECOMP = {"projector": 0, "s_sdg": 1}
MERGE_FORM = {"auto": 0, "fma": 1, "tf32x3": 2, "bf16x3": 3, "ozaki": 4, "f16x3": 5}
GATE_KIND = {"U3": 0, "H": 1, "X": 2, "Z": 3, "S": 4, "SDG": 5, "T": 6, "TDG": 7, "CZ": 8, "CX": 9,
             "SWAP": 10, "ISWAP": 11, "CAN": 12}
TWO_QUBIT = ("CZ", "CX", "SWAP", "ISWAP", "CAN")


class CGate(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("q0", c_int32), ("q1", c_int32), ("reserved", c_int32),
                ("theta", c_double), ("phi", c_double), ("lam", c_double)]


class CPlanInfo(ctypes.Structure):
    _fields_ = [
        ("q", c_int32), ("n_seg", c_int32), ("c_total", c_int32), ("precision", c_int32),
        ("decomp", c_int32),
        ("seg_qubits", c_int32 * CC_MAX_SEGMENTS),
        ("seg_start", c_int32 * CC_MAX_SEGMENTS),
        ("seg_cuts", c_int32 * CC_MAX_SEGMENTS),
        ("seg_passes", c_int32 * CC_MAX_SEGMENTS),
        ("seg_ops", c_int32 * CC_MAX_SEGMENTS),
        ("seg_offset", c_int64 * CC_MAX_SEGMENTS),
        ("n_sub", c_int64),
        ("seg_buf_bytes", c_uint64), ("psi_bytes", c_uint64), ("workspace_bytes", c_uint64),
        ("table_bytes", c_uint64), ("cut_bits", c_int32), ("reserved0", c_int32),
    ]


class CBatchInfo(ctypes.Structure):
    _fields_ = [
        ("n_circ", c_int32), ("precision", c_int32), ("tile_bits", c_int32),
        ("merge_rows", c_int32), ("n_jobs", c_int32), ("merge_levels", c_int32),
        ("n_items", c_int64), ("n_sub", c_int64),
        ("seg_buf_bytes", c_uint64), ("psi_bytes", c_uint64), ("workspace_bytes", c_uint64),
        ("block", c_int32), ("grid", c_int32),
    ]


class CutsimError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {message}")


_SIGNATURES = {
    "cc_plan_create": (c_int32, [POINTER(CGate), c_int32, c_int32, POINTER(c_int32), c_int32,
                                 c_int32, c_int32, POINTER(c_void_p)]),
    "cc_plan_info": (c_int32, [c_void_p, POINTER(CPlanInfo)]),
    "cc_plan_cut": (c_int32, [c_void_p, c_int32, POINTER(c_int32), POINTER(c_int32),
                              POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)]),
    "cc_plan_destroy": (None, [c_void_p]),
    "cc_simulate_segments": (c_int32, [c_void_p, c_void_p, c_uint64, c_void_p]),
    "cc_merge": (c_int32, [c_void_p, c_void_p, c_uint64, c_void_p, c_uint64, c_void_p, c_uint64,
                           c_int32, c_void_p]),
    "cc_uncut_create": (c_int32, [POINTER(CGate), c_int32, c_int32, c_int32, POINTER(c_void_p)]),
    "cc_uncut_info": (c_int32, [c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)]),
    "cc_program_image": (c_int32, [POINTER(CGate), c_int32, c_int32, c_int32, c_int32,
                                   POINTER(c_int64), POINTER(c_int64), POINTER(c_double),
                                   POINTER(c_int64)]),
    "cc_plan_program_image": (c_int32, [POINTER(CGate), c_int32, c_int32, POINTER(c_int32),
                                        c_int32, c_int32, c_int32, c_int32, c_int32,
                                        POINTER(c_int64), POINTER(c_int64), POINTER(c_double),
                                        POINTER(c_int64)]),
    "cc_simulate_uncut": (c_int32, [c_void_p, c_void_p, c_uint64, c_void_p]),
    "cc_uncut_destroy": (None, [c_void_p]),
    "cc_compare": (c_int32, [c_void_p, c_void_p, c_int64, c_int32, POINTER(c_double), c_void_p]),
    "cc_gather": (c_int32, [c_void_p, c_int64, c_int32, POINTER(c_int64), c_int64, c_void_p,
                            c_void_p]),
    "cc_gather_static": (c_int32, [c_void_p, c_int64, c_int32, POINTER(c_int64), c_int64,
                                   c_void_p, c_void_p]),
    "cc_kak_gates": (c_int32, [POINTER(c_double), c_int32, c_int32, POINTER(CGate),
                               POINTER(c_int32)]),
    "cc_batch_create": (c_int32, [POINTER(CGate), POINTER(c_int64), c_int32, POINTER(c_int32),
                                  POINTER(c_int32), POINTER(c_int32), c_int32, c_int32, c_int32,
                                  c_int32, POINTER(c_void_p)]),
    "cc_batch_info": (c_int32, [c_void_p, POINTER(CBatchInfo)]),
    "cc_batch_circuit": (c_int32, [c_void_p, c_int32, POINTER(c_int64), POINTER(c_int32),
                                   POINTER(c_int32), POINTER(c_int64)]),
    "cc_batch_run": (c_int32, [c_void_p, c_void_p, c_uint64, c_void_p, c_uint64, c_void_p,
                               c_uint64, c_void_p, c_void_p]),
    "cc_batch_capture": (c_int32, [c_void_p, c_void_p, c_uint64, c_void_p, c_uint64, c_void_p,
                                   c_uint64, c_void_p, c_void_p]),
    "cc_batch_launch": (c_int32, [c_void_p, c_void_p]),
    "cc_batch_autotune": (c_int32, [c_void_p, c_void_p, c_uint64, c_void_p, c_uint64, c_void_p,
                                    c_uint64, c_void_p, c_int32, POINTER(c_int32),
                                    POINTER(c_int32), POINTER(c_int32), POINTER(ctypes.c_float)]),
    "cc_batch_destroy": (None, [c_void_p]),
    "cc_mlp_param_count": (c_int64, [POINTER(c_int32), c_int32]),
    "cc_mlp_work_bytes": (c_uint64, [POINTER(c_int32), c_int32, c_int64]),
    "cc_mlp_forward": (c_int32, [POINTER(c_int32), c_int32, c_void_p, c_void_p, c_int64, c_void_p,
                                 c_void_p, c_uint64, c_void_p]),
    "cc_mlp_train": (c_int32, [POINTER(c_int32), c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_int64, c_int32, ctypes.c_float, c_void_p, c_void_p,
                               c_uint64, c_void_p]),
    "cc_check_wait_expiry": (c_int32, [c_int32, c_void_p]),
    "cc_copy_to_host": (c_int32, [c_void_p, c_void_p, c_uint64, c_void_p]),
    "cc_sync": (c_int32, [c_void_p]),
    "cc_last_error": (c_char_p, []),
    "cc_version": (c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def lib():
    """The loaded library (loaded once); raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -m paper_2603_01443_gb300.build)")
            handle = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def check(status: int, where: str) -> None:
    if status != 0:
        raise CutsimError(status, where, lib().cc_last_error().decode(errors="replace"))


class GateArray:
    """A circuit packed once into a cc_gate array (reusable across calls)."""

    def __init__(self, gates):
        self.n = len(gates)
        self.data = gate_array(gates)


def gate_array(gates):
    """Pack gates (objects with kind, q0, q1, theta, phi, lam) into a cc_gate array."""
    arr = (CGate * max(len(gates), 1))()
    for i, g in enumerate(gates):
        arr[i].kind = GATE_KIND[g.kind]
        arr[i].q0 = g.q0
        arr[i].q1 = g.q1 if g.kind in TWO_QUBIT else -1
        arr[i].reserved = 0
        arr[i].theta = g.theta
        arr[i].phi = g.phi
        arr[i].lam = g.lam
    return arr


def header_functions(path: str = HEADER):
    """Names of the functions declared in include/cutsim.h."""
    import re

    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cc_[a-z_0-9]+)\s*\(", text)))
