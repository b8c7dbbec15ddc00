"""FP64 verification quantities between two state vectors.

Reconstruction is exact up to rounding (Sec. III), so the reported numbers are
max |a - b| (which sees a global phase error), max |b| (the scale the tolerance
is relative to), the fidelity |<a|b>|^2 and the squared norms.
"""

from __future__ import annotations

import numpy as np


def compare(a: np.ndarray, b: np.ndarray) -> dict:
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    if a.shape != b.shape:
        raise ValueError("shape mismatch")
    inner = np.vdot(a, b)
    na = float(np.vdot(a, a).real)
    nb = float(np.vdot(b, b).real)
    return {
        "max_abs_diff": float(np.max(np.abs(a - b))) if a.size else 0.0,
        "max_abs_b": float(np.max(np.abs(b))) if b.size else 0.0,
        "inner_re": float(inner.real),
        "inner_im": float(inner.imag),
        "norm2_a": na,
        "norm2_b": nb,
        "fidelity": float(abs(inner) ** 2 / (na * nb)) if na > 0 and nb > 0 else 0.0,
    }
