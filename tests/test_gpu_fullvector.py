"""Full-vector parity with the FP64 oracle at q = 24 and q = 26.

The oracle's state is its own literal Algorithms 1-3 in complex128 (every
subcircuit simulated from |0>, every Kronecker term summed), which the CPU
pins tie to the uncut definition (cut == uncut, closed forms).  Every one of
the 2^q amplitudes of the GPU result is compared, relative to max |psi|, and
the fidelity over the whole vector is checked, in complex64 (AUTO merge: the
tensor-core 3xTF32 form at these K) and complex128.
"""

import pytest
import torch

import workload as w
from oracle import cutting as ct
from gpu_util import TOL, assert_parity, gpu_cut

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("q,n,c,prec,form,decomp", [
    (24, 2, 6, "c64", "auto", "projector"),
    (26, 2, 4, "c64", "auto", "s_sdg"),
    (24, 2, 6, "c128", "auto", "projector"),
    (26, 2, 4, "c128", "auto", "projector"),
    (24, 3, 4, "c64", "auto", "projector"),
    (24, 3, 4, "c128", "auto", "s_sdg"),
])
def test_full_vector_vs_oracle(cuda_lib, q, n, c, prec, form, decomp):
    segs = w.equal_partition(q, n)
    gates = w.brickwork_cut(q, 16, 100 + q + c, segs, w.split_cuts(c, n))
    psi, _, plan = gpu_cut(gates, q, segs, decomp, prec, form)
    assert plan.info["c_total"] == c
    got = psi.cpu().numpy()
    del psi
    torch.cuda.empty_cache()
    ref, _, _ = ct.cut_simulate(q, gates, segs, decomp)
    assert_parity(got, ref, prec, f"q={q} n={n} c={c} {prec} {form}")
