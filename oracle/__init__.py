"""FP64 CPU oracle for circuit cutting in state-vector simulation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2603_01443_gb300``) never imports or calls it and shares no code with
it: gate matrices, decompositions, simulation and merging are all written out
here independently, in plain numpy complex128, in the paper's order and
notation, with no blocking, fusion or reordering.

Modules
-------
statevector  -- gate definitions and gate-by-gate state-vector simulation (the
                uncut reference T_orig = O(2^q D), Sec. III.A).
cutting      -- Algorithm 1 (preprocessing), Algorithm 2 (subcircuit
                simulation), Algorithm 3 (merging) and a per-amplitude form of
                the Algorithm 3 sum for vectors too large to materialise.
thresholds   -- the cost-model thresholds (Eqs. 12-15, Table II).
reductions   -- the FP64 verification quantities (max |d psi|, fidelity, norm).
mlp          -- the planner network's forward pass, loss gradient and Adam
                steps in FP64 (pinned by finite differences and closed forms).

Parity status: every function is pinned by the ``-m "not gpu"`` tests (closed
forms, brute-force unitaries, cut == uncut, the Table II values); none is
"parity unpinned".
"""

from . import statevector, cutting, thresholds, reductions, mlp  # noqa: F401
