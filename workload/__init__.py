"""Seeded synthetic circuit generators.

This package is the one module that both the CUDA path and the FP64 oracle
import.  It only draws gate lists and sample indices from a counter-based
generator; it holds none of the cutting method's arithmetic (no gate matrices,
no decompositions, no state vectors).
"""

from .circuits import (  # noqa: F401
    Gate,
    SplitMix64,
    GATE_KINDS,
    ONE_QUBIT_KINDS,
    TWO_QUBIT_KINDS,
    RANK4_KINDS,
    ALL_TWO_QUBIT_KINDS,
    equal_partition,
    cut_layers,
    brickwork,
    brickwork_cut,
    staircase,
    staircase_depth,
    ghz,
    graph_state,
    random_circuit,
    sample_indices,
    split_cuts,
    BatchItem,
    uneven_sizes,
    uneven_batch,
)
