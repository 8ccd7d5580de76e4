"""Incremental all-pairs SimRank on one GB300 (sm_103a).

The computation lives in the CUDA library ``libsimrank.so`` (C ABI in
``include/simrank.h``); this package is its thin Python binding.
"""
from ._binding import (  # noqa: F401
    SimRank,
    MultiSimRank,
    SimrankError,
    Config,
    Update,
    Stats,
    SIGNATURES,
    LIB_PATH,
    lib,
    default_config,
    updates_array,
    plan_batch,
    MODE_DENSE,
    MODE_COLUMN,
    APPLY_UNIT,
    APPLY_SINK_BLOCKS,
    APPLY_ONE_SHOT,
    SUPDATE_FUSED,
    SUPDATE_PLAIN,
    INIT_SWEEPS,
    INIT_FOREST,
    INIT_COMPONENTS,
)
