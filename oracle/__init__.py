"""Plain FP64 CPU oracle of the single-chain slip-spring model (arXiv:1106.2899).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg use it to check and time the CUDA library.  It shares no code
with that library and the product path never imports it.

Functions whose parity is not pinned by a `-m "not gpu"` test: none (each
docstring in oracle.py and each comment in ss_oracle.c names its pin).
"""
from .oracle import (  # noqa: F401
    CORR_P,
    OPS_CATEGORIES,
    Ensemble,
    Params,
    corr_counts,
    corr_lags,
    corr_series,
    decode_block,
    init_chain,
    norm_ppf,
    op_counts,
    philox,
    step_chain,
    stress,
)
