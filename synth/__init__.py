"""Seeded synthetic SCCS inputs shared by the tests, the benchmark and the oracle checks.

This package only draws data (patients, eras, offsets, drug indicators, event counts).
It holds none of the fitting method's arithmetic, and it imports neither the CUDA
package nor the oracle.
"""
from .sccs_synth import (  # noqa: F401
    SCCSData,
    make_dataset,
    tiny_fit_config,
    mid_fit_config,
    paper_scale_config,
    large_columns_config,
    batched_fit_configs,
    batched_fit_plan,
    batched_fit_one,
    serving_pool_plan,
    serving_outcome,
    serving_requests,
    PRIOR_VARIANCE_GRID,
    cv_folds,
    fold_weights,
    bootstrap_weights,
    CONFIGS,
)
