"""GB300 (sm_103a) BSCCS cyclic-coordinate-descent MAP fit (arXiv 1208.0945, Section 2).

The compute lives in libsccs.so (hand-written CUDA behind the C ABI of include/sccs.h);
`sccs` is its ctypes binding.  Importing this package fails if the library is not built.
"""
from .sccs import (  # noqa: F401
    EXPORTED,
    FitServer,
    sccs_poll,
    sccs_server_create,
    sccs_server_destroy,
    sccs_server_get_stats,
    sccs_submit,
    SCCSError,
    SCCSModel,
    sccs_check_wait_timeout,
    sccs_create,
    sccs_destroy,
    sccs_fit,
    sccs_fit_batch,
    sccs_get_beta,
    sccs_get_info,
    sccs_grad_hess,
    sccs_grad_hess_noalloc,
    sccs_heldout_loglik,
    sccs_last_error,
    sccs_logpost,
    sccs_set_prior,
    sccs_version,
)
