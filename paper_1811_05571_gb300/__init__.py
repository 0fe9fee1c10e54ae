"""GB300 (sm_103a) norm-1 ADMM for g = Hu + w in its consensus, sectioning and
consensus-and-sectioning forms (Heredia-Juesas et al., Sections III-A..C).

The numerical work lives in the CUDA library ``libadmm.so`` (C ABI in
``include/admm.h``); this package only builds it, loads it and marshals
arguments.  Importing is cheap; the library is loaded (and built from
``csrc/`` when a source is newer than the binary) on first use, and any
failure to build or load raises instead of falling back to other code.
"""

from ._binding import (  # noqa: F401
    ADMM_C64, ADMM_C128, ADMM_OK, ADMM_EINVAL, ADMM_ENOMEM, ADMM_ECUDA, ADMM_ENOTPD,
    ADMM_ENONFINITE, ADMM_ETIMEOUT, ADMM_EUNSUPPORTED, ADMM_EDIVERGED,
    ADMM_OPT_TIMEOUT_NS, ADMM_OPT_HIST_CAP, ADMM_OPT_BARRIER_EXTRA, ADMM_OPT_TRACE_ITERS,
    ADMM_OPT_L2_KEEP_BYTES, ADMM_OPT_H_FP16, ADMM_OPT_L2_PREFETCH_BYTES, ADMM_OPT_RECORD_ITERS,
    ADMM_OPT_DIR_FACTOR_PASS, ABI_VERSION,
    ADMM_FORM_LEMMA, ADMM_FORM_DIRECT, ADMM_FORM_AUTO,
    AdmmError, load, library_path,
    admm_abi_version, admm_strerror, admm_partition, admm_comm_elements, admm_plan, admm_setup, admm_setup_form, admm_iterate,
    admm_solve, admm_get_v, admm_get_u, admm_get_residuals, admm_set_g, admm_set_lambda,
    admm_set_rho, admm_reset, admm_get_state, admm_set_state, admm_get_info, admm_set_option,
    admm_get_trace, admm_status, admm_destroy, admm_solve_small_noalloc,
    admm_batch_setup, admm_batch_set_g, admm_batch_iterate, admm_batch_get_v, admm_batch_get_residuals,
    admm_batch_reset, admm_batch_forward, admm_batch_adjoint, admm_batch_status, admm_batch_get_info,
    admm_batch_destroy, admm_batch_record, admm_batch_backward, admm_batch_tune, admm_tune, admm_backward,
    admm_group_setup, admm_group_iterate, admm_group_info, admm_group_destroy,
)
from .solver import BatchSolver, Group, UnrolledADMM  # noqa: F401
from .solver import Solver  # noqa: F401
