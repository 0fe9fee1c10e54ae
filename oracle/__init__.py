"""FP64 CPU oracle for the consensus / sectioning / consensus-and-sectioning
norm-1 ADMM (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it and
shares no code with it.
"""

from .admm_fp64 import (  # noqa: F401
    OracleResult,
    soft_threshold,
    balanced_blocks,
    BlockSolver,
    lasso_admm,
    consensus_admm,
    sectioning_admm,
    cs_admm,
    run_split,
    stop_test,
    threshold_margin,
    comm_elements,
    lemma_applies,
)
from . import quantize  # noqa: F401,E402
from . import adjoint  # noqa: F401,E402
