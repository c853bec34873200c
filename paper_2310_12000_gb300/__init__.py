"""Python binding of libvl, the GB300 iterative Vecchia-Laplace library.

Argument marshalling only: every computation runs in the CUDA kernels behind the
C ABI declared in ``include/vl.h``. Arrays may be numpy arrays (host) or torch
tensors (host or CUDA); they are passed by pointer. The first call that needs the
library (``library()``, ``Context()``) loads ``_build/libvl.so`` and raises ImportError
if it has not been built (there is no CPU fallback);
``paper_2310_12000_gb300.build.build()`` compiles it with nvcc.

The calls mirror the ABI and the paper's problem statement:

    ctx = Context()                                       # device memory, stream
    fac = ctx.build_factor(locs, order, cov, sigma2, rho, m)     # Section 2.1
    st = fac.find_mode(lik, y, F)                         # Eq. newton
    lml = st.log_marglik()                                # Eqs. VLA_loss, def_SLQ
    mean, var = st.pred_var(test_locs)                    # Algorithm simAlgo
"""
from __future__ import annotations

from ._lib import (COV_EXPONENTIAL, COV_MATERN15, FP32_REFINE, FP64, LIK_BERNOULLI_LOGIT, LIK_GAMMA_LOG,
                   LIK_POISSON_LOG, OP_A, OP_A2, OP_B, OP_BINV, OP_BT, OP_BTINV, OP_PINV, OP_SIGMA,
                   PREC_LRAC, PREC_LVA, PREC_VADU, SOLVE_AUTO, SOLVE_CLUSTER, SOLVE_GRID, SOLVE_GRID_ALL, SOLVE_SHARED, SOLVE_TILE,
                   Batch, Context, Factor, Opts, State, Stats, VLError, lib_path, library, tune_report,
                   tune_reset)

__all__ = [
    "Context", "Factor", "State", "Batch", "Opts", "Stats", "VLError", "library", "lib_path", "tune_report", "tune_reset",
    "COV_EXPONENTIAL", "COV_MATERN15", "LIK_BERNOULLI_LOGIT", "LIK_POISSON_LOG", "LIK_GAMMA_LOG",
    "PREC_VADU", "PREC_LVA", "PREC_LRAC", "FP64", "FP32_REFINE",
    "OP_A", "OP_PINV", "OP_B", "OP_BT", "OP_BINV", "OP_BTINV", "OP_SIGMA", "OP_A2",
    "SOLVE_AUTO", "SOLVE_SHARED", "SOLVE_CLUSTER", "SOLVE_GRID", "SOLVE_GRID_ALL", "SOLVE_TILE",
]
