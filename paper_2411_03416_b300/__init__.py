"""B300-native (sm_103a) P-GVIMP: parallel proximal Gaussian variational
inference motion planning (arXiv 2411.03416).

The hot path -- GP prior build, marginal recovery on the chain, factor
quadrature, gradient assembly, the KL-proximal update with its step-size
search, and the SLR outer loop -- runs in hand-written CUDA kernels behind the
C ABI in include/pgvimp.h; this package is its thin ctypes binding.
"""
from ._lib import (PREC_MIXED, PREC_MIXED_DF, PREC_PLAIN_FP64, Batch, Context, PgvimpError, PlanResult, Server,  # noqa: F401
                   lib, solve,
                   version)

__all__ = ["Batch", "Context", "PgvimpError", "PlanResult", "PREC_MIXED", "PREC_MIXED_DF", "PREC_PLAIN_FP64", "Server", "lib", "solve",
           "version"]
