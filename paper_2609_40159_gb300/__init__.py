"""GB300-native (sm_103a) sparse triangular solve over the dependency DAG.

Level-set analysis, equation rewriting, level-scheduled / synchronisation-free
/ block-local solves, batched solves and their adjoints, all in hand-written
CUDA behind the C ABI of include/sptrsv.h.  Importing the package does not
touch the GPU; the first call that needs the library loads
``libsptrsv_gb300.so`` and raises if it has not been built.
"""
from . import _lib
from ._lib import SpTRSVError
from .api import (Analysis, BatchPlan, Handle, Matrix, Plan, UpperPlan, analyze, handle, level_summary, rewrite,
                  transpose, validate)
from .autograd import BatchSpTRSVFunction, SpTRSVFunction, batch_solve, solve
from .env import EnvConfig, RewriteEnv

__all__ = [
    "_lib", "SpTRSVError", "Analysis", "BatchPlan", "Handle", "Matrix", "Plan", "analyze", "handle", "rewrite",
    "validate", "level_summary", "transpose", "UpperPlan", "SpTRSVFunction", "BatchSpTRSVFunction", "solve", "batch_solve",
    "EnvConfig", "RewriteEnv",
]
