"""GB300-native micro-macro parareal for slow-fast SDEs (arXiv:1912.09240).

The compute path is libpr.so (CUDA for sm_103a, C ABI in include/pr.h);
``_lib`` binds it with ctypes and ``parareal`` sequences it.  Importing this
package does not load the library; the first call does, and raises if the
library has not been built.
"""
from ._lib import (  # noqa: F401
    Grid, Model, Rng, PrError, PR_F32, PR_F64, PR_MODEL_OU, PR_MODEL_DOUBLE_WELL, PR_MODEL_DW_MULTI,
    PR_ITER_QUANTILE, PR_ITER_ADD, PR_ITER_MULT, PR_ITER_ROT, PR_ITER_NONE, PR_QMODE_TWO_SIDED,
    PR_QMODE_MIDPOINT,
)

__version__ = "0.1.0"
