"""GB300-native two-sided Lanczos sign function sgn(H(mu)) x and its derivative
d_t sgn(H(mu)) x for the finite-density Wilson kernel H(mu) = gamma5 Dw(mu) (Puhr &
Buividovich, Lattice 2016).  The compute path is the CUDA library liblq.so (C ABI in
include/lq.h); `lq` is its ctypes binding, `build` compiles it for sm_103a."""
from . import lq  # noqa: F401
from .lq import (Context, LQError, LQ_FP64, LQ_MIXED, LQ_DIR_MU, LQ_DIR_SU3, LQ_DIR_U1)  # noqa: F401
