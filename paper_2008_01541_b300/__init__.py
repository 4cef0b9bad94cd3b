"""B300-native localized-collision Projective Dynamics (Wang et al., SCA 2020).

The compute path is the CUDA library libpd.so (C ABI in include/pd.h); this
package is only its ctypes binding.  Importing it loads the library and fails
loudly if it has not been built.
"""
from ._lib import lib, PDError, FP64, FP32_IR, TF32_IR, BF16_IR, PCG_WARM, LIB_PATH  # noqa: F401
from .solver import Solver, host_schur  # noqa: F401
