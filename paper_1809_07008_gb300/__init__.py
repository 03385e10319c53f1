"""GB300-native (sm_103a) coupled LBM-DEM step with the immersed moving boundary.

The compute path is the CUDA library ``libimblbm.so`` (C ABI in
``include/imblbm.h``); :mod:`.binding` is its ctypes binding.  Importing this
package loads nothing: the library is built and loaded on first use and every
call fails loudly when it or a CUDA device is missing.  :mod:`.autodiff` wraps the
library's drag gradient as a ``torch.autograd.Function`` (imported on demand).
"""
from .binding import (BC_INLET_OUTLET, BC_PERIODIC, BC_WALL, EPS_EXACT, EPS_SUBCELL, EXPORTS,
                      STORE_BF16, STORE_FP16, STORE_FP32, Batch, ImbError, Lattice, Lattice3, binomial_schedule,
                      default_params, library_path, load)

__all__ = ["Lattice", "Lattice3", "Batch", "ImbError", "load", "library_path", "default_params", "EXPORTS", "binomial_schedule",
           "BC_PERIODIC", "BC_WALL", "BC_INLET_OUTLET", "STORE_FP32", "STORE_FP16", "STORE_BF16",
           "EPS_EXACT", "EPS_SUBCELL"]
