"""B300-native batched drone physics step (Crazyflow, arXiv 2606.01478).

The hot path is the CUDA library ``libcrazyflow_b300.so`` (C-ABI declared in
include/crazyflow.h); this package is its thin binding.  Importing the
package does not load the library; ``Sim(...)`` does, and raises if it is
missing.  There is no CPU fallback.
"""
from ._lib import (ABSTRACTED, CTRL_ATTITUDE, CTRL_POSITION, CTRL_ROTOR_SPEED, EULER,
                   FIRST_PRINCIPLES, RK4, SimError, load)
from .sim import Sim, pack_params, select_elites

__all__ = ["Sim", "SimError", "load", "pack_params", "select_elites", "FIRST_PRINCIPLES", "ABSTRACTED", "EULER",
           "RK4", "CTRL_ROTOR_SPEED", "CTRL_ATTITUDE", "CTRL_POSITION"]
