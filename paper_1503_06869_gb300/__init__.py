"""GB300 library for the lattice Boltzmann method with fully resolved moving
rigid particles (Bartuschat et al., Sec. 4): C interface in ``include/lbm.h``,
CUDA kernels in ``csrc/``, ctypes binding in ``lbm``."""
from . import lbm  # noqa: F401
from .lbm import Simulation, load  # noqa: F401
