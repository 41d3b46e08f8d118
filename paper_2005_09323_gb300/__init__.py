"""GB300-native ensemble lattice-Boltzmann rare-event sampling (Lestang,
Bouchet & Leveque, arXiv 2005.09323): a C-ABI CUDA library (liblbmrare.so,
include/lbmrare.h) and its Python binding."""
from . import lbmrare  # noqa: F401
from .lbmrare import LbmError, config  # noqa: F401
