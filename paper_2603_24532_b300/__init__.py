"""B300-native (sm_103a) Monte Carlo evaluation of zero-temperature Hugenholtz
diagrams for the nuclear equation of state (arXiv:2603.24532): a C-ABI CUDA
library (include/mbpt.h, csrc/) and its thin Python binding (mbpt.py)."""
from . import mbpt  # noqa: F401
