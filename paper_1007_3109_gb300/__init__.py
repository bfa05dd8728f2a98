"""GB300-native lattice-Boltzmann reaction-diffusion step (sm_103a).

The compute path lives in ``csrc/`` and is exposed by the C ABI declared in
``include/lb_rd.h``; ``binding`` is the thin ctypes layer over it.
"""
from . import inputs  # noqa: F401
