"""FP64 CPU oracle of the lattice-Boltzmann reaction-diffusion method.

Test infrastructure only: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the library under
``paper_1007_3109_gb300`` never does.  It shares no code with the CUDA path.
"""
from .lbrd_oracle import *  # noqa: F401,F403
