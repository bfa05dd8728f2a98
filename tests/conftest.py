import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# The oracle's OpenMP threads meet at a barrier every time step.  On a host
# whose cores are shared with other machines, spinning at those barriers
# while a descheduled thread is missing slows the long oracle runs of the
# tests by an order of magnitude; threads that sleep while they wait do not.
# Read by the OpenMP runtime when the oracle library loads (before any test).
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
