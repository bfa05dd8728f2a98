"""lb_rd_step_noalloc: the fused step for callers that cannot allocate device
memory (for example a real-time loop whose memory was all reserved at
start-up, or a plugin that may only use buffers its host application gives
it).  Its reduction scratch lives in a static device array, so the only
memory it touches is the caller's.

Checked through the C ABI against the existing entry point (lb_rd_step on a
handle) on two calls in a row: the states must agree bit for bit (the same
per-site arithmetic) and the FP64 masses to 1e-12 relative (the same sums in
a different grouping).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1007_3109_gb300 import binding as B
from paper_1007_3109_gb300 import inputs

pytestmark = pytest.mark.gpu

CKPT_HEADER = 56  # bytes before the state in an lb_rd_save buffer


def _state_bytes(ckpt, nspecies, nx, ny, precision):
    pitch = (nx + 31) // 32 * 32
    rho_bytes = nspecies * ny * pitch * (8 if precision == "fp64" else 4)
    return bytes(ckpt[CKPT_HEADER:len(ckpt) - rho_bytes])


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp32_bf16dev"])
def test_noalloc_step_matches_lb_rd_step_on_two_calls(precision):
    import torch

    nx, ny = 200, 96
    rho0 = inputs.rho0_square(nx, ny, seed=31, side=30)
    kw = dict(lattice="D2Q9", nspecies=2, nx=nx, ny=ny, tau=[0.8, 0.65], reaction="gray_scott", F=0.04, k=0.06,
              precision=precision)
    cfg = B.make_config(**kw)
    with B.Simulation(**kw, track_mass=True) as sim:
        sim.init(rho0).step(3)
        start = _state_bytes(sim.save(), 2, nx, ny, precision)
        expected_states, expected_mass = [], []
        for _ in range(2):
            sim.step(1)
            expected_mass.append(sim.mass())
            expected_states.append(_state_bytes(sim.save(), 2, nx, ny, precision))

    # caller-owned device buffers (allocated by the caller, not by the library)
    a = torch.frombuffer(bytearray(start), dtype=torch.uint8).cuda()
    b = torch.empty_like(a)
    mass = torch.zeros(2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    bufs = [(a, b), (b, a)]
    for call, (src, dst) in enumerate(bufs):
        B.lb_rd_step_noalloc(cfg, src.data_ptr(), dst.data_ptr(), mass.data_ptr())
        torch.cuda.synchronize()
        got_state = dst.cpu().numpy().tobytes()
        assert got_state == expected_states[call], f"state differs on call {call + 1}"
        np.testing.assert_allclose(mass.cpu().numpy(), expected_mass[call], rtol=1e-12)


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    cfg = B.make_config(lattice="D2Q9", nspecies=2, nx=8192, ny=8192, tau=[0.8, 0.65], reaction="gray_scott",
                        F=0.037, k=0.06, precision="fp32")
    with pytest.raises(B.LbRdError) as ei:
        B.lb_rd_step_noalloc(cfg, 16, 32, 64)  # rejected before any pointer is used
    assert ei.value.status == B.LB_RD_EINVAL
    assert "static scratch" in str(ei.value) and "65536" in str(ei.value)
