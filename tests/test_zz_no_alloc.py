"""lb_rd_step_noalloc: the fused step for callers that cannot allocate device
memory (for example a real-time loop whose memory was all reserved at
start-up, or a plugin that may only use buffers its host application gives
it).  Its reduction scratch lives in a static device array, so the only
memory it touches is the caller's.

Checked through the C ABI against the existing entry point (lb_rd_step on a
handle) on two calls in a row: the states must agree bit for bit (the same
per-site arithmetic) and the FP64 masses to 1e-12 relative (the same sums in
a different grouping).  The cases cover both lattices, one and two species,
every storage format, a width that is not a multiple of the tile, and a grid
whose (tile, species) count is exactly the scratch limit, so that the last
partial-sum slot and the arrival counter placed right after it are used.

The file is named so that pytest collects it last: the static scratch array
is shared by every call in the process, and if one of these tests fails, a
run that stops at the first failure has then already run every other test.
Each test also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1007_3109_gb300 import binding as B
from paper_1007_3109_gb300 import inputs

pytestmark = pytest.mark.gpu

CKPT_HEADER = 56  # bytes before the state in an lb_rd_save buffer
SLOTS = 65536     # (tile, species) partial sums the static scratch holds


def _state_bytes(ckpt, nspecies, nx, ny, precision):
    pitch = (nx + 31) // 32 * 32
    rho_bytes = nspecies * ny * pitch * (8 if precision == "fp64" else 4)
    return bytes(ckpt[CKPT_HEADER:len(ckpt) - rho_bytes])


def _check_two_calls(kw, rho0, warm=3):
    import torch

    S, nx, ny, precision = kw["nspecies"], kw["nx"], kw["ny"], kw["precision"]
    cfg = B.make_config(**kw)
    with B.Simulation(**kw, track_mass=True) as sim:
        sim.init(rho0).step(warm)
        start = _state_bytes(sim.save(), S, nx, ny, precision)
        expected_states, expected_mass = [], []
        for _ in range(2):
            sim.step(1)
            expected_mass.append(sim.mass())
            expected_states.append(_state_bytes(sim.save(), S, nx, ny, precision))

    # caller-owned device buffers (allocated by the caller, not by the library); the
    # row padding (pitch beyond nx) is never written, so the destination starts
    # zeroed like a handle's buffers and the whole buffers can be compared
    a = torch.frombuffer(bytearray(start), dtype=torch.uint8).cuda()
    b = torch.zeros_like(a)
    mass = torch.zeros(S, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for call, (src, dst) in enumerate([(a, b), (b, a)]):
        B.lb_rd_step_noalloc(cfg, src.data_ptr(), dst.data_ptr(), mass.data_ptr())
        torch.cuda.synchronize()
        got_state = dst.cpu().numpy().tobytes()
        assert got_state == expected_states[call], f"state differs on call {call + 1}"
        np.testing.assert_allclose(mass.cpu().numpy(), expected_mass[call], rtol=1e-12)


@pytest.mark.parametrize("lattice", ["D2Q9", "D2Q5"])
@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp32_bf16dev", "fp32_fp16dev"])
def test_noalloc_step_matches_lb_rd_step_on_two_calls(lattice, precision):
    nx, ny = 200, 96
    rho0 = inputs.rho0_square(nx, ny, seed=31, side=30)
    kw = dict(lattice=lattice, nspecies=2, nx=nx, ny=ny, tau=[0.8, 0.65], reaction="gray_scott", F=0.04, k=0.06,
              precision=precision)
    _check_two_calls(kw, rho0)


@pytest.mark.parametrize("precision,nx,ny", [("fp32", 131, 45), ("fp64", 131, 45), ("fp32_bf16dev", 68, 7)])
def test_noalloc_one_species_linear_reaction(precision, nx, ny):
    """One species with the transformation source (Sec. II.B), widths that
    leave a ragged last tile."""
    rho0 = inputs.rho0_cosine(nx, ny, seed=32, noise=1e-3)
    kw = dict(lattice="D2Q9", nspecies=1, nx=nx, ny=ny, tau=[1.1], reaction="linear", kappa=0.01,
              precision=precision)
    _check_two_calls(kw, rho0)


def test_noalloc_grid_at_the_scratch_limit():
    """FP64 tiles are 32 x 4 sites: 2048 x 2048 with two species needs
    64 * 512 * 2 = 65536 partial sums, the whole array (the last block writes
    the last slot, and the counter sits right after it)."""
    nx = ny = 2048
    assert (nx // 32) * (ny // 4) * 2 == SLOTS
    rho0 = inputs.rho0_square(nx, ny, seed=33, side=200)
    kw = dict(lattice="D2Q9", nspecies=2, nx=nx, ny=ny, tau=[0.8, 0.65], reaction="gray_scott", F=0.04, k=0.06,
              precision="fp64")
    _check_two_calls(kw, rho0, warm=1)


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    """One row of FP64 tiles more than the limit (2048 x 2052: 64 * 513 * 2 =
    65664 partial sums) is rejected with EINVAL before any launch; the
    buffers are real device allocations of the state's size, so a call that
    got past the check would still stay inside them."""
    import torch

    nx, ny = 2048, 2052
    assert (nx // 32) * ((ny + 3) // 4) * 2 > SLOTS
    cfg = B.make_config(lattice="D2Q9", nspecies=2, nx=nx, ny=ny, tau=[0.8, 0.65], reaction="gray_scott",
                        F=0.037, k=0.06, precision="fp64")
    nbytes = 2 * 9 * ny * ((nx + 31) // 32 * 32) * 8
    src = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    dst = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    mass = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(B.LbRdError) as ei:
        B.lb_rd_step_noalloc(cfg, src.data_ptr(), dst.data_ptr(), mass.data_ptr())
    assert ei.value.status == B.LB_RD_EINVAL
    assert "static scratch" in str(ei.value) and "65536" in str(ei.value)
    torch.cuda.synchronize()
    assert int(dst.count_nonzero()) == 0  # nothing ran
