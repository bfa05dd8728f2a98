"""Failure detection on the GPU without a fault: a bounded device-side wait
that runs out returns an error status the host reads, and the context stays
usable.  The wait is made to run out by expecting 16 bytes that are never
copied (a barrier that nothing completes); it gives up after about a second."""
import numpy as np
import pytest

from paper_1007_3109_gb300 import binding as B
from paper_1007_3109_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.timeout(120)
@pytest.mark.parametrize("variant", ["bulk256_s2", "tb2_352x512_s2", "tb2w_288x256_s2x2"])
def test_bounded_wait_reports_timeout_and_context_survives(variant):
    nx, ny = 512, 24
    rho0 = inputs.rho0_square(nx, ny, seed=77, side=8)
    kw = dict(lattice="D2Q9", nspecies=2, nx=nx, ny=ny, tau=[0.8, 0.65], reaction="gray_scott", F=0.04, k=0.06,
              precision="fp32")
    names = [B.lb_rd_variant_name("fp32", v) for v in range(B.lb_rd_variant_count("fp32"))]
    with B.Simulation(**kw) as sim, B.Simulation(**kw) as ref:
        sim.set_variant(names.index(variant))
        sim.init(rho0)
        B.lb_rd_debug_inject_wait_timeout(sim.h, True)
        sim.step(5)
        with pytest.raises(B.LbRdError) as ei:
            sim.moments()
        assert ei.value.status == B.LB_RD_ETIMEOUT
        # the context is usable: re-initialise and compare with a clean handle
        sim.init(rho0).step(5)
        ref.init(rho0).step(5)
        np.testing.assert_array_equal(sim.moments()[0], ref.moments()[0])
