"""In-place (AA) streaming: one state copy, steps alternating between
neighbour reads with swapped writes back to the neighbours (t even) and
site-local reads and writes (t odd).

The per-site arithmetic is the ping-pong kernels', so every in-place run must
give the same bits as the two-copy run of the same config (densities,
distributions f*(t) at even and odd t, masses), and FP64 the oracle's bits.
Checkpoints keep the layout; the in-place handle allocates one copy.
"""
import numpy as np
import pytest

import oracle as orc
from oracle import Reaction
from paper_1007_3109_gb300 import binding as B
from paper_1007_3109_gb300 import inputs

pytestmark = pytest.mark.gpu

NET3 = ([0.3, 0.05, 0.02, 0.01, 0.07], [(1, 1, 0), (0, 0, 1), (0, 0, 1), (0, 0, 0), (0, 2, 0)],
        [(-1, -1, 1), (1, 1, -1), (0, 0, -1), (1, 0, 0), (0, -1, 0)])

CASES = [
    # name, lattice, S, kwargs, shape
    ("gs_fp32", "D2Q9", 2, dict(tau=[0.8, 0.65], reaction="gray_scott", F=0.04, k=0.06, precision="fp32"), (70, 37)),
    ("gs_fp64", "D2Q9", 2, dict(tau=[0.8, 0.65], reaction="gray_scott", F=0.04, k=0.06, precision="fp64"), (33, 20)),
    ("linear_d2q5_fp32", "D2Q5", 1, dict(tau=[0.9], reaction="linear", kappa=0.01, precision="fp32"), (129, 4)),
    ("net3_fp64", "D2Q9", 3, dict(tau=[0.7, 0.9, 1.4], reaction="mass_action", network=NET3, precision="fp64"),
     (40, 16)),
    ("coupled4_fp32", "D2Q9", 4, dict(tau=[0.8, 0.65, 0.8, 0.65], reaction="mass_action",
                                      network=inputs.coupled_gs_network(), precision="fp32"), (64, 30)),
    ("tiny_fp32", "D2Q9", 2, dict(tau=[0.8, 0.65], reaction="gray_scott", F=0.04, k=0.06, precision="fp32"), (1, 1)),
]


def _rho0(S, nx, ny, seed):
    if S == 2:
        return inputs.rho0_square(nx, ny, seed=seed, side=max(1, min(nx, ny) // 3))
    rng = np.random.default_rng(seed)
    return 0.2 + rng.random((S, ny, nx))


@pytest.mark.parametrize("steps", [1, 2, 7, 40])
@pytest.mark.parametrize("name,lat,S,kw,shape", CASES, ids=[c[0] for c in CASES])
def test_inplace_equals_pingpong_bitwise(name, lat, S, kw, shape, steps):
    nx, ny = shape
    rho0 = _rho0(S, nx, ny, seed=len(name) + steps)
    out = {}
    for inplace in (False, True):
        with B.Simulation(lat, S, nx, ny, track_mass=True, inplace=inplace, **kw) as sim:
            sim.init(rho0).step(steps // 2).step(steps - steps // 2)
            rho, mass = sim.moments()
            f = sim.distributions()
            out[inplace] = (rho, mass, f)
    np.testing.assert_array_equal(out[True][0], out[False][0])
    np.testing.assert_array_equal(out[True][2], out[False][2])
    np.testing.assert_allclose(out[True][1], out[False][1], rtol=1e-6 if kw["precision"] == "fp32" else 1e-13)


def test_inplace_fp64_equals_oracle_and_checkpoints():
    nx, ny, S = 45, 21, 2
    rho0 = _rho0(S, nx, ny, seed=4)
    taus = [0.8, 0.65]
    ref = orc.density("D2Q9", orc.run("D2Q9", taus, Reaction("gray_scott", F=0.04, k=0.06),
                                      orc.init("D2Q9", rho0), 33))
    kw = dict(tau=taus, reaction="gray_scott", F=0.04, k=0.06, precision="fp64", inplace=True)
    with B.Simulation("D2Q9", S, nx, ny, **kw) as a, B.Simulation("D2Q9", S, nx, ny, **kw) as b:
        a.init(rho0).step(13)  # odd time: pushed-and-swapped layout
        blob = a.save()
        a.step(20)
        np.testing.assert_array_equal(a.moments()[0], ref)
        b.init(rho0)
        b.restore(blob)
        b.step(20)
        np.testing.assert_array_equal(b.moments()[0], ref)
    with B.Simulation("D2Q9", S, nx, ny, **dict(kw, inplace=False)) as c:
        c.init(rho0).step(13)
        with pytest.raises(B.LbRdError):
            c.restore(blob)  # the layouts differ


@pytest.mark.parametrize("name,lat,S,kw,shape", [c for c in CASES if c[3]["precision"] == "fp32"],
                         ids=[c[0] for c in CASES if c[3]["precision"] == "fp32"])
@pytest.mark.parametrize("steps", [1, 6])
def test_every_inplace_variant_equals_pingpong(name, lat, S, kw, shape, steps):
    """Each FP32 in-place launch variant (1, 2 or 4 sites per thread; the
    vector forms assemble the pushed columns with shuffles and edge-lane
    scalar stores) gives the ping-pong bits, at odd and even times."""
    nx, ny = shape
    if nx % 4:
        nx += 4 - nx % 4  # the vector variants need nx % 4 == 0
    rho0 = _rho0(S, nx, ny, seed=steps)
    with B.Simulation(lat, S, nx, ny, track_mass=True, **kw) as ref:
        ref.init(rho0).step(steps)
        want_rho, want_f = ref.moments()[0], ref.distributions()
    with B.Simulation(lat, S, nx, ny, track_mass=True, inplace=True, **kw) as sim:
        n = B.lb_rd_handle_variant_count(sim.h)
        names = [B.lb_rd_handle_variant_name(sim.h, v) for v in range(n)]
        assert names[0] == "aa_1site" and n >= 3
        for v in range(n):
            B.lb_rd_set_variant(sim.h, v)
            sim.init(rho0).step(steps)
            np.testing.assert_array_equal(sim.moments()[0], want_rho, err_msg=names[v])
            np.testing.assert_array_equal(sim.distributions(), want_f, err_msg=names[v])


def test_inplace_autotune_leaves_the_state_alone():
    nx, ny = 256, 64
    rho0 = _rho0(2, nx, ny, seed=5)
    kw = dict(tau=[0.8, 0.65], reaction="gray_scott", F=0.04, k=0.06, precision="fp32")
    with B.Simulation("D2Q9", 2, nx, ny, inplace=True, **kw) as sim, B.Simulation("D2Q9", 2, nx, ny, **kw) as ref:
        sim.init(rho0).step(5)
        best, times = B.lb_rd_autotune(sim.h, iters=3)
        assert 0 <= best < B.lb_rd_handle_variant_count(sim.h) and times[best] > 0
        sim.step(4)
        ref.init(rho0).step(9)
        np.testing.assert_array_equal(sim.moments()[0], ref.moments()[0])
