"""Up to four species and mass-action networks on the GPU (the general
kernel), against the FP64 oracle.

FP64 performs the oracle's operations in the oracle's order: bitwise equal
densities.  FP32 within 2e-5 relative (the same bound as the two-species
FP32 path over a few hundred steps).  Also: conservation under a
conservative network with the fused mass diagnostic, checkpoint/restore and
the single launch variant.
"""
import zlib

import numpy as np
import pytest

import oracle as orc
from oracle import Reaction
from paper_1007_3109_gb300 import binding as B
from paper_1007_3109_gb300 import inputs

pytestmark = pytest.mark.gpu

NET3 = ([0.3, 0.05, 0.02, 0.01, 0.07], [(1, 1, 0), (0, 0, 1), (0, 0, 1), (0, 0, 0), (0, 2, 0)],
        [(-1, -1, 1), (1, 1, -1), (0, 0, -1), (1, 0, 0), (0, -1, 0)])
CYCLE4 = ([0.02, 0.03, 0.05, 0.01, 0.04], [(1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (2, 0, 0, 0)],
          [(-1, 1, 0, 0), (0, -1, 1, 0), (0, 0, -1, 1), (1, 0, 0, -1), (-1, 1, 0, 0)])
LOGISTIC1 = ([0.05, 0.05], [(1,), (2,)], [(1,), (-1,)])  # A -> 2A, 2A -> A: rho' = r rho (1 - rho)
GS_NET = ([1.0, 0.04, 0.04, 0.1], [(1, 2), (0, 0), (1, 0), (0, 1)], [(-1, 1), (1, 0), (-1, 0), (0, -1)])

CASES = [
    ("net3_d2q9", "D2Q9", 3, NET3, (0.7, 0.9, 1.4), (37, 23)),
    ("net3_d2q5", "D2Q5", 3, NET3, (0.6, 1.1, 0.8), (130, 7)),
    ("cycle4_d2q9", "D2Q9", 4, CYCLE4, (0.6, 0.8, 1.0, 1.7), (64, 33)),
    ("coupled_gs4", "D2Q9", 4, inputs.coupled_gs_network(), (0.8, 0.65, 0.8, 0.65), (96, 40)),
    ("logistic1", "D2Q9", 1, LOGISTIC1, (0.9,), (50, 3)),
    ("gs_as_network", "D2Q9", 2, GS_NET, (0.8, 0.65), (48, 48)),
    ("diffusion4", "D2Q5", 4, None, (0.55, 0.8, 1.0, 3.0), (1, 1)),
]


def _rho0(S, nx, ny, seed):
    rng = np.random.default_rng(seed)
    return 0.2 + rng.random((S, ny, nx))


def _oracle(lat, S, net, taus, rho0, steps):
    reac = Reaction.network(*net) if net else Reaction("none")
    return orc.density(lat, orc.run(lat, list(taus), reac, orc.init(lat, rho0), steps))


def _gpu(lat, S, net, taus, rho0, steps, precision, track_mass=False):
    kw = dict(reaction="mass_action", network=net) if net else dict(reaction="none")
    ny, nx = rho0.shape[1:]
    with B.Simulation(lat, S, nx, ny, list(taus), precision=precision, track_mass=track_mass, **kw) as sim:
        sim.init(rho0).step(steps)
        return sim.moments()


@pytest.mark.parametrize("name,lat,S,net,taus,shape", CASES, ids=[c[0] for c in CASES])
def test_fp64_bitwise_equal_to_oracle(name, lat, S, net, taus, shape):
    rho0 = _rho0(S, *shape, seed=zlib.crc32(name.encode()) % 1000)
    ref = _oracle(lat, S, net, taus, rho0, 60)
    rho, mass = _gpu(lat, S, net, taus, rho0, 60, "fp64")
    np.testing.assert_array_equal(rho, ref)
    np.testing.assert_allclose(mass, ref.sum(axis=(1, 2)), rtol=1e-12)


@pytest.mark.parametrize("name,lat,S,net,taus,shape", CASES, ids=[c[0] for c in CASES])
def test_fp32_within_tolerance(name, lat, S, net, taus, shape):
    rho0 = _rho0(S, *shape, seed=zlib.crc32(name.encode()) % 1000)
    ref = _oracle(lat, S, net, taus, rho0, 200)
    rho, _ = _gpu(lat, S, net, taus, rho0, 200, "fp32")
    err = np.max(np.abs(rho - ref)) / np.max(np.abs(ref))
    assert err < 2e-5, err


def test_conservative_network_keeps_total_mass_fused_diagnostic():
    rho0 = _rho0(4, 200, 120, seed=7)
    m0 = rho0.sum()
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-6)):
        kw = dict(reaction="mass_action", network=CYCLE4)
        with B.Simulation("D2Q9", 4, 200, 120, [0.6, 0.8, 1.0, 1.7], precision=prec, track_mass=True, **kw) as sim:
            sim.init(rho0).step(300)
            m = sim.mass()
            assert abs(m.sum() - m0) / m0 < tol, (prec, m.sum(), m0)
            assert np.max(np.abs(m - rho0.sum(axis=(1, 2)))) > 1.0  # the species did react


def test_checkpoint_and_single_variant():
    rho0 = _rho0(3, 70, 20, seed=9)
    kw = dict(reaction="mass_action", network=NET3)
    with B.Simulation("D2Q9", 3, 70, 20, [0.7, 0.9, 1.4], precision="fp64", **kw) as a, \
            B.Simulation("D2Q9", 3, 70, 20, [0.7, 0.9, 1.4], precision="fp64", **kw) as b:
        a.init(rho0).step(15)
        blob = a.save()
        a.step(15)
        b.init(rho0)
        b.restore(blob)
        b.step(15)
        np.testing.assert_array_equal(a.moments()[0], b.moments()[0])
        best, times = B.lb_rd_autotune(a.h, iters=2)
        assert best == 0 and len([t for t in times if t is not None and t >= 0]) >= 1
        with pytest.raises(B.LbRdError):
            B.lb_rd_set_variant(a.h, 1)


@pytest.mark.parametrize("S,net,taus", [(4, inputs.coupled_gs_network(), (0.8, 0.65, 0.8, 0.65)),
                                        (3, NET3, (0.7, 0.9, 1.4)), (1, LOGISTIC1, (0.9,))])
@pytest.mark.parametrize("nx,ny", [(64, 48), (516, 9), (8, 3)])
def test_every_general_fp32_variant_is_bitwise_identical(S, net, taus, nx, ny):
    rho0 = _rho0(S, nx, ny, seed=nx + ny)
    with B.Simulation("D2Q9", S, nx, ny, list(taus), reaction="mass_action", network=net, precision="fp32",
                      track_mass=True) as sim:
        n = B.lb_rd_handle_variant_count(sim.h)
        names = [B.lb_rd_handle_variant_name(sim.h, v) for v in range(n)]
        assert names[0] == "general_1site" and len(set(names)) == n
        ref = None
        for v in range(n):
            try:
                B.lb_rd_set_variant(sim.h, v)
            except B.LbRdError:
                assert nx % 4, names[v]  # only the 4-site variant needs nx % 4 == 0 here
                continue
            sim.init(rho0).step(25)
            rho, mass = sim.moments()
            if ref is None:
                ref = (rho, mass)
            else:
                np.testing.assert_array_equal(rho, ref[0], err_msg=names[v])
                np.testing.assert_allclose(mass, ref[1], rtol=1e-6)
