"""Batched simulations: one persistent launch per step over all instances.

Each instance must compute exactly what a single handle with its config
computes (same tile body, same arithmetic): bitwise.  The phase-diagram sweep
(1024 instances of 256^2, F in [0.01, 0.08], k in [0.03, 0.07]) runs at full
size and sampled instances are checked against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle as orc
from oracle import Reaction
from paper_1007_3109_gb300 import binding as B
from paper_1007_3109_gb300 import inputs

pytestmark = pytest.mark.gpu


def _configs(precision="fp32"):
    shapes = [(64, 48), (100, 37), (36, 70), (8, 3), (256, 16)]
    out = []
    for j, (nx, ny) in enumerate(shapes):
        if precision.endswith("dev") and nx % 4:
            continue
        out.append(dict(lattice="D2Q9", nspecies=2, nx=nx, ny=ny, tau=[0.8 + 0.05 * j, 0.65], reaction="gray_scott",
                        F=0.03 + 0.004 * j, k=0.06 - 0.002 * j, precision=precision))
    return out


def _rho0(c, j):
    return inputs.rho0_square(c["nx"], c["ny"], seed=50 + j, side=max(2, min(c["nx"], c["ny"]) // 3))


def _single(c, rho0, steps):
    with B.Simulation(**c) as sim:
        sim.init(rho0).step(steps)
        return sim.moments()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_bf16dev", "fp32_fp16dev"])
@pytest.mark.parametrize("graph", [0, 8])
def test_batch_instances_equal_single_handles(precision, graph):
    """One step per launch (the FP32 default, K steps per launch, is tested
    below)."""
    cfgs = _configs(precision)
    steps = 57
    with B.Batch(cfgs) as b:
        b.set_graph(graph)
        b.set_steps_per_launch(1)
        for j, c in enumerate(cfgs):
            b.init(j, _rho0(c, j))
        b.step(20).step(steps - 20)
        assert b.time == steps
        for j, c in enumerate(cfgs):
            rho, mass = b.moments(j)
            ref_rho, ref_mass = _single(c, _rho0(c, j), steps)
            np.testing.assert_array_equal(rho, ref_rho, err_msg=f"instance {j}")
            np.testing.assert_allclose(mass, ref_mass, rtol=1e-14)


def test_batch_fp64_equals_oracle_bitwise():
    """FP64 instances of mixed sizes, tau and reactions against the oracle,
    element by element (the FP64 update rounds every operation on its own in
    the oracle's order)."""
    cases = [dict(nx=100, ny=100, tau=[0.56, 0.56], reaction="linear", kappa=0.01),
             dict(nx=37, ny=5, tau=[0.9, 1.3], reaction="gray_scott", F=0.04, k=0.06),
             dict(nx=300, ny=3, tau=[1.0, 0.7], reaction="none"),
             dict(nx=1, ny=1, tau=[0.8, 0.8], reaction="linear", kappa=0.1)]
    cfgs = [dict(lattice="D2Q9", nspecies=2, precision="fp64", **c) for c in cases]
    steps = 41
    with B.Batch(cfgs) as b:
        rho0s = []
        for j, c in enumerate(cfgs):
            rho0 = inputs.rho0_square(c["nx"], c["ny"], seed=900 + j, side=max(1, c["nx"] // 4))
            rho0s.append(rho0)
            b.init(j, rho0)
        b.step(steps)
        for j, (c, case) in enumerate(zip(cfgs, cases)):
            rho, _ = b.moments(j)
            reac = Reaction(case["reaction"], kappa=case.get("kappa", 0.0), F=case.get("F", 0.0), k=case.get("k", 0.0))
            ref = orc.density("D2Q9", orc.run("D2Q9", c["tau"], reac, orc.init("D2Q9", rho0s[j]), steps))
            np.testing.assert_array_equal(rho, ref, err_msg=f"instance {j}")


def test_batch_rejects_mixed():
    cfgs = _configs()
    bad = [dict(cfgs[0]), dict(cfgs[1], lattice="D2Q5")]
    with pytest.raises(B.LbRdError):
        B.Batch(bad)
    with pytest.raises(B.LbRdError):
        B.Batch([dict(cfgs[0]), dict(cfgs[1], precision="fp64")])
    with B.Batch(cfgs[:2]) as b:
        b.init(0, _rho0(cfgs[0], 0))
        with pytest.raises(B.LbRdError):
            b.step(1)  # instance 1 not initialised


def test_phase_diagram_sweep_full_size_sampled():
    """gs_sweep_256 at full size (1024 x 256^2, FP32) in the configuration the
    batched benchmark times; sampled instances checked against the oracle."""
    w = inputs.WORKLOADS["gs_sweep_256"]
    F, k = inputs.sweep_params()
    taus = [float(t) for t in orc.tau_from_diffusion(np.array(w["D"]))]
    n, T = w["nx"], 30
    cfgs = [dict(lattice="D2Q9", nspecies=2, nx=n, ny=n, tau=taus, reaction="gray_scott", F=float(F[i]),
                 k=float(k[i]), precision="fp32") for i in range(w["instances"])]
    with B.Batch(cfgs) as b:
        for i in range(len(cfgs)):
            b.init(i, inputs.rho0_square(n, n, seed=w["seed"] + i))
        b.step(T)
        for i in (0, 517, 1023):
            rho, _ = b.moments(i)
            rho0 = inputs.rho0_square(n, n, seed=w["seed"] + i)
            reac = Reaction("gray_scott", F=float(F[i]), k=float(k[i]))
            ref = orc.density("D2Q9", orc.run("D2Q9", taus, reac, orc.init("D2Q9", rho0), T))
            err = np.max(np.abs(rho - ref), axis=(1, 2)) / np.maximum(np.max(np.abs(ref), axis=(1, 2)), 1e-4)
            assert np.all(err <= 5e-5), (i, err)


def test_batch_with_inplace_instances_equals_single_handles():
    """A batch mixing one-copy (in-place) and two-copy FP32 instances: every
    instance gives the bits of a single two-copy handle, at odd and even
    batch times, with and without graphs."""
    extra = dict(_configs("fp32")[0], nx=70, ny=9)  # nx % 4 != 0: one site per thread in place
    cfgs = _configs("fp32") + [extra, dict(extra, nx=37, ny=5)]
    cfgs = [dict(c, inplace=(j != 1)) for j, c in enumerate(cfgs)]
    for graph, steps in ((0, 23), (8, 40)):
        with B.Batch(cfgs) as b:
            b.set_graph(graph)
            for j, c in enumerate(cfgs):
                b.init(j, _rho0(c, j))
            b.step(steps)
            for j, c in enumerate(cfgs):
                rho, _ = b.moments(j)
                ref_rho, _ = _single(dict(c, inplace=False), _rho0(c, j), steps)
                np.testing.assert_array_equal(rho, ref_rho, err_msg=f"instance {j} graph {graph}")


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q5"])
@pytest.mark.parametrize("graph", [0, 8, 6])
@pytest.mark.parametrize("steps", [1, 2, 7, 40])
def test_batch_two_steps_per_launch_equals_single_handles(lat, graph, steps):
    """Instances with nx a multiple of 256 can run the two-step kernel over
    the whole list; each instance gives the bits
    of a single handle, whatever the graph length (6: an odd number of
    two-step launches per graph) and step count (odd counts end with single
    steps)."""
    shapes = [(256, 40), (512, 16), (256, 3), (768, 9)]
    cfgs = [dict(lattice=lat, nspecies=2, nx=nx, ny=ny, tau=[0.8 + 0.05 * j, 0.65], reaction="gray_scott",
                 F=0.03 + 0.004 * j, k=0.06 - 0.002 * j, precision="fp32") for j, (nx, ny) in enumerate(shapes)]
    with B.Batch(cfgs) as b:
        b.set_graph(graph)
        b.set_steps_per_launch(2)
        for j, c in enumerate(cfgs):
            b.init(j, _rho0(c, j))
        b.step(steps).step(steps)
        _, launches = B.lb_rd_batch_get_time(b.b)
        for j, c in enumerate(cfgs):
            rho, _ = b.moments(j)
            ref_rho, _ = _single(c, _rho0(c, j), 2 * steps)
            np.testing.assert_array_equal(rho, ref_rho, err_msg=f"instance {j}")
    if steps >= 7:
        assert launches < 2 * steps  # two steps per launch were used


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q5"])
@pytest.mark.parametrize("K", [2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("staging", ["16-byte", "4-byte"])
@pytest.mark.parametrize("graph", [0, 8, 12])
def test_batch_k_steps_per_launch_equals_single_handles(lat, K, staging, graph):
    """K = 2 .. 8 steps per launch run the depth-K kernel over the (band,
    strip) units of all instances (ragged strips, bands of a few rows; K = 2
    here too, as not every nx is a multiple of 256); each call of 21 steps
    runs 21 // K launches of K steps and one of the 21 % K left (a single
    step for one), the last writing the densities; each instance gives the
    bits of a single handle.  All nx multiples of 4: the 16-byte staging;
    otherwise 4-byte copies.  Graph 12: an odd number of K-step launches per
    graph for K = 4 and 8."""
    shapes = [(64, 48), (100, 37), (36, 70), (8, 3), (256, 16)]
    if staging == "4-byte":
        shapes += [(70, 9), (33, 20)]
    cfgs = [dict(lattice=lat, nspecies=2, nx=nx, ny=ny, tau=[0.8 + 0.05 * j, 0.65], reaction="gray_scott",
                 F=0.03 + 0.004 * j, k=0.06 - 0.002 * j, precision="fp32") for j, (nx, ny) in enumerate(shapes)]
    steps = 21
    with B.Batch(cfgs) as b:
        b.set_graph(graph)
        b.set_steps_per_launch(K)
        for j, c in enumerate(cfgs):
            b.init(j, _rho0(c, j))
        b.step(steps).step(steps)
        _, launches = B.lb_rd_batch_get_time(b.b)
        for j, c in enumerate(cfgs):
            rho, _ = b.moments(j)
            ref_rho, _ = _single(c, _rho0(c, j), 2 * steps)
            np.testing.assert_array_equal(rho, ref_rho, err_msg=f"instance {j}")
    # one init launch per instance; per call 21 // K launches of K steps and one for the 21 % K left
    assert launches == len(cfgs) + 2 * (steps // K + (1 if steps % K else 0))


@pytest.mark.parametrize("precision", ["fp32_bf16dev", "fp32_fp16dev"])
@pytest.mark.parametrize("K", [2, 3, 4, 5])
@pytest.mark.parametrize("shapes", [[(64, 48), (100, 37), (36, 70), (8, 3), (256, 16), (68, 9)],
                                    [(64, 48), (104, 37), (40, 70), (8, 3), (256, 16), (72, 9)]],
                         ids=["nx%4", "nx%8"])
def test_batch_half_k_steps_per_launch_equals_single_handles(precision, K, shapes):
    """16-bit deviation storage: K = 2 .. 5 steps per launch run a depth-K
    kernel over the (band, strip) units of all instances (each level holds
    rho* and the deviations rounded as a single step stores them; the
    two-column kernel when every instance has nx % 8 == 0); each instance
    gives the bits of a single handle (which runs single steps), over calls
    of 21 steps (21 // K launches of K and one of the rest)."""
    cfgs = [dict(lattice="D2Q9", nspecies=2, nx=nx, ny=ny, tau=[0.8 + 0.05 * j, 0.65], reaction="gray_scott",
                 F=0.03 + 0.004 * j, k=0.06 - 0.002 * j, precision=precision) for j, (nx, ny) in enumerate(shapes)]
    steps = 21
    with B.Batch(cfgs) as b:
        b.set_steps_per_launch(K)
        for j, c in enumerate(cfgs):
            b.init(j, _rho0(c, j))
        b.step(steps).step(steps)
        _, launches = B.lb_rd_batch_get_time(b.b)
        for j, c in enumerate(cfgs):
            rho, _ = b.moments(j)
            ref_rho, _ = _single(dict(c, tb_depth=1), _rho0(c, j), 2 * steps)
            np.testing.assert_array_equal(rho, ref_rho, err_msg=f"instance {j}")
    assert launches == len(cfgs) + 2 * (steps // K + (1 if steps % K else 0))


def test_batch_steps_per_launch_switch():
    cfgs = _configs("fp32")  # includes nx not a multiple of 256
    with B.Batch(cfgs) as b:
        b.set_steps_per_launch(2)  # the depth-K kernel of two steps (the two-step kernel needs nx % 256 == 0)
        b.set_steps_per_launch(1)
        b.set_steps_per_launch(6)  # the depth-K kernel takes any nx
        b.set_steps_per_launch(3)
        for k in (0, 9, 16, -1):
            with pytest.raises(B.LbRdError):
                b.set_steps_per_launch(k)
    ip = [dict(c, inplace=True) for c in _configs("fp32")[:2]]
    with B.Batch(ip) as b:
        for k in (2, 4):
            with pytest.raises(B.LbRdError):
                b.set_steps_per_launch(k)  # in-place instances: one state copy
