"""Serving loop: continuous batching of simulation requests.

Requests that arrive while others run are admitted between ticks as slots and
memory free up; every result must be bitwise what a single handle with the
same config computes (the same result alone and in the mix).
"""
import time

import numpy as np
import pytest

from paper_1007_3109_gb300 import binding as B
from paper_1007_3109_gb300 import inputs

pytestmark = pytest.mark.gpu


def _request(j, side, scale, steps):
    D = (0.1 * scale, 0.05 * scale)
    kw = dict(lattice="D2Q9", nspecies=2, nx=side, ny=side, tau=[3 * D[0] + 0.5, 3 * D[1] + 0.5],
              reaction="gray_scott", F=0.04, k=0.06, precision="fp32")
    rho0 = inputs.rho0_square(side, side, seed=300 + j, side=max(2, side // 4))
    return kw, rho0, steps


def _alone(kw, rho0, steps):
    with B.Simulation(**kw) as sim:
        sim.init(rho0).step(steps)
        return sim.moments()


def _wait(srv, ticket, S, side, timeout=120.0):
    rho = np.empty((S, side, side))
    mass = np.empty(S)
    t0 = time.time()
    while True:
        rc, st = B.lb_rd_poll(srv, ticket, rho, mass)
        if rc != B.LB_RD_EPENDING:
            return rc, rho, mass, st
        assert time.time() - t0 < timeout, "request did not finish"
        time.sleep(0.002)


def test_results_identical_alone_and_in_the_mix():
    reqs = [_request(0, 64, 1, 150), _request(1, 100, 2, 37), _request(2, 36, 4, 260), _request(3, 128, 1, 64),
            _request(4, 70, 2, 1), _request(5, 256, 1, 90), _request(6, 12, 1, 500), _request(7, 96, 4, 77)]
    srv = B.lb_rd_server_create(hbm_budget_bytes=1 << 30, max_slots=5, steps_per_tick=16)
    try:
        tickets = []
        for j, (kw, rho0, steps) in enumerate(reqs):
            tickets.append(B.lb_rd_submit(srv, B.make_config(**kw), rho0, steps))
            if j % 3 == 2:
                time.sleep(0.01)  # later requests arrive while earlier ones run
        for (kw, rho0, steps), t in zip(reqs, tickets):
            rc, rho, mass, st = _wait(srv, t, 2, kw["nx"])
            assert rc == B.LB_RD_OK
            ref_rho, ref_mass = _alone(kw, rho0, steps)
            np.testing.assert_array_equal(rho, ref_rho)
            np.testing.assert_allclose(mass, ref_mass, rtol=1e-14)
            assert st["arrival_ns"] <= st["start_ns"] <= st["end_ns"] and st["steps"] == steps
        stats = B.lb_rd_server_stats(srv)
        assert stats["finished"] == len(reqs)
        # continuous batching: fewer batched launches than the summed step counts
        assert stats["launches"] < sum(r[2] for r in reqs)
        with pytest.raises(B.LbRdError) as ei:
            B.lb_rd_poll(srv, tickets[0])
        assert ei.value.status == B.LB_RD_ENOTFOUND
    finally:
        B.lb_rd_server_destroy(srv)


@pytest.mark.parametrize("tick", [5, 16, 64])
def test_d2q5_k_step_ticks_equal_single_handles(tick):
    """A D2Q5 server: ticks advance the resident requests by six-step
    launches of the two-column depth-K kernel (nx % 4 != 0 among them: the
    chunks at the periodic seam copied column by column) and one launch of
    the steps left; every result is bitwise a single handle's."""
    sides = [(64, 41), (36, 17), (70, 9), (128, 30)]
    reqs = []
    for j, (side, steps) in enumerate(sides):
        kw, rho0, _ = _request(j, side, 1 + j % 2, steps)
        reqs.append((dict(kw, lattice="D2Q5"), rho0, steps))
    srv = B.lb_rd_server_create(hbm_budget_bytes=1 << 30, max_slots=4, steps_per_tick=tick, lattice="D2Q5")
    try:
        tickets = [B.lb_rd_submit(srv, B.make_config(**kw), rho0, steps) for kw, rho0, steps in reqs]
        for (kw, rho0, steps), t in zip(reqs, tickets):
            rc, rho, mass, _ = _wait(srv, t, 2, kw["nx"])
            assert rc == B.LB_RD_OK
            ref_rho, _ = _alone(kw, rho0, steps)
            np.testing.assert_array_equal(rho, ref_rho)
        if tick > 5:
            assert B.lb_rd_server_stats(srv)["launches"] < sum(r[2] for r in reqs) // 2
    finally:
        B.lb_rd_server_destroy(srv)


@pytest.mark.parametrize("tick,launches", [(64, 13), (65, 13), (13, 3), (6, 2), (5, 1), (1, 1)])
def test_d2q9_tick_launches(tick, launches):
    """One D2Q9 request of `tick` steps (the two-column depth-K kernel,
    K = 5) is one tick: tick // 5 five-step launches and one launch of the
    tick % 5 steps left (a single step when one is left), the last writing
    the densities: a 64-step tick is twelve five-step launches and one
    four-step launch, with no single step.  The result is bitwise a single
    handle's."""
    kw, rho0, _ = _request(3, 96, 1, tick)
    srv = B.lb_rd_server_create(hbm_budget_bytes=1 << 30, max_slots=4, steps_per_tick=tick)
    try:
        t = B.lb_rd_submit(srv, B.make_config(**kw), rho0, tick)
        rc, rho, mass, _ = _wait(srv, t, 2, kw["nx"])
        assert rc == B.LB_RD_OK
        ref_rho, ref_mass = _alone(kw, rho0, tick)
        np.testing.assert_array_equal(rho, ref_rho)
        np.testing.assert_allclose(mass, ref_mass, rtol=1e-12)
        st = B.lb_rd_server_stats(srv)
        assert (st["ticks"], st["launches"]) == (1, launches)
    finally:
        B.lb_rd_server_destroy(srv)


def test_memory_budget_queues_and_rejects():
    kw, rho0, _ = _request(10, 128, 1, 40)
    need = 2 * 2 * 9 * 128 * 128 * 4 + 2 * 128 * 128 * 4
    srv = B.lb_rd_server_create(hbm_budget_bytes=int(need * 1.5), max_slots=8, steps_per_tick=8)
    try:
        # fits only one at a time: the second waits for the first to finish
        t1 = B.lb_rd_submit(srv, B.make_config(**kw), rho0, 40)
        t2 = B.lb_rd_submit(srv, B.make_config(**kw), rho0, 40)
        big_kw, big_rho, _ = _request(11, 512, 1, 5)
        t3 = B.lb_rd_submit(srv, B.make_config(**big_kw), big_rho, 5)  # larger than the whole budget
        B.lb_rd_server_drain(srv, 60000)
        rc1, r1, _, s1 = _wait(srv, t1, 2, 128)
        rc2, r2, _, s2 = _wait(srv, t2, 2, 128)
        assert rc1 == rc2 == B.LB_RD_OK
        np.testing.assert_array_equal(r1, r2)
        assert s2["start_ns"] >= s1["end_ns"] - 5_000_000  # admitted after the first released its memory
        rc3, _, _, s3 = _wait(srv, t3, 2, 512)
        assert rc3 == B.LB_RD_ENOMEM and s3["status"] == B.LB_RD_ENOMEM
    finally:
        B.lb_rd_server_destroy(srv)


def test_submit_validation():
    srv = B.lb_rd_server_create(hbm_budget_bytes=1 << 28, max_slots=2, steps_per_tick=4)
    try:
        kw, rho0, _ = _request(20, 32, 1, 10)
        with pytest.raises(B.LbRdError):
            B.lb_rd_submit(srv, B.make_config(**dict(kw, precision="fp32_bf16dev")), rho0, 10)
        with pytest.raises(B.LbRdError):
            B.lb_rd_submit(srv, B.make_config(**kw), rho0, 0)
        with pytest.raises(B.LbRdError):
            B.lb_rd_submit(srv, B.make_config(**dict(kw, tau=[0.5, 0.6])), rho0, 10)
        t = B.lb_rd_submit(srv, B.make_config(**kw), rho0, 10)
        rc, _, _, _ = _wait(srv, t, 2, 32)
        assert rc == B.LB_RD_OK
    finally:
        B.lb_rd_server_destroy(srv)


def test_destroy_with_requests_in_flight():
    srv = B.lb_rd_server_create(hbm_budget_bytes=1 << 30, max_slots=4, steps_per_tick=4)
    kw, rho0, _ = _request(30, 256, 1, 10)
    for _ in range(6):
        B.lb_rd_submit(srv, B.make_config(**kw), rho0, 2000)
    time.sleep(0.05)
    B.lb_rd_server_destroy(srv)  # must not hang or fault


def test_fp64_server_equals_oracle_bitwise():
    """An FP64 server: requests of different sizes, relaxation times and step
    counts (a point-source sweep over D at D t = const, Sec. II.B) finish at
    different ticks; each result equals the oracle element by element."""
    import oracle as orc
    from oracle import Reaction

    srv = B.lb_rd_server_create(hbm_budget_bytes=1 << 28, max_slots=3, steps_per_tick=16, precision="fp64")
    try:
        jobs = []
        for j, D in enumerate((0.02, 0.04, 0.1, 1.0 / 6.0)):
            L = 40 + 10 * j
            rho0 = np.zeros((2, L, L))
            rho0[0, L // 2, L // 2] = 1.0
            tau = 3.0 * D + 0.5
            kw = dict(lattice="D2Q9", nspecies=2, nx=L, ny=L, tau=[tau, tau], reaction="linear", kappa=0.01,
                      precision="fp64")
            steps = int(round(2.0 / D))
            jobs.append((kw, rho0, steps, B.lb_rd_submit(srv, B.make_config(**kw), rho0, steps)))
        for kw, rho0, steps, t in jobs:
            rc, rho, mass, st = _wait(srv, t, 2, kw["nx"])
            assert rc == B.LB_RD_OK and st["steps"] == steps
            ref = orc.density("D2Q9", orc.run("D2Q9", kw["tau"], Reaction("linear", kappa=0.01),
                                              orc.init("D2Q9", rho0), steps))
            np.testing.assert_array_equal(rho, ref)
            # A -> B conserves the total: sum of both species stays 1
            assert abs(mass.sum() - 1.0) < 1e-13
    finally:
        B.lb_rd_server_destroy(srv)


def test_inplace_requests_mix_and_double_the_residents():
    """In-place (one state copy) FP32 requests next to two-copy ones give the
    single-handle bits; under a budget that holds one two-copy request, two
    in-place requests are resident at once."""
    kw, rho0, _ = _request(40, 128, 1, 60)
    kw2, rho2, _ = _request(41, 70, 2, 45)  # nx % 4 != 0: one site per thread
    reqs = [(dict(kw, inplace=True), rho0, 60), (kw, rho0, 61), (dict(kw, inplace=True), rho0, 33),
            (dict(kw2, inplace=True), rho2, 45)]
    srv = B.lb_rd_server_create(hbm_budget_bytes=1 << 30, max_slots=4, steps_per_tick=16)
    try:
        ts = [B.lb_rd_submit(srv, B.make_config(**c), r, n) for c, r, n in reqs]
        for (c, r, n), t in zip(reqs, ts):
            rc, rho, _, _ = _wait(srv, t, 2, c["nx"])
            assert rc == B.LB_RD_OK
            ref, _ = _alone(dict(c, inplace=False), r, n)
            np.testing.assert_array_equal(rho, ref)
    finally:
        B.lb_rd_server_destroy(srv)
    state = 2 * 9 * 128 * 128 * 4
    rho_b = 2 * 128 * 128 * 4
    budget = int(2 * (state + rho_b) * 1.02)  # two one-copy requests, but one two-copy request only
    for inplace, concurrent in ((True, True), (False, False)):
        srv = B.lb_rd_server_create(hbm_budget_bytes=budget, max_slots=4, steps_per_tick=8)
        try:
            c = dict(kw, inplace=inplace)
            t1 = B.lb_rd_submit(srv, B.make_config(**c), rho0, 400)
            t2 = B.lb_rd_submit(srv, B.make_config(**c), rho0, 400)
            B.lb_rd_server_drain(srv, 60000)
            _, r1, _, s1 = _wait(srv, t1, 2, 128)
            _, r2, _, s2 = _wait(srv, t2, 2, 128)
            np.testing.assert_array_equal(r1, r2)
            assert (s2["start_ns"] < s1["end_ns"]) == concurrent, (inplace, s1, s2)
        finally:
            B.lb_rd_server_destroy(srv)


@pytest.mark.parametrize("precision", ["fp32_bf16dev", "fp32_fp16dev"])
@pytest.mark.parametrize("sides", [[(64, 41), (36, 17), (68, 9), (128, 30)], [(64, 41), (40, 17), (72, 9), (128, 30)]],
                         ids=["nx%4", "nx%8"])
def test_half_storage_requests_equal_single_handles(precision, sides):
    """A server of 16-bit deviation storage: ticks run a 16-bit depth-K
    kernel over all resident requests (the one-column kernel, K = 4 steps per
    launch, unless every request has nx % 8 == 0: the two-column kernel, K =
    5), one launch for the rest; every result is bitwise a single handle's
    (which runs single steps: each level rounds the deviations as a single
    step stores them)."""
    reqs = []
    for j, (side, steps) in enumerate(sides):
        kw, rho0, _ = _request(60 + j, side, 1 + j % 2, steps)
        reqs.append((dict(kw, precision=precision), rho0, steps))
    srv = B.lb_rd_server_create(hbm_budget_bytes=1 << 30, max_slots=4, steps_per_tick=16, precision=precision)
    try:
        tickets = [B.lb_rd_submit(srv, B.make_config(**kw), rho0, steps) for kw, rho0, steps in reqs]
        for (kw, rho0, steps), t in zip(reqs, tickets):
            rc, rho, mass, _ = _wait(srv, t, 2, kw["nx"])
            assert rc == B.LB_RD_OK
            ref_rho, _ = _alone(dict(kw, tb_depth=1), rho0, steps)
            np.testing.assert_array_equal(rho, ref_rho)
        assert B.lb_rd_server_stats(srv)["launches"] < sum(r[2] for r in reqs) // 2
    finally:
        B.lb_rd_server_destroy(srv)


def test_least_remaining_work_ticks():
    """tick_sites > 0: each tick advances the requests with the least
    remaining work (sites x steps left) first, enough of them to make up
    tick_sites sites; the others wait.  Every request still finishes with
    the bits of a single handle, and a short request submitted beside long
    ones finishes first."""
    reqs = [_request(70, 128, 1, 600), _request(71, 128, 2, 600), _request(72, 96, 1, 20),
            _request(73, 64, 4, 300), _request(74, 100, 1, 45)]
    srv = B.lb_rd_server_create(hbm_budget_bytes=1 << 30, max_slots=8, steps_per_tick=16, tick_sites=20000)
    try:
        tickets = [B.lb_rd_submit(srv, B.make_config(**kw), rho0, steps) for kw, rho0, steps in reqs]
        ends = {}
        for (kw, rho0, steps), t in zip(reqs, tickets):
            rc, rho, _, st = _wait(srv, t, 2, kw["nx"])
            assert rc == B.LB_RD_OK and st["steps"] == steps
            ref_rho, _ = _alone(kw, rho0, steps)
            np.testing.assert_array_equal(rho, ref_rho)
            ends[steps] = st["end_ns"]
        assert ends[20] < ends[600]
    finally:
        B.lb_rd_server_destroy(srv)
