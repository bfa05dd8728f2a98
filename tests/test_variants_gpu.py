"""Launch variants and the autotuner.

Every FP32 launch variant (tile shape, register budget, cache policy, TMA
bulk-copy staging, temporal blocking of 2 .. 8 steps per launch)
performs the same per-site operations in the same order, so their states
must agree bit for bit; the autotuner must not advance or change the
simulation state.
"""
import re

import numpy as np
import pytest

from paper_1007_3109_gb300 import binding as B
from paper_1007_3109_gb300 import inputs

pytestmark = pytest.mark.gpu

GRIDS = [("D2Q9", 2, 64, 48, "gray_scott"), ("D2Q9", 2, 1000, 50, "gray_scott"), ("D2Q5", 2, 1024, 20, "gray_scott"),
         ("D2Q9", 1, 8, 3, "linear"), ("D2Q9", 2, 70, 37, "gray_scott"), ("D2Q9", 2, 4, 5, "gray_scott"),
         ("D2Q9", 2, 512, 40, "gray_scott"), ("D2Q5", 1, 256, 9, "linear"), ("D2Q9", 2, 512, 3, "gray_scott")]


def _run(lat, S, nx, ny, reac, variant, steps=25):
    rho0 = inputs.rho0_square(nx, ny, seed=41, side=max(2, min(nx, ny) // 3))[:S] if S == 2 else \
        inputs.rho0_cosine(nx, ny, seed=41, noise=1e-3)
    kw = dict(F=0.04, k=0.06) if reac == "gray_scott" else dict(kappa=0.01)
    with B.Simulation(lat, S, nx, ny, [0.8, 0.65][:S], reac, precision="fp32", track_mass=True, **kw) as sim:
        try:
            sim.set_variant(variant)
        except B.LbRdError as err:  # the variant does not fit this grid
            assert err.status == B.LB_RD_EINVAL
            return None
        sim.init(rho0).step(steps)
        rho, mass = sim.moments()
        f = sim.distributions()
    return rho, mass, f


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: f"{g[0]}-S{g[1]}-{g[2]}x{g[3]}")
def test_every_fp32_variant_is_bitwise_identical(grid):
    lat, S, nx, ny, reac = grid
    ref = _run(lat, S, nx, ny, reac, 0)
    ran = 0
    for v in range(1, B.lb_rd_variant_count("fp32")):
        name = B.lb_rd_variant_name("fp32", v)
        out = _run(lat, S, nx, ny, reac, v)
        if out is None:
            # bulk-copy variants and deep<K>v*_ variants (16-byte staging) need nx % 4 == 0, two-step variants
            # (tb2[iw]_<threads>x<strip>_...) nx % strip == 0; the other deep<K>_ variants fit any grid
            m = re.match(r"tb2[iw]?_\d+x(\d+)_", name)
            assert ((name.startswith("bulk") or re.match(r"deep\dv", name)) and nx % 4) or \
                (m and nx % int(m.group(1))), name
            continue
        ran += 1
        rho, mass, f = out
        np.testing.assert_array_equal(rho, ref[0], err_msg=name)
        np.testing.assert_array_equal(f, ref[2], err_msg=name)
        # the fused mass adds FP32 per-tile partials in FP64: variants group them differently
        np.testing.assert_allclose(mass, ref[1], rtol=1e-6, err_msg=name)
    if nx % 512 == 0:
        assert ran == B.lb_rd_variant_count("fp32") - 1  # every variant ran, two-step ones included


@pytest.mark.parametrize("grid", [("D2Q9", 2, 70, 37, "gray_scott"), ("D2Q5", 2, 100, 9, "gray_scott"),
                                  ("D2Q9", 1, 33, 17, "linear"), ("D2Q9", 2, 100, 37, "gray_scott"),
                                  ("D2Q9", 2, 12, 5, "gray_scott"), ("D2Q5", 2, 44, 13, "linear")],
                         ids=lambda g: f"{g[0]}-S{g[1]}-{g[2]}x{g[3]}-{g[4]}")
def test_k_step_variants_over_step_counts(grid):
    """deep<K>_ variants advance K steps per launch and cover the last steps
    of a call with launches of fewer steps: every step count gives the bits of
    single steps (ragged last strip, bands of a few rows), and the densities
    the last launch writes equal those of single steps."""
    lat, S, nx, ny, reac = grid
    names = [B.lb_rd_variant_name("fp32", v) for v in range(B.lb_rd_variant_count("fp32"))]
    deep = [v for v, n in enumerate(names) if n.startswith("deep")]
    assert sorted({B.variant_steps(names[v]) for v in deep}) == [1, 2, 3, 4, 5, 6, 7, 8]
    assert any(re.match(r"deep\dv", names[v]) for v in deep)
    for steps in (1, 2, 7, 8, 9, 17, 33):
        ref = _run(lat, S, nx, ny, reac, 0, steps=steps)
        for v in deep:
            out = _run(lat, S, nx, ny, reac, v, steps=steps)
            if out is None:  # 16-byte staging needs nx % 4 == 0
                assert re.match(r"deep\dv", names[v]) and nx % 4, names[v]
                continue
            rho, mass, f = out
            np.testing.assert_array_equal(f, ref[2], err_msg=f"{names[v]} steps={steps}")
            np.testing.assert_array_equal(rho, ref[0], err_msg=f"{names[v]} steps={steps}")
            np.testing.assert_allclose(mass, ref[1], rtol=1e-6, err_msg=f"{names[v]} steps={steps}")


@pytest.mark.parametrize("nx,ny", [(64, 48), (70, 37)])
def test_k_step_calls_end_on_a_launch_that_writes_rho(nx, ny):
    """With a depth-K variant, the launches of a call (per
    lb_rd_launch_times) add up to its steps and run at most one single step
    (the plan minimises the estimated time: several single steps never are);
    a call of 20 = 4 x 5 steps runs no single step.  When the last launch has
    two or more steps it writes rho(t), so lb_rd_moments then launches only
    the export; after a last single step rho(t) is recomputed from the other
    copy (one more launch).  Densities, masses and distributions equal those
    of single steps after every call."""
    rho0 = inputs.rho0_square(nx, ny, seed=44, side=max(2, min(nx, ny) // 3))
    kw = dict(lattice="D2Q9", nspecies=2, nx=nx, ny=ny, tau=[0.8, 0.65], reaction="gray_scott", F=0.04, k=0.06,
              precision="fp32", track_mass=True)
    names = [B.lb_rd_variant_name("fp32", v) for v in range(B.lb_rd_variant_count("fp32"))]
    for name in ("deep6v_128_minb2", "deep8_128_minb2", "deep4_128_minb3"):
        if name.startswith("deep6v") and nx % 4:
            continue
        with B.Simulation(**kw) as sim, B.Simulation(**kw) as ref:
            sim.set_variant(names.index(name))
            sim.init(rho0)
            ref.init(rho0)
            B.lb_rd_set_timing(sim.h, True)
            prev = 0
            for n in (2, 7, 20, 33, 1, 13):
                sim.step(n)
                ref.step(n)
                _, steps, var = B.lb_rd_launch_times(sim.h)
                new, prev = steps[prev:], len(steps)
                assert sum(new) == n and new.count(1) <= 1, (name, n, new)
                assert all(B.variant_steps(names[v]) == d for v, d in zip(var, steps)), (name, n)
                if n == 20:
                    assert 1 not in new, (name, new)
                l0 = B.lb_rd_launch_count(sim.h)
                rho, mass = sim.moments()
                launched = B.lb_rd_launch_count(sim.h) - l0
                assert launched == (1 if new[-1] >= 2 else 2), (name, n, new, launched)
                rref, mref = ref.moments()
                np.testing.assert_array_equal(rho, rref, err_msg=f"{name} after {n}")
                np.testing.assert_allclose(mass, mref, rtol=1e-6)
                np.testing.assert_array_equal(sim.distributions(), ref.distributions())


def test_tb_depth_config_field():
    """lb_rd_config.tb_depth selects the steps per launch at creation: a
    depth-K variant of that many steps (the same bits as single steps), 1 a
    single-step variant; EINVAL where no variant of that depth fits."""
    nx, ny = 68, 21
    rho0 = inputs.rho0_square(nx, ny, seed=45, side=7)
    kw = dict(lattice="D2Q9", nspecies=2, nx=nx, ny=ny, tau=[0.8, 0.65], reaction="gray_scott", F=0.04, k=0.06,
              precision="fp32")
    with B.Simulation(**kw, tb_depth=1) as ref:
        ref.init(rho0).step(23)
        want = ref.moments()[0]
        assert B.variant_steps(B.lb_rd_handle_variant_name(ref.h, B.lb_rd_get_variant(ref.h))) == 1
    for d in range(2, 9):
        with B.Simulation(**kw, tb_depth=d) as sim:
            assert B.variant_steps(B.lb_rd_handle_variant_name(sim.h, B.lb_rd_get_variant(sim.h))) == d
            sim.init(rho0).step(23)
            np.testing.assert_array_equal(sim.moments()[0], want, err_msg=f"tb_depth {d}")
    with pytest.raises(B.LbRdError) as ei:
        B.Simulation(**dict(kw, nx=70), tb_depth=7)  # depth 7 only with 16-byte staging (nx % 4 == 0)
    assert ei.value.status == B.LB_RD_EINVAL


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q5"])
@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (7, 1), (2, 3), (5, 2)])
def test_degenerate_grids_every_variant(lat, shape):
    """Grids narrower or lower than one halo: the periodic wrap of the
    multi-step kernels (true modulo, several periods inside one warp) gives
    the bits of single steps."""
    nx, ny = shape
    rng = np.random.default_rng(1000 + nx * 31 + ny)
    rho0 = np.stack([0.5 + 0.5 * rng.random((ny, nx)), 0.25 * rng.random((ny, nx))])
    names = [B.lb_rd_variant_name("fp32", v) for v in range(B.lb_rd_variant_count("fp32"))]
    ref = None
    for v, name in enumerate(names):
        with B.Simulation(lat, 2, nx, ny, [0.8, 0.65], "gray_scott", F=0.04, k=0.06, precision="fp32") as sim:
            try:
                sim.set_variant(v)
            except B.LbRdError:
                continue  # the variant does not fit this grid
            sim.init(rho0).step(19)
            f = sim.distributions()
        if ref is None:
            ref = f
        else:
            np.testing.assert_array_equal(f, ref, err_msg=name)
    assert ref is not None


def test_autotune_leaves_the_state_unchanged():
    nx, ny = 512, 256
    rho0 = inputs.rho0_square(nx, ny, seed=42)
    kw = dict(lattice="D2Q9", nspecies=2, nx=nx, ny=ny, tau=[0.8, 0.65], reaction="gray_scott", F=0.04, k=0.06,
              precision="fp32")
    with B.Simulation(**kw) as a, B.Simulation(**kw) as b:
        a.init(rho0).step(10)
        before = a.moments()[0]
        best, times = a.autotune(iters=3)
        assert a.time == 10
        np.testing.assert_array_equal(a.moments()[0], before)
        n = B.lb_rd_variant_count("fp32")
        assert 0 <= best < n and times[best] > 0
        assert all(times[v] > 0 or times[v] == -1.0 for v in range(n))
        assert B.lb_rd_get_variant(a.h) == best
        a.step(20)
        b.init(rho0).step(30)
        np.testing.assert_array_equal(a.moments()[0], b.moments()[0])


@pytest.mark.parametrize("precision", ["fp32_bf16dev", "fp32_fp16dev"])
@pytest.mark.parametrize("nx,ny", [(64, 48), (512, 20), (12, 3)])
def test_every_half_variant_is_bitwise_identical(precision, nx, ny):
    rho0 = inputs.rho0_square(nx, ny, seed=43, side=max(2, min(nx, ny) // 3))
    kw = dict(lattice="D2Q9", nspecies=2, nx=nx, ny=ny, tau=[0.8, 0.65], reaction="gray_scott", F=0.04, k=0.06,
              precision=precision)
    outs = []
    for v in range(B.lb_rd_variant_count(precision)):
        name = B.lb_rd_variant_name(precision, v)
        with B.Simulation(**kw) as sim:
            try:
                sim.set_variant(v)
            except B.LbRdError as err:  # two columns per lane (hpair<K>_) need nx % 8 == 0
                assert err.status == B.LB_RD_EINVAL and name.startswith("hpair") and nx % 8, name
                continue
            sim.init(rho0).step(21)
            outs.append((name, sim.moments()[0], sim.distributions()))
    for name, rho, f in outs[1:]:
        np.testing.assert_array_equal(rho, outs[0][1], err_msg=name)
        np.testing.assert_array_equal(f, outs[0][2], err_msg=name)


@pytest.mark.parametrize("precision", ["fp32_bf16dev", "fp32_fp16dev"])
@pytest.mark.parametrize("grid", [("D2Q5", 2, 136, 11, "gray_scott"), ("D2Q9", 1, 72, 9, "linear"),
                                  ("D2Q9", 2, 8, 5, "gray_scott"), ("D2Q9", 2, 120, 70, "gray_scott")],
                         ids=lambda g: f"{g[0]}-S{g[1]}-{g[2]}x{g[3]}-{g[4]}")
def test_half_two_column_variants_over_lattices(precision, grid):
    """The two-column 16-bit depth-K kernels (hpair<K>_) on D2Q5, one species
    with the linear source (the reaction kind tested per site), the smallest
    grid (nx = 8: the 64-column window spans eight periods) and several
    strips and bands: the bits of single steps, over a call of 23 steps."""
    lat, S, nx, ny, reac = grid
    rho0 = inputs.rho0_square(nx, ny, seed=47, side=max(2, min(nx, ny) // 3))[:S]
    taus = [0.8, 0.65][:S]
    kw = dict(lattice=lat, nspecies=S, nx=nx, ny=ny, tau=taus, reaction=reac, F=0.04, k=0.06, kappa=0.01,
              precision=precision)
    names = [B.lb_rd_variant_name(precision, v) for v in range(B.lb_rd_variant_count(precision))]
    with B.Simulation(**kw) as ref:
        ref.set_variant(0)
        ref.init(rho0).step(23)
        want_rho, want_f = ref.moments()[0], ref.distributions()
    ran = 0
    for v, name in enumerate(names):
        if not name.startswith("hpair"):
            continue
        with B.Simulation(**kw) as sim:
            sim.set_variant(v)
            sim.init(rho0).step(23)
            np.testing.assert_array_equal(sim.moments()[0], want_rho, err_msg=name)
            np.testing.assert_array_equal(sim.distributions(), want_f, err_msg=name)
        ran += 1
    assert ran == 6
