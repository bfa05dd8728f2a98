"""The C ABI without a GPU: the library loads, exports every declared entry
point, and validates configurations on the host."""
import os
import re

import pytest

from paper_1007_3109_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^LB_RD_API\s+[\w\s\*]*?\b(lb_rd_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return B.lib()


def test_header_declares_the_paper_entry_points():
    names = declared_symbols()
    for required in ("lb_rd_create", "lb_rd_init", "lb_rd_step", "lb_rd_moments", "lb_rd_submit", "lb_rd_poll",
                     "lb_rd_batch_create", "lb_rd_batch_step", "lb_rd_autotune", "lb_rd_step_noalloc"):
        assert required in names, required


def test_library_exports_every_declared_symbol(lib):
    exported = set(os.popen(f"nm -D --defined-only {B.LIB_PATH}").read().split())
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    for n in declared_symbols():
        assert hasattr(lib, n)


def test_version_and_tau_map(lib):
    assert "sm_103a" in B.lb_rd_version()
    assert B.lb_rd_tau_from_diffusion(0.1) == pytest.approx(0.8)
    assert B.lb_rd_tau_from_diffusion(1.0 / 6.0) == 1.0


def _cfg(**kw):
    base = dict(lattice="D2Q9", nspecies=2, nx=64, ny=48, tau=(0.8, 0.65), reaction="gray_scott", F=0.04, k=0.06,
                precision="fp32")
    base.update(kw)
    return B.make_config(**base)


@pytest.mark.parametrize("kw,msg", [
    (dict(tau=(0.5, 0.65)), "tau[0]"),
    (dict(tau=(0.8, 0.4)), "tau[1]"),
    (dict(nspecies=5, tau=(0.8,) * 4), "nspecies"),
    (dict(nspecies=3, tau=(0.8,) * 3), "Gray-Scott"),
    (dict(nspecies=3, tau=(0.8,) * 3, reaction="linear"), "A -> B"),
    (dict(nspecies=3, tau=(0.8, 0.7, 0.4)), "tau[2]"),
    (dict(nspecies=1, reaction="gray_scott"), "Gray-Scott"),
    (dict(reaction="mass_action"), "nreactions"),
    (dict(reaction="mass_action", network=([-1.0], [(1, 0)], [(-1, 1)])), "rate"),
    (dict(reaction="mass_action", network=([1.0], [(4, 0)], [(-1, 1)])), "order"),
    (dict(reaction="mass_action", network=([1.0], [(1, 0)], [(-5, 1)])), "change"),
    (dict(reaction="mass_action", network=([1.0], [(1, 0, 1)], [(-1, 1, 0)])), "beyond nspecies"),
    (dict(reaction="mass_action", network=([1.0], [(1, 0)], [(-1, 1)]), precision="fp32_bf16dev"), "FP64 or FP32"),
    (dict(nspecies=4, tau=(0.8,) * 4, reaction="none", precision="fp32_fp16dev"), "FP64 or FP32"),
    (dict(nx=0), "nx"),
    (dict(ny=70000), "nx and ny"),
    (dict(lattice=7), "lattice"),
    (dict(precision=9), "precision"),
    (dict(reaction=5), "reaction"),
    (dict(tb_depth=9), "tb_depth"),
    (dict(tb_depth=-1), "tb_depth"),
    (dict(tb_depth=4, precision="fp64"), "tb_depth > 1"),
    (dict(tb_depth=2, inplace=True), "tb_depth > 1"),
    (dict(tb_depth=3, nspecies=3, tau=(0.8,) * 3, reaction="none"), "tb_depth > 1"),
])
def test_config_validation_rejects(lib, kw, msg):
    with pytest.raises(B.LbRdError) as ei:
        B.lb_rd_check_config(_cfg(**kw))
    assert ei.value.status == B.LB_RD_EINVAL
    assert msg in str(ei.value)


def test_config_validation_accepts_networks_and_four_species(lib):
    net = ([0.3, 0.01], [(1, 1, 0, 0), (0, 0, 1, 0)], [(-1, -1, 1, 0), (0, 0, -1, 1)])
    n4 = B.lb_rd_check_config(_cfg(nspecies=4, tau=(0.8, 0.7, 0.9, 1.2), reaction="mass_action", network=net))
    n2 = B.lb_rd_check_config(_cfg())
    assert n4 > 1.9 * n2
    B.lb_rd_check_config(_cfg(nspecies=3, tau=(0.8,) * 3, reaction="none", precision="fp64"))


def test_config_validation_accepts_and_sizes(lib):
    n = B.lb_rd_check_config(_cfg())
    # two FP32 copies of 2 x 9 planes of 48 x 64 plus the rho cache
    assert n >= 2 * 2 * 9 * 48 * 64 * 4 + 2 * 48 * 64 * 4
    n64 = B.lb_rd_check_config(_cfg(precision="fp64"))
    assert n64 > n
    nh = B.lb_rd_check_config(_cfg(precision="fp32_bf16dev"))
    assert nh < n
    # steps per launch do not change the memory (the last field of the struct reaches the library)
    for d in range(9):
        assert B.lb_rd_check_config(_cfg(tb_depth=d)) == n
    assert B.lb_rd_check_config(_cfg(tb_depth=1, precision="fp64")) == n64


def test_server_and_batch_reject_bad_configs_on_the_host(lib):
    # validation happens before any device call
    cfg = B.lb_rd_server_config(0, 4, 8, 0, 2, 1, None)
    out = B.c_void_p()
    assert lib.lb_rd_server_create(B.ctypes.byref(cfg), B.ctypes.byref(out)) == B.LB_RD_EINVAL
    cfg = B.lb_rd_server_config(1 << 30, 4, 8, 0, 2, 7, None)  # unknown precision
    assert lib.lb_rd_server_create(B.ctypes.byref(cfg), B.ctypes.byref(out)) == B.LB_RD_EINVAL
    cfg = B.lb_rd_server_config(1 << 30, 4, 8, 0, 3, 0, None)  # three species
    assert lib.lb_rd_server_create(B.ctypes.byref(cfg), B.ctypes.byref(out)) == B.LB_RD_EINVAL
    cfg = B.lb_rd_server_config(1 << 30, 4, 8, 0, 2, 1, None, -1)  # negative tick_sites
    assert lib.lb_rd_server_create(B.ctypes.byref(cfg), B.ctypes.byref(out)) == B.LB_RD_EINVAL
    assert lib.lb_rd_batch_create(None, 0, B.ctypes.byref(out)) == B.LB_RD_EINVAL
    assert lib.lb_rd_poll(None, 1, None, None, None) == B.LB_RD_EINVAL


def test_variant_table_on_the_host(lib):
    n = B.lb_rd_variant_count("fp32")
    names = [B.lb_rd_variant_name("fp32", v) for v in range(n)]
    assert len(set(names)) == n and names[0] == "64x2_minb4"
    assert any(x.startswith("bulk") for x in names) and any(x.startswith("tb2") for x in names)
    steps = [B.variant_steps(x) for x in names if x.startswith("deep")]
    assert sorted(set(steps)) == list(range(1, 9))
    assert sum(B.variant_steps(x) == 1 for x in names) == 15  # 14 one-step kernels and deep1_
    assert all(B.variant_steps(x) == int(x[4]) for x in names if x.startswith("deep"))
    assert B.lb_rd_variant_count("fp64") == 1
    half = [B.lb_rd_variant_name("fp32_bf16dev", v) for v in range(B.lb_rd_variant_count("fp32_bf16dev"))]
    assert half == [B.lb_rd_variant_name("fp32_fp16dev", v) for v in range(len(half))]
    assert sorted(set(B.variant_steps(x) for x in half)) == [1, 2, 3, 4, 5, 6]
    assert all(B.variant_steps(x) == int(x[5]) for x in half if x.startswith(("hdeep", "hpair")))


def test_null_arguments_are_errors_not_crashes(lib):
    assert lib.lb_rd_create(None, None) == B.LB_RD_EINVAL
    assert lib.lb_rd_step(None, 1) == B.LB_RD_EINVAL
    assert lib.lb_rd_moments(None, None, None, 0) == B.LB_RD_EINVAL
    assert lib.lb_rd_destroy(None) == B.LB_RD_OK


def test_inplace_config_validation_and_size(lib):
    base = dict(lattice="D2Q9", nspecies=2, nx=512, ny=512, tau=[0.8, 0.65], reaction="gray_scott", F=0.04, k=0.06,
                precision="fp32")
    two = B.lb_rd_check_config(B.make_config(**base))
    one = B.lb_rd_check_config(B.make_config(**base, inplace=True))
    assert two - one == 2 * 9 * 512 * 512 * 4  # one state copy instead of two
    with pytest.raises(B.LbRdError) as ei:
        B.lb_rd_check_config(B.make_config(**dict(base, precision="fp32_bf16dev"), inplace=True))
    assert "in-place" in str(ei.value)
    cfg = B.make_config(**base)
    cfg.streaming = 2
    with pytest.raises(B.LbRdError):
        B.lb_rd_check_config(cfg)
    out = B.c_void_p()
    # batches take in-place FP32 instances only (checked before any device call)
    for bad in (dict(base, precision="fp64"),):
        cfgs = (B.lb_rd_config * 1)(B.make_config(**bad, inplace=True))
        assert lib.lb_rd_batch_create(cfgs, 1, B.ctypes.byref(out)) == B.LB_RD_EINVAL
