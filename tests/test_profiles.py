"""The per-kernel DRAM traffic table the benchmark reports from: every entry
names source files that exist, matches the current source (an entry of a
kernel changed since its capture must be removed, not kept), points at a
committed capture summary, and holds figures consistent with one read and
one write of the state per launch."""
import importlib.util
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
BYTES_PER_SITE = {("D2Q9", "fp32"): 144, ("D2Q5", "fp32"): 80, ("D2Q9", "fp32_bf16dev"): 80,
                  ("D2Q9", "fp32_fp16dev"): 80, ("D2Q5", "fp32_bf16dev"): 48, ("D2Q5", "fp32_fp16dev"): 48}


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def entries():
    with open(TRAFFIC) as fh:
        d = json.load(fh)
    return sorted((k, v) for k, v in d.items() if not k.startswith("_"))


def test_table_has_the_default_kernels():
    keys = {k for k, _ in entries()}
    assert "gs_8192/D2Q9/fp32/deep5vw_256_minb1" in keys


@pytest.mark.parametrize("key,ent", entries(), ids=[k for k, _ in entries()])
def test_entry_matches_current_source(bench, key, ent):
    srcs = [ent["src"]] if isinstance(ent["src"], str) else ent["src"]
    for name in srcs:
        assert os.path.exists(os.path.join(ROOT, "paper_1007_3109_gb300", "csrc", name)), name
    assert bench._src_hash(ent["src"]) == ent["src_sha"], f"{key}: kernel source changed since the capture"


@pytest.mark.parametrize("key,ent", entries(), ids=[k for k, _ in entries()])
def test_entry_is_consistent(bench, key, ent):
    workload, lattice, precision, variant = key.split("/")
    assert workload == "gs_8192" and ent["n"] == 8192
    assert os.path.exists(os.path.join(ROOT, ent["capture"])), ent["capture"]
    alg = BYTES_PER_SITE[(lattice, precision)] * ent["n"] ** 2
    assert ent["algorithmic_bytes_per_launch"] == alg
    assert bench.BYTES_PER_SITE[(lattice, precision, 2)] * ent["n"] ** 2 == alg
    # one read and one write of the state per launch, within the halo and
    # partial-line overheads the captures show
    assert 0.95 < ent["bytes_per_launch"] / alg < 1.15
    m = re.match(r"(?:h?deep|hpair)(\d+)", variant)
    assert ent["steps_per_launch"] == (int(m.group(1)) if m else 1)
    assert ent["warp_inst_per_launch"] > 0
