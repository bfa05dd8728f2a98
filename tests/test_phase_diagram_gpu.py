"""Phase-diagram sweep (1024 Gray-Scott instances of 256^2 on the 32 x 32
(F, k) grid, noisy-square init, 10000 steps) in one batch per storage
format, every instance labelled by linear theory (Sec. III.B-C) and by its
simulated outcome (decayed to the trivial state, uniform, or a pattern with
its dominant wavelength, Eq. reac_diff35).

What linear theory fixes, checked on every instance of the FP32 run:
* a uniform end state is a linearly stable fixed point: the instance's
  larger-v state is labelled "stable" and the field sits on it;
* a decayed instance sits on the trivial state u = 1, v = 0.
Equal accuracy of the storage formats: FP32, bf16 and fp16 deviation
storage give the same outcome on at least 99 % of the instances, and the
median wavelength difference over pattern instances is below 1 %
(chaotic and still-spreading patterns differ pointwise, so single
wavelengths are not compared there).
Sampled instances (uniform, decayed and three stationary patterns) are run
by the FP64 oracle over the full 10000 steps: same outcome, same uniform
state, wavelength within 2 %.
"""
import numpy as np
import pytest

import oracle as orc
from oracle import Reaction
from paper_1007_3109_gb300 import analysis, inputs, studies

pytestmark = pytest.mark.gpu

T = 10000
W = inputs.WORKLOADS["gs_sweep_256"]
N = W["nx"]
F, K = inputs.sweep_params()
SAMPLES = (514, 1023, 470, 341, 208)  # uniform, decayed, three stationary patterns


@pytest.fixture(scope="module")
def runs():
    out = {}
    for prec in ("fp32", "fp32_bf16dev", "fp32_fp16dev"):
        r = studies.phase_diagram(prec, T, keep=SAMPLES if prec == "fp32" else ())
        out[prec] = (r["outcome"], r["fields"])
    return out


def test_uniform_and_decayed_states_agree_with_linear_theory(runs):
    res, _ = runs["fp32"]
    counts = {}
    for i, o in enumerate(res):
        c = analysis.gs_classify(float(F[i]), float(K[i]), *W["D"])
        counts[o["outcome"]] = counts.get(o["outcome"], 0) + 1
        if o["outcome"] == "uniform":
            assert c["label"] == "stable", (i, c)
            u, v = c["state"]
            assert abs(o["umean"] - u) < 1e-5 and abs(o["mean"] - v) < 1e-5, (i, o, c)
        elif o["outcome"] == "decayed":
            assert abs(o["umean"] - 1.0) < 1e-3, (i, o)
    assert min(counts.get(x, 0) for x in ("decayed", "uniform", "pattern")) > 50, counts


@pytest.mark.parametrize("prec", ["fp32_bf16dev", "fp32_fp16dev"])
def test_storage_formats_give_the_same_phase_diagram(runs, prec):
    ref, _ = runs["fp32"]
    got, _ = runs[prec]
    same = sum(a["outcome"] == b["outcome"] for a, b in zip(ref, got))
    assert same >= 0.99 * len(ref), same
    rel = [abs(a["wavelength"] - b["wavelength"]) / a["wavelength"] for a, b in zip(ref, got)
           if a["outcome"] == b["outcome"] == "pattern"]
    assert len(rel) > 50 and np.median(rel) < 0.01, (len(rel), np.median(rel))


def test_sampled_instances_against_the_oracle(runs):
    res, keep = runs["fp32"]
    taus = [float(t) for t in orc.tau_from_diffusion(np.array(W["D"]))]
    for i in SAMPLES:
        rho0 = inputs.rho0_square(N, N, seed=W["seed"] + i)
        ref = orc.density("D2Q9", orc.run("D2Q9", taus, Reaction("gray_scott", F=float(F[i]), k=float(K[i])),
                                          orc.init("D2Q9", rho0), T))
        o_ref = analysis.pattern_outcome(ref[1])
        assert res[i]["outcome"] == o_ref["outcome"], (i, res[i], o_ref)
        if o_ref["outcome"] == "pattern":
            assert res[i]["wavelength"] == pytest.approx(o_ref["wavelength"], rel=0.02), (i, res[i], o_ref)
        else:
            np.testing.assert_allclose(keep[i], ref, atol=1e-5, err_msg=f"instance {i}")
