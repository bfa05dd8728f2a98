"""The point-source convergence study of Sec. II.B on the FP64 path.

A unit mass of species A at the centre of a periodic L x L box diffuses and
turns into B at rate kappa (Eq. reac_diff2, R_A = -kappa rho_A,
R_B = +kappa rho_A, D_B = D_A).  The density of A after t steps is compared
with the unbounded-plane solution (Eq. reac_diff5) by the relative error
E_rho; every run of a sweep is compared at the same physical time
(D t = const: the same spread of the source), so t = round(Dt / D).

All runs of a study are requests to one FP64 server: they advance together,
one batched launch per step, each at its own size, relaxation time, rate
and step count, and each result is bitwise what a single FP64 handle gives.

* ``truncation_sweep``: E_rho over a grid of (D, kappa) (Fig. 1c-d, Fig. 2),
  with the minimising D per kappa.
* ``diffusive_refinement``: the same physical problem on L, 2 L, 4 L ...
  sites (dx halved, dt quartered: D fixed in lattice units, kappa / 4 and
  4 t per level); the ratio of successive errors measures the order.

And the Gray-Scott phase diagram (Sec. III.B-D, Fig. 6): ``phase_diagram``
runs the (F, k) sweep as one batch and labels every instance both by linear
theory and by its simulated outcome.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import analysis
from . import binding as B


def point_source_request(L: int, D: float, kappa: float, steps: int) -> tuple[dict, np.ndarray]:
    """Config and initial densities of one run: rho_A = 1 at (L/2, L/2),
    zero elsewhere; rho_B = 0; tau_A = tau_B from D."""
    rho0 = np.zeros((2, L, L))
    rho0[0, L // 2, L // 2] = 1.0
    tau = B.lb_rd_tau_from_diffusion(D)
    cfg = dict(lattice="D2Q9", nspecies=2, nx=L, ny=L, tau=[tau, tau], reaction="linear", kappa=float(kappa),
               precision="fp64")
    return cfg, rho0


def run_requests(runs, max_slots: int = 256, steps_per_tick: int = 64, budget: int = 64 << 30):
    """Run [(cfg, rho0, steps)] through one FP64 server.  Returns the list of
    (rho, mass) in input order and the wall time in seconds (submit of the
    first request to the result of the last on the host)."""
    out = [None] * len(runs)
    with B.Server(budget, max_slots=max_slots, steps_per_tick=steps_per_tick, nspecies=2,
                  precision="fp64") as srv:
        t0 = time.perf_counter()
        tickets = [srv.submit(rho0, steps, **cfg) for cfg, rho0, steps in runs]
        for j, t in enumerate(tickets):
            rho, mass, _ = srv.result(t)
            out[j] = (rho, mass)
        wall = time.perf_counter() - t0
        stats = srv.stats()
    return out, wall, stats


def _steps(D: float, Dt: float) -> int:
    return max(1, int(round(Dt / D)))


def truncation_sweep(Ds, kappas, L: int = 100, Dt: float = 8.0, keep_fields: bool = False) -> dict:
    """E_rho(D, kappa) at D t = Dt on an L x L box.

    Returns {"D", "kappa", "steps" (per D), "E" [kappa][D], "D_min" and
    "E_min" per kappa, "mass" [kappa][D][species], "site_steps",
    "wall_s", "launches"} (+ "rho" [kappa][D] of A when keep_fields)."""
    Ds = [float(d) for d in Ds]
    kappas = [float(k) for k in kappas]
    runs = []
    for kap in kappas:
        for D in Ds:
            cfg, rho0 = point_source_request(L, D, kap, _steps(D, Dt))
            runs.append((cfg, rho0, _steps(D, Dt)))
    results, wall, stats = run_requests(runs)
    E = np.empty((len(kappas), len(Ds)))
    mass = np.empty((len(kappas), len(Ds), 2))
    fields = []
    for a, kap in enumerate(kappas):
        row = []
        for b, D in enumerate(Ds):
            rho, m = results[a * len(Ds) + b]
            t = _steps(D, Dt)
            an = analysis.point_source(L, L, L // 2, L // 2, D, kap, t)
            E[a, b] = analysis.relative_error(an, rho[0])
            mass[a, b] = m
            if keep_fields:
                row.append(rho[0])
        fields.append(row)
    imin = np.argmin(E, axis=1)
    out = {"D": Ds, "kappa": kappas, "steps": [_steps(D, Dt) for D in Ds], "E": E,
           "D_min": [Ds[i] for i in imin], "E_min": [float(E[a, i]) for a, i in enumerate(imin)], "mass": mass,
           "site_steps": int(sum(L * L * s for _, _, s in runs)), "wall_s": wall, "launches": stats["launches"]}
    if keep_fields:
        out["rho"] = fields
    return out


def diffusive_refinement(D: float, kappa: float, L0: int = 50, t0: int = 100, levels: int = 3) -> dict:
    """E_rho of one physical problem on L0 * 2^l sites, l < levels: kappa / 4^l,
    t0 * 4^l steps.  Returns {"L", "steps", "kappa", "E", "ratio" (E_l / E_l+1),
    "order" (log2 of the ratios), "site_steps", "wall_s"}."""
    runs, Ls, steps, kaps = [], [], [], []
    for l in range(levels):
        L, t, kap = L0 * 2 ** l, t0 * 4 ** l, kappa / 4 ** l
        cfg, rho0 = point_source_request(L, D, kap, t)
        runs.append((cfg, rho0, t))
        Ls.append(L)
        steps.append(t)
        kaps.append(kap)
    results, wall, _ = run_requests(runs)
    E = [analysis.relative_error(analysis.point_source(L, L, L // 2, L // 2, D, kap, t), r[0][0])
         for (L, t, kap), r in zip(zip(Ls, steps, kaps), results)]
    ratio = [E[i] / E[i + 1] for i in range(levels - 1)]
    return {"L": Ls, "steps": steps, "kappa": kaps, "E": E, "ratio": ratio,
            "order": [math.log2(r) for r in ratio], "site_steps": int(sum(L * L * t for L, t in zip(Ls, steps))),
            "wall_s": wall}


def loglog_slope(x, y) -> float:
    """Least-squares slope of log y against log x."""
    lx, ly = np.log(np.asarray(x, dtype=np.float64)), np.log(np.asarray(y, dtype=np.float64))
    return float(np.polyfit(lx, ly, 1)[0])


def phase_diagram(precision: str = "fp32", steps: int | None = None, keep=(), n_grid: int = 32) -> dict:
    """The Gray-Scott (F, k) sweep gs_sweep_256 in one batch: n_grid^2
    instances of 256^2 sites (F in [0.01, 0.08], k in [0.03, 0.07],
    D = (0.1, 0.05)), noisy-square init, ``steps`` steps (10000), then each
    instance's outcome (``analysis.pattern_outcome`` of its v field, plus the
    mean of u) and linear-theory label
    (``analysis.gs_classify``).  Returns {"F", "k", "outcome" (list of
    dicts), "label", "fields" {index: rho} for the indices in ``keep``,
    "step_s" (device time of the stepping, CUDA events), "site_steps",
    "launches" (batched kernel launches of the stepping)}."""
    import torch

    from . import inputs
    w = inputs.WORKLOADS["gs_sweep_256"]
    side, D, seed = w["nx"], w["D"], w["seed"]
    steps = w["steps"] if steps is None else steps
    F, k = inputs.sweep_params(n_grid)
    taus = [B.lb_rd_tau_from_diffusion(d) for d in D]
    cfgs = [dict(lattice="D2Q9", nspecies=2, nx=side, ny=side, tau=taus, reaction="gray_scott", F=float(F[i]),
                 k=float(k[i]), precision=precision) for i in range(len(F))]
    outcome, fields = [], {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with B.Batch(cfgs) as b:
        for i in range(len(F)):
            b.init(i, inputs.rho0_square(side, side, seed=seed + i))
        torch.cuda.synchronize()
        _, l0 = B.lb_rd_batch_get_time(b.b)
        e0.record()
        b.step(steps)
        e1.record()
        torch.cuda.synchronize()
        step_s = e0.elapsed_time(e1) / 1e3
        launches = B.lb_rd_batch_get_time(b.b)[1] - l0
        for i in range(len(F)):
            rho, _ = b.moments(i)
            o = analysis.pattern_outcome(rho[1])
            o["umean"] = float(rho[0].mean())
            outcome.append(o)
            if i in keep:
                fields[i] = rho
    labels = [analysis.gs_classify(float(F[i]), float(k[i]), *D)["label"] for i in range(len(F))]
    return {"F": F, "k": k, "outcome": outcome, "label": labels, "fields": fields, "step_s": step_s,
            "site_steps": int(len(F) * side * side * steps), "launches": int(launches)}


def outcome_map(res: dict, n_grid: int = 32) -> list[str]:
    """Rows of the (F, k) map, largest F first: '.' decayed, 'u' uniform,
    'P' pattern; k grows to the right."""
    sym = {"decayed": ".", "uniform": "u", "pattern": "P"}
    g = [sym[o["outcome"]] for o in res["outcome"]]
    return ["".join(g[i * n_grid:(i + 1) * n_grid]) for i in range(n_grid - 1, -1, -1)]
