"""Benchmark of the fused LB reaction-diffusion step on GB300.

Workload (default): gs_8192 -- Gray-Scott, two species, D2Q9, 8192 x 8192
periodic, FP32, D_u = 0.1, D_v = 0.05, F = 0.037, k = 0.06, 256 random
16 x 16 spots (u = 0.5, v = 0.25) plus 1 % noise.  One benchmark step is one
LB time step over the whole grid: one launch of the fused kernel (pull-stream,
rho_s = sum_i f_i,s, Gray-Scott source, BGK relaxation, store) with the FP64
mass reduction of rho_s fused in.  The state (9.66 GB in two copies) is far
larger than L2, so no L2 flush is needed between steps.

Metric: MLUPS = species x sites x steps / s / 1e6 (species-site updates).

Printed: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle (the reference for this method) on a bounded window of the same
workload on the host cores instead.

Multi-GPU: the method has no exchange step here; N ranks run N independent
replicas (weak scaling) and the value is the sum over ranks of the work
divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1007_3109_gb300 import inputs  # noqa: E402

# Algorithmic bytes per site per step (read + write every stored value once).
BYTES_PER_SITE = {("D2Q9", "fp32", 2): 144, ("D2Q5", "fp32", 2): 80, ("D2Q9", "fp64", 2): 288,
                  ("D2Q9", "fp32_bf16dev", 2): 80, ("D2Q9", "fp32_fp16dev", 2): 80,
                  ("D2Q5", "fp32_bf16dev", 2): 48, ("D2Q5", "fp32_fp16dev", 2): 48}

# DRAM traffic per launch of the step kernel from an ncu capture (see
# profiles/), valid only for the kernel source it was taken on.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def _src_hash(names):
    """Hash of a kernel's source files (its own file and the headers that hold
    its arithmetic), in the order listed."""
    h = hashlib.sha256()
    for name in [names] if isinstance(names, str) else names:
        with open(os.path.join(ROOT, "paper_1007_3109_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


def reduce_over_ranks(ms: float, work: float, dist=None, device="cpu"):
    """Replicas: the job's time is the slowest rank's, its work the sum over
    ranks.  Returns (max ms, total work); without a process group, the inputs."""
    if dist is None or not dist.is_initialized():
        return ms, work
    import torch
    t_ms = torch.tensor([ms], dtype=torch.float64, device=device)
    t_w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
    dist.all_reduce(t_w, op=dist.ReduceOp.SUM)
    return float(t_ms.item()), float(t_w.item())


def workload_params(name: str, lattice: str, tau_from_diffusion):
    w = inputs.WORKLOADS[name]
    return w, [float(tau_from_diffusion(D)) for D in w["D"]]


def run_cpu_oracle_sample(name, lattice, window, steps):
    """The FP64 oracle, as it stands, on a periodic window of the workload."""
    import oracle as orc
    w, taus = workload_params(name, lattice, orc.tau_from_diffusion)
    n = w["nx"]
    rho_full_rows = inputs.rho0_spots(n, n, w["seed"], rows=slice(0, window))
    rho0 = np.ascontiguousarray(rho_full_rows[:, :window, :window])
    reac = orc.Reaction("gray_scott", F=w["reaction"]["F"], k=w["reaction"]["k"])
    f = orc.init(lattice, rho0)
    f = orc.step(lattice, taus, reac, f)  # warm the library and the pages
    t0 = time.perf_counter()
    f = orc.run(lattice, taus, reac, f, steps)
    dt = time.perf_counter() - t0
    ssu = 2 * window * window * steps
    return ssu, dt, orc.threads()


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as orc
    lattice = args.lattice
    w, taus = workload_params(args.workload, lattice, orc.tau_from_diffusion)
    window = args.ref_window
    n = w["nx"]
    rho0 = np.ascontiguousarray(inputs.rho0_spots(n, n, w["seed"], rows=slice(0, window))[:, :window, :window])
    reac = orc.Reaction("gray_scott", F=w["reaction"]["F"], k=w["reaction"]["k"])
    f = orc.init(lattice, rho0)
    for _ in range(args.warmup):
        f = orc.step(lattice, taus, reac, f)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = orc.step(lattice, taus, reac, f)
    dt = time.perf_counter() - t0
    mlups = 2 * window * window * args.steps / dt / 1e6
    sample = f"{window}x{window} periodic window of {args.workload} ({lattice}, 2 species, FP64), one oracle step per bench step"
    line = {"metric": "MLUPS", "value": mlups, "unit": "MLUPS (species-site updates/s / 1e6)", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "lattice": lattice, "nx": window, "ny": window, "species": 2,
                       "precision": "fp64", "sample_of": f"{n}x{n}"},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": orc.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def batch_mode(args):
    """gs_sweep_256: 1024 Gray-Scott instances of 256^2 on the (F, k) grid, one
    persistent launch per step over all of them (graph-captured), against a
    plain loop that steps every instance through its own handle."""
    import torch
    from paper_1007_3109_gb300 import binding as B
    torch.cuda.set_device(0)
    w = inputs.WORKLOADS["gs_sweep_256"]
    F, k = inputs.sweep_params()
    n = w["nx"]
    ninst = args.instances or w["instances"]
    taus = [float(B.lb_rd_tau_from_diffusion(D)) for D in w["D"]]
    cfgs = [dict(lattice=args.lattice, nspecies=2, nx=n, ny=n, tau=taus, reaction="gray_scott", F=float(F[i]),
                 k=float(k[i]), precision=args.precision) for i in range(ninst)]
    rho0s = [inputs.rho0_square(n, n, seed=w["seed"] + i) for i in range(ninst)]
    K, W = args.steps, args.warmup
    ssu = 2 * n * n * ninst * K
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per_launch = {}
    with B.Batch(cfgs) as b:
        for i in range(ninst):
            b.init(i, rho0s[i])
        # 1, 2 (every nx a multiple of 256), 4, 5, 6, 8 time steps per launch; the fastest is the result
        for spl in [int(x) for x in args.batch_k.split(",")]:
            try:
                b.set_steps_per_launch(spl)
            except B.LbRdError:
                continue
            b.step(W)
            torch.cuda.synchronize()
            _, l0 = B.lb_rd_batch_get_time(b.b)
            ev0.record()
            b.step(K)
            ev1.record()
            torch.cuda.synchronize()
            _, l1 = B.lb_rd_batch_get_time(b.b)
            per_launch[spl] = (ev0.elapsed_time(ev1), l1 - l0)
        steps_per_launch = min(per_launch, key=lambda kk: per_launch[kk][0])
        batched_ms, launches = per_launch[steps_per_launch]
        mass0 = b.moments(0)[1]
        t_batch = B.lb_rd_batch_get_time(b.b)[0]
    # plain loop: every instance through its own handle, instance after instance,
    # with the autotuner's choice for 256^2 (one handle tuned; handles created
    # afterwards start from its choice, K-step variants included)
    first = B.Simulation(**cfgs[0])
    first.init(rho0s[0])
    B.lb_rd_autotune(first.h, iters=5)
    loop_variant = B.lb_rd_handle_variant_name(first.h, B.lb_rd_get_variant(first.h))
    sims = [first] + [B.Simulation(**c) for c in cfgs[1:]]
    for sim, r in zip(sims, rho0s):
        sim.init(r).step(t_batch - K)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0.record()
    for sim in sims:
        sim.step(K)
    ev1.record()
    torch.cuda.synchronize()
    loop_ms = ev0.elapsed_time(ev1)
    loop_wall = (time.perf_counter() - t0) * 1e3
    np.testing.assert_allclose(sims[0].mass(), mass0, rtol=1e-12)
    for sim in sims:
        sim.close()
    peak, peak_kind = measured_peaks()
    bps = BYTES_PER_SITE[(args.lattice, args.precision, 2)]
    line = {"metric": "MLUPS", "value": ssu / (batched_ms / 1e3) / 1e6, "unit": "MLUPS (species-site updates/s / 1e6)",
            "n_gpus": 1, "steps": K, "warmup": W, "ms_per_step": batched_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else args.precision,
            "data": "synthetic",
            "config": {"workload": "gs_sweep_256", "lattice": args.lattice, "instances": ninst, "nx": n, "ny": n,
                       "species": 2, "precision": args.precision, "graph_steps": 64,
                       "steps_per_launch": steps_per_launch,
                       "batched_ms_per_step_by_steps_per_launch": {str(k): v[0] / K for k, v in per_launch.items()},
                       "l2": f"no flush: state of {2 * ninst * sim_state_bytes(args.lattice, args.precision, n) / 1e9:.2f} GB"},
            "roofline": {"bound": "hbm", "achieved": bps * n * n * ninst / (batched_ms / launches / 1e3) / 1e9,
                         "peak": peak, "unit": "GB/s", "peak_kind": peak_kind,
                         "bytes_per_site_per_launch": bps, "steps_per_launch": K / launches,
                         "effective_per_step_GBs": bps * n * n * ninst / (batched_ms / K / 1e3) / 1e9},
            "plain_loop": {"value": ssu / (loop_ms / 1e3) / 1e6, "ms_per_step": loop_ms / K,
                           "wall_ms_per_step": loop_wall / K, "variant": loop_variant},
            "speedup_vs_plain_loop": loop_ms / batched_ms, "gpu_launches": int(launches)}
    line["roofline"]["frac"] = line["roofline"]["achieved"] / peak
    if not args.no_cpu:
        # the FP64 oracle, as it stands, on the first 16 instances of the sweep
        import oracle as orc
        from oracle import Reaction
        nsample = min(16, ninst)
        otaus = [float(t) for t in orc.tau_from_diffusion(np.array(w["D"]))]
        t_cpu, ssu_cpu = 0.0, 0
        for i in range(nsample):
            f = orc.init(args.lattice, rho0s[i])
            reac = Reaction("gray_scott", F=float(F[i]), k=float(k[i]))
            t0 = time.perf_counter()
            orc.run(args.lattice, otaus, reac, f, args.cpu_steps)
            t_cpu += time.perf_counter() - t0
            ssu_cpu += 2 * n * n * args.cpu_steps
        line["cpu_baseline"] = {"value": ssu_cpu / t_cpu / 1e6, "unit": "MLUPS", "cores": orc.threads(),
                                "kind": "oracle",
                                "sample": f"{nsample} instances of gs_sweep_256 (256^2, their own F and k), "
                                          f"{args.cpu_steps} FP64 oracle steps each ({t_cpu:.1f} s)"}
    print(json.dumps(line))
    return 0


def serving_mode(args):
    """gs_serving: a seeded Poisson stream of Gray-Scott requests (side in
    [64, 2048], diffusion scale in {1, 2, 4}, steps uniform in [1e3, 5e4]
    times --steps-scale) replayed in real time against the continuous-batching
    server and against a serial first-in first-out loop of plain handles."""
    import torch
    from paper_1007_3109_gb300 import binding as B
    torch.cuda.set_device(0)
    w = inputs.WORKLOADS["gs_serving"]
    nreq = args.requests
    req = inputs.serving_requests(nreq, w["seed"], rate=1.0)
    steps = np.maximum(1, np.round(req["steps"] * args.steps_scale)).astype(np.int64)
    sides, scales = req["side"], req["scale"]
    ssu = 2 * sides.astype(np.float64) ** 2 * steps
    capacity = args.capacity_mlups * 1e6  # SSU/s the server sustains on this stream (a saturated run's figure)
    rate = args.load * capacity / ssu.mean()
    # the seeded unit-rate stream, rescaled; load 0: every request submitted at once (saturation)
    arrivals = req["arrival_s"] / rate if args.load > 0 else np.zeros(nreq)
    F, k = w["reaction"]["F"], w["reaction"]["k"]

    def cfg(j, server=True):
        D = np.array(w["D"]) * scales[j]
        # --inplace: the server keeps one state copy per request
        inplace = bool(server and args.inplace)
        return dict(lattice="D2Q9", nspecies=2, nx=int(sides[j]), ny=int(sides[j]),
                    tau=[float(B.lb_rd_tau_from_diffusion(d)) for d in D], reaction="gray_scott", F=F, k=k,
                    precision="fp32", inplace=inplace)

    rho0s = [inputs.rho0_square(int(sides[j]), int(sides[j]), seed=w["seed"] + j) for j in range(nreq)]

    # continuous batching
    srv = B.lb_rd_server_create(hbm_budget_bytes=int(args.budget_gb * 1e9), max_slots=args.slots,
                                steps_per_tick=args.tick, tick_sites=args.tick_sites)
    t0 = time.perf_counter()
    tickets = []
    for j in range(nreq):
        dt = arrivals[j] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        tickets.append(B.lb_rd_submit(srv, B.make_config(**cfg(j)), rho0s[j], int(steps[j])))
    B.lb_rd_server_drain(srv, 3_600_000)
    lat, ends, starts0 = [], [], None
    for j, t in enumerate(tickets):
        rc, st = B.lb_rd_poll(srv, t)
        assert rc == B.LB_RD_OK, rc
        lat.append((st["end_ns"] - st["arrival_ns"]) / 1e9)
        ends.append(st["end_ns"])
        starts0 = st["arrival_ns"] if starts0 is None else min(starts0, st["arrival_ns"])
    stats = B.lb_rd_server_stats(srv)
    B.lb_rd_server_destroy(srv)
    makespan = (max(ends) - starts0) / 1e9
    fifo = None
    if not args.no_fifo:
        fifo = fifo_loop(args, B, cfg, sides, rho0s, steps, arrivals, nreq)
    total = ssu.sum()
    line = {"metric": "MLUPS", "value": total / makespan / 1e6, "unit": "MLUPS (species-site updates/s / 1e6)",
            "n_gpus": 1, "steps": int(steps.sum()), "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "gs_serving", "requests": nreq, "steps_scale": args.steps_scale,
                       "load": args.load, "capacity_mlups": args.capacity_mlups, "budget_gb": args.budget_gb,
                       "slots": args.slots, "steps_per_tick": args.tick, "tick_sites": args.tick_sites,
                       "arrival_rate_per_s": rate if args.load > 0 else None,
                       "inplace_requests": int(sum(1 for j in range(nreq) if cfg(j)["inplace"])),
                       "total_ssu": float(total), "makespan_s": makespan},
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(np.max(lat))},
            "server": stats, "gpu_launches": stats["launches"]}
    if fifo is not None:
        lat_fifo, makespan_fifo = fifo
        line["fifo_plain_loop"] = {"value": total / makespan_fifo / 1e6, "makespan_s": makespan_fifo,
                                   "latency_s": {"p50": float(np.percentile(lat_fifo, 50)),
                                                 "p99": float(np.percentile(lat_fifo, 99))},
                                   "handles": "autotuned per grid side before the replay (untimed)"}
    print(json.dumps(line))
    return 0


def fifo_loop(args, B, cfg, sides, rho0s, steps, arrivals, nreq):
    """The serving stream replayed against a serial first-in first-out loop
    of plain handles: (latencies, makespan)."""
    # serial FIFO plain loop on the same stream; every grid side tuned beforehand
    # (untimed), so each handle starts from the autotuner's choice for its
    # shape, K-step variants included
    for side in sorted(set(int(x) for x in sides)):
        j = int(np.nonzero(sides == side)[0][0])
        with B.Simulation(**cfg(j, server=False)) as sim:
            sim.init(rho0s[j])
            B.lb_rd_autotune(sim.h, iters=args.fifo_tune_iters)
    t0 = time.perf_counter()
    lat_fifo = []
    for j in range(nreq):
        dt = arrivals[j] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        with B.Simulation(**cfg(j, server=False)) as sim:
            sim.init(rho0s[j]).step(int(steps[j]))
            sim.moments()
        lat_fifo.append(time.perf_counter() - t0 - arrivals[j])
    return lat_fifo, time.perf_counter() - t0


def truncation_mode(args):
    """Point-source convergence study (Sec. II.B, Figs. 1-2) on the FP64 path:
    E_rho over a (D, kappa) grid at D t = 8 on 100^2 sites, and a diffusive
    refinement from 50^2 to 800^2; every run is a request to one FP64 server
    (batched launches).  The value is the study's species-site updates per
    second of wall time, submit to results on the host."""
    import torch
    from paper_1007_3109_gb300 import studies
    torch.cuda.set_device(0)
    Ds = [float(d) for d in np.geomspace(0.004, 0.3, 40)]
    kappas = (0.0025, 0.005, 0.0075, 0.01, 0.015, 0.02, 0.033)
    studies.truncation_sweep(Ds[-4:], kappas[:1], L=100, Dt=8.0)  # warm-up: library load, pools
    sw = studies.truncation_sweep(Ds, kappas, L=100, Dt=8.0)
    rf = studies.diffusive_refinement(0.05, 0.04, L0=50, t0=40, levels=5)
    E = sw["E"]
    branch = {}
    for a, kap in enumerate(kappas):
        loc = [i for i in range(1, len(Ds) - 1) if E[a, i] < E[a, i - 1] and E[a, i] < E[a, i + 1]]
        branch[str(kap)] = [{"D": Ds[i], "E": float(E[a, i])} for i in loc]
    slopes = {}
    for D in (0.02, 0.05, 0.1):
        b = int(np.argmin(np.abs(np.array(Ds) - D)))
        slopes[f"{Ds[b]:.4f}"] = studies.loglog_slope(kappas, E[:, b])
    ssu = 2 * (sw["site_steps"] + rf["site_steps"])
    wall = sw["wall_s"] + rf["wall_s"]
    line = {"metric": "MLUPS", "value": ssu / wall / 1e6, "unit": "MLUPS (species-site updates/s / 1e6)",
            "n_gpus": 1, "steps": int(sum(sw["steps"]) * len(kappas) + sum(rf["steps"])), "warmup": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "point_source_sweep", "L": 100, "Dt": 8.0, "D": [Ds[0], Ds[-1], len(Ds)],
                       "kappa": list(kappas), "refinement_L": rf["L"], "runs": len(Ds) * len(kappas) + len(rf["L"]),
                       "timing": "wall clock, submit of the first request to the last result on the host"},
            "study": {"E_min_global": {str(k): {"D": sw["D_min"][a], "E": sw["E_min"][a]} for a, k in enumerate(kappas)},
                      "local_minima": branch, "slope_E_vs_kappa": slopes,
                      "refinement": {"L": rf["L"], "E": rf["E"], "ratio": rf["ratio"], "order": rf["order"]}},
            "gpu_launches": int(sw["launches"])}
    if not args.no_cpu:
        import oracle as orc
        from oracle import Reaction
        t0 = time.perf_counter()
        cpu_ssu = 0
        for D in Ds[12:]:
            t = max(1, int(round(8.0 / D)))
            rho0 = np.zeros((2, 100, 100))
            rho0[0, 50, 50] = 1.0
            tau = float(orc.tau_from_diffusion(D))
            orc.density("D2Q9", orc.run("D2Q9", [tau, tau], Reaction("linear", kappa=0.01), orc.init("D2Q9", rho0), t))
            cpu_ssu += 2 * 100 * 100 * t
        cpu_s = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": cpu_ssu / cpu_s / 1e6, "unit": line["unit"], "cores": orc.threads(),
                                "kind": "oracle",
                                "sample": f"kappa = 0.01 row, {len(Ds) - 12} D values >= {Ds[12]:.4f}, 100^2, FP64"}
    print(json.dumps(line))
    return 0


def network_mode(args):
    """gs2x_8192: four species (two Gray-Scott pairs exchanging v) as a
    mass-action network of 10 steps, FP32, through the general kernel (one
    thread per site), K steps timed with CUDA events on the launching stream."""
    import torch
    from paper_1007_3109_gb300 import binding as B
    torch.cuda.set_device(0)
    w = inputs.WORKLOADS["gs2x_8192"]
    n = args.n or w["nx"]
    S = w["nspecies"]
    taus = [float(B.lb_rd_tau_from_diffusion(D)) for D in w["D"]]
    net = inputs.coupled_gs_network()
    prec = args.precision if args.precision in ("fp32", "fp64") else "fp32"
    rho0 = inputs.initial_density("gs2x_8192", nx=n, ny=n)
    stream = torch.cuda.current_stream()
    sim = B.Simulation("D2Q9", S, n, n, taus, "mass_action", precision=prec, track_mass=True,
                       stream=stream.cuda_stream, network=net, inplace=args.inplace)
    sim.init(torch.from_numpy(rho0).cuda())
    sim.step(args.warmup)
    nvar = B.lb_rd_handle_variant_count(sim.h)
    names = [B.lb_rd_handle_variant_name(sim.h, v) for v in range(nvar)]
    best, times = B.lb_rd_autotune(sim.h, iters=args.tune_iters or 5)
    tuning = {names[v]: (round(times[v], 4) if times[v] >= 0 else None) for v in range(nvar)}
    sim.step(3)
    torch.cuda.synchronize()
    launches0 = B.lb_rd_launch_count(sim.h)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        ev0.record(stream)
        B.lb_rd_step(sim.h, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = B.lb_rd_launch_count(sim.h) - launches0
    mass = sim.mass()
    assert np.all(np.isfinite(mass))
    sim.close()
    bps = S * 9 * (8 if prec == "fp64" else 4) * 2
    peak, peak_kind = measured_peaks()
    achieved = bps * n * n / (ms / 1e3 / args.steps) / 1e9
    line = {"metric": "MLUPS", "value": S * n * n * args.steps / (ms / 1e3) / 1e6,
            "unit": "MLUPS (species-site updates/s / 1e6)", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": "gs2x_8192", "nx": n, "ny": n, "species": S, "reaction_steps": len(net[0]),
                       "precision": prec, "variant": names[best], "autotune_ms_per_step": tuning,
                       "streaming": "in-place (AA), one state copy" if args.inplace else "ping-pong, two state copies",
                       "l2": f"no flush: state of {(0.5 if args.inplace else 1) * bps * n * n / 1e9:.1f} GB >> 129 MB L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": f"general:{names[best]} ({prec}, D2Q9, {S} species)",
                         "bytes_per_site_per_launch": bps, "peak_kind": peak_kind},
            "gpu_launches": int(launches), "clocks": clocks.summary()}
    if not args.no_cpu:
        import oracle as orc
        from oracle import Reaction
        win = args.cpu_window // 2
        r0 = np.ascontiguousarray(rho0[:, :win, :win])
        reac = Reaction.network(*net)
        f = orc.init("D2Q9", r0)
        t0 = time.perf_counter()
        orc.run("D2Q9", taus, reac, f, args.cpu_steps)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": S * win * win * args.cpu_steps / dt / 1e6, "unit": "MLUPS",
                                "cores": orc.threads(), "kind": "oracle",
                                "sample": f"{win}x{win} periodic window, {args.cpu_steps} FP64 oracle steps"}
    print(json.dumps(line))
    return 0


def parity_mode(args):
    """The parity workloads at their full step counts on the GPU and on the
    FP64 oracle: decay_128 (one species, linear reaction, D2Q9 and D2Q5,
    FP64, 2000 steps) and gs_512 (Gray-Scott 512^2, FP64 and FP32, 20000
    steps).  Parity: FP64 bit for bit over the whole run; FP32 pointwise after
    1000 steps (maximum relative error per species <= 1e-3) and, as the
    pattern then diverges under rounding, by its dominant wavelength after
    the full run (within 2 %: the library's structure-factor peak of the GPU
    field against the oracle's of its own field).  The GPU states fit in L2,
    so the GPU is timed on a sample of single steps, each after a 512 MB
    write that evicts L2, with CUDA events around every step; the oracle on
    its full runs (host cores)."""
    import torch
    import oracle as orc
    from oracle import Reaction
    from paper_1007_3109_gb300 import analysis
    from paper_1007_3109_gb300 import binding as B
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    cases = [("decay_128", "D2Q9", "fp64"), ("decay_128", "D2Q5", "fp64"), ("gs_512", "D2Q9", "fp64"),
             ("gs_512", "D2Q9", "fp32")]
    out, oracle_runs = {}, {}
    for name, lat, prec in cases:
        w = inputs.WORKLOADS[name]
        steps = args.parity_steps or w["steps"]
        early = min(1000, steps)
        n, S, r = w["nx"], w["nspecies"], w["reaction"]
        rho0 = inputs.initial_density(name)
        if (name, lat) not in oracle_runs:
            otaus = [float(t) for t in orc.tau_from_diffusion(np.array(w["D"]))]
            reac = (Reaction("linear", kappa=r["kappa"]) if r["kind"] == "linear"
                    else Reaction("gray_scott", F=r["F"], k=r["k"]))
            f = orc.init(lat, rho0)
            t0 = time.perf_counter()
            f = orc.run(lat, otaus, reac, f, early)
            dt = time.perf_counter() - t0
            ref_early = orc.density(lat, f)
            t0 = time.perf_counter()
            f = orc.run(lat, otaus, reac, f, steps - early)
            dt += time.perf_counter() - t0
            oracle_runs[(name, lat)] = (ref_early, orc.density(lat, f), S * n * n * steps / dt / 1e6, dt)
        ref_early, ref, oracle_mlups, oracle_s = oracle_runs[(name, lat)]
        gtaus = [float(B.lb_rd_tau_from_diffusion(D)) for D in w["D"]]
        kw = dict(kappa=r["kappa"]) if r["kind"] == "linear" else dict(F=r["F"], k=r["k"])
        with B.Simulation(lat, S, n, n, gtaus, r["kind"], precision=prec, stream=stream.cuda_stream, **kw) as sim:
            sim.init(rho0).step(early)
            rho_early, _ = sim.moments()
            sim.step(steps - early)
            rho, _ = sim.moments()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.parity_timed)]
            for e0, e1 in evs:
                flush.zero_()  # same stream: the step starts with L2 holding none of the state
                e0.record(stream)
                B.lb_rd_step(sim.h, 1)
                e1.record(stream)
            torch.cuda.synchronize()
            step_ms = sum(e0.elapsed_time(e1) for e0, e1 in evs) / len(evs)

        def rel(a, b):
            return (np.max(np.abs(a - b), axis=(1, 2)) / np.max(np.abs(b), axis=(1, 2))).tolist()
        case = {"steps": steps, "bitwise_equal_to_oracle": bool(np.array_equal(rho, ref)),
                f"max_rel_err_after_{early}_steps": rel(rho_early, ref_early), "max_rel_err_full_run": rel(rho, ref),
                "gpu_mlups": S * n * n / (step_ms / 1e3) / 1e6, "gpu_ms_per_step": step_ms,
                "oracle_mlups": oracle_mlups, "oracle_s_full_run": oracle_s}
        if prec == "fp64":
            assert case["bitwise_equal_to_oracle"], (name, lat, case)
        else:
            assert max(case[f"max_rel_err_after_{early}_steps"]) <= 1e-3, (name, lat, prec, case)
            lam_gpu = analysis.dominant_wavelength(rho[S - 1])["wavelength"]
            lam_ref = orc.structure_factor_peak(ref[S - 1])["wavelength"]
            case["wavelength_gpu_oracle"] = [lam_gpu, lam_ref]
            assert abs(lam_gpu - lam_ref) <= 0.02 * lam_ref, (name, lat, prec, lam_gpu, lam_ref)
        out[f"{name}/{lat}/{prec}"] = case
    main_case = out["gs_512/D2Q9/fp64"]
    line = {"metric": "MLUPS", "value": main_case["gpu_mlups"], "unit": "MLUPS (species-site updates/s / 1e6)",
            "n_gpus": 1, "steps": args.parity_timed, "warmup": 0, "ms_per_step": main_case["gpu_ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "gs_512 (FP64; decay_128 and FP32 in cases)",
                       "l2": "flushed before every timed step (512 MB write on the stream)",
                       "timed": f"{args.parity_timed} single steps after the full run"},
            "cases": out,
            "cpu_baseline": {"value": main_case["oracle_mlups"], "unit": "MLUPS", "cores": orc.threads(),
                             "kind": "oracle",
                             "sample": f"the full {main_case['steps']}-step gs_512 run "
                                       f"({main_case['oracle_s_full_run']:.1f} s)"},
            "gpu_launches": int(args.parity_timed)}
    print(json.dumps(line))
    return 0


def phase_mode(args):
    """gs_sweep_256 as a phase diagram (Sec. III.B-D, Fig. 6): the 1024-instance
    (F, k) sweep for its full 10000 steps in one batch per storage format;
    every instance labelled by linear theory and by its simulated outcome.
    The value is the FP32 batch's MLUPS over the stepping (CUDA events)."""
    import torch
    from paper_1007_3109_gb300 import studies
    torch.cuda.set_device(0)
    steps = args.phase_steps
    res = {p: studies.phase_diagram(p, steps) for p in ("fp32", "fp32_bf16dev", "fp32_fp16dev")}
    ref = res["fp32"]
    table = {}
    for lab, o in zip(ref["label"], ref["outcome"]):
        table.setdefault(lab, {}).setdefault(o["outcome"], 0)
        table[lab][o["outcome"]] += 1
    agree = {}
    for p in ("fp32_bf16dev", "fp32_fp16dev"):
        same = sum(a["outcome"] == b["outcome"] for a, b in zip(ref["outcome"], res[p]["outcome"]))
        rel = [abs(a["wavelength"] - b["wavelength"]) / a["wavelength"]
               for a, b in zip(ref["outcome"], res[p]["outcome"]) if a["outcome"] == b["outcome"] == "pattern"]
        agree[p] = {"same_outcome": same, "pattern_instances": len(rel),
                    "wavelength_rel_diff": {"median": float(np.median(rel)), "p90": float(np.percentile(rel, 90)),
                                            "within_2pct": float(np.mean(np.array(rel) <= 0.02))}}
    ssu = 2 * ref["site_steps"]
    line = {"metric": "MLUPS", "value": ssu / ref["step_s"] / 1e6, "unit": "MLUPS (species-site updates/s / 1e6)",
            "n_gpus": 1, "steps": steps, "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "gs_sweep_256", "instances": len(ref["F"]), "steps": steps},
            "by_precision_mlups": {p: 2 * r["site_steps"] / r["step_s"] / 1e6 for p, r in res.items()},
            "theory_vs_outcome": table, "precision_agreement": agree,
            "map": studies.outcome_map(ref), "gpu_launches": int(ref["launches"]),
            "gpu_launches_by_precision": {p: r["launches"] for p, r in res.items()}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gs_8192")
    ap.add_argument("--lattice", default="D2Q9", choices=["D2Q9", "D2Q5"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp32_bf16dev", "fp32_fp16dev"])
    ap.add_argument("--n", type=int, default=0, help="grid side override (same recipe, smaller grid)")
    ap.add_argument("--ref-window", type=int, default=512)
    ap.add_argument("--cpu-window", type=int, default=1024)
    ap.add_argument("--cpu-steps", type=int, default=2000,
                    help="FP64 oracle steps of the CPU baseline sample (about 10-30 s on the host cores)")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="steps of each end-to-end repetition (0: the workload's full run, 10000 for gs_8192)")
    ap.add_argument("--batch-steps", type=int, default=20,
                    help="steps of the gs_sweep_256 batched sub-measure beside the headline (0: skip)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--tune-iters", type=int, default=10)
    ap.add_argument("--mode", default="step",
                    choices=["step", "batch", "serving", "truncation", "phase", "network", "parity"])
    ap.add_argument("--parity-steps", type=int, default=0, help="parity mode: steps of the full runs (0: the workload's)")
    ap.add_argument("--parity-timed", type=int, default=200, help="parity mode: timed single steps (L2 flushed)")
    ap.add_argument("--phase-steps", type=int, default=10000)
    ap.add_argument("--inplace", action="store_true", help="one state copy (AA streaming)")
    ap.add_argument("--variant", default="", help="force a launch variant by name (after the autotune sweep)")
    ap.add_argument("--instances", type=int, default=0)
    ap.add_argument("--batch-k", default="1,2,4,5,6,8",
                    help="batch mode: time steps per launch to time (comma-separated); the fastest is the result")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--steps-scale", type=float, default=0.05)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--capacity-mlups", type=float, default=75000.0)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--slots", type=int, default=64)
    ap.add_argument("--tick", type=int, default=64)
    ap.add_argument("--no-fifo", action="store_true", help="serving mode: skip the FIFO plain-loop baseline")
    ap.add_argument("--tick-sites", type=int, default=0,
                    help="serving mode: ticks advance the least-remaining-work requests making up this many sites "
                         "(0: every resident request, every tick)")
    ap.add_argument("--fifo-tune-iters", type=int, default=1,
                    help="serving mode: autotuner iterations per grid side for the FIFO loop's handles")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)
    if args.mode == "batch":
        return batch_mode(args)
    if args.mode == "serving":
        return serving_mode(args)
    if args.mode == "truncation":
        return truncation_mode(args)
    if args.mode == "phase":
        return phase_mode(args)
    if args.mode == "network":
        return network_mode(args)
    if args.mode == "parity":
        return parity_mode(args)

    import torch
    from paper_1007_3109_gb300 import binding as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w, taus = workload_params(args.workload, args.lattice, B.lb_rd_tau_from_diffusion)
    n = args.n or w["nx"]
    F, k = w["reaction"]["F"], w["reaction"]["k"]
    rho0 = inputs.initial_density(args.workload, nx=n, ny=n)
    stream = torch.cuda.current_stream()
    sim = B.Simulation(args.lattice, 2, n, n, taus, "gray_scott", F=F, k=k, precision=args.precision,
                       track_mass=True, stream=stream.cuda_stream, inplace=args.inplace)
    rho0_dev = torch.from_numpy(rho0).cuda()
    sim.init(rho0_dev)
    nvar = B.lb_rd_handle_variant_count(sim.h)
    names = [B.lb_rd_handle_variant_name(sim.h, v) for v in range(nvar)]
    if args.variant:
        B.lb_rd_set_variant(sim.h, names.index(args.variant))
    sim.step(args.warmup)
    tuning = {}
    if args.tune_iters > 0:
        # project autotuner: every launch variant timed on this state (not advanced)
        best, times = B.lb_rd_autotune(sim.h, iters=args.tune_iters)
        tuning = {names[v]: (round(times[v], 4) if times[v] >= 0 else None) for v in range(nvar)}
    if args.variant:
        B.lb_rd_set_variant(sim.h, names.index(args.variant))
    best = B.lb_rd_get_variant(sim.h)
    sim.step(3)
    barrier()

    # -- device-timed region: K step launches and nothing else, bracketed by
    # CUDA events on the launching stream ------------------------------------
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # The clock samples (every 200 ms) span the timed region and, under the
    # same load, an untimed stretch of the same calls before it and the
    # per-launch-timed repeats after it: a short timed region alone can fall
    # between two samples.
    with ClockSampler(local) as clocks:
        t_pre = time.perf_counter()
        while time.perf_counter() - t_pre < 0.5:
            B.lb_rd_step(sim.h, args.steps)
            torch.cuda.synchronize()
        launches0 = B.lb_rd_launch_count(sim.h)
        barrier()
        ev0.record(stream)
        B.lb_rd_step(sim.h, args.steps)
        ev1.record(stream)
        barrier()
        launches = B.lb_rd_launch_count(sim.h) - launches0
        # the timed call repeated with per-launch CUDA events on the launching
        # stream (lb_rd_launch_times): the same launch plan, each launch timed
        # on its own; enough repetitions for >= 30 launches of the dominant kernel
        reps = max(1, -(-30 // max(launches, 1)))
        B.lb_rd_set_timing(sim.h, True)
        t_rep = time.perf_counter()
        while True:
            for _ in range(reps):
                B.lb_rd_step(sim.h, args.steps)
            torch.cuda.synchronize()
            if time.perf_counter() - t_rep >= 0.5:
                break
        l_ms, l_steps, l_var = B.lb_rd_launch_times(sim.h)
        B.lb_rd_set_timing(sim.h, False)
    ms_total = ev0.elapsed_time(ev1)
    steps_per_launch = args.steps / max(launches, 1)
    sites = n * n
    ssu_per_step = 2 * sites
    ms_total, work = reduce_over_ranks(ms_total, float(ssu_per_step * args.steps), dist, "cuda")
    mass = sim.mass()
    assert np.all(np.isfinite(mass)), "non-finite mass"
    value = work / (ms_total / 1e3) / 1e6

    # -- roofline of the dominant kernel -----------------------------------------
    # From the per-launch events above: the dominant kernel is the (variant,
    # steps per launch) pair with the most device time; its achieved bandwidth
    # is the algorithmic bytes of one launch (one read and one write of the
    # state, bps per site) over its mean launch time.
    peak, peak_kind = measured_peaks()
    bps = BYTES_PER_SITE[(args.lattice, args.precision, 2)]
    reps = len(l_ms) // max(launches, 1)
    by_kernel = {}
    for t, d, v in zip(l_ms, l_steps, l_var):
        e = by_kernel.setdefault((names[v], d), [0.0, 0])
        e[0] += t
        e[1] += 1
    (variant_name, dom_steps), (dom_ms, dom_n) = max(by_kernel.items(), key=lambda kv: kv[1][0])
    avg_launch_s = dom_ms / dom_n / 1e3
    achieved = bps * sites / avg_launch_s / 1e9
    effective = bps * sites * args.steps / (ms_total / 1e3) / 1e9
    launch_plan = {f"{k[0]} ({k[1]} steps)": {"launches_per_call": v[1] // reps, "mean_ms": v[0] / v[1],
                                              "share": v[0] / sum(x[0] for x in by_kernel.values())}
                   for k, v in sorted(by_kernel.items(), key=lambda kv: -kv[1][0])}
    traffic = inst_per_launch = None
    if os.path.exists(TRAFFIC_FILE):
        with open(TRAFFIC_FILE) as fh:
            tr = json.load(fh)
        ent = tr.get(f"{args.workload}/{args.lattice}/{args.precision}/{variant_name}")
        if ent and ent.get("n") == n and ent.get("src_sha") == _src_hash(ent["src"]):
            traffic = ent["bytes_per_launch"]
            inst_per_launch = ent.get("warp_inst_per_launch")
    # Instruction-issue roofline of the same kernel (the limiter of a K-step
    # launch): warp instructions per launch from the ncu capture over the
    # live launch time, against SMs x 4 schedulers x 1 instruction per clock
    # at the median SM clock sampled during the timed region.
    clk = clocks.summary()
    issue = None
    if inst_per_launch and clk.get("sm_mhz"):
        issue_peak = torch.cuda.get_device_properties(0).multi_processor_count * 4 * clk["sm_mhz"] * 1e6
        issue_ach = inst_per_launch / avg_launch_s
        issue = {"achieved": issue_ach, "peak": issue_peak, "unit": "warp instructions/s", "frac": issue_ach / issue_peak,
                 "inst_per_launch": inst_per_launch,
                 "source": "ncu smsp__inst_executed.sum of this kernel (profiles/traffic.json); peak = SMs x 4 x SM clock"}
    single = None
    if tuning:
        ones = {k: v for k, v in tuning.items() if v and B.variant_steps(k) == 1}
        if ones:
            k1 = min(ones, key=ones.get)
            gbs = bps * sites / (ones[k1] / 1e3) / 1e9
            single = {"variant": k1, "ms_per_step": ones[k1], "GBs": gbs, "frac": gbs / peak,
                      "source": "autotuner, CUDA events"}
    # Temporal-blocking depth sweep: per steps-per-launch K, the fastest variant
    # of the autotuner's sweep (K = 1: every single-step kernel).  A K-step
    # launch moves the state once (bps per site), so its HBM use per launch is
    # bps * sites / (K * ms per step).
    depth = {}
    for name, ms in tuning.items():
        if not ms:
            continue
        kk = B.variant_steps(name)
        if kk not in depth or ms < depth[kk]["ms_per_step"]:
            depth[kk] = {"variant": name, "ms_per_step": ms}
    for kk, d in depth.items():
        gbs = bps * sites / (d["ms_per_step"] * kk / 1e3) / 1e9
        d.update({"MLUPS": ssu_per_step / (d["ms_per_step"] / 1e3) / 1e6, "hbm_GBs_per_launch": gbs,
                  "hbm_frac_per_launch": gbs / peak})
    depth = {str(kk): depth[kk] for kk in sorted(depth)}

    # -- end to end through the C ABI with host buffers --------------------------
    del rho0_dev
    pinned_in = torch.from_numpy(rho0).pin_memory()
    pinned_out = torch.empty(rho0.shape, dtype=torch.float64).pin_memory()
    mass_out = np.empty(2)
    rho_in_np, rho_out_np = pinned_in.numpy(), pinned_out.numpy()
    # Three repetitions of the workload as a user runs it (each: host rho0 in,
    # the configuration's full run of e2e_steps steps, host rho out); the median
    # over them, each the slowest rank's time, is the result: the host copies
    # share the machine's memory system with other jobs.
    e2e_steps = args.e2e_steps or int(w["steps"])
    e2e_reps = []
    for _ in range(3):
        barrier()
        t0 = time.perf_counter()
        B.lb_rd_init(sim.h, rho_in_np)
        B.lb_rd_step(sim.h, e2e_steps)
        B.lb_rd_moments(sim.h, rho_out_np, mass_out)
        rep_ms, e2e_work = reduce_over_ranks((time.perf_counter() - t0) * 1e3,
                                             float(ssu_per_step * e2e_steps), dist, "cuda")
        barrier()
        e2e_reps.append(e2e_work / (rep_ms / 1e3) / 1e6)
    e2e_mlups = float(np.median(e2e_reps))
    h2d = rho0.nbytes / e2e_steps
    d2h = (rho0.nbytes + mass_out.nbytes) / e2e_steps

    state_gb = (1 if args.inplace else 2) * sim_state_bytes(args.lattice, args.precision, n) / 1e9
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS (species-site updates/s / 1e6)", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp32_bf16dev": "f32+bf16", "fp32_fp16dev": "f32+f16"}[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload, "lattice": args.lattice, "nx": n, "ny": n, "species": 2,
                   "precision": args.precision, "lb_steps_per_step": 1,
                   "mass_diagnostic": "fused into every launch (every step, or every K-th step with K steps per launch)",
                   "l2": (f"no flush: state of {state_gb:.2f} GB >> 129 MB L2" if state_gb > 0.5 else
                          f"state of {state_gb * 1e3:.1f} MB resident in the 129 MB L2 (no flush)"),
                   "parallelism": f"replicas x{world}",
                   "variant": variant_name, "autotune_ms_per_step": tuning,
                   "streaming": "in-place (AA), one state copy" if args.inplace else "ping-pong, two state copies"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": f"step_{args.precision}:{variant_name}",
                     "steps_per_launch": dom_steps, "bytes_per_site_per_launch": bps,
                     "avg_launch_ms": avg_launch_s * 1e3, "launches_timed": dom_n,
                     "timing": f"per-launch CUDA events on the launching stream, the timed call repeated {reps}x",
                     "clock_samples": "nvidia-smi every 200 ms over the timed region, 0.5 s of the same calls before "
                                      "it and the per-launch-timed repeats after it",
                     "launch_plan": launch_plan, "mean_steps_per_launch": steps_per_launch,
                     "effective_per_step_GBs": effective, "effective_frac": effective / peak,
                     "peak_kind": peak_kind, "single_step": single,
                     # a K-step launch moves the state once for K steps: it is bound by instruction
                     # issue (ncu: issue active well above DRAM throughput), not by HBM alone
                     "limiter": ("instruction issue and HBM (state moved once per launch of %d steps)" % dom_steps
                                 if dom_steps > 1 else "hbm bandwidth"),
                     "issue": issue},
        "depth_sweep": depth or None,
        "e2e": {"value": e2e_mlups, "unit": "MLUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "lb_steps": e2e_steps, "path": "lb_rd_init(host) + lb_rd_step + lb_rd_moments(host)",
                "repetitions": e2e_reps, "statistic": "median"},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        ssu, dt, cores = run_cpu_oracle_sample(args.workload, args.lattice, args.cpu_window, args.cpu_steps)
        line["cpu_baseline"] = {"value": ssu / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                                "sample": f"{args.cpu_window}x{args.cpu_window} periodic window of {args.workload}, "
                                          f"{args.cpu_steps} FP64 oracle steps ({dt:.1f} s)"}
        import oracle as orc
        all_cores = orc.threads()
        orc.set_threads(1)
        ssu1, dt1, _ = run_cpu_oracle_sample(args.workload, args.lattice, args.cpu_window // 4, args.cpu_steps // 2)
        orc.set_threads(all_cores)
        line["cpu_baseline"]["single_core"] = {
            "value": ssu1 / dt1 / 1e6, "unit": "MLUPS", "cores": 1,
            "sample": f"{args.cpu_window // 4}x{args.cpu_window // 4} window, {args.cpu_steps // 2} steps ({dt1:.1f} s)"}
    sim.close()
    if rank == 0 and args.batch_steps > 0 and args.lattice == "D2Q9" and args.precision == "fp32":
        line["batched"] = batched_sub_measure(args)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def batched_sub_measure(args):
    """gs_sweep_256 beside the headline: 1024 Gray-Scott instances of 256^2 on
    the (F, k) grid of the phase-diagram sweep (Sec. III), FP32, advanced
    args.batch_steps steps (i) batched: the library's default depth-K
    launches over the combined unit list of all instances, and (ii) by the
    plain loop, every instance through its own handle, instance after
    instance, each handle with the autotuner's choice for 256^2 (K-step
    variants included).  Both timed with CUDA events on the launching stream
    after args.warmup steps; the sampled instances of the two must agree bit
    for bit (equal accuracy)."""
    import torch
    from paper_1007_3109_gb300 import binding as B
    w = inputs.WORKLOADS["gs_sweep_256"]
    F, k = inputs.sweep_params()
    n, ninst = w["nx"], w["instances"]
    taus = [float(B.lb_rd_tau_from_diffusion(D)) for D in w["D"]]
    cfgs = [dict(lattice="D2Q9", nspecies=2, nx=n, ny=n, tau=taus, reaction="gray_scott", F=float(F[i]),
                 k=float(k[i]), precision="fp32") for i in range(ninst)]
    rho0s = [inputs.rho0_square(n, n, seed=w["seed"] + i) for i in range(ninst)]
    K, W = args.batch_steps, args.warmup
    samples = [0, ninst // 3, ninst - 1]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with B.Batch(cfgs) as b:
        for i in range(ninst):
            b.init(i, rho0s[i])
        b.step(W)
        torch.cuda.synchronize()
        _, l0 = B.lb_rd_batch_get_time(b.b)
        ev0.record()
        b.step(K)
        ev1.record()
        torch.cuda.synchronize()
        _, l1 = B.lb_rd_batch_get_time(b.b)
        batched_ms = ev0.elapsed_time(ev1)
        rho_b = [b.moments(i)[0] for i in samples]
    # the plain loop: tune one 256^2 handle; handles created afterwards start from its choice
    first = B.Simulation(**cfgs[0])
    first.init(rho0s[0])
    B.lb_rd_autotune(first.h, iters=5)
    sims = [first] + [B.Simulation(**c) for c in cfgs[1:]]
    for sim, r in zip(sims, rho0s):
        sim.init(r).step(W)
    variant = B.lb_rd_handle_variant_name(first.h, B.lb_rd_get_variant(first.h))
    torch.cuda.synchronize()
    c0 = sum(B.lb_rd_launch_count(sim.h) for sim in sims)
    ev0.record()
    for sim in sims:
        sim.step(K)
    ev1.record()
    torch.cuda.synchronize()
    loop_ms = ev0.elapsed_time(ev1)
    loop_launches = sum(B.lb_rd_launch_count(sim.h) for sim in sims) - c0
    same = all(np.array_equal(sims[i].moments()[0], rb) for i, rb in zip(samples, rho_b))
    for sim in sims:
        sim.close()
    ssu = 2 * n * n * ninst * K
    return {"workload": "gs_sweep_256", "instances": ninst, "nx": n, "ny": n, "steps": K, "warmup": W,
            "value": ssu / (batched_ms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": batched_ms / K,
            "gpu_launches": int(l1 - l0),
            "plain_loop": {"value": ssu / (loop_ms / 1e3) / 1e6, "ms_per_step": loop_ms / K,
                           "variant": variant, "gpu_launches": int(loop_launches)},
            "speedup_vs_plain_loop": loop_ms / batched_ms,
            "bitwise_equal_sampled": bool(same), "sampled_instances": samples,
            "l2": "no flush: state of 9.66 GB (two copies) per form >> 129 MB L2"}


def sim_state_bytes(lattice, precision, n):
    Q = 9 if lattice == "D2Q9" else 5
    per = {"fp32": 4 * Q, "fp64": 8 * Q}.get(precision, 4 + 2 * (Q - 1))
    return 2 * per * n * n


if __name__ == "__main__":
    sys.exit(main())
