#!/usr/bin/env python3
"""Benchmark of the grouped cPINN / XPINN training step on GB300.

One step = one pass of the whole hot path over all subdomains: interface
exchange, jets (value, first and second input derivatives) through every
subdomain's network at its residual, data and interface points, PDE residual
and interface terms, reverse pass, fixed-order gradient reduction and Adam.

Headline workload (the largest single-GPU configuration): XPINN inverse
diffusion on a seeded star polygon, 10 Voronoi regions x 256 independent
copies (2,560 subdomains, two networks each: u 2->40x5->1 and K 2->20x4->1
softplus, tanh/sin/cos with trained slopes), 30k residual points per region:
76.8 M residual points and 20.7 M parameters per step.  Its inputs (0.9 GB of
points and forcing, 0.3 GB of parameters and Adam moments) exceed L2; L2 is
also flushed (a 256 MB write) before every timed step, and each step is timed
alone with CUDA events on the launching stream.

The same JSON line carries, as extra keys: the per-subdomain launch loop of
the same kernels on the headline workload; the XPINN Poisson (16 uneven
subdomains) and Kovasznay cPINN (64 x 50k points) workloads, grouped and
looped; the Burgers cPINN configuration's Adam steps per second; the serving
mix (query and training-step requests, p50/p99 latency); the FP64 oracle on
the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                  [--workload c4|c2|c3|c1|...]

With N > 1 (torchrun) every rank trains its own replica (replicas only: the
path has no cross-GPU exchange); value = all ranks' residual points / the
slowest rank's time.  --impl reference times the FP64 CPU oracle instead.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "residual pts/s (jet fwd+bwd) grouped vs per-subdomain loop; query p50/p99 ms"

# DRAM traffic of the jet kernel, per workload, from one ncu capture each
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch; see profiles/).
# A key is reported only while the kernel source and the launch options are
# the ones that were measured.  Where the full launch is too large to capture,
# a reduced copy of the workload was captured and its traffic is scaled to the
# full launch by residual points ("scaled_from"): the traffic is the saved
# jets and the gradient slices, both in proportion to the points processed.
TRAFFIC = {
    # one launch of the reduced copy (160 subdomains, 4.8 M residual points):
    # 0.921 GB read + 17.893 GB written; x16 to the full 76.8 M points
    "c4": {"sha": "e80959e32d830038", "scaled_from": "c4s", "scale": 16,
           "options": {"points_per_thread": 1, "threads_per_cta": 256, "items_per_cta": 32,
                       "max_points_per_tile": 0},
           "bytes_per_launch": 16 * (920784640 + 17893173248)},
}
FP32_LANES_PER_SM = 128      # FFMA lanes per SM (4 partitions x 32)


def workload(name):
    from paper_2104_10013_gb300 import problems as P
    if name == "c2":
        return P.poisson_xpinn(), ("XPINN Poisson -lap u = f on the unit square, 16 subdomains of an uneven "
                                   "4x4 grid, depth 4-6 x width 20-80 tanh MLPs and 2k-20k residual points "
                                   "per subdomain (seed 0), 200 points per interface")
    if name == "c1":
        return P.burgers_cpinn(), "cPINN Burgers, 4 x-slabs, 2->20x3->1, 1000 residual pts each"
    if name == "c3":
        return P.kovasznay_cpinn(), "cPINN Kovasznay NS Re=40, 8x8 grid, 2->64x6->3, 50k residual pts each"
    if name == "c3s":
        return P.kovasznay_cpinn(nx=4, ny=4, n_res=20000), ("the Kovasznay cPINN workload reduced for counter "
                                                            "captures: 4x4 grid, 2->64x6->3, 20k residual pts each")
    if name == "tablevb":
        return P.burgers_spacetime(4, 2), ("XPINN space-time Burgers, 4 x 2 subdomains, 2->20x5->1, 80k residual pts "
                                           "in total, 20 pts per interface (Table TableVB)")
    if name == "c4":
        return P.diffusion_xpinn(), ("XPINN inverse diffusion div(K grad u) = f on a seeded star polygon, "
                                     "10 Voronoi regions x 256 independent copies (2,560 subdomains), "
                                     "u: 2->40x5->1 and K: 2->20x4->1 softplus per region, hidden activation "
                                     "tanh/sin/cos by region with trained slopes (Table Table_USmap), "
                                     "30k residual pts and 500 noisy u observations per region")
    if name == "c4s":
        return P.diffusion_xpinn(n_copies=16), ("the inverse-diffusion workload reduced for counter captures: "
                                                "16 copies of the 10 regions (160 subdomains), same networks "
                                                "and per-region points")
    if name == "c2a":
        import dataclasses
        pb = P.poisson_xpinn()
        for s in pb.subs:
            s.nets = [dataclasses.replace(n, adaptive=True) for n in s.nets]
        return pb, ("the default XPINN Poisson workload with trainable layer-wise slopes n a^k (Sec. 3) "
                    "in every tanh network")
    raise SystemExit(f"unknown workload {name}")


# jet components propagated at residual points, per PDE and network:
# Burgers (u, u_x, u_t, u_xx); Poisson, NS and the inverse-diffusion u-net
# (u, u_x, u_y, u_xx + u_yy) as Laplacian jets; the diffusion K-net (K, K_x, K_y)
K_RES = {0: (4,), 1: (4,), 2: (4,), 3: (4, 3)}


def algorithmic_flops(pb, subset=None):
    """6 K M FLOP per residual point (forward W h, reverse W^T z-bar and
    z-bar h^T, FMA = 2 FLOP), M = sum over layers k >= 2 of N_k N_{k-1};
    over the subdomains in `subset` (indices), else all."""
    tot = 0.0
    for q, s in enumerate(pb.subs):
        if subset is not None and q not in subset:
            continue
        for net, K in zip(s.nets, K_RES[pb.pde]):
            w = net.widths
            M = sum(w[k] * w[k - 1] for k in range(2, len(w)))
            tot += 6.0 * K * M * s.res_xy.shape[0]
    return tot


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_id}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.3)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if "Active" in v and "Not" not in v})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].strip().replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def time_steps(torch, s, stream, flush, steps):
    """Time `steps` single steps, each alone: flush L2, then events around
    the step on its stream.  Returns (step ms list, jet-kernel ms list); the
    tensor-core kernel's ms of each step, when it runs, go to s.tc_ms."""
    step_ms, jet_ms = [], []
    has_tc = s.plan_counts()[1] > 0 and s.options()["schedule"] == 0
    if has_tc:
        s.tc_ms = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0.record(stream)
        s.step(1, losses=None, stream=stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        jet_ms.append(float(s.phase_times()[2]))
        if has_tc:
            s.tc_ms.append(s.tc_kernel_ms())
    return step_ms, jet_ms


def serving(X, n_req, max_query, seed=0, budget=8 << 30):
    """Continuous-batching server over three trained models (Burgers cPINN,
    XPINN Poisson, Kovasznay cPINN with 2k points per subdomain) under a
    Poisson-arrival mix: 80% evaluation queries (log-uniform 1..max_query
    points, derivative order 0-2, routed on the device) and 20% training
    requests on a private fork of 1-64 subdomains (at most the model's) with
    1k-50k residual points each.  Arrivals at 70% of the closed-loop capacity;
    latency = submit -> completion; results are drained as they complete."""
    from paper_2104_10013_gb300 import problems as P
    rng = np.random.default_rng(seed)
    pbs = [P.burgers_cpinn(), P.poisson_xpinn(), P.kovasznay_cpinn(n_res=2000)]
    models = [X.Solver(pb) for pb in pbs]
    for m in models:
        m.step(20, losses=None)                       # "trained" models
        m.sync()
    # point pools: requests take slices (no per-request generation)
    pool = []
    for pb in pbs:
        x0, x1, y0, y1 = pb.meta["xcuts"][0], pb.meta["xcuts"][-1], pb.meta["ycuts"][0], pb.meta["ycuts"][-1]
        pool.append(np.stack([rng.uniform(x0, x1, max_query), rng.uniform(y0, y1, max_query)], 1).astype(np.float32))
    sub_pool = []
    for pb in pbs:
        per = []
        for sd in pb.subs:
            x0, x1, y0, y1 = sd.rect
            per.append(np.stack([rng.uniform(x0, x1, 50000), rng.uniform(y0, y1, 50000)], 1).astype(np.float32))
        sub_pool.append(per)

    def make():
        m = int(rng.integers(0, 3))
        if rng.random() < 0.2:
            k = int(rng.integers(1, min(64, pbs[m].n_sub) + 1))
            sel = sorted(rng.choice(pbs[m].n_sub, k, replace=False).tolist())
            xy = []
            for q in sel:
                n = int(rng.integers(1000, 50001))
                o = int(rng.integers(0, 50000 - n + 1))
                xy.append(sub_pool[m][q][o:o + n])
            return ("fork", m, sel, xy, sum(len(a) for a in xy))
        n = int(10 ** rng.uniform(0, np.log10(max_query)))
        o = int(rng.integers(0, max_query - n + 1))
        return ("eval", m, pool[m][o:o + n], int(rng.integers(0, 3)), n)

    def submit(srv, r):
        if r[0] == "fork":
            return srv.submit_fork(r[1], r[2], r[3], None, 1)
        return srv.submit_eval(r[1], r[2], r[3])

    srv = X.Server(models, hbm_budget=budget)
    # closed-loop capacity: keep 8 requests in flight
    cap_reqs = [make() for _ in range(max(40, n_req // 10))]
    t0 = time.perf_counter()
    inflight, k = [], 0
    while k < len(cap_reqs) or inflight:
        while k < len(cap_reqs) and len(inflight) < 8:
            inflight.append(submit(srv, cap_reqs[k])); k += 1
        srv.wait(inflight.pop(0))
    cap = len(cap_reqs) / (time.perf_counter() - t0)
    lam = 0.7 * cap
    gaps = rng.exponential(1.0 / lam, n_req)
    pending = {}                  # ticket -> (kind, points)
    res = []

    def drain():
        for t in list(pending):
            r = srv.poll(t)
            if r is not None:
                kind, pts = pending.pop(t)
                res.append((kind, pts, r["status"], r["latency_ms"], r["batch"], r["tick_requests"], r["error"]))

    t_start = time.perf_counter()
    t_next = t_start
    for g in gaps:
        r = make()
        t_next += g
        while time.perf_counter() < t_next:
            drain()
            time.sleep(min(2e-4, max(0.0, t_next - time.perf_counter())))
        pending[submit(srv, r)] = (r[0], r[4])
    while pending:
        drain()
        time.sleep(1e-4)
    wall = time.perf_counter() - t_start
    srv.close()
    for m in models:
        m.close()
    bad = [x for x in res if x[2] != 0]
    if bad:
        raise RuntimeError(f"serving: {len(bad)} requests failed, first: {bad[0][6]}")
    lat = np.array([x[3] for x in res])
    ev = np.array([x[3] for x in res if x[0] == "eval"])
    fk = np.array([x[3] for x in res if x[0] == "fork"])
    pts = sum(x[1] for x in res)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "eval_p50_ms": float(np.percentile(ev, 50)), "eval_p99_ms": float(np.percentile(ev, 99)),
            "step_p50_ms": float(np.percentile(fk, 50)) if len(fk) else None,
            "step_p99_ms": float(np.percentile(fk, 99)) if len(fk) else None,
            "sustained_pts_per_s": pts / wall, "requests": n_req, "evals": int(len(ev)), "steps": int(len(fk)),
            "wall_s": wall, "arrival_rate_per_s": lam, "capacity_req_per_s": cap,
            "max_batch": int(max(x[4] for x in res)), "max_tick_requests": int(max(x[5] for x in res)),
            "mean_tick_requests": float(np.mean([x[5] for x in res])),
            "device_pool_bytes": budget,
            "mix": f"80% evaluation queries (log-uniform 1..{max_query} pts, order 0-2), 20% one-step "
                   "training requests on a private fork of 1-64 subdomains x 1k-50k residual pts, over "
                   "Burgers cPINN / Poisson XPINN / Kovasznay cPINN models; Poisson arrivals at 70% of "
                   "closed-loop capacity; points/s counts evaluated and trained points"}


def cpu_baseline(pb, seconds):
    """The FP64 oracle, as it stands, on this host's cores: gradients of whole
    subdomains of the same workload in turn until `seconds` have passed."""
    import torch
    from oracle import Oracle
    orc = Oracle(pb)
    theta = pb.packed_params()
    pts, t_tot, qs = 0, 0.0, []
    q = 0
    while t_tot < seconds and len(qs) < 4 * pb.n_sub:
        t0 = time.perf_counter()
        orc.grad(theta, subset=[q])
        t_tot += time.perf_counter() - t0
        pts += pb.subs[q].res_xy.shape[0]
        qs.append(q)
        q = (q + 1) % pb.n_sub
    # the same oracle on one core, for a short sample (the smallest subdomain,
    # when it is small enough to finish in seconds on one core)
    n_thr = torch.get_num_threads()
    q1 = int(np.argmin([sd.res_xy.shape[0] for sd in pb.subs]))
    one = None
    if pb.subs[q1].res_xy.shape[0] <= 5000:
        torch.set_num_threads(1)
        try:
            t0 = time.perf_counter()
            orc.grad(theta, subset=[q1])
            t1 = time.perf_counter() - t0
        finally:
            torch.set_num_threads(n_thr)
        one = {"value": pb.subs[q1].res_xy.shape[0] / t1, "unit": "pts/s",
               "sample": f"subdomain {q1}, {pb.subs[q1].res_xy.shape[0]} residual points, one thread"}
    return {"value": pts / t_tot, "unit": "pts/s", "cores": n_thr, "kind": "oracle",
            "sample": f"FP64 oracle gradients of {len(qs)} whole subdomains of the same workload, taken in "
                      f"turn (q = 0, 1, ...), {pts} residual points in {t_tot:.1f} s",
            "one_core": one}


def whole_job(total_ms, world, n_res, steps, dist=None, device="cpu"):
    """Replicas only: every rank trained its own copy of the workload (n_res
    residual points per step) for `steps` steps in total_ms.  The job's time
    is the slowest rank's; value = all ranks' residual points / that time.
    Returns (value in pts/s, ms per step)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * n_res * steps / (total_ms / 1e3), total_ms / steps


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    pb, desc = workload(args.workload)
    from oracle import Oracle
    orc = Oracle(pb)
    theta = pb.packed_params()
    q = 0
    for _ in range(args.warmup):
        orc.grad(theta, subset=[q]); q = (q + 1) % pb.n_sub
    pts, t_tot = 0, 0.0
    t_start = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        orc.grad(theta, subset=[q])
        t_tot += time.perf_counter() - t0
        pts += pb.subs[q].res_xy.shape[0]
        q = (q + 1) % pb.n_sub
    v = pts / t_tot
    sample = (f"each step: FP64 oracle gradient of one whole subdomain of the workload (subdomains in turn), "
              f"{pts} residual points over {args.steps} steps")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "pts/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc},
        "cpu_baseline": {"value": v, "unit": "pts/s", "cores": torch.get_num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t_start}))


# Tuned options recorded on this machine's GB300 (bench.py --write-tune-cache),
# per problem signature and shape class; problems not in it are tuned live.
TUNE_CACHE = os.path.join(ROOT, "paper_2104_10013_gb300", "tuning_gb300.json")
_tune_args = {"cache": TUNE_CACHE if os.path.exists(TUNE_CACHE) else None, "write": False}


def tuned_solver(X, pb, autotune, opts=None):
    """A Solver with profile_phases on (the phase timer gives the jet
    kernel's device time) and, unless disabled, autotuned tile options."""
    s = X.Solver(pb)
    s.set_options(profile_phases=1, **(opts or {}))
    tune = None
    if autotune:
        t0 = time.perf_counter()
        tune = dict(s.autotune(steps=3, **_tune_args))
        tune["seconds"] = time.perf_counter() - t0
        tune["cache"] = _tune_args["cache"] is not None and tune["seconds"] < 1.0
        s.set_options(profile_phases=1)
    return s, tune


def roofline(pb, jet_ms, n_sm, name, s):
    """Achieved algorithmic FP32 FLOP/s of the jet kernel against the derived
    FFMA peak, with the ncu traffic of the same launch when it was captured."""
    import hashlib
    flops = algorithmic_flops(pb)
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    peak = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = flops / (jet_ms / 1e3) / 1e12
    src = os.path.join(ROOT, "paper_2104_10013_gb300", "csrc", "jet_step.cuh")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    t = TRAFFIC.get(name)
    opts = s.options()
    traffic = None
    traffic_note = None
    if t and t["sha"] == sha and all(opts.get(k) == v for k, v in t["options"].items()):
        traffic = t["bytes_per_launch"]
        if "scaled_from" in t:
            traffic_note = (f"DRAM bytes of one launch of the reduced workload '{t['scaled_from']}' "
                            f"(same kernel and options) x {t['scale']}, the ratio of residual points")
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_note": traffic_note,
            "kernel": "xp::jet_step_kernel (exchange, residual, data and interface items)",
            "kernel_ms": jet_ms, "flop_per_launch": flops,
            "flop_per_point": "6 K M per residual point of every network (K jet components: 4 for the "
                              "u-network (Laplacian jets) and Burgers, 3 for the K-network; M = sum over "
                              "layers k >= 2 of N_k N_{k-1})",
            "peak_note": f"FP32 FFMA peak derived: {n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 FLOP x "
                         f"{sm_max:.0f} MHz (max SM clock in MEASURED_PEAKS.json)"}


# TF32 dense tensor rate relative to BF16 (nominal 1.1 vs 2.25 PFLOP/s per GPU)
TF32_OVER_BF16 = 1.1 / 2.25


def roofline_tc(pb, s, step_ms):
    """The tensor-core training kernel (residual items of the networks of
    hidden widths train_tensor_cores..64) against the TF32 tensor peak: the
    measured BF16 burst figure times the nominal TF32/BF16 ratio.  achieved =
    the algorithmic 6 K M FLOP per residual point of the subdomains it trains
    (unpadded widths) / its CUDA-event time; the executed tensor work counts
    the hidden-to-hidden layers at the padded width, three TF32 products for
    the forward and reverse contractions and four for the weight gradient."""
    n_items, n_tc, n_tc_sub = s.plan_counts()
    if not n_tc:
        return None
    tc_ms = float(np.mean(s.tc_ms)) if getattr(s, "tc_ms", None) else s.tc_kernel_ms()
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops")
    peak = bf16 * TF32_OVER_BF16 if bf16 else 1900.0 * TF32_OVER_BF16
    on = s.tc_subdomains()
    flops = algorithmic_flops(pb, {q for q in range(pb.n_sub) if on[q]})
    # on the tensor pipe: the hidden-to-hidden layers at the padded width 64,
    # three products forward and reverse and four for the weight gradient
    executed = sum(10.0 / 3.0 * 6 * 4 * (len(sd.nets[0].widths) - 3) * 64 * 64 * sd.res_xy.shape[0]
                   for q, sd in enumerate(pb.subs) if on[q])
    achieved = flops / (tc_ms / 1e3) / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "kernel": "xp::step_tc_kernel (residual items, tcgen05 kind::tf32)", "kernel_ms": tc_ms,
            "kernel_share_of_step": tc_ms / step_ms, "items": n_tc, "subdomains": n_tc_sub,
            "flop_per_launch": flops, "executed_tensor_flop_per_launch": executed,
            "peak_note": ("TF32 dense peak = measured BF16 burst (MEASURED_PEAKS.json) x 1.1/2.25, the nominal "
                          "TF32/BF16 ratio" if bf16 else "fallback 1.9 PFLOP/s BF16 x 1.1/2.25")}


def loop_compare(torch, s, stream, flush, steps, ipcs, n_res, grouped_ms):
    """The per-subdomain launch loop (schedule 1) of the same kernels on the
    same handle, at its own best items-per-CTA; the grouped options are
    restored afterwards."""
    grouped_opts = s.options()
    best = None
    for ipc in ipcs:
        s.set_options(schedule=1, items_per_cta=ipc)
        s.step(1, losses=None, stream=stream.cuda_stream)
        lms, _ = time_steps(torch, s, stream, flush, steps)
        if best is None or np.sum(lms) < np.sum(best[1]):
            best = (ipc, lms)
    s.sync(stream.cuda_stream)
    ipc, lms = best
    lval = n_res * len(lms) / (np.sum(lms) / 1e3)
    s.set_options(**grouped_opts)
    return {"value": lval, "unit": "pts/s", "ms_per_step": float(np.mean(lms)), "items_per_cta": ipc,
            "steps": len(lms), "grouped_speedup": lval and (n_res / (grouped_ms / 1e3)) / lval}


def extra_workload(torch, X, name, stream, flush, steps, loop_steps, n_sm):
    """Grouped step (autotuned) and per-subdomain loop of one more workload."""
    pb, desc = workload(name)
    s, tune = tuned_solver(X, pb, True)
    for _ in range(3):
        s.step(1, losses=None, stream=stream.cuda_stream)
    step_ms, jet_ms = time_steps(torch, s, stream, flush, steps)
    s.sync(stream.cuda_stream)
    ms = float(np.mean(step_ms))
    out = {"workload": desc, "value": pb.n_res / (ms / 1e3), "unit": "pts/s", "ms_per_step": ms,
           "steps": steps, "residual_pts_per_step": pb.n_res, "options": s.options(),
           "roofline": roofline(pb, float(np.mean(jet_ms)), n_sm, name, s)}
    tc = roofline_tc(pb, s, ms)
    if tc:
        # the residual items run on the tensor cores: their kernel is the one
        # to hold against its roofline; the FP32 line covers the whole phase
        out["roofline_fp32_phase"] = out.pop("roofline")
        out["roofline"] = tc
    if loop_steps:
        out["loop"] = loop_compare(torch, s, stream, flush, loop_steps, (4, 16, 64), pb.n_res, ms)
    s.close()
    return out


def eval_tensor_cores(torch, X, stream, flush, n_pts=1 << 20, reps=10, orders=(0, 1, 2)):
    """Routed evaluation (Eq. FSol) of the Kovasznay cPINN model (64
    subdomains, 2->64x6->3) at n_pts uniform query points on the device,
    derivative orders 0-2, the tensor-core kernel against the FP32 jet
    kernel on the same handle, buffers and points.  Per order and path:
    the whole xpinn_eval_ws call (route, plan, bucket, evaluation kernel,
    gather) and the evaluation kernel alone, both CUDA-event medians over
    `reps` calls with L2 flushed before each; the tensor-core kernel's
    roofline is its algorithmic contraction FLOPs (2 K per point per weight of
    the hidden-to-hidden layers) against the dense TF32 rate."""
    pb, _ = workload("c3")
    s = X.Solver(pb)
    s.step(5, losses=None, stream=stream.cuda_stream)
    s.set_options(profile_phases=1)
    rng = np.random.default_rng(11)
    xy = np.stack([rng.uniform(-0.5, 1.0, n_pts), rng.uniform(-0.5, 1.5, n_pts)], 1).astype(np.float32)
    dxy = torch.from_numpy(xy).cuda()
    m_h = sum(n.widths[k] * n.widths[k - 1] for n in pb.subs[0].nets for k in range(2, len(n.widths) - 1))
    peaks = measured_peaks()
    tf32 = peaks.get("bf16_tflops", 1900.0) * (1.1 / 2.25)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    out = {"workload": "Kovasznay cPINN model, 64 subdomains 2->64x6->3 tanh, %d uniform query points, "
                       "device buffers (xpinn_eval_ws)" % n_pts, "orders": {}}
    for order in orders:
        K = (1, 3, 5)[order]
        ws = torch.empty(s.eval_workspace_size(n_pts, order), dtype=torch.uint8, device="cuda")
        dout = torch.empty((n_pts, 3 * K), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        res = {}
        for tc in (0, 1):
            s.set_options(eval_tensor_cores=tc)
            with torch.cuda.stream(stream):   # eval_ws runs on the current stream
                for _ in range(3):
                    s.eval_ws(0, dxy, order, dout, ws)
            call_ms, kern_ms = [], []
            for _ in range(reps):
                with torch.cuda.stream(stream):
                    flush.zero_()
                    e0.record(stream)
                    s.eval_ws(0, dxy, order, dout, ws)
                    e1.record(stream)
                e1.synchronize()
                call_ms.append(e0.elapsed_time(e1))
                kern_ms.append(s.eval_kernel_ms())
            s.sync(stream.cuda_stream)
            c, k = float(np.median(call_ms)), float(np.median(kern_ms))
            res["tensor_cores" if tc else "fp32_jet_kernel"] = {
                "call_ms": c, "kernel_ms": k, "pts_per_s": n_pts / (c / 1e3)}
        t = res["tensor_cores"]
        flops = 2.0 * K * m_h * n_pts
        t["roofline"] = {"bound": "tensor", "achieved": flops / (t["kernel_ms"] / 1e3) / 1e12, "peak": tf32,
                         "unit": "TFLOP/s", "frac": flops / (t["kernel_ms"] / 1e3) / 1e12 / tf32,
                         "traffic": None,
                         "peak_note": "dense TF32: measured bf16 burst x 1.1/2.25 (nominal ratio); the "
                                      "kernel issues three TF32 products per term (hi/lo split), so its "
                                      "algorithmic fraction is at most 1/3"}
        res["kernel_speedup"] = res["fp32_jet_kernel"]["kernel_ms"] / t["kernel_ms"]
        res["call_speedup"] = res["fp32_jet_kernel"]["call_ms"] / t["call_ms"]
        out["orders"][str(order)] = res
    s.set_options(eval_tensor_cores=0)
    s.close()
    return out


def adam_steps_per_s(torch, X, stream, n=320):
    """Adam steps per second of the Burgers cPINN configuration (4 x 1000
    residual points, launch-bound): n training steps back to back in one
    call (replayed from a graph of 16 steps), timed with CUDA events; the
    problem stays in L2 as it does in a training run."""
    pb, desc = workload("c1")
    s = X.Solver(pb)
    tune = s.autotune(steps=5, **_tune_args)   # small sub-tiles spread the 4,000 points over the SMs
    s.set_options(profile_phases=0)
    s.step(64, losses=None, stream=stream.cuda_stream)
    s.sync(stream.cuda_stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(n, losses=None, stream=stream.cuda_stream)
    e1.record(stream)
    e1.synchronize()
    s.sync(stream.cuda_stream)
    ms = e0.elapsed_time(e1)
    s.close()
    return {"workload": desc, "value": n / (ms / 1e3), "unit": "Adam steps/s", "steps": n,
            "ms_per_step": ms / n, "residual_pts_per_s": pb.n_res * n / (ms / 1e3),
            "options": tune.get("options"), "class_caps": tune.get("class_caps"),
            "note": "steps back to back in one xpinn_step call, graphs of 16 steps; L2 not flushed"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="c4")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-loop", action="store_true")
    ap.add_argument("--loop-steps", type=int, default=0, help="timed loop steps (0: 2 for c4, else --steps)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads and Adam steps/s")
    ap.add_argument("--only-eval", action="store_true",
                    help="run only the tensor-core vs FP32 evaluation comparison and print its JSON")
    ap.add_argument("--eval-points", type=int, default=1 << 20, help="query points of that comparison")
    ap.add_argument("--eval-orders", default="0,1,2", help="derivative orders of that comparison")
    ap.add_argument("--pt", type=int, default=0, help="points per thread in the register tile (0: library default)")
    ap.add_argument("--items-per-cta", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA (0: library default)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--train-tensor-cores", type=int, default=-1,
                    help="option train_tensor_cores of the timed workload (-1: library default)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=10000)
    ap.add_argument("--serving-max-query", type=int, default=1000000)
    ap.add_argument("--write-tune-cache", default=None,
                    help="time every workload's options and record them in this JSON file")
    args = ap.parse_args()
    if args.write_tune_cache:
        _tune_args.update(cache=args.write_tune_cache, write=True)
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2104_10013_gb300 import build as B
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    from paper_2104_10013_gb300 import xpinn as X
    X.load()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    eval_orders = tuple(int(o) for o in args.eval_orders.split(","))
    if args.only_eval:
        stream = torch.cuda.Stream()
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        print(json.dumps(eval_tensor_cores(torch, X, stream, flush, n_pts=args.eval_points, orders=eval_orders)))
        return

    pb, desc = workload(args.workload)
    n_res = pb.n_res
    opts = {}
    if args.pt:
        opts["points_per_thread"] = args.pt
    if args.items_per_cta:
        opts["items_per_cta"] = args.items_per_cta
    if args.threads:
        opts["threads_per_cta"] = args.threads
    autotune = not args.no_autotune and not opts
    s, tune = tuned_solver(X, pb, autotune, opts)
    if args.train_tensor_cores >= 0:
        s.set_options(train_tensor_cores=args.train_tensor_cores)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        s.step(1, losses=None, stream=stream.cuda_stream)
    s.sync(stream.cuda_stream)
    torch.cuda.synchronize()

    # ---- timed region: K grouped steps
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = str(local)
    clocks = Clocks(gpu_id)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, jet_ms = time_steps(torch, s, stream, flush, args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    s.sync(stream.cuda_stream)      # raises if a device wait gave up or a loss became non-finite
    value, ms_step = whole_job(float(np.sum(step_ms)), world, n_res, args.steps, dist, "cuda")
    # our kernels per step: step_begin, pack_weights (when some network has a
    # hidden-to-hidden layer), the jet kernel, reduce_adam
    launches_per_step = 3 + int(any(len(n.widths) > 3 for sd in pb.subs for n in sd.nets))
    roof = roofline(pb, float(np.mean(jet_ms)), n_sm, args.workload, s)
    roof["kernel_share_of_step"] = roof["kernel_ms"] / ms_step

    out = {"metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": desc, "n_sub": pb.n_sub, "residual_pts_per_step": n_res,
                      "params": pb.n_params,
                      "l2": "inputs larger than L2, and L2 flushed (256 MB write) before every timed step",
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                      "options": s.options(), "autotune": tune},
           "adam_steps_per_s": 1e3 / ms_step, "roofline": roof, "gpu_launches": launches_per_step * args.steps,
           "clocks": clk}

    # ---- per-subdomain launch loop, same kernels, same GPU.  Its items are
    # cut at its own best granularity (more items per subdomain fill more
    # CTAs of each per-subdomain launch), not the grouped schedule's.
    if not args.no_loop:
        big = n_res > 10_000_000
        lsteps = args.loop_steps or (2 if big else args.steps)
        out["loop"] = loop_compare(torch, s, stream, flush, lsteps, (64,) if big else (4, 16, 64), n_res, ms_step)

    # ---- end to end through the public API with host buffers
    if not args.no_e2e:
        xy = torch.from_numpy(np.concatenate([sd.res_xy for sd in pb.subs])).pin_memory()
        f = torch.from_numpy(np.concatenate([sd.res_f for sd in pb.subs])).pin_memory()
        losses = torch.empty((1, pb.n_sub, 5), dtype=torch.float32).pin_memory()
        e_steps = max(3, min(args.steps, 10)) if n_res > 10_000_000 else args.steps
        for _ in range(2):
            s.set_residual_points(xy, f)
            s.step(1, losses=losses)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            s.set_residual_points(xy, f)
            s.step(1, losses=losses)
        e2e_s = time.perf_counter() - t0
        out["e2e"] = {"value": n_res * e_steps / e2e_s * world, "unit": "pts/s", "steps": e_steps,
                      "h2d_bytes_per_step": int(xy.numel() * 4 + f.numel() * 4),
                      "d2h_bytes_per_step": int(losses.numel() * 4),
                      "ms_per_step": 1e3 * e2e_s / e_steps,
                      "path": "xpinn_set_residual_points (pinned host points and forcing) + xpinn_step with "
                              "host losses, wall clock"}
    s.close()

    if not args.no_extras and world == 1 and args.workload == "c4":
        out["workloads"] = {
            "c2": extra_workload(torch, X, "c2", stream, flush, args.steps, 0 if args.no_loop else args.steps, n_sm),
            "c3": extra_workload(torch, X, "c3", stream, flush, 5, 0 if args.no_loop else 3, n_sm),
        }
        out["adam_steps"] = adam_steps_per_s(torch, X, stream)
        out["eval_tensor_cores"] = eval_tensor_cores(torch, X, stream, flush, n_pts=args.eval_points,
                                                     orders=eval_orders)

    if not args.no_serving:
        out["serving"] = serving(X, args.serving_requests, args.serving_max_query)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(pb, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
