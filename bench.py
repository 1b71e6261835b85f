#!/usr/bin/env python
"""Benchmark of the alternating-projection hot path on one or more GPUs.

One step = one whole pass of the hot path on one synthetic problem: scale the
inputs and build the FP64 block-Cholesky cache (ap_create), then run Alg. 1 with
the fused residual update, Gauss-Southwell selection and the FP32 recompute
that refines and certifies (ap_solve).

Workload of the timed steps (default): n = 262,144, d = 3, X ~ N(0, I),
Matern-5/2 ARD with lengthscales log-uniform in [0.3, 3], noise 1e-2, blocks of
4096, B = [y, 15 Rademacher probes], every column to ||r|| / ||b|| <= 1e-3,
capped at 30 epochs (the tolerance is out of AP's reach on this workload).

value = kernel-matrix entries evaluated per second over the whole step (the
n*b entries of the cache plus n*b per AP step plus n^2 per FP32 recompute).

Also in the line: the other form on the same workload; e2e = the same step
through the host-buffer entry point ap_solve_host with its copies timed;
time-to-tolerance of the FP32 form on n = 4096 (RBF, tol 1e-6) and of both forms
on n = 2,097,152 (d = 11, RBF ARD, noise 1e-3, blocks of 8192, y column to 1e-2);
the MLL gradient on n = 131,072 (Matern-3/2, 31 probes); a serving replay; the
FP64 oracle on the host cores (cpu_baseline).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload and prints the same kind of line.
Multi-GPU (torchrun): independent replicas, one problem per rank, no
collective on the data path; value = all ranks' entries / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

METRIC = "AP time-to-tol & kernel-entries/s, BF16+refine vs FP32; serve p50/p99"
T_START = time.perf_counter()
# forms of the residual update: FP32 SIMT, tensor-core BF16 hi/lo
FORMS = {"fp32": lambda ap: ap.AP_FP32, "bf16": lambda ap: ap.AP_BF16_REFINE}
DTYPES = {"fp32": "f32", "bf16": "bf16"}
FP32_LANES_PER_SM = 128
NUM_SMS = 152


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def workload(name: str, sub: int, n: int = 0):
    kw = {"n": n} if n else {}
    if name == "matern52_ard":
        return wl.matern52_ard(sub=sub, **kw)
    if name == "small_rbf":
        return wl.small_rbf(sub=sub, **kw)
    if name == "rbf_ard_large":
        return wl.rbf_ard_large(sub=sub, **kw)
    raise SystemExit(f"unknown workload {name}")


def describe(p, args) -> dict:
    return {"workload": f"{p.name}: {wl.KERNEL_NAMES[p.kernel]} ARD, n={p.n}, d={p.d}, b={p.block}, "
                        f"c={p.c} (y + {p.c - 1} Rademacher probes), noise={p.noise:g}, "
                        f"every column to ||r||/||b|| <= {p.tol:g}",
            "n": p.n, "d": p.d, "block": p.block, "rhs": p.c, "tol": p.tol,
            "kernel": wl.KERNEL_NAMES[p.kernel], "precision": args.precision, "stop": "max_rel",
            "min_epochs": args.min_epochs, "max_epochs": args.max_epochs,
            "l2": "inputs larger than L2 each step: the FP64 factor workspace and the FP32 "
                  "inverse-factor cache are streamed through HBM",
            "parallelism": "replicas (one independent problem per GPU)"}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = {"kmv_fp32_update": ["kmv_fp32.cuh", "ap_internal.cuh"],
                  "kmv_tc_update": ["kmv_tc.cu", "tcgen05.cuh", "kmv_fp32.cuh", "ap_internal.cuh"]}


def kernel_src_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2310_17137_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_from_profiles(kernel: str, workload_name: str, precision: str, n_launch_units: float):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary,
    or None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f)
    ent = t.get(f"{kernel}:{workload_name}:{precision}")
    if not ent or ent.get("src_hash") != kernel_src_hash(kernel):
        return None
    return ent["dram_bytes_per_launch"] * n_launch_units / ent.get("units_per_launch", n_launch_units)


def aggregate(ms: float, units: float, dist, device):
    """Whole-job numbers of a multi-rank run: the slowest rank's time and the sum
    of the units all ranks processed (replicas: no data-path collective)."""
    import torch
    ms_t = torch.tensor([ms], device=device, dtype=torch.float64)
    u_t = torch.tensor([units], device=device, dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u_t, op=dist.ReduceOp.SUM)
    return float(ms_t.item()), float(u_t.item())


def run_ours(args, rank: int, world: int):
    import torch

    import paper_2310_17137_gb300 as ap

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    p = workload(args.workload, sub=rank, n=args.n)
    prec = FORMS[args.precision](ap)
    hyper = ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise, p.mean)
    X = torch.from_numpy(p.X).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    W = torch.empty_like(B)
    stream = torch.cuda.current_stream(dev)

    def opts(pr=None):
        return ap.ap_opts_default(block=p.block, tol=p.tol, stop=ap.AP_STOP_MAX_REL, min_epochs=args.min_epochs,
                                  max_epochs=args.max_epochs, precision=prec if pr is None else pr, profile=1,
                                  refine_every=args.refine_every, stream=stream.cuda_stream)

    def one_step(pr=None):
        ctx = ap.ap_create(X, hyper, opts(pr))
        st, _, info, _ = ap.ap_solve(ctx, B, W=W)
        launches = ap.ap_launch_count(ctx)
        ap.ap_destroy(ctx)
        return st, info, launches

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index) if rank == 0 else None
    if sampler:
        sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos, launches, statuses = [], 0, []
    for _ in range(args.steps):
        st, info, nl = one_step()
        infos.append(info)
        statuses.append(st)
        launches += nl
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    cache_entries = float(p.n) * float(p.block)
    entries = sum(cache_entries + i["kernel_entries"] for i in infos)
    ms_max, total_entries = aggregate(e0.elapsed_time(e1), entries, dist, dev)
    value = total_entries / (ms_max * 1e-3)

    # the other forms on the same problem, timed the same way
    compare = None
    if not args.no_compare:
        compare = {}
        for name in FORMS:
            if name == args.precision:
                continue
            other = FORMS[name](ap)
            one_step(other)
            torch.cuda.synchronize()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            cinfos = []
            csteps = min(args.steps, args.compare_steps)
            for _ in range(csteps):
                _, ci, _ = one_step(other)
                cinfos.append(ci)
            c1.record(stream)
            torch.cuda.synchronize()
            cms = c0.elapsed_time(c1) / csteps
            cent = sum(float(p.n) * float(p.block) + i["kernel_entries"] for i in cinfos) / csteps
            compare[name] = {"ms_per_step": cms, "kernel_entries_per_s": cent / (cms * 1e-3),
                             "update_kernel_ms": cinfos[-1]["t_update_s"] / max(1, cinfos[-1]["n_update"]) * 1e3,
                             "solve_s": statistics.median(i["t_solve_s"] for i in cinfos),
                             "rel_res_y": cinfos[-1]["rel_res_true"][0],
                             "rel_res_max": max(cinfos[-1]["rel_res_true"]),
                             "epochs": cinfos[-1]["epochs"], "refinements": cinfos[-1]["refinements"],
                             "steps_timed": csteps}

    # end to end through the public API with host buffers (pinned), copies timed
    e2e_value, e2e_steps = None, 0
    if not args.no_e2e:
        e2e_value, e2e_steps = end_to_end(ap, torch, p, hyper, opts, dev, stream, args, dist)
    ttt = None
    if rank == 0 and not args.no_ttt:
        ttt = time_to_tol_small(ap, torch, dev, stream)
    mll = None
    if rank == 0 and not args.no_mll:
        mll = mll_grad_timing(ap, torch, dev, stream)
    # the long legs run only while the whole run stays inside its time budget
    # (estimates from measured runs on this workload: 13.5 min and 3 min)
    def budget_left() -> float:
        return args.time_budget_s - (time.perf_counter() - T_START)

    ttt_large = None
    if rank == 0 and not args.no_ttt_large:
        ttt_large = (time_to_tol_large(ap, torch, dev, stream, args) if budget_left() > 900
                     else {"skipped": f"time budget ({args.time_budget_s:.0f} s) nearly used"})
    serve = None
    if rank == 0 and not args.no_serve_replay:
        serve = (serving_replay(ap, args, args.serve_replay_requests, args.serve_max_epochs) if budget_left() > 240
                 else {"skipped": f"time budget ({args.time_budget_s:.0f} s) nearly used"})

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = result_line(ap, p, args, world, ms_max, value, infos, statuses, launches, clocks, e2e_value, ttt,
                       e2e_steps)
    line["other_forms"] = compare
    line["mll_grad"] = mll
    line["time_to_tol_large"] = ttt_large
    line["serving"] = serve
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, infos[-1]["epochs"], args)
        if not args.no_ttt:
            line["cpu_baseline"]["time_to_tol_small"] = oracle_time_to_tol_small()
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def end_to_end(ap, torch, p, hyper, opts, dev, stream, args, dist):
    """The same step through the one-shot host-buffer entry point ap_solve_host:
    X and B copied in from page-locked host memory, the cache built, Alg. 1 run,
    W copied out, every step inside the timed region."""
    Xh = torch.from_numpy(p.X).pin_memory()
    Bh = torch.from_numpy(p.B).pin_memory()
    Wh = torch.empty(p.B.shape, dtype=torch.float32).pin_memory()
    Xn, Bn, Wn = Xh.numpy(), Bh.numpy(), Wh.numpy()
    steps = min(args.steps, args.e2e_steps)
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    e2e_entries = 0.0
    cache_entries = float(p.n) * float(p.block)
    for _ in range(steps):
        _, _, info = ap.ap_solve_host(Xn, Bn, hyper, opts(), W=Wn)
        e2e_entries += cache_entries + info["kernel_entries"]
    e3.record(stream)
    torch.cuda.synchronize()
    e2e_ms, e2e_entries = aggregate(e2.elapsed_time(e3), e2e_entries, dist, dev)
    return e2e_entries / (e2e_ms * 1e-3), steps


def time_to_tol_small(ap, torch, dev, stream) -> dict:
    """Time-to-tol of the plain FP32 solve on n = 4096 (RBF l = 0.5, noise 0.1,
    blocks of 512, tol 1e-6, certified by the compensated FP32 recompute):
    the configuration where AP reaches its tolerance within the epoch cap."""
    p = wl.small_rbf()
    X = torch.from_numpy(p.X).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    hyper = ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise, p.mean)
    times, infos = [], []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = ap.ap_create(X, hyper, ap.ap_opts_default(block=p.block, tol=p.tol, stop=ap.AP_STOP_MAX_REL,
                                                        max_epochs=100000, stream=stream.cuda_stream))
        st, W, info, _ = ap.ap_solve(ctx, B)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        infos.append(info)
        ap.ap_destroy(ctx)
    i = infos[-1]
    return {"workload": "small_rbf n=4096 d=8 b=512 c=1 tol=1e-6 (FP32 form, compensated certification)",
            "time_to_tol_s": statistics.median(times), "epochs": i["epochs"], "refinements": i["refinements"],
            "rel_res_true": i["rel_res_true"][0], "status": ap.ap_status_str(st)}


def time_to_tol_large(ap, torch, dev, stream, args) -> dict:
    """Time-to-tolerance of both forms on n = 2,097,152, d = 11, X ~ U[-1,1]^11,
    RBF ARD (lengthscales log-uniform in [0.2, 2]), noise 1e-3, blocks of 8192,
    B = [y, 15 Rademacher probes]: each form runs Alg. 1 until the y column's
    relative residual, recomputed over all n^2 entries in FP32 (the
    certification the solver applies whenever its rule holds), is at most
    1e-2.  One run per form, the Cholesky cache included; kernel blocks are
    never stored."""
    p = wl.rbf_ard_large()
    X = torch.from_numpy(p.X).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    hyper = ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise, p.mean)
    out = {"workload": f"{p.name}: RBF ARD, n={p.n}, d={p.d}, b={p.block}, c={p.c} (y + {p.c - 1} probes), "
                       f"noise={p.noise:g}, y column to ||r||/||y|| <= {p.tol:g} (FP32 recompute)"}
    for name in ("bf16", "fp32"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = ap.ap_create(X, hyper, ap.ap_opts_default(block=p.block, tol=p.tol, stop=ap.AP_STOP_Y_REL, min_epochs=1,
                                                        max_epochs=args.ttt_large_max_epochs,
                                                        precision=FORMS[name](ap), refine_every=args.refine_every,
                                                        residual_mode=ap.AP_RESID_FP32, profile=1,
                                                        stream=stream.cuda_stream))
        st, _, info, _ = ap.ap_solve(ctx, B)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        ap.ap_destroy(ctx)
        out[name] = {"time_to_tol_s": t, "status": ap.ap_status_str(st), "epochs": info["epochs"],
                     "refinements": info["refinements"], "fp32_epochs": info["fp32_epochs"],
                     "cache_s": info["t_cache_s"], "solve_s": info["t_solve_s"], "refine_s": info["t_refine_s"],
                     "rel_res_y": info["rel_res_true"][0], "rel_res_max": max(info["rel_res_true"][:p.c]),
                     "update_kernel_ms": info["t_update_s"] / max(1, info["n_update"]) * 1e3}
    out["speedup_bf16_vs_fp32"] = out["fp32"]["time_to_tol_s"] / out["bf16"]["time_to_tol_s"]
    del X, B
    torch.cuda.empty_cache()
    return out


def serving_replay(ap, args, n_requests: int, max_epochs: int) -> dict:
    """Replay of the serving workload (Poisson arrivals at `rate`/s, n
    log-uniform in [2^10, 2^18], d in {3..20}, RBF or Matern-5/2, tolerance
    1e-2 or 1e-4, half of the requests in the tensor-core form, solve +
    posterior mean on 1024 test points, 120 GB budget): latency percentiles,
    solves/s, and every request that did not reach its tolerance."""
    trace = wl.serving_trace(n_requests=n_requests, rate=args.serve_rate)
    data = [wl.request_data(r, m_test=1024) for r in trace]
    srv = ap.ApServer(hbm_budget=int(args.serve_budget_gb * (1 << 30)), slots=args.serve_slots)
    t0 = time.perf_counter()
    ids = []
    for r, (X, y, Xt) in zip(trace, data):
        delay = r.arrival_s - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        h = ap.Hyper(r.kernel, r.lengthscale, r.outputscale, r.noise, 0.0)
        prec = ap.AP_BF16_REFINE if r.low_precision else ap.AP_FP32
        ids.append(srv.submit(X, y, Xt, h, block=min(r.n, 4096), tol=r.tol, stop=ap.AP_STOP_Y_REL, min_epochs=1,
                              max_epochs=max_epochs, precision=prec))
    res = [srv.wait(i, timeout_s=3600.0) for i in ids]
    wall = time.perf_counter() - t0
    srv.close()
    lat = np.array([x["latency_s"] for x in res])
    missed = [{"n": r.n, "d": r.d, "tol": r.tol, "form": "bf16" if r.low_precision else "fp32",
               "rel_res": x["rel_res"], "epochs": x["epochs"], "status": ap.ap_status_str(x["status"])}
              for r, x in zip(trace, res) if x["status"] != ap.AP_OK]
    return {"requests": len(res), "solves_per_s": len(res) / wall, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "mean_queue_s": float(np.mean([x["queue_s"] for x in res])),
            "wall_s": wall, "converged": len(res) - len(missed), "max_epochs": max_epochs, "not_converged": missed,
            "config": f"{len(res)} requests, Poisson {args.serve_rate}/s, n logU[2^10, 2^18], d U{{3..20}}, RBF or "
                      f"Matern-5/2, tol {{1e-2, 1e-4}} on the y column, solve + mean on 1024 test points, half in "
                      f"the tensor-core form, {args.serve_budget_gb:g} GB budget, {args.serve_slots} slots"}


def mll_grad_timing(ap, torch, dev, stream) -> dict:
    """One stochastic MLL gradient (Eq. loss_grad_unbiased) on n = 131,072,
    d = 8, Matern-3/2 ARD, noise 0.05, 31 Rademacher probes, blocks of 4096:
    cache + AP solve of the 32 right-hand sides to the paper's training
    tolerance (mean relative residual < 1, at least 11 epochs) in the
    tensor-core form + the fused derivative quadratic forms.  Median of 3."""
    p = wl.matern32_grad()
    X = torch.from_numpy(p.X).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    Z = torch.from_numpy(np.ascontiguousarray(p.B[:, 1:])).to(dev)
    hyper = ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise, p.mean)
    times, infos, grads = [], [], []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = ap.ap_create(X, hyper, ap.ap_opts_default(block=p.block, tol=p.tol, stop=ap.AP_STOP_MEAN_REL,
                                                        min_epochs=11, max_epochs=1000,
                                                        precision=ap.AP_BF16_REFINE, refine_every=10,
                                                        stream=stream.cuda_stream))
        st, g, info = ap.ap_mll_grad(ctx, y, p.c - 1, Z)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        infos.append(info)
        grads.append(g)
        ap.ap_destroy(ctx)
    i = infos[-1]
    return {"workload": f"{p.name}: Matern-3/2 ARD, n={p.n}, d={p.d}, b={p.block}, 31 probes, noise={p.noise:g}, "
                        "training tolerance 1 (mean rule, >= 11 epochs), BF16+refine solve",
            "time_s": statistics.median(times), "cache_s": i["t_cache_s"], "solve_s": i["t_solve_s"],
            "epochs": i["epochs"], "status": ap.ap_status_str(st),
            "grad_norm": float(np.linalg.norm(grads[-1].astype(np.float64)))}


def result_line(ap, p, args, world, ms_max, value, infos, statuses, launches, clocks, e2e_value, ttt,
                e2e_steps=0) -> dict:
    peaks = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    last = infos[-1]
    n_up = max(1, last["n_update"])
    t_launch = last["t_update_s"] / n_up
    units = float(p.n) * float(p.block)
    sfu = ap.ap_sfu_rates() if args.precision != "fp32" else (32.0, 16.0)
    roof = roofline(p, args, t_launch, units, sm_max, sfu)
    roof["sfu_rates_per_clk_sm"] = {"exp2": sfu[0], "sqrt": sfu[1]} if args.precision != "fp32" else None
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "kernel-entries/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPES[args.precision],
        "data": "synthetic (seeded NumPy PCG64; stands in for the paper's UCI sets)",
        "config": describe(p, args),
        "epochs": [i["epochs"] for i in infos],
        "refinements": [i["refinements"] for i in infos],
        "fp32_epochs": [i["fp32_epochs"] for i in infos],
        "refine_s": statistics.median(i["t_refine_s"] for i in infos),
        "status": [ap.ap_status_str(s) for s in statuses],
        "rel_res_max": max(max(i["rel_res_true"]) for i in infos),
        "rel_res_y": infos[-1]["rel_res_true"][0],
        "cache_s": statistics.median(i["t_cache_s"] for i in infos),
        "solve_s": statistics.median(i["t_solve_s"] for i in infos),
        "iteration_entries_per_s": statistics.median(i["entries_per_s"] for i in infos),
        "update_kernel_ms": t_launch * 1e3,
        "blocksolve_kernel_ms": last["t_blocksolve_s"] / n_up * 1e3,
        "roofline": roof,
        "e2e": None if e2e_value is None else {
            "value": e2e_value, "unit": "kernel-entries/s",
            "h2d_bytes_per_step": int(p.X.nbytes + p.B.nbytes), "d2h_bytes_per_step": int(p.B.nbytes),
            "api": "ap_solve_host (host buffers, page-locked)", "steps": e2e_steps},
        "gpu_launches": launches,
        "clocks": clocks,
        "time_to_tol_small": ttt,
    }
    return line


# MUFU results per clock per SM on GB300.  ncu's pct-of-peak for the XU pipe
# (28 % at 7.75 results/clk/SM measured on the tensor-core update kernel) puts
# the pipe's peak at ~32/clk/SM (Blackwell Ultra doubled the SFU rate).


def roofline(p, args, t_launch: float, units: float, sm_max: float, sfu=(32.0, 16.0)) -> dict:
    """Roofline of the dominant kernel (the fused residual update of one AP step)."""
    if args.precision == "fp32":
        flops_per_entry = 2 * p.c + 3 * p.d
        achieved = units * flops_per_entry / t_launch / 1e12 if t_launch > 0 else None
        peak = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": traffic_from_profiles("kmv_fp32_update", args.workload, "fp32", units),
                "kernel": "kmv_fp32_kernel (fused residual update, one AP step)",
                "per_unit": f"{flops_per_entry} FP32 flop per kernel entry (2c contraction + 3d distance)",
                "peak_note": f"FP32 FMA pipe: {NUM_SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x "
                             f"{sm_max:.0f} MHz (derived from unit counts and max clock)"}
    # SFU operations per entry: exp2 for every kernel, sqrt for the Matern ones.
    # Peak: the measured per-clock rates of this GPU (ap_sfu_rates) at the
    # maximum SM clock; for the Matern mix (one of each per entry) the pipe
    # completes 2 / (1/r_exp2 + 1/r_sqrt) operations per clock and SM.
    r_ex2, r_sqrt = sfu
    if p.kernel == wl.RBF:
        ops, per_clk = 1, r_ex2
        mix = f"exp2 {r_ex2:.1f}/clk/SM"
    else:
        ops, per_clk = 2, 2.0 / (1.0 / r_ex2 + 1.0 / r_sqrt)
        mix = f"1:1 exp2 ({r_ex2:.1f}/clk/SM) + sqrt ({r_sqrt:.1f}/clk/SM) = {per_clk:.2f}/clk/SM"
    achieved = units * ops / t_launch / 1e12 if t_launch > 0 else None
    peak = NUM_SMS * per_clk * sm_max * 1e6 / 1e12
    kd = 16 if p.d + 2 <= 16 else 32
    cp = max(16, p.c)
    # distance: three FP16 hi/lo products of K = kd; contraction: three BF16 hi/lo
    # products of K = 1 per entry and C columns
    tensor_flops = 3 * 2 * kd + 3 * 2 * cp
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic_from_profiles("kmv_tc_update", args.workload, args.precision, units),
            "kernel": "kmv_tc_kernel (tcgen05 fused residual update, one AP step)",
            "per_unit": f"{ops} SFU op(s) per kernel entry; units are tera-ops/s of the SFU pipe",
            "peak_note": f"SFU pipe measured on this GPU by ap_sfu_rates: {mix}, x {NUM_SMS} SMs x "
                         f"{sm_max:.0f} MHz",
            "tensor_tflops": units * tensor_flops / t_launch / 1e12 if t_launch > 0 else None,
            "tensor_flops_per_entry": tensor_flops}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_time_to_tol_small() -> dict:
    """The FP64 oracle's own time-to-tolerance on n = 4096, d = 8, RBF l = 0.5,
    noise 0.1, blocks of 512, tol 1e-6 (every column), measured outright."""
    import oracle
    p = wl.small_rbf()
    t0 = time.perf_counter()
    r = oracle.ap_solve(oracle.Hyper.of(p), p.X.astype(np.float64), p.B.astype(np.float64), p.block,
                        stop=oracle.STOP_MAX_REL, tol=p.tol, min_epochs=11, max_epochs=100000)
    return {"workload": "small_rbf n=4096 d=8 b=512 c=1 tol=1e-6", "time_to_tol_s": time.perf_counter() - t0,
            "epochs": r.epochs, "converged": r.status == oracle.OK, "rel_res": float(r.rel[0]),
            "cores": oracle.num_threads()}


def cpu_baseline(p, epochs: int, args) -> dict:
    """The FP64 oracle as it stands on the host cores, on a bounded sample of the
    same workload: one AP residual update over a row sample (the hot loop of
    Alg. 1) and the Cholesky factorisation of one diagonal block; time-to-tol
    is extrapolated to the whole step with the epoch count of the GPU run."""
    import oracle
    h = oracle.Hyper.of(p)
    X = p.X.astype(np.float64)
    rows = min(p.n, args.cpu_rows)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(p.n, rows, replace=False)).astype(np.int64)
    b = p.block
    delta = rng.standard_normal((b, p.c))
    R = np.zeros((p.n, p.c))
    t0 = time.perf_counter()
    oracle.block_update(h, X, 0, delta, R, rows=idx)
    t_upd = time.perf_counter() - t0
    ent_per_s = rows * b / t_upd
    Kii = oracle.gram(h, X[:b], X[:b], row0=0, col0=0)
    t0 = time.perf_counter()
    oracle.cholesky(Kii)
    t_chol = time.perf_counter() - t0
    m = -(-p.n // b)
    steps = epochs * m
    entries = float(p.n) * b + steps * float(p.n) * b + float(p.n) ** 2
    t_total = m * t_chol + (steps * float(p.n) * b + float(p.n) ** 2) / ent_per_s
    return {"value": entries / t_total, "unit": "kernel-entries/s", "cores": oracle.num_threads(),
            "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"one residual update (Eq. text_update_of_r) over {rows} of {p.n} rows x b={b} "
                      f"({t_upd:.1f} s) + FP64 Cholesky of one {b}x{b} block ({t_chol:.1f} s); "
                      f"time-to-tol extrapolated to {m} blocks and {epochs} epochs = {t_total:.0f} s",
            "time_to_tol_s_extrapolated": t_total}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    import oracle
    p = workload(args.workload, sub=0, n=args.n)
    epochs = args.max_epochs
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.warmup + args.steps):
        vals.append(cpu_baseline(p, epochs, args))
    t_all = time.perf_counter() - t_all
    timed = vals[args.warmup:]
    v = statistics.median(x["value"] for x in timed)
    line = {
        "metric": METRIC, "impl": "reference", "value": v, "unit": "kernel-entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.median(x["time_to_tol_s_extrapolated"] for x in timed) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded NumPy PCG64)", "config": describe(p, args),
        "cpu_baseline": {"value": v, "unit": "kernel-entries/s", "cores": oracle.num_threads(),
                         "cpu_model": cpu_model(), "kind": "oracle", "sample": timed[-1]["sample"]},
        "e2e": {"value": v, "unit": "kernel-entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": t_all,
    }
    print(json.dumps(line), flush=True)


def run_serving(args) -> None:
    """The full serving replay (`--serve`): 512 requests by default."""
    import paper_2310_17137_gb300 as ap
    out = serving_replay(ap, args, args.serve_requests, args.serve_max_epochs)
    line = {"metric": METRIC, "mode": "serving", "value": out["solves_per_s"], "unit": "solves/s", **out}
    print(json.dumps(line), flush=True)


def run_study(args) -> None:
    """Selection rules and block sizes on the same kernels (the shape of the
    paper's Sec. 3 block-selection comparison and of its block-size study), on
    the Matern-5/2 generator at n = 65,536 in the tensor-core form: the true
    relative residual after 1..32 epochs for Gauss-Southwell, cyclic and random
    selection (b = 2048), and time and residual after 16 epochs for b = 1024 ..
    8192 (cache included)."""
    import torch
    import paper_2310_17137_gb300 as ap
    dev = torch.device("cuda", 0)
    p = wl.matern52_ard(n=args.study_n)
    X = torch.from_numpy(p.X).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    hyper = ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise, p.mean)
    rules = {"gauss_southwell": ap.AP_SEL_GS, "cyclic": ap.AP_SEL_CYCLIC, "random": ap.AP_SEL_RANDOM}
    epochs = [1, 2, 4, 8, 16, 32]
    sel = {}
    for name, rule in rules.items():
        rows = []
        for e in epochs:
            ctx = ap.ap_create(X, hyper, ap.ap_opts_default(block=2048, select=rule, tol=1e-30, min_epochs=e,
                                                            max_epochs=e, precision=ap.AP_BF16_REFINE,
                                                            refine_every=10, seed=5))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, _, info, _ = ap.ap_solve(ctx, B)
            torch.cuda.synchronize()
            rows.append({"epochs": e, "rel_res_y": info["rel_res_true"][0],
                         "rel_res_max": max(info["rel_res_true"][:p.c]), "solve_s": time.perf_counter() - t0})
            ap.ap_destroy(ctx)
        sel[name] = rows
    bs = []
    for b in [1024, 2048, 4096, 8192]:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = ap.ap_create(X, hyper, ap.ap_opts_default(block=b, tol=1e-30, min_epochs=16, max_epochs=16,
                                                        precision=ap.AP_BF16_REFINE, refine_every=10))
        _, _, info, _ = ap.ap_solve(ctx, B)
        torch.cuda.synchronize()
        bs.append({"block": b, "time_s": time.perf_counter() - t0, "cache_s": info["t_cache_s"],
                   "solve_s": info["t_solve_s"], "rel_res_y": info["rel_res_true"][0],
                   "rel_res_max": max(info["rel_res_true"][:p.c])})
        ap.ap_destroy(ctx)
    print(json.dumps({"metric": METRIC, "mode": "study", "workload": f"{p.name} ({wl.KERNEL_NAMES[p.kernel]} ARD, "
                      f"c={p.c}, noise={p.noise:g}), BF16+refine form", "selection": sel, "block_size": bs}),
          flush=True)


def main():
    ap_ = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap_.add_argument("--gpus", type=int, default=1)
    ap_.add_argument("--steps", type=int, default=3)
    ap_.add_argument("--warmup", type=int, default=3)
    ap_.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap_.add_argument("--workload", default="matern52_ard")
    ap_.add_argument("--precision", choices=sorted(FORMS), default="bf16",
                     help="form of the timed steps: bf16 = tensor-core BF16 hi/lo with FP32 refinement, "
                          "fp32 = FP32 SIMT")
    ap_.add_argument("--refine-every", type=int, default=10)
    ap_.add_argument("--no-compare", action="store_true", help="skip the timed runs of the other forms")
    ap_.add_argument("--min-epochs", type=int, default=11)
    ap_.add_argument("--max-epochs", type=int, default=30,
                     help="epoch cap per solve (the configured tolerance is out of AP's reach on "
                          "this workload within any practical cap; see the time_to_tol_small key)")
    ap_.add_argument("--n", type=int, default=0, help="override n (profiling on a smaller case)")
    ap_.add_argument("--cpu-rows", type=int, default=65536)
    ap_.add_argument("--no-cpu-baseline", action="store_true")
    ap_.add_argument("--no-e2e", action="store_true")
    ap_.add_argument("--no-ttt", action="store_true")
    ap_.add_argument("--no-mll", action="store_true", help="skip the MLL-gradient timing")
    ap_.add_argument("--no-ttt-large", action="store_true",
                     help="skip the time-to-tolerance runs on the n = 2,097,152 RBF workload")
    ap_.add_argument("--ttt-large-max-epochs", type=int, default=400)
    ap_.add_argument("--no-serve-replay", action="store_true", help="skip the reduced serving replay")
    ap_.add_argument("--serve-replay-requests", type=int, default=48)
    ap_.add_argument("--time-budget-s", type=float, default=1500.0,
                     help="skip the time-to-tolerance and serving legs when they would not fit")
    ap_.add_argument("--compare-steps", type=int, default=3, help="timed steps of the other form")
    ap_.add_argument("--e2e-steps", type=int, default=5, help="timed steps of the end-to-end leg")
    ap_.add_argument("--serve", action="store_true", help="replay the serving workload instead")
    ap_.add_argument("--study", action="store_true", help="selection rules and block sizes instead")
    ap_.add_argument("--study-n", type=int, default=65536)
    ap_.add_argument("--serve-requests", type=int, default=512)
    ap_.add_argument("--serve-rate", type=float, default=40.0)
    ap_.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap_.add_argument("--serve-slots", type=int, default=8)
    ap_.add_argument("--serve-max-epochs", type=int, default=300)
    args = ap_.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if args.gpus == 1 else 1))
    if args.serve:
        if rank == 0:
            run_serving(args)
    elif args.study:
        if rank == 0:
            run_study(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
