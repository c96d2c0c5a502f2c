#!/usr/bin/env python
"""CP-ALS benchmark on GB300: sweeps/s and MTTKRP TFLOP/s, MSDT / PP vs DT.

Default workload: order-4 dense FP32 tensor 128^4 (268M entries, 1.07 GB) =
sum of R = 64 rank-one terms with U[0,1) factors plus Gaussian noise at 1e-3
of the tensor norm; R = 64, U[0,1) initial factors.  A step is one sweep of
the multi-sweep dimension tree (N = 4 factor updates: first-level TTM when a
root is due, mTTVs, FP64 Hadamard/Cholesky/solve/Gram, residual terms).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  With N > 1 (torchrun) every rank decomposes
its own tensor (replicas; the engine runs on one GPU per problem) and `value`
sums the ranks' sweeps/s over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: dims, R, law, eta, seed
    "c2": dict(dims=(128, 128, 128, 128), R=64, law="uniform", eta=1e-3, seed=20101205 + 1000,
               desc="order-4 dense FP32 128^4, rank-64 U[0,1) factors + 1e-3 noise, R=64"),
    "c1": dict(dims=(64, 64, 64), R=16, law="uniform", eta=1e-2, seed=20101205,
               desc="order-3 dense 64^3, rank-16 U[0,1) factors + 1e-2 noise, R=16"),
    "c3": dict(dims=(1024, 1024, 1024), R=256, law="gaussian", eta=1e-2, seed=20101205 + 2000,
               desc="order-3 dense FP32 1024^3, rank-256 N(0,1) factors + 1e-2 noise, R=256"),
    "c4": dict(dims=(160, 160, 160, 160), R=100, law="collinear", eta=1e-3, C=0.9,
               seed=20101205 + 3000,
               desc="order-4 dense FP32 160^4, rank-100 collinear (cos 0.9) factors + 1e-3 noise"),
}
METRIC = "ALS sweep/s (MSDT) on 1 GPU, order-4 128^4 R=64"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=list(WORKLOADS))
    ap.add_argument("--prec", default="bf16x3", choices=["fp32", "tf32", "bf16x3", "bf16", "tf32x3"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return dict(PEAKS_FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                mhz.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        mhz.sort()
        med = mhz[len(mhz) // 2] if mhz else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(mhz)}


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


def oracle_sweeps(T64, A0, seconds, route="msdt"):
    """Time the FP64 oracle (as it stands) on the same tensor: sweeps/s over a bounded sample."""
    from oracle import cp_oracle as co
    A = [a.copy() for a in A0]
    n, t0 = 0, time.perf_counter()
    while True:
        res = co.cp_als(T64, A, 1, route=route)
        A = res.A
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return n / el, n, el


def make_inputs(wl, device):
    import synth
    return synth.make_problem_device(wl["seed"], wl["dims"], wl["R"], law=wl["law"], eta=wl["eta"],
                                     C=wl.get("C"), device=device)


def run_reference(args, wl, rank):
    """Reference arm: the FP64 CPU oracle timed on the host cores (rank 0 only)."""
    import numpy as np
    import torch
    if rank != 0:
        return
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    T, F, A0 = make_inputs(wl, dev)
    T64 = T.cpu().numpy().astype(np.float64)
    del T
    from oracle import cp_oracle as co
    A = [a.copy() for a in A0]
    for _ in range(args.warmup):
        A = co.cp_als(T64, A, 1, route="msdt").A
    t0 = time.perf_counter()
    for _ in range(args.steps):
        A = co.cp_als(T64, A, 1, route="msdt").A
    el = time.perf_counter() - t0
    v = args.steps / el
    cores = cpu_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "sweep/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "sweep": "msdt"},
        "cpu_baseline": {"value": v, "unit": "sweep/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} FP64 oracle MSDT sweeps on the full tensor"},
        "e2e": {"value": v, "unit": "sweep/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl, rank)
        return

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    import paper_2010_12056_gb300 as pkg
    import __graft_entry__ as ge
    ge.build()

    dims, R = wl["dims"], wl["R"]
    N = len(dims)
    numel = int(np.prod(dims))
    T, F, A0 = make_inputs(wl, "cuda")
    stream = torch.cuda.current_stream()
    ctx = pkg.CPContext(T, R, A0=A0, prec=args.prec, stream=stream)

    # ---------------------------------------------------------------- MSDT (the step)
    ctx.sweep_msdt(args.warmup)
    st0 = ctx.stats()
    clk = ClockSampler(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    ctx.sweep_msdt(args.steps)
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    st1 = ctx.stats()
    launches = int(st1["launches"] - st0["launches"])
    flops = (st1["ttm_flops"] - st0["ttm_flops"]) + (st1["mttv_flops"] - st0["mttv_flops"])
    msdt_sps = args.steps / (ms / 1e3)
    value = msdt_sps * world
    mttkrp_tflops = flops / (ms / 1e3) / 1e12
    fit_formula = ctx.fit(exact=False)[0]
    fit_direct = ctx.fit(exact=True)[0]

    # ---------------------------------------------------------------- DT on the same problem
    ctx_dt = pkg.CPContext(T, R, A0=A0, prec=args.prec, stream=stream)
    ctx_dt.sweep_dt(args.warmup)
    barrier()
    e0.record(stream)
    ctx_dt.sweep_dt(args.steps)
    e1.record(stream)
    barrier()
    ms_dt = max_over_ranks(e0.elapsed_time(e1))
    dt_sps = args.steps / (ms_dt / 1e3)
    ctx_dt.close()

    # ---------------------------------------------------------------- TTM roofline
    peaks, peak_kind = load_peaks()
    mode = N - 1
    X = torch.empty(numel // dims[mode] * R, dtype=torch.float32, device="cuda")
    for _ in range(3):
        ctx.ttm(mode, out=X)
    nrep = max(5, args.steps)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(nrep):
        ctx.ttm(mode, out=X)
    e1.record(stream)
    torch.cuda.synchronize()
    ttm_ms = e0.elapsed_time(e1) / nrep
    ttm_bytes = 4.0 * numel + 4.0 * (numel // dims[mode]) * R
    ttm_flops = 2.0 * numel * R
    del X
    if args.prec == "fp32":
        sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        roofline = {"bound": "alu", "achieved": ttm_flops / (ttm_ms / 1e3) / 1e12, "peak": alu_peak,
                    "unit": "TFLOP/s", "frac": None, "traffic": None,
                    "kernel": "ttm_simt", "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz} MHz"}
    else:
        ach = ttm_bytes / (ttm_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": None, "traffic": None, "kernel": "ttm_tc",
                    "peak_source": f"hbm_gbs of {peak_kind}"}
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    roofline["ms_per_launch"] = ttm_ms
    roofline["algorithmic_bytes"] = ttm_bytes
    roofline["algorithmic_flops"] = ttm_flops

    # ---------------------------------------------------------------- PP (approximated sweeps)
    ctx_pp = pkg.CPContext(T, R, A0=A0, prec=args.prec, stream=stream)
    ctx_pp.sweep_msdt(max(2, args.warmup))
    ctx_pp.sweep_pp(3, eps=0.99)           # regular sweep, PP init, first approximated sweep
    tr0 = len(ctx_pp.trace())
    t0 = time.perf_counter()
    ctx_pp.sweep_pp(args.steps, eps=0.99)
    torch.cuda.synchronize()
    wall_pp = time.perf_counter() - t0
    tr = ctx_pp.trace()[tr0:]
    pp_ms = [t["ms"] for t in tr if t["kind"] == "pp"]
    pp_info = {"approx_sweeps": len(pp_ms),
               "approx_sweep_ms": (sum(pp_ms) / len(pp_ms)) if pp_ms else None,
               "approx_sweeps_per_s_wall": len(tr) / wall_pp,
               "init_count": ctx_pp.stats()["pp_init"]}
    ctx_pp.close()

    # ---------------------------------------------------------------- e2e (host buffers)
    e2e = None
    if not args.no_e2e:
        Th = torch.empty(dims, dtype=torch.float32, pin_memory=True)
        Th.copy_(T.cpu())
        ctx_e = pkg.CPContext(T, R, A0=A0, prec=args.prec, stream=stream)
        ctx_e.sweep_msdt(1)
        barrier()
        t0 = time.perf_counter()
        fits = []
        for _ in range(args.steps):
            T.copy_(Th, non_blocking=True)     # this step's input, host -> device
            ctx_e.sweep_msdt(1)
            fits.append(ctx_e.fit(exact=False)[0])  # the step's result, device -> host
        barrier()
        el = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": world * args.steps / el, "unit": "sweep/s",
               "h2d_bytes_per_step": 4 * numel, "d2h_bytes_per_step": 8}
        ctx_e.close()
        del Th

    # ---------------------------------------------------------------- CPU baseline (oracle)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and args.gpus == 1:
        T64 = T.cpu().numpy().astype(np.float64)
        v, n, el = oracle_sweeps(T64, A0, args.cpu_seconds)
        cpu = {"value": v, "unit": "sweep/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{n} FP64 oracle MSDT sweeps of the full tensor ({el:.1f} s)"}
        del T64

    line = {
        "metric": METRIC, "value": value, "unit": "sweep/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "precision": {"ttm": args.prec, "mttv": "f32", "gram_cholesky_solve_residual": "f64"},
        "data": "synthetic",
        "config": {"workload": wl["desc"], "dims": list(dims), "R": R, "sweep": "msdt",
                   "l2": "inputs larger than L2 (tensor 1.07 GB, root 537 MB)"
                   if args.workload == "c2" else "see dims"},
        "mttkrp_tflops": mttkrp_tflops,
        "dt_sweeps_per_s": dt_sps * world,
        "msdt_time_over_dt": (ms / args.steps) / (ms_dt / args.steps),
        "fit": {"formula": fit_formula, "direct": fit_direct, "after_sweeps": args.warmup + args.steps},
        "solves_fp64": int(st1["solves_fp64"]),
        "pp": pp_info,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": launches,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
