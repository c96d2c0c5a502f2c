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
    # synthetic stand-ins with the mode sizes and ranks of the paper's application
    # tensors (Sec. V-A; the datasets themselves are not used): U[0,1) factors, whose
    # columns are collinear (expected cosine 0.75), plus 1e-3 noise
    "coil": dict(dims=(128, 128, 3, 7200), R=20, law="uniform", eta=1e-3, seed=20101205 + 6000,
                 desc="order-4 FP32 128x128x3x7200 (image-set shape), rank-20 U[0,1) factors + 1e-3 noise"),
    "timelapse": dict(dims=(1024, 1344, 33, 9), R=50, law="uniform", eta=1e-3, seed=20101205 + 7000,
                      desc="order-4 FP32 1024x1344x33x9 (hyperspectral time-lapse shape), rank-50 U[0,1) "
                           "factors + 1e-3 noise"),
    # rank 256 against modes of 280: U[0,1) factors that collinear drive ALS into
    # singular normal equations, so this stand-in draws N(0,1) factors
    "chem": dict(dims=(4520, 280, 280), R=256, law="gaussian", eta=1e-3, seed=20101205 + 8000,
                 desc="order-3 FP32 4520x280x280 (density-fitting tensor shape), rank-256 N(0,1) factors "
                      "+ 1e-3 noise (the paper uses ranks 300-1000)"),
}
STANDINS = ("coil", "timelapse", "chem")
METRIC = "ALS sweep/s (MSDT) on 1 GPU, order-4 128^4 R=64"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# DRAM bytes per launch of the last-mode TTM on 128^4 R=64 from ncu captures of
# the current kernel, by precision (profiles/ttm_tc_*_c2.md); a precision whose
# kernel changed since its capture has no entry (traffic null)
TRAFFIC_C2 = {"f16x3": 1.073848e9 + 0.500767e9}
FIT_SWEEPS = 20     # the fit check: direct residual after this many MSDT sweeps from A0
FIT_TOL = 1e-6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=list(WORKLOADS) + ["policy", "collinearity"])
    ap.add_argument("--prec", default="f16x3", choices=["fp32", "tf32", "bf16x3", "bf16", "tf32x3", "f16x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    # learned PP policy experiment (--workload policy)
    ap.add_argument("--train-tensors", type=int, default=512)
    ap.add_argument("--eval-tensors", type=int, default=64)
    ap.add_argument("--probe-sweeps", type=int, default=40)
    ap.add_argument("--target-sweeps", type=int, default=60)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--policy-dims", default="256,256,256")
    ap.add_argument("--policy-law", default="collinear", choices=["collinear", "uniform"])
    # collinearity study (--workload collinearity; Sec. V-A tensors with given collinearity)
    ap.add_argument("--col-seeds", type=int, default=3, help="tensors per collinearity bin")
    ap.add_argument("--col-size", type=int, default=1600)
    ap.add_argument("--col-rank", type=int, default=400)
    ap.add_argument("--col-bins", default="0,0.2,0.4,0.6,0.8,1.0")
    ap.add_argument("--col-exact", default="dt,msdt", help="exact routes timed beside PP")
    ap.add_argument("--ttm-only", action="store_true",
                    help="time only one first-level TTM (cp_ttm, --ttm-mode) and exit")
    ap.add_argument("--ttm-mode", type=int, default=-1, help="mode of --ttm-only (default: the last)")
    ap.add_argument("--presplit", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="R > 128: T's stored 16-bit parts (cp_set_option CP_OPT_TTM_PRESPLIT; "
                         "0 off, 1 256-column passes, 2 128-column passes; -1 the library's default)")
    ap.add_argument("--dims", default=None, help="override the workload's mode sizes, e.g. 512,512,512")
    ap.add_argument("--rank", type=int, default=None, help="override the workload's rank")
    ap.add_argument("--law", default=None, choices=["uniform", "gaussian", "collinear"])
    ap.add_argument("--pp-sweeps", type=int, default=-1,
                    help="PP (eps = 0.1) vs exact MSDT over this many sweeps (default: 100 for c4, else 0)")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return dict(PEAKS_FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms.  Samples taken
    between mark_start() and mark_stop() (the timed region) are summarised; when
    that region is shorter than the sampling period, the samples of the whole
    GPU-busy window around it (mark_window_start/stop: the timed region followed
    by the schedule and roofline loops on the same workload) stand in, and the
    summary says which."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.t = None
        self.t0 = self.t1 = None
        self.w0 = self.w1 = None

    def mark_window_start(self):
        self.w0 = time.time()

    def mark_window_stop(self):
        self.w1 = time.time()

    def start(self, wait_s=3.0):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        t_end = time.time() + wait_s   # the first sample shows the sampler is running
        while not self.rows and time.time() < t_end:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append((time.time(), parts))

    def mark_start(self):
        self.t0 = time.time()

    def mark_stop(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        rows = self.rows
        source = "all samples"
        if self.t0 is not None and self.t1 is not None:
            inside = [r for r in rows if self.t0 <= r[0] <= self.t1 + 0.05]
            if inside:
                rows, source = inside, "timed region"
            elif self.w0 is not None and self.w1 is not None:
                rows = [r for r in rows if self.w0 <= r[0] <= self.w1]
                source = "benchmark window (timed region shorter than the 50 ms sampling period)"
            else:
                rows = [r for r in rows if r[0] >= self.t0][:1]
                source = "first sample after the timed region"
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, r in rows:
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
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(mhz),
                "source": source}


class Ranks:
    """Rank bookkeeping of the replica benchmark: every rank decomposes its own
    tensor; timing takes a barrier on both sides and the maximum over ranks.
    `dist` is torch.distributed (initialised) or None for one process."""

    def __init__(self, dist=None, device="cuda"):
        self.dist = dist
        self.device = device

    def _sync(self):
        if self.device == "cuda":
            import torch
            torch.cuda.synchronize()

    def barrier(self):
        self._sync()
        if self.dist is not None:
            self.dist.barrier()
        self._sync()

    def max(self, x):
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def replica_rate(steps, ms_max, world):
    """Whole-job sweeps/s: every rank ran `steps` sweeps; the slowest rank's time counts."""
    return world * steps / (ms_max / 1e3)


def cpu_threads():
    """Host cores the oracle's BLAS may use: every core of the box (nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def make_inputs(wl, device):
    import synth
    return synth.make_problem_device(wl["seed"], wl["dims"], wl["R"], law=wl["law"], eta=wl["eta"],
                                     C=wl.get("C"), device=device)


def run_reference(args, wl, rank, budget_s=60.0):
    """Reference arm: the FP64 CPU oracle timed on the host cores (rank 0 only).

    A step is one oracle MSDT sweep of the full tensor; the sample is bounded:
    sweeps run until --steps are done or about budget_s seconds have passed (at
    least one), after at most one warm-up sweep, and the line says how many ran."""
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
    for _ in range(min(args.warmup, 1)):
        A = co.cp_als(T64, A, 1, route="msdt").A
    n, t0 = 0, time.perf_counter()
    while n < args.steps:
        A = co.cp_als(T64, A, 1, route="msdt").A
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    v = n / el
    cores = cpu_threads()
    sample = f"{n} of {args.steps} FP64 oracle MSDT sweeps on the full tensor ({el:.1f} s, budget {budget_s:.0f} s)"
    nwarm = min(args.warmup, 1)
    r_direct = co.residual_direct(T64, A)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "sweep/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / n,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "sweep": "msdt"},
        "cpu_baseline": {"value": v, "unit": "sweep/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "sweep/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "fit": {"direct": r_direct, "after_sweeps": nwarm + n},
    }
    print(json.dumps(line), flush=True)


def policy_problem(i, dims, base_seed, law="collinear"):
    """The i-th tensor of the policy study: rank-R factors, R in {16, 32, 64}, noise
    log-uniform in [1e-4, 1e-2] (draws from a seeded generator).  law "collinear":
    pairwise cosine U[0.5, 0.95] (needs every mode >= R); "uniform": U[0,1) factors
    (expected cosine 0.75), for shapes with small modes."""
    import numpy as np
    import synth
    g = np.random.default_rng(base_seed + i)
    R = (16, 32, 64)[i % 3]
    C = float(g.uniform(0.5, 0.95))
    eta = float(10.0 ** g.uniform(-4.0, -2.0))
    if law == "collinear":
        T, _, _ = synth.make_problem_device(base_seed + i, list(dims), R, law="collinear", eta=eta, C=C)
    else:
        T, _, _ = synth.make_problem_device(base_seed + i, list(dims), R, law=law, eta=eta)
        C = 0.75
    return T, R, C, eta


def run_policy(args):
    """Learned PP policy: traces from the training tensors (cp_pp_probe), training with the
    library's kernels, then device time to reach exact MSDT's fit after --target-sweeps sweeps
    on held-out tensors for exact MSDT, Alg. 2 with eps = 0.1, and the learned policy."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2010_12056_gb300 import policy as pol
    import paper_2010_12056_gb300 as pkg
    dims = tuple(int(x) for x in args.policy_dims.split(","))
    train_seed, eval_seed = 20101205 + 4000, 20101205 + 5000
    t0 = time.perf_counter()
    Xs, ys = [], []
    for i in range(args.train_tensors):
        T, R, C, eta = policy_problem(i, dims, train_seed, args.policy_law)
        X, y, _ = pol.collect(T, R, args.probe_sweeps, prec=args.prec, seed=1 + i, min_gain=1e-9)
        Xs.append(X)
        ys.append(y)
        del T
    X = np.concatenate(Xs)
    y = np.concatenate(ys)
    t_collect = time.perf_counter() - t0
    t0 = time.perf_counter()
    policy = pol.train(X, y, steps=args.train_steps, lr=3e-3, seed=0)
    t_train = time.perf_counter() - t0
    acc = pol.accuracy(policy, X, y)
    res = {"msdt": [], "pp": [], "policy": []}
    per = []
    for i in range(args.eval_tensors):
        T, R, C, eta = policy_problem(i, dims, eval_seed, args.policy_law)
        ctx = pkg.CPContext(T, R, prec=args.prec, seed=7 + i)
        ctx.sweep_msdt(args.target_sweeps)
        target = ctx.fit(exact=True)[1] + 1e-6   # equal fit: within 1e-6
        ctx.close()
        row = {"R": R, "C": round(C, 3), "eta": eta, "target_resid": target}
        for m in ("msdt", "pp", "policy"):
            ms, k, r, tr = pol.time_to_target(T, R, m, target, 3 * args.target_sweeps, prec=args.prec,
                                              seed=7 + i, eps=0.1, policy=policy if m == "policy" else None)
            res[m].append(ms)
            row[m] = {"ms": ms, "sweeps": k,
                      "approx": sum(t.get("kind") == "pp" for t in tr),
                      "rolled_back": sum(t.get("rolled_back", 0) for t in tr)}
            if tr and "error" in tr[-1]:
                row[m]["error"] = tr[-1]["error"]
        per.append(row)
        del T
    tot = {m: float(np.sum(v)) for m, v in res.items()}
    reached = {m: int(np.sum(np.isfinite(v))) for m, v in res.items()}
    both = np.isfinite(res["msdt"]) & np.isfinite(res["pp"]) & np.isfinite(res["policy"])
    common = {m: float(np.sum(np.asarray(v)[both])) for m, v in res.items()}
    wins = {m: 0 for m in res}
    for i in range(len(res["msdt"])):
        wins[min(res, key=lambda m: res[m][i])] += 1
    line = {
        "metric": "device time to exact MSDT's fit after %d sweeps (+1e-6), held-out tensors" % args.target_sweeps,
        "value": tot["policy"], "unit": "ms (sum over held-out tensors)", "n_gpus": 1,
        "higher_is_better": False, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "learned PP policy, %s %s tensors" % ("x".join(map(str, dims)),
                                                                    args.policy_law),
                   "train_tensors": args.train_tensors, "eval_tensors": args.eval_tensors,
                   "probe_sweeps": args.probe_sweeps, "train_steps": args.train_steps, "prec": args.prec},
        "total_ms": tot, "reached": reached, "wins": wins,
        "total_ms_where_all_reached": common, "all_reached": int(both.sum()),
        "policy_vs_pp": tot["pp"] / tot["policy"] if tot["policy"] > 0 else None,
        "policy_vs_msdt": tot["msdt"] / tot["policy"] if tot["policy"] > 0 else None,
        "train": {"samples": int(len(y)), "positive": float(np.mean(y)) if len(y) else None,
                  "accuracy": acc, "collect_s": t_collect, "train_s": t_train},
        "per_tensor": per,
    }
    print(json.dumps(line), flush=True)


def run_collinearity(args):
    """The paper's collinearity study on one GPU (Sec. V-A, Fig. 4, Table 3): order-3
    tensors s^3 = [[A, A, A]] from rank-R factors whose columns have pairwise cosine
    C drawn uniformly from each bin [a, b) (no noise: CP rank at most R), U[0,1)
    initial factors; PP-CP-ALS (Alg. 2) with tolerance 0.2 and exact sweeps, each
    stopped when the relative residual changes by at most 1e-5 between sweeps or
    after 300 sweeps (Sec. V-C).  Reports per bin the sweep counts of Table 3
    (exact sweeps inside PP, PP initializations, approximated sweeps), the device
    time to stop and the final direct fit of every method."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2010_12056_gb300 as pkg
    import synth
    s, R = args.col_size, args.col_rank
    edges = [float(x) for x in args.col_bins.split(",")]
    exact_routes = [x for x in args.col_exact.split(",") if x]
    bins = []
    for b in range(len(edges) - 1):
        a, e = edges[b], edges[b + 1]
        runs = []
        for i in range(args.col_seeds):
            seed = 20101205 + 9000 + 100 * b + i
            g = np.random.default_rng(seed)
            C = float(g.uniform(a, e))
            C = min(C, 0.999)
            T, _, A0 = synth.make_problem_device(seed, [s, s, s], R, law="collinear", C=C, eta=0.0)
            torch.cuda.synchronize()
            run = {"C": C, "seed": seed}
            for route in exact_routes + ["pp"]:
                ctx = pkg.CPContext(T, R, A0=A0, prec=args.prec, pp_eps=0.2, delta=1e-5, max_sweeps=300)
                err = None
                try:
                    ctx.run(route)
                except pkg.CPError as ex:
                    err = str(ex)
                tr = ctx.trace()
                rec = {"sweeps": len(tr), "ms": sum(t["ms"] for t in tr), "error": err}
                try:
                    rec["fit_direct"] = ctx.fit(exact=True)[0]
                except pkg.CPError as ex:
                    rec["fit_direct"] = None
                if route == "pp":
                    rec["als"] = sum(1 for t in tr if t["kind"] != "pp")
                    rec["pp_init"] = sum(t["pp_init"] for t in tr)
                    rec["pp_approx"] = sum(1 for t in tr if t["kind"] == "pp")
                run[route] = rec
                ctx.close()
            del T
            torch.cuda.empty_cache()
            runs.append(run)
            print(json.dumps({"bin": [a, e], **run}), flush=True)

        def mean(key, route):
            v = [r[route][key] for r in runs if r[route].get(key) is not None]
            return float(np.mean(v)) if v else None
        summary = {"bin": [a, e], "tensors": len(runs),
                   "num_als": mean("als", "pp"), "num_pp_init": mean("pp_init", "pp"),
                   "num_pp_approx": mean("pp_approx", "pp"), "pp_ms": mean("ms", "pp"),
                   "pp_fit": mean("fit_direct", "pp")}
        for route in exact_routes:
            summary[f"{route}_sweeps"] = mean("sweeps", route)
            summary[f"{route}_ms"] = mean("ms", route)
            summary[f"{route}_fit"] = mean("fit_direct", route)
            sp = [r[route]["ms"] / r["pp"]["ms"] for r in runs if r["pp"]["ms"] > 0]
            summary[f"speedup_pp_over_{route}_median"] = float(np.median(sp)) if sp else None
        bins.append(summary)
    print(json.dumps({"metric": "collinearity study: PP (eps 0.2) vs exact sweeps, time to stop",
                      "config": {"dims": [s, s, s], "R": R, "eps": 0.2, "delta": 1e-5, "max_sweeps": 300,
                                 "tensors_per_bin": args.col_seeds, "prec": args.prec, "noise": 0.0},
                      "bins": bins}), flush=True)


def run_ttm_only(args, wl):
    """Time cp_ttm of the last mode (the kernel the sweeps launch) on one workload."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2010_12056_gb300 as pkg
    dims, R = wl["dims"], wl["R"]
    numel = int(np.prod(dims))
    T, _, A0 = make_inputs(wl, "cuda")
    ctx = pkg.CPContext(T, R, A0=A0, prec=args.prec)
    if args.presplit >= 0:
        ctx.set_option("ttm_presplit", args.presplit)
    mode = args.ttm_mode if args.ttm_mode >= 0 else len(dims) - 1
    X = torch.empty(numel // dims[mode] * R, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        ctx.ttm(mode, out=X)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        ctx.ttm(mode, out=X)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    st = ctx.stats()
    print(json.dumps({"metric": "first-level TTM time", "value": ms, "unit": "ms", "workload": wl["desc"],
                      "prec": args.prec, "mode": mode, "tflops_algorithmic": 2.0 * numel * R / (ms / 1e3) / 1e12,
                      "gbs_algorithmic": (4.0 * numel + 4.0 * numel // dims[mode] * R) / (ms / 1e3) / 1e9,
                      "tensor_core_launches": st["ttm_tensor_core"],
                      "stored_parts_launches": st["ttm_stored_parts"]}), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.workload == "policy":
        if int(os.environ.get("RANK", "0")) == 0:
            run_policy(args)
        return
    if args.workload == "collinearity":
        if int(os.environ.get("RANK", "0")) == 0:
            run_collinearity(args)
        return
    wl = dict(WORKLOADS[args.workload])
    if args.dims or args.rank or args.law:
        if args.dims:
            wl["dims"] = tuple(int(x) for x in args.dims.split(","))
        if args.rank:
            wl["R"] = args.rank
        if args.law:
            wl["law"] = args.law
        wl["desc"] = "custom: dims %s, R = %d, %s factors + %g noise" % (
            "x".join(map(str, wl["dims"])), wl["R"], wl["law"], wl["eta"])
    if args.ttm_only:
        run_ttm_only(args, wl)
        return
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

    ranks = Ranks(dist, "cuda")
    barrier, max_over_ranks = ranks.barrier, ranks.max

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
    clk.mark_window_start()
    clk.mark_start()
    e0.record(stream)
    ctx.sweep_msdt(args.steps)
    e1.record(stream)
    barrier()
    clk.mark_stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    st1 = ctx.stats()
    launches = int(st1["launches"] - st0["launches"])
    flops = (st1["ttm_flops"] - st0["ttm_flops"]) + (st1["mttv_flops"] - st0["mttv_flops"])
    msdt_sps = args.steps / (ms / 1e3)
    value = replica_rate(args.steps, ms, world)
    mttkrp_tflops = flops / (ms / 1e3) / 1e12
    fit_formula = ctx.fit(exact=False)[0]
    fit_direct = ctx.fit(exact=True)[0]

    # ---------------------------------------------------------------- other schedules, same problem
    def timed_sweeps(route, **options):
        """sweeps/s of `route` from the same start, with cp_set_option switches."""
        c2 = pkg.CPContext(T, R, A0=A0, prec=args.prec, stream=stream)
        for k, v in options.items():
            c2.set_option(k, v)
        run = c2.sweep_dt if route == "dt" else c2.sweep_msdt
        run(args.warmup)
        barrier()
        e0.record(stream)
        run(args.steps)
        e1.record(stream)
        barrier()
        t = max_over_ranks(e0.elapsed_time(e1))
        c2.close()
        return args.steps / (t / 1e3)

    dt_sps = timed_sweeps("dt")
    schedules = {
        "msdt": msdt_sps,
        "dt_fused": dt_sps,
        # Fig. 1a literally: first-level TTM, then one multi-TTV per level
        "dt_unfused": timed_sweeps("dt", fuse_dt=False),
        # the TTM epilogue also forms the first child of roots T x_0 and T x_{N-1}
        "msdt_fused_child": timed_sweeps("msdt", fuse_child=True),
        # second child contracted on a side stream during the next update (6 blocks/SM)
        "msdt_lookahead": timed_sweeps("msdt", lookahead=6),
    }
    if N >= 4:
        # upper two levels combined (Sec. IV): level-2 roots straight from T, s^(N-2) R memory
        schedules["msdt_levels2"] = timed_sweeps("msdt", msdt_levels=2)

    # ---------------------------------------------------------------- TTM roofline
    peaks, peak_kind = load_peaks()
    # the last mode, unless it has no tensor-core plan (uneven shapes: a small last
    # mode or a row stride that TMA cannot address); then the largest mode that has one
    mode = N - 1
    used_tc = False
    for m in [N - 1] + sorted(range(N - 1), key=lambda k: -dims[k]):
        n0 = ctx.stats()["ttm_tensor_core"]
        Xm = torch.empty(numel // dims[m] * R, dtype=torch.float32, device="cuda")
        ctx.ttm(m, out=Xm)
        del Xm
        if ctx.stats()["ttm_tensor_core"] > n0:
            mode, used_tc = m, True
            break
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
    clk.mark_window_stop()
    clocks = clk.stop()
    if args.prec == "fp32" or not used_tc:
        sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        roofline = {"bound": "alu", "achieved": ttm_flops / (ttm_ms / 1e3) / 1e12, "peak": alu_peak,
                    "unit": "TFLOP/s", "frac": None, "traffic": None,
                    "kernel": "ttm_simt", "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz} MHz"}
    else:
        # tensor peak for the algorithmic flops of this mode: x3 modes issue three
        # products per term; tf32 runs at half the bf16 rate (nominal ratio)
        nprod = 3 if args.prec in ("bf16x3", "tf32x3", "f16x3") else 1
        rate = 1.0 if args.prec in ("bf16x3", "bf16", "f16x3") else 0.5
        tpeak = peaks["bf16_tflops"] * rate / nprod
        t_hbm = ttm_bytes / (peaks["hbm_gbs"] * 1e9)
        t_tc = ttm_flops / (tpeak * 1e12)
        if t_tc > t_hbm:
            roofline = {"bound": "tensor", "achieved": ttm_flops / (ttm_ms / 1e3) / 1e12, "peak": tpeak,
                        "unit": "TFLOP/s", "frac": None, "traffic": None, "kernel": "ttm_tc",
                        "peak_source": f"bf16_tflops of {peak_kind} x {rate} / {nprod} products per term"}
        else:
            ach = ttm_bytes / (ttm_ms / 1e3) / 1e9
            roofline = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": None, "traffic": None, "kernel": "ttm_tc",
                        "peak_source": f"hbm_gbs of {peak_kind}"}
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    if args.workload == "c2" and args.prec in TRAFFIC_C2 and not (args.dims or args.rank or args.law):
        # DRAM bytes per launch of this kernel on this workload, from one ncu capture
        # (dram__bytes_read.sum + dram__bytes_write.sum)
        roofline["traffic"] = TRAFFIC_C2[args.prec]
        roofline["traffic_source"] = "ncu dram__bytes_read+write of k_ttm_tc on 128^4 R=64, one launch"

    roofline["mode"] = mode
    roofline["ms_per_launch"] = ttm_ms
    roofline["algorithmic_bytes"] = ttm_bytes
    roofline["algorithmic_flops"] = ttm_flops

    # ---------------------------------------------------------------- PP (approximated sweeps)
    # operators built explicitly after the warm-up, then a bounded run of Alg. 2
    # with a loose tolerance (0.5) so that most sweeps are approximated
    ctx_pp = pkg.CPContext(T, R, A0=A0, prec=args.prec, stream=stream)
    ctx_pp.sweep_msdt(max(2, args.warmup))
    npp_run = min(args.steps, 20)
    pp_info = {"eps": 0.5, "sweeps": npp_run}
    try:
        ctx_pp.pp_init()
        tr0 = len(ctx_pp.trace())
        t0 = time.perf_counter()
        ctx_pp.sweep_pp(npp_run, eps=0.5)
        torch.cuda.synchronize()
        wall_pp = time.perf_counter() - t0
        tr = ctx_pp.trace()[tr0:]
        pp_ms = [t["ms"] for t in tr if t["kind"] == "pp" and not t["pp_init"]]
        pp_info.update({"approx_sweeps": len(pp_ms),
                        "approx_sweep_ms": (sum(pp_ms) / len(pp_ms)) if pp_ms else None,
                        "sweeps_per_s_wall": len(tr) / wall_pp,
                        "init_count": ctx_pp.stats()["pp_init"]})
    except pkg.CPError as e:
        pp_info["error"] = str(e)
    ctx_pp.close()

    # ---------------------------------------------------------------- PP vs exact MSDT (Alg. 2, eps 0.1)
    # target: exact MSDT's direct residual after npp sweeps, plus the fit tolerance
    # 1e-6; each method runs from the same start until its direct residual reaches
    # it (at most 3 npp sweeps); time = device time of its sweeps (operator builds
    # included, the per-sweep residual check not)
    npp = args.pp_sweeps if args.pp_sweeps >= 0 else (100 if args.workload in ("c4",) + STANDINS else 0)
    pp_vs = None
    if npp > 0:
        from paper_2010_12056_gb300 import policy as pol
        c2 = pkg.CPContext(T, R, A0=A0, prec=args.prec, stream=stream)
        c2.sweep_msdt(npp)
        target = c2.fit(exact=True)[1] + 1e-6
        c2.close()
        pp_vs = {"target": "exact MSDT's direct residual after %d sweeps + 1e-6" % npp, "eps": 0.1,
                 "target_resid": target}
        for name in ("msdt", "pp"):
            ms, k, r, tr = pol.time_to_target(T, R, name, target, 3 * npp, prec=args.prec, A0=A0, eps=0.1)
            apx = [t["ms"] for t in tr if t.get("kind") == "pp" and not t.get("pp_init")]
            ini = [t["ms"] for t in tr if t.get("pp_init")]
            reg = [t["ms"] for t in tr if t.get("kind") in ("msdt", "pp-regular")]
            pp_vs[name] = {"ms_to_target": ms if ms != float("inf") else None, "reached": ms != float("inf"),
                           "sweeps": k, "resid": r, "approx_sweeps": len(apx), "inits": len(ini),
                           "regular_sweeps": len(reg),
                           "approx_sweep_ms": (sum(apx) / len(apx)) if apx else None,
                           "sweep_with_init_ms": (sum(ini) / len(ini)) if ini else None,
                           "regular_sweep_ms": (sum(reg) / len(reg)) if reg else None}
        if pp_vs["msdt"]["reached"] and pp_vs["pp"]["reached"]:
            pp_vs["speedup_pp_over_msdt"] = pp_vs["msdt"]["ms_to_target"] / pp_vs["pp"]["ms_to_target"]

    # ---------------------------------------------------------------- e2e (host buffers, C ABI)
    # every step hands the library this step's tensor in pinned host memory
    # (cp_load_tensor: host -> device copy, cached nodes dropped), runs one MSDT
    # sweep and reads the step's fit back (cp_fit: device -> host)
    e2e = None
    if not args.no_e2e:
        Th = torch.empty(dims, dtype=torch.float32, pin_memory=True)
        Th.copy_(T.cpu())
        ctx_e = pkg.CPContext(Th, R, A0=A0, prec=args.prec, stream=stream)
        ctx_e.sweep_msdt(1)
        barrier()
        t0 = time.perf_counter()
        fits = []
        for _ in range(args.steps):
            ctx_e.load_tensor(Th)
            ctx_e.sweep_msdt(1)
            fits.append(ctx_e.fit(exact=False)[0])
        barrier()
        el = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": world * args.steps / el, "unit": "sweep/s",
               "h2d_bytes_per_step": 4 * numel, "d2h_bytes_per_step": 16,
               "path": "cp_load_tensor(host) + cp_sweep_msdt(1) + cp_fit per step"}
        ctx_e.close()
        del Th

    # ---------------------------------------------------------------- fit check and CPU baseline (oracle)
    # the GPU's direct residual after FIT_SWEEPS MSDT sweeps from A0 against the FP64
    # oracle's after the same sweeps on the same FP32 bytes; the oracle run is also
    # the timed CPU baseline
    cpu = None
    fit_vs = None
    if rank == 0 and not args.no_cpu_baseline and args.gpus == 1:
        cf = pkg.CPContext(T, R, A0=A0, prec=args.prec, stream=stream)
        cf.sweep_msdt(FIT_SWEEPS)
        r_gpu = cf.fit(exact=True)[1]
        cf.close()
        from oracle import cp_oracle as co
        T64 = T.cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        ref = co.cp_als(T64, A0, FIT_SWEEPS, route="msdt")
        el = time.perf_counter() - t0
        r_orc = co.residual_direct(T64, ref.A)
        del T64
        fit_vs = {"sweeps": FIT_SWEEPS, "route": "msdt", "resid_gpu": r_gpu, "resid_oracle": r_orc,
                  "abs_diff": abs(r_gpu - r_orc), "tol": FIT_TOL, "pass": abs(r_gpu - r_orc) <= FIT_TOL}
        cpu = {"value": FIT_SWEEPS / el, "unit": "sweep/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{FIT_SWEEPS} FP64 oracle MSDT sweeps of the full tensor from A0 ({el:.1f} s)"}

    line = {
        "metric": METRIC if args.workload == "c2" and not (args.dims or args.rank or args.law)
        else "ALS sweep/s (MSDT) on 1 GPU, " + wl["desc"], "value": value, "unit": "sweep/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "precision": {"ttm": args.prec, "mttv": "f32", "gram_cholesky_solve_residual": "f64"},
        "data": "synthetic",
        "config": {"workload": wl["desc"], "dims": list(dims), "R": R, "sweep": "msdt",
                   "l2": "inputs larger than L2 (tensor 1.07 GB, root 537 MB)"
                   if args.workload == "c2" else "see dims"},
        "mttkrp_tflops": mttkrp_tflops,
        "dt_sweeps_per_s": dt_sps * world,
        "msdt_time_over_dt": dt_sps / msdt_sps,
        "msdt_time_over_dt_unfused": schedules["dt_unfused"] / msdt_sps,
        "schedules_sweeps_per_s": schedules,
        "fit": {"formula": fit_formula, "direct": fit_direct, "after_sweeps": args.warmup + args.steps},
        "fit_vs_oracle": fit_vs,
        "solves_fp64": int(st1["solves_fp64"]),
        "pp": pp_info,
        "pp_vs_msdt": pp_vs,
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
