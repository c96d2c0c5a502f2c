"""Learned PP-regime policy: trace collection, training and evaluation.

The paper steers pairwise perturbation with one hand-set tolerance (Alg. 2:
approximate while every ||dA(i)||_F < eps ||A(i)||_F, otherwise one regular
sweep and a rebuild of the operators).  This module replaces that rule by the
library's 8 -> 64 -> 64 -> 1 network, with no counterpart in the paper:

* ``collect`` labels the PP choices of every sweep state with cp_pp_probe
  (each choice is run from the same state and judged by the direct residual),
* ``train`` fits the network with the library's own forward/backward/Adam
  kernels (cp_policy_train),
* ``time_to_target`` measures the device time a method needs to reach a given
  direct residual, summing the trace's per-sweep event times (which include
  operator builds, network queries and the judge).

Everything numerical runs in libcpals.so; this module only sequences calls and
holds the collected features on the device.
"""
from __future__ import annotations

import numpy as np

from . import CPContext, N_POLICY_PARAMS, Policy

FEATURES = ["sweep/100", "L(max step)", "L(max |A-Ap|)", "L(|dr|/r)", "L(r)",
            "since build/10", "last approximated", "L(V share)"]
# hidden sizes of the network (fixed by the library's kernels)
_SHAPES = [(64, 8), (64,), (64, 64), (64,), (64,), (1,)]
_FAN_IN = [8, None, 64, None, 64, None]


def init_theta(seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, in the library's parameter order."""
    rng = np.random.default_rng(seed)
    parts = []
    for shp, fan in zip(_SHAPES, _FAN_IN):
        n = int(np.prod(shp))
        parts.append(rng.uniform(-1.0, 1.0, n) / np.sqrt(fan) if fan else np.zeros(n))
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == N_POLICY_PARAMS
    return theta


def collect(T, R, sweeps, prec="f16x3", seed=1, follow=-1, min_gain=0.0):
    """Probe `sweeps` consecutive states of one decomposition of T.

    Returns (X, y, recs): one sample per labelled choice (current operators when
    they exist, rebuilt operators always) and the raw probe records.  Stops early
    once a regular sweep lowers the residual by less than min_gain * r0.
    """
    ctx = CPContext(T, R, prec=prec, seed=seed)
    X, y, recs = [], [], []
    try:
        for _ in range(sweeps):
            rec = ctx.probe(follow)
            recs.append(rec)
            if rec["has_ops"]:
                X.append(rec["feat_cur"])
                y.append(rec["label_cur"])
            X.append(rec["feat_new"])
            y.append(rec["label_new"])
            if rec["r0"] - rec["r_exact"] < min_gain * rec["r0"]:
                break
    finally:
        ctx.close()
    return np.array(X, np.float32).reshape(-1, 8), np.array(y, np.float32), recs


def train(X, y, steps=2000, lr=3e-3, seed=0, theta=None, chunk=200):
    """Full-batch Adam on (X, y) with the library's kernels; returns the trained Policy.

    Samples of the rarer label are repeated so that both labels carry equal
    weight in the loss.
    """
    import torch
    X = np.asarray(X, np.float32)
    y = np.asarray(y, np.float32)
    pos, neg = np.flatnonzero(y > 0.5), np.flatnonzero(y <= 0.5)
    if len(pos) and len(neg):
        rng = np.random.default_rng(seed)
        small, big = (pos, neg) if len(pos) < len(neg) else (neg, pos)
        extra = rng.choice(small, len(big) - len(small), replace=True)
        idx = np.concatenate([big, small, extra])
        X, y = X[idx], y[idx]
    pol = Policy(init_theta(seed) if theta is None else theta)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        pol.train(Xd, yd, k, lr)
        done += k
    torch.cuda.synchronize()
    return pol


def accuracy(pol, X, y):
    import torch
    if len(y) == 0:
        return float("nan")
    p = pol.forward(torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()).cpu().numpy()
    return float(np.mean((p >= 0.5) == (np.asarray(y) > 0.5)))


def time_to_target(T, R, method, target_resid, max_sweeps, prec="f16x3", seed=1, eps=0.1,
                   policy=None, judge_every=5, A0=None):
    """Device milliseconds until the direct residual first drops to target_resid.

    method: "msdt" (regular sweeps), "pp" (Alg. 2 with tolerance eps) or
    "policy" (cp_sweep_pp with the network).  The residual check after each
    sweep is outside the timed work.  Returns (ms or inf, sweeps, final resid,
    trace).  A0: initial factors (default: U[0,1) from `seed`).
    """
    from . import CPError
    ctx = CPContext(T, R, A0=A0, prec=prec, seed=seed, judge_every=judge_every)
    try:
        r = 1.0
        for k in range(max_sweeps):
            try:
                if method == "msdt":
                    ctx.sweep_msdt(1)
                elif method == "pp":
                    ctx.sweep_pp(1, eps)
                elif method == "policy":
                    ctx.sweep_pp(1, eps, policy)
                else:
                    raise ValueError(method)
                _, r = ctx.fit(exact=True)
            except CPError as e:
                # the iteration broke down (e.g. diverging factors): target not reached
                return float("inf"), k + 1, float("nan"), ctx.trace() + [{"error": str(e)}]
            if r <= target_resid:
                tr = ctx.trace()
                return sum(t["ms"] for t in tr), k + 1, r, tr
        return float("inf"), max_sweeps, r, ctx.trace()
    finally:
        ctx.close()
