"""The learned PP policy on the GPU: network kernels vs the FP64 oracle, branch
probing vs plain runs, and the policy-driven regime control with its judge.

Tolerances: the network runs in FP32 (tanh/exp of FP32 arguments), so scores are
compared to 1e-5 absolute and gradients to 1e-4 relative (Frobenius) against the
FP64 oracle; Adam steps to 1e-5 absolute.  Probing restores factors exactly, so
probe-driven trajectories match plain runs to 1e-12.
"""
import numpy as np
import pytest

import synth
from oracle import mlp_oracle as mo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge
    ge.build()
    import paper_2010_12056_gb300 as p
    return p


def net_inputs(seed, B):
    X = (2.0 * synth.uniform(seed, 0, B * 8) - 1.0).reshape(B, 8) * 1.5
    y = (synth.uniform(seed, 1, B) < 0.4).astype(np.float64)
    theta = mo.init_params(synth.uniform(seed, 2, mo.N_PARAMS))
    theta[mo.N_PARAMS - 129:mo.N_PARAMS - 65] += 0.05   # non-zero b2
    return X.astype(np.float32), y.astype(np.float32), theta.astype(np.float32)


@pytest.mark.parametrize("B", [1, 2, 37, 1000])
def test_forward_matches_oracle(pkg, B):
    X, _, theta = net_inputs(3 + B, B)
    pol = pkg.Policy(theta)
    p = pol.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    ref = mo.predict(theta.astype(np.float64), X.astype(np.float64))
    assert np.abs(p - ref).max() <= 1e-5
    pol.close()


@pytest.mark.parametrize("B", [1, 7, 300, 2000])
def test_grad_matches_oracle(pkg, B):
    X, y, theta = net_inputs(11 + B, B)
    pol = pkg.Policy(theta)
    loss, g = pol.grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    lref, gref = mo.grad(theta.astype(np.float64), X.astype(np.float64), y.astype(np.float64))
    assert abs(float(loss.item()) - lref) <= 1e-5 * max(1.0, abs(lref))
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)
    pol.close()


def test_adam_steps_match_oracle(pkg):
    X, y, theta = net_inputs(5, 64)
    pol = pkg.Policy(theta)
    pol.train(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), 3, lr=1e-2)
    got = pol.get().astype(np.float64)
    th = theta.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for t in range(1, 4):
        _, g = mo.grad(th, X.astype(np.float64), y.astype(np.float64))
        th, m, v = mo.adam_step(th, g, m, v, t, lr=1e-2)
    assert np.abs(got - th).max() <= 1e-5
    pol.close()


def test_training_fits_a_separable_rule(pkg):
    X, _, theta = net_inputs(9, 512)
    y = (X[:, 0] + 0.5 * X[:, 3] > 0.1).astype(np.float32)
    pol = pkg.Policy(theta)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    l0, _ = pol.grad(Xd, yd)
    pol.train(Xd, yd, 400, lr=1e-2)
    l1, _ = pol.grad(Xd, yd)
    acc = float(((pol.forward(Xd).cpu().numpy() >= 0.5) == (y > 0.5)).mean())
    assert l1.item() < 0.3 * l0.item()
    assert acc >= 0.97
    pol.close()


# ------------------------------------------------------------ regime control
def pp_problem(seed=7, dims=(40, 36, 44), R=6, C=0.8, eta=1e-3):
    T, _, _ = synth.make_problem(seed, list(dims), R, law="collinear", eta=eta, C=C)
    return torch.from_numpy(np.ascontiguousarray(T.astype(np.float32))).cuda(), R


def factors_close(a, b, tol=1e-12):
    return all(np.linalg.norm(x - y) <= tol * np.linalg.norm(y) for x, y in zip(a, b))


def test_probe_follow_regular_equals_msdt(pkg):
    T, R = pp_problem()
    a = pkg.CPContext(T, R, prec="fp32", seed=3)
    b = pkg.CPContext(T, R, prec="fp32", seed=3)
    for _ in range(4):
        rec = a.probe(0)
        assert rec["followed"] == 0
    b.sweep_msdt(4)
    assert factors_close(a.factors(), b.factors())
    ra = [t["resid"] for t in a.trace()]
    rb = [t["resid"] for t in b.trace()]
    assert len(ra) == 4 and np.allclose(ra, rb, rtol=0, atol=1e-13)
    # the probe's regular branch is the residual the plain run reaches
    assert abs(rec["r_exact"] - b.fit(exact=True)[1]) <= 1e-12
    a.close()
    b.close()


def test_probe_branches_equal_plain_runs(pkg):
    T, R = pp_problem(seed=8)
    a = pkg.CPContext(T, R, prec="fp32", seed=4)
    b = pkg.CPContext(T, R, prec="fp32", seed=4)
    recs = [a.probe(0), a.probe(2), a.probe(1)]
    assert [r["followed"] for r in recs] == [0, 2, 1]
    assert recs[0]["has_ops"] == 0 and np.isnan(recs[0]["r_cur"])
    assert recs[2]["has_ops"] == 1
    b.sweep_msdt(1)
    b.pp_init()
    b.sweep_pp(1, 0.5)          # operators fresh: dA = 0 passes any tolerance
    rb1 = b.fit(exact=True)[1]
    assert abs(recs[1]["r_new"] - rb1) <= 1e-12
    b.sweep_pp(1, 0.999)
    assert [t["kind"] for t in b.trace()] == ["msdt", "pp", "pp"]
    assert abs(recs[2]["r_cur"] - b.fit(exact=True)[1]) <= 1e-12
    assert factors_close(a.factors(), b.factors())
    for r in recs:
        slack = 0.1 * max(0.0, r["r0"] - r["r_exact"]) + 1e-9 * r["r0"]
        assert r["label_new"] == int(r["r_new"] - r["r_exact"] <= slack)
        if r["has_ops"]:
            assert r["label_cur"] == int(r["r_cur"] - r["r_exact"] <= slack)
    a.close()
    b.close()


def test_policy_features_layout(pkg):
    T, R = pp_problem(seed=9)
    a = pkg.CPContext(T, R, prec="fp32", seed=5)
    fc, fn = a.policy_features()
    assert fc[0] == 0 and fc[2] == -1 and fc[5] == 3 and fc[6] == 0 and fc[7] == -1
    assert fn[2] == -1 and fn[5] == 0
    a.sweep_msdt(2)
    a.pp_init()
    a.sweep_pp(1, 0.5)
    fc, fn = a.policy_features()
    tr = a.trace()
    step = max(tr[-1]["max_rel_step"], 1e-12)
    assert abs(fc[0] - 0.03) < 1e-6
    assert abs(fc[1] - (np.log10(min(step, 1.0)) / 6 + 1)) < 1e-5
    assert -1 < fc[2] < 1 and fc[6] == 1 and abs(fc[5] - 0.1) < 1e-6
    assert abs(fc[4] - (np.log10(tr[-1]["resid"]) / 6 + 1)) < 1e-5
    assert fn[2] == -1 and fn[5] == 0 and fn[7] == -1
    a.close()


def const_policy(pkg, logit):
    th = np.zeros(mo.N_PARAMS, np.float32)
    th[-1] = logit
    return pkg.Policy(th)


def test_policy_always_regular_equals_msdt(pkg):
    T, R = pp_problem(seed=10)
    a = pkg.CPContext(T, R, prec="fp32", seed=6, judge_every=5)
    b = pkg.CPContext(T, R, prec="fp32", seed=6)
    pol = const_policy(pkg, -20.0)
    a.sweep_pp(10, 0.1, pol)
    b.sweep_msdt(10)
    assert factors_close(a.factors(), b.factors())
    tr = a.trace()
    assert [t["kind"] for t in tr] == ["pp-regular"] * 10
    assert all(t["decided_by"] == 1 and t["p_cur"] < 1e-6 and t["rolled_back"] == 0 for t in tr)
    assert a.stats()["rollbacks"] == 0
    pol.close()
    a.close()
    b.close()


def test_policy_judge_never_lets_the_residual_rise(pkg):
    """A policy that always approximates, judged every sweep: the judged
    (direct) residual never rises by more than the judge's noise allowance
    (1e-5 relative) whatever the network says."""
    T, R = pp_problem(seed=11, C=0.9)
    a = pkg.CPContext(T, R, prec="fp32", seed=7, judge_every=1, policy_gate=False)
    pol = const_policy(pkg, 20.0)
    rs = [a.fit(exact=True)[1]]
    for _ in range(25):
        a.sweep_pp(1, 0.1, pol)
        rs.append(a.fit(exact=True)[1])
    rs = np.array(rs)
    assert np.all(rs[1:] <= rs[:-1] * (1 + 1e-5))
    tr = a.trace()
    st = a.stats()
    assert st["sweeps_pp"] > 0
    nrb = sum(t["rolled_back"] for t in tr)
    assert (nrb > 0) == (st["rollbacks"] > 0)
    # after a rollback the next sweep is a regular one
    for i, t in enumerate(tr[:-1]):
        if t["rolled_back"] and not tr[i + 1]["rolled_back"]:
            assert tr[i + 1]["decided_by"] == 2 and tr[i + 1]["kind"] == "pp-regular"
    pol.close()
    a.close()


def test_policy_gate_keeps_small_problems_regular(pkg):
    """On a tensor this small an approximated sweep saves almost no MTTKRP
    traffic, so the gated policy never consults the network and runs the
    regular sweeps of MSDT, whatever the network would say."""
    T, R = pp_problem(seed=12)
    a = pkg.CPContext(T, R, prec="fp32", seed=8, judge_every=5)
    b = pkg.CPContext(T, R, prec="fp32", seed=8)
    pol = const_policy(pkg, 20.0)
    a.sweep_pp(8, 0.1, pol)
    b.sweep_msdt(8)
    assert a.stats()["sweeps_pp"] == 0
    assert all(t["kind"] == "pp-regular" and t["p_cur"] == -1 for t in a.trace())
    assert factors_close(a.factors(), b.factors())
    pol.close()
    a.close()
    b.close()
