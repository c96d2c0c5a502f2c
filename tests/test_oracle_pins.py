"""Pins of the FP64 oracle against facts the paper and mathematics fix (no GPU).

Each test checks the oracle against something other than itself: brute force,
closed forms, invariants the paper states, special cases that reduce to a
textbook routine, and the structures printed in Fig. 1a, Fig. 2 and Table 1.
"""
import math

import numpy as np
import pytest

import synth
from oracle import cp_oracle as co
from oracle import mlp_oracle as mo
from tests.conftest import golden

# ----------------------------------------------------------------------------- generator


def test_philox_known_answers():
    for line in open(golden("philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out = synth.philox4x32_10(*w[:6])
        assert [int(x) for x in out] == w[6:]


def test_uniform_range_and_moments():
    u = synth.uniform(7, 3, 200001)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3
    # element i does not depend on how many are drawn
    assert np.array_equal(synth.uniform(7, 3, 11), u[:11])


def test_collinear_factors_exact_gram():
    C = 0.9
    F = synth.collinear_factors(11, [20, 17, 16], 16, C)
    K = (1 - C) * np.eye(16) + C * np.ones((16, 16))
    for A in F:
        assert np.abs(A.T @ A - K).max() < 1e-12


def test_noise_ratio_exact():
    F = synth.uniform_factors(5, [6, 7, 8], 3)
    T = synth.cp_full(F)
    Tn = synth.add_noise(T, 1e-2, 5, 64)
    ratio = np.linalg.norm((Tn - T).ravel()) / np.linalg.norm(T.ravel())
    assert abs(ratio - 1e-2) < 1e-12


@pytest.mark.parametrize("dims,R", [((9, 5, 4, 3), 4), ((7, 6, 5), 3)])
def test_device_generator_slices_equal_one_product(dims, R):
    """The large-tensor generator builds [[A]] in mode-0 slices when its Khatri-Rao rows
    would be large; slices of 1, 2 and 3 mode-0 indices give the tensor of one product,
    and that tensor is the definition sum_r prod_n A(n)[i_n, r] (no noise)."""
    torch = pytest.importorskip("torch")
    whole, F, _ = synth.make_problem_device(31, dims, R, device="cpu")
    ref = synth.cp_full(F).astype(np.float32)
    assert np.array_equal(whole.numpy(), ref) or np.abs(whole.numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
    inner = int(np.prod(dims[1:-1]))
    for rows in (1, 2, 3):
        sliced, _, _ = synth.make_problem_device(31, dims, R, device="cpu", slab_elems=rows * inner * R)
        assert np.array_equal(sliced.numpy(), whole.numpy())


# ----------------------------------------------------------------------------- MTTKRP


@pytest.mark.parametrize("dims", [(3, 4, 5), (2, 3, 4, 3), (2, 2, 3, 2, 3)])
def test_mttkrp_definition_matches_bruteforce(dims):
    R = 3
    T = synth.normal(1, 0, int(np.prod(dims))).reshape(dims)
    A = synth.gaussian_factors(2, dims, R)
    for n in range(len(dims)):
        Mb = co.mttkrp_bruteforce(T, A, n)
        M = co.mttkrp(T, A, n)
        assert np.abs(M - Mb).max() <= 1e-12 * max(1.0, np.abs(Mb).max())


def test_mttkrp_order2_is_matrix_product():
    """N = 2: M^(1) = T A(2) and M^(2) = T^T A(1), a plain matrix product."""
    T = synth.normal(3, 0, 7 * 5).reshape(7, 5)
    A = synth.gaussian_factors(4, (7, 5), 4)
    assert np.allclose(co.mttkrp(T, A, 0), T @ A[1], rtol=0, atol=1e-13)
    assert np.allclose(co.mttkrp(T, A, 1), T.T @ A[0], rtol=0, atol=1e-13)


@pytest.mark.parametrize("dims", [(4, 5, 6), (3, 4, 3, 5), (3, 2, 3, 2, 3)])
@pytest.mark.parametrize("route", ["dt", "msdt"])
def test_tree_mttkrps_equal_definition(dims, route):
    """Each tree-built M^(n) equals the definition with the factors current at that moment."""
    N = len(dims)
    A = synth.uniform_factors(5, dims, 4)
    T = synth.normal(6, 0, int(np.prod(dims))).reshape(dims)
    gen = co.dt_updates(T, A) if route == "dt" else co.msdt_updates(T, A, 3 * N)
    count = 0
    for n, M in gen:
        ref = co.mttkrp(T, A, n)
        assert np.abs(M - ref).max() <= 1e-12 * np.abs(ref).max()
        # perturb A[n] like an update would, so later nodes must see the new factor
        A[n] = A[n] * 0.5 + 0.1 * synth.uniform(7, count, A[n].size).reshape(A[n].shape)
        count += 1
    assert count == (N if route == "dt" else 3 * N)


def _edges_1based(edges):
    out = []
    for parent, child in edges:
        p = "T" if parent == "T" else ",".join(str(m + 1) for m in parent)
        out.append((p, ",".join(str(m + 1) for m in child)))
    return out


def _read_edges(name):
    out = []
    for line in open(golden(name)):
        if line.startswith("#") or not line.strip():
            continue
        p, c = [x.strip() for x in line.split("->")]
        out.append((p, c))
    return out


def test_dt_tree_is_fig1a():
    dims = (3, 3, 3, 3)
    A = synth.uniform_factors(1, dims, 2)
    T = synth.normal(1, 0, 81).reshape(dims)
    ctr = co.Counters()
    for n, M in co.dt_updates(T, A, ctr):
        pass
    assert sorted(_edges_1based(ctr.edges)) == sorted(_read_edges("dt_tree_n4_fig1a.txt"))
    assert ctr.ttm_modes == [3, 0]


def test_msdt_tree_is_fig2():
    dims = (3, 3, 3, 3)
    A = synth.uniform_factors(1, dims, 2)
    T = synth.normal(1, 0, 81).reshape(dims)
    ctr = co.Counters()
    for n, M in co.msdt_updates(T, A, 12, ctr):
        pass
    assert sorted(_edges_1based(ctr.edges)) == sorted(_read_edges("msdt_tree_n4_fig2.txt"))
    assert ctr.ttm_modes == [3, 2, 1, 0]


def test_first_level_ttm_counts_table1():
    for line in open(golden("cost_table1.txt")):
        if line.startswith("#") or not line.strip():
            continue
        N, sweeps, dt_ttms, msdt_ttms = map(int, line.split())
        dims = (2,) * N
        T = synth.normal(2, 0, 2 ** N).reshape(dims)
        r_dt = co.cp_als(T, synth.uniform_factors(3, dims, 2), sweeps, route="dt")
        r_ms = co.cp_als(T, synth.uniform_factors(3, dims, 2), sweeps, route="msdt")
        assert r_dt.counters.ttm == dt_ttms
        assert r_ms.counters.ttm == msdt_ttms
        s = 2
        assert r_ms.counters.ttm_flops == pytest.approx(2 * N / (N - 1) * s ** N * 2 * sweeps)
        assert r_dt.counters.ttm_flops == pytest.approx(4 * s ** N * 2 * sweeps)


@pytest.mark.parametrize("dims,levels", [((4, 5, 3, 6), 2), ((3, 4, 3, 4, 3), 2), ((3, 4, 3, 4, 3), 3),
                                         ((3, 3, 2, 3, 3, 2), 4)])
def test_combined_level_msdt_mttkrps_equal_definition(dims, levels):
    """Multi-sweep tree with the upper `levels` levels combined (Sec. IV): every
    MTTKRP equals the definition with the factors current at that moment."""
    N = len(dims)
    A = synth.uniform_factors(5, dims, 4)
    T = synth.normal(6, 0, int(np.prod(dims))).reshape(dims)
    n_upd = 2 * N * (N - levels)
    count = 0
    for n, M in co.msdt_updates(T, A, n_upd, levels=levels):
        assert n == count % N                       # updates stay in mode order
        ref = co.mttkrp(T, A, n)
        assert np.abs(M - ref).max() <= 1e-12 * np.abs(ref).max()
        A[n] = A[n] * 0.5 + 0.1 * synth.uniform(8, count, A[n].size).reshape(A[n].shape)
        count += 1
    assert count == n_upd


@pytest.mark.parametrize("N,levels", [(4, 2), (5, 2), (5, 3), (6, 2), (6, 4)])
def test_combined_level_msdt_costs(N, levels):
    """Sec. IV: with the upper l levels combined, one pass over T per N - l updates
    (2N/(N-l) s^N R flops per sweep, counted once per pass) and auxiliary memory of
    s^(N-l) R: the largest intermediate the tree forms."""
    s, R = 3, 2
    dims = (s,) * N
    T = synth.normal(9, 0, s ** N).reshape(dims)
    A = synth.uniform_factors(10, dims, R)
    ctr = co.Counters()
    sweeps = N - levels                          # a whole number of subtrees
    biggest = 0
    for n, M in co.msdt_updates(T, A, sweeps * N, ctr, levels=levels):
        pass
    assert ctr.ttm == N
    assert ctr.ttm_flops == pytest.approx(2 * N / (N - levels) * s ** N * R * sweeps)
    # every first-level node keeps N - l modes
    kept = [child for parent, child in ctr.edges if parent == "T"]
    assert all(len(k) == N - levels for k in kept)
    # each root contracts the l modes updated just before its subtree, all distinct
    for j, modes in enumerate(ctr.ttm_modes):
        t0 = j * (N - levels)
        want = sorted((t0 - 1 - i) % N for i in range(levels))
        assert sorted(modes if isinstance(modes, tuple) else (modes,)) == want
    with pytest.raises(ValueError):
        next(co.msdt_updates(T, A, 1, levels=N - 1))


@pytest.mark.parametrize("dims,levels", [((5, 4, 6, 3), 2), ((3, 4, 3, 5, 3), 3)])
def test_combined_level_msdt_trajectory_is_als(dims, levels):
    T, F, A0 = synth.make_problem(41, dims, 3, eta=0.1)
    a = co.cp_als(T, A0, 8, route="naive")
    c = co.cp_als(T, A0, 8, route="msdt", levels=levels)
    for n in range(len(dims)):
        assert np.abs(a.A[n] - c.A[n]).max() < 1e-10 * np.abs(a.A[n]).max()
    assert np.allclose(a.resid, c.resid, rtol=0, atol=1e-12)


# ----------------------------------------------------------------------------- solve / residual


def test_cholesky_solve_equals_pinv_and_lstsq():
    A = synth.gaussian_factors(8, (30, 30), 6)
    G = (A[0].T @ A[0]) * (A[1].T @ A[1])
    M = synth.normal(9, 0, 12 * 6).reshape(12, 6)
    X = co.solve_normal(M, G)
    assert np.abs(X @ G - M).max() < 1e-10 * np.abs(M).max()
    assert np.abs(X - M @ np.linalg.pinv(G)).max() < 1e-12 * np.abs(X).max()
    # rank-deficient Gamma: the pseudo-inverse branch = minimum-norm least squares
    B = synth.normal(10, 0, 6 * 3).reshape(6, 3)
    Gd = B @ B.T                                   # rank 3, PSD, Cholesky fails
    Xd = co.solve_normal(M, Gd)
    ref = np.linalg.lstsq(Gd, M.T, rcond=None)[0].T
    assert np.abs(Xd - ref).max() < 1e-8 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("dims", [(5, 6, 7), (4, 3, 5, 4)])
def test_residual_formula_equals_direct(dims):
    R = 3
    A = synth.uniform_factors(12, dims, R)
    T = synth.normal(13, 0, int(np.prod(dims))).reshape(dims) + synth.cp_full(A)
    N = len(dims)
    S = [co.gram(a) for a in A]
    G = co.hadamard_except(S, N - 1)
    M = co.mttkrp(T, A, N - 1)
    r1 = co.residual_formula(float(np.sum(T * T)), G, A[N - 1], M)
    assert abs(r1 - co.residual_direct(T, A)) < 1e-10


def test_cp_full_matches_generator_rank_one_sum():
    A = synth.gaussian_factors(14, (3, 4, 2), 2)
    T = co.cp_full(A)
    i, j, k = 2, 1, 1
    assert T[i, j, k] == pytest.approx(sum(A[0][i, r] * A[1][j, r] * A[2][k, r] for r in range(2)))
    assert np.abs(T - synth.cp_full(A)).max() < 1e-13


# ----------------------------------------------------------------------------- CP-ALS


def test_als_direct_residual_monotone():
    """ALS decreases the residual monotonically (Sec. I)."""
    dims, R = (8, 9, 10), 4
    T, F, A0 = synth.make_problem(20, dims, R, eta=0.05)
    A = [a.copy() for a in A0]
    prev = co.residual_direct(T, A)
    for _ in range(15):
        A = co.cp_als(T, A, 1).A
        r = co.residual_direct(T, A)
        assert r <= prev + 1e-13
        prev = r


def test_als_exact_recovery_noiseless():
    """Noiseless rank-R tensors with well-conditioned factors are recovered (fit -> 1)."""
    ok = 0
    for seed in range(10):
        dims, R = (10, 11, 12), 3
        T, F, A0 = synth.make_problem(100 + seed, dims, R, law="gaussian")
        res = co.cp_als(T, A0, 500, delta=1e-13)
        if co.residual_direct(T, res.A) < 1e-8:
            ok += 1
    assert ok >= 8


def test_als_order2_reaches_eckart_young():
    """N = 2: the ALS fixed point is the best rank-R approximation (Eckart-Young)."""
    s1, s2, R = 12, 9, 3
    U, _ = np.linalg.qr(synth.normal(30, 0, s1 * s1).reshape(s1, s1))
    V, _ = np.linalg.qr(synth.normal(30, 1, s2 * s2).reshape(s2, s2))
    sig = np.array([10.0, 8.0, 6.0, 2.0, 1.5, 1.0, 0.5, 0.3, 0.1])
    T = (U[:, :s2] * sig) @ V.T
    res = co.cp_als(T, synth.uniform_factors(31, (s1, s2), R), 300)
    opt = math.sqrt(np.sum(sig[R:] ** 2)) / math.sqrt(np.sum(sig ** 2))
    assert abs(co.residual_direct(T, res.A) - opt) < 1e-10
    assert abs(res.resid[-1] - opt) < 1e-8


@pytest.mark.parametrize("dims", [(6, 7, 8), (4, 5, 4, 5)])
def test_dt_msdt_naive_trajectories_identical(dims):
    """MSDT gives exactly the results of the standard dimension tree (Sec. I, III)."""
    T, F, A0 = synth.make_problem(40, dims, 3, eta=0.1)
    a = co.cp_als(T, A0, 10, route="naive")
    b = co.cp_als(T, A0, 10, route="dt")
    c = co.cp_als(T, A0, 10, route="msdt")
    for n in range(len(dims)):
        sc = np.abs(a.A[n]).max()
        assert np.abs(a.A[n] - b.A[n]).max() < 1e-10 * sc
        assert np.abs(a.A[n] - c.A[n]).max() < 1e-10 * sc
    assert np.allclose(a.resid, c.resid, rtol=0, atol=1e-12)


# ----------------------------------------------------------------------------- PP


def _pp_setup(dims, R, seed, t, T=None, only=None):
    Ap = synth.uniform_factors(seed, dims, R)
    D = synth.gaussian_factors(seed + 1, dims, R)
    A = [Ap[i] + (t * D[i] if (only is None or i == only) else 0.0) for i in range(len(dims))]
    if T is None:
        T = synth.normal(seed + 2, 0, int(np.prod(dims))).reshape(dims)
    return T, Ap, A


def _pp_err(T, Ap, A, n):
    pairs, Mp = co.pp_operators(T, Ap)
    dA = [A[i] - Ap[i] for i in range(len(A))]
    S = [co.gram(a) for a in A]
    Mt = co.pp_mttkrp(pairs, Mp, A, dA, S, n)
    M = co.mttkrp(T, A, n)
    return np.abs(Mt - M).max() / np.abs(M).max(), Mt, M


@pytest.mark.parametrize("dims", [(5, 6, 7), (4, 5, 3, 4)])
def test_pp_zero_perturbation_is_exact(dims):
    T, Ap, A = _pp_setup(dims, 3, 50, 0.0)
    for n in range(len(dims)):
        e, Mt, M = _pp_err(T, Ap, A, n)
        assert e < 1e-13


@pytest.mark.parametrize("dims", [(5, 6, 7), (4, 5, 3, 4)])
def test_pp_single_factor_perturbation_is_exact(dims):
    """Multilinearity: with one dA(i) != 0 the first-order term is the whole change."""
    for only in range(len(dims)):
        T, Ap, A = _pp_setup(dims, 3, 60, 0.3, only=only)
        for n in range(len(dims)):
            e, _, _ = _pp_err(T, Ap, A, n)
            assert e < 1e-12


def test_pp_order3_exact_on_cp_tensor():
    """N = 3, T = [[A]] with the current factors: V equals the second-order term exactly."""
    dims = (5, 6, 7)
    _, Ap, A = _pp_setup(dims, 3, 70, 0.2)
    T = co.cp_full(A)
    for n in range(3):
        e, _, _ = _pp_err(T, Ap, A, n)
        assert e < 1e-12


def _slope(ts, errs):
    return np.polyfit(np.log(ts), np.log(errs), 1)[0]


def test_pp_error_order():
    """||M~ - M|| ~ t^2 for N = 3 with a general T; ~ t^3 for N = 4 with T = [[A]]."""
    ts = np.array([1e-1, 5e-2, 2.5e-2, 1.25e-2])
    e3 = [_pp_err(*_pp_setup((5, 6, 7), 3, 80, t), 0)[0] for t in ts]
    assert abs(_slope(ts, e3) - 2.0) < 0.1
    e4 = []
    for t in ts:
        _, Ap, A = _pp_setup((4, 5, 4, 5), 3, 90, t)
        e4.append(_pp_err(co.cp_full(A), Ap, A, 1)[0])
    assert abs(_slope(ts, e4) - 3.0) < 0.1


def test_pp_loop_tiny_eps_is_plain_als():
    T, F, A0 = synth.make_problem(95, (6, 7, 8), 3, eta=0.05)
    a = co.cp_als(T, A0, 8)
    b = co.pp_cp_als(T, A0, 8, eps=1e-12)
    assert b.kinds == ["als"] * 8 and b.n_pp_init == 0
    assert np.allclose(a.resid, b.resid, rtol=0, atol=1e-14)


def test_pp_loop_enters_and_tracks_als():
    """With eps = 0.1 PP is entered near convergence and the fit follows exact ALS closely."""
    T, F, A0 = synth.make_problem(96, (12, 13, 14), 4, eta=1e-3)
    a = co.cp_als(T, A0, 40)
    b = co.pp_cp_als(T, A0, 40, eps=0.1)
    assert b.n_pp_init >= 1 and "pp" in b.kinds
    assert b.kinds[0] == "als"                       # dA <- A initially: first sweep is exact
    assert abs(b.resid[-1] - a.resid[-1]) < 1e-3


def _scripted_pp(monkeypatch, steps, eps=0.1, dims=(5, 6, 7), R=2):
    """Run the oracle's Alg. 2 loop with the normal-equation solve replaced by a
    script: update n of sweep k returns A(n) * (1 + steps[k]).  Every factor then
    changes by exactly steps[k] / (1 + steps[k]) relative in a sweep, so the
    regime tests of Alg. 2 see prescribed values, whatever the contractions
    compute.  Returns the result and the factors each operator build started from."""
    T = synth.normal(300, 0, int(np.prod(dims))).reshape(dims)
    A0 = synth.uniform_factors(301, dims, R)
    N = len(dims)
    cur = [a.copy() for a in A0]
    calls = {"k": 0}

    def fake_solve(M, G):
        k, n = divmod(calls["k"], N)
        calls["k"] += 1
        cur[n] = cur[n] * (1.0 + steps[k])
        return cur[n].copy()

    builds = []
    real_ops = co.pp_operators

    def spy_ops(Tt, Ap):
        builds.append([a.copy() for a in Ap])
        return real_ops(Tt, Ap)

    monkeypatch.setattr(co, "solve_normal", fake_solve)
    monkeypatch.setattr(co, "pp_operators", spy_ops)
    res = co.pp_cp_als(T, A0, len(steps), eps=eps)
    return res, builds, A0


def _grow(A0, factor):
    return [a * factor for a in A0]


def test_pp_control_follows_alg2_on_a_script(monkeypatch):
    """Alg. 2's regime logic, sweep by sweep, on scripted relative changes (eps 0.1):
      0  dA = A (start): regular                        step 0.5  -> change 0.333
      1  0.333 >= eps: regular                         step 0.05 -> change 0.048
      2  0.048 < eps: build operators (A_p = A), PP    step 0.04 -> A - A_p 0.038
      3  0.038 < eps: stay in PP                       step 0.04 -> 0.075
      4  0.075 < eps: stay in PP                       step 0.04 -> 0.111
      5  0.111 >= eps: leave, one regular sweep        step 0.02 -> change 0.0196
      6  that sweep's change 0.0196 < eps: rebuild, PP step 0.3  -> 0.231
      7  0.231 >= eps: leave, regular                  step 0.2  -> change 0.167
      8  0.167 >= eps: regular again                   step 0.01 -> change 0.0099
      9  rebuild, PP
    A PP initialization is not a sweep: ten sweeps, three builds."""
    steps = [0.5, 0.05, 0.04, 0.04, 0.04, 0.02, 0.3, 0.2, 0.01, 0.01]
    res, builds, A0 = _scripted_pp(monkeypatch, steps)
    assert res.kinds == ["als", "als", "pp", "pp", "pp", "als", "pp", "als", "als", "pp"]
    assert len(res.kinds) == len(res.resid) == len(steps)
    assert res.n_pp_init == 3 == len(builds)
    # each build starts from the factors of that moment (A_p = A, Alg. 2's operator build)
    for b, k in zip(builds, (2, 6, 9)):
        g = float(np.prod([1.0 + x for x in steps[:k]]))
        for n in range(3):
            assert np.allclose(b[n], A0[n] * g, rtol=1e-14, atol=0)
    # the final factors are the scripted ones (PP sweeps write A(n), dA = A - A_p)
    g = float(np.prod([1.0 + x for x in steps]))
    for n in range(3):
        assert np.allclose(res.A[n], A0[n] * g, rtol=1e-14, atol=0)


def test_pp_control_reentry_uses_the_regular_sweeps_change(monkeypatch):
    """After leaving PP, the entry test uses the change made by the regular sweep
    (Alg. 2, after a regular sweep), not A - A_p of the old operators: here the accumulated
    A - A_p (0.3 after the regular sweep) would keep it out, the sweep's own change
    (0.01) lets it back in with new operators."""
    steps = [0.5, 0.05, 0.09, 0.09, 0.01, 0.01]
    res, builds, _ = _scripted_pp(monkeypatch, steps)
    # 0 als (dA = A), 1 als (0.333), 2 build + pp (0.048), 3 pp (A - A_p 0.083),
    # 4 leave: als (A - A_p 0.158), 5 re-enter on the regular change 0.0099: build + pp
    assert res.kinds == ["als", "als", "pp", "pp", "als", "pp"]
    assert res.n_pp_init == 2


def test_pp_control_tests_every_factor(monkeypatch):
    """The test is ||dA(i)|| < eps ||A(i)|| for every i: one factor above eps keeps
    the sweep regular (entry) or ends the approximation (stay)."""
    dims, R, N = (5, 6, 7), 2, 3
    T = synth.normal(302, 0, int(np.prod(dims))).reshape(dims)
    A0 = synth.uniform_factors(303, dims, R)
    # relative step of factor n in sweep k (new = old (1 + step))
    steps = [[1.0, 1.0, 1.0],          # 0 regular (dA = A)
             [0.01, 0.25, 0.01],       # 1 regular (0.5 >= eps); factor 1 changes 0.2
             [0.01, 0.01, 0.01],       # 2 regular: factor 1 alone is above eps
             [0.001, 0.001, 0.2],      # 3 build + PP; factor 2 drifts 0.167 from A_p
             [0.01, 0.01, 0.01]]       # 4 regular: factor 2 alone is above eps
    cur = [a.copy() for a in A0]
    calls = {"k": 0}

    def fake_solve(M, G):
        k, n = divmod(calls["k"], N)
        calls["k"] += 1
        cur[n] = cur[n] * (1.0 + steps[k][n])
        return cur[n].copy()

    monkeypatch.setattr(co, "solve_normal", fake_solve)
    res = co.pp_cp_als(T, A0, len(steps), eps=0.1)
    assert res.kinds == ["als", "als", "als", "pp", "als"]
    assert res.n_pp_init == 1


# ----------------------------------------------------------------------------- MLP


def test_mlp_param_count_and_fd_gradient():
    assert mo.N_PARAMS == 4801
    theta = mo.init_params(synth.uniform(200, 0, mo.N_PARAMS))
    X = synth.normal(201, 0, 16 * 8).reshape(16, 8)
    y = (synth.uniform(202, 0, 16) < 0.5).astype(float)
    L, g = mo.grad(theta, X, y)
    assert L == pytest.approx(mo.loss(theta, X, y), abs=1e-14)
    idx = np.linspace(0, mo.N_PARAMS - 1, 97).astype(int)
    h = 1e-6
    for i in idx:
        e = np.zeros(mo.N_PARAMS)
        e[i] = h
        fd = (mo.loss(theta + e, X, y) - mo.loss(theta - e, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9


def test_mlp_loss_closed_forms():
    """Zero weights: p = 1/2 and the loss is log 2; a single sample gives dL/db3 = p - y."""
    theta = np.zeros(mo.N_PARAMS)
    X = synth.normal(203, 0, 5 * 8).reshape(5, 8)
    assert mo.loss(theta, X, np.ones(5)) == pytest.approx(math.log(2.0), abs=1e-15)
    L, g = mo.grad(theta, X[:1], np.array([1.0]))
    assert g[-1] == pytest.approx(0.5 - 1.0, abs=1e-15)


def test_adam_first_step_is_signed_lr():
    """With bias correction the first Adam step is -lr * g / (|g| + eps), about lr * sign(g)."""
    g = np.array([3.0, -0.5, 1e-3])
    th, m, v = mo.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-8)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
