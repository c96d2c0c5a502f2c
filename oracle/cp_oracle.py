"""FP64 CPU oracle for CP-ALS with dimension trees, MSDT and pairwise perturbation.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module; the GPU library never calls it.  It is
deliberately plain and slow: NumPy in float64, one library matmul/tensordot
per contraction, no blocking or fusion, so each function can be checked
against the paper by eye.

Conventions.  A tensor is a C-order ndarray (last index fastest).  Modes are
0-based (the paper's mode n is index n-1 here).  A factor A[n] is s_n x R.  An
intermediate of the dimension tree (Sec. II-C, Eq. tensors-cp) is an ndarray
whose axes are the kept modes in increasing order followed by the rank axis r.

Readings of the paper that this oracle takes (each listed in the design notes):
  * Eq. (residual) prints ||T||_F under the square root; the identity needs the
    squared norm, so ||T||_F^2 is used and the radicand is clamped at 0.
  * Alg. 1 writes A = M Gamma^dagger; Gamma is SPD for full-column-rank
    factors, so a Cholesky solve is used, falling back to an eigenvalue
    pseudo-inverse (cut-off lambda < R * 2^-52 * lambda_max) if Cholesky fails.
  * The dimension tree splits an ordered leaf list L into L1 = first
    ceil(|L|/2) leaves and L2 = the rest (Fig. 1a for N=4; any binary split has
    the same leading cost).  The first child contracts L2 starting from its last
    mode, the second child contracts L1 starting from its first mode, which
    reproduces Fig. 1a and Fig. 2.
  * MSDT (Sec. III, Fig. 2): root modes N-1, N-2, ..., 0, N-1, ... (0-based);
    root m = T x_m A[m] serves updates m+1, ..., m+N-1 (mod N) with a binary
    dimension tree over those leaves in that order.
  * PP (Alg. 2, Eqs. ppupdate, U_ni, V_nij, ds): M_p^(n,i) with n > i is the
    transposed view of M_p^(i,n); A[n] inside V^(n) is its value before its own
    update in the current approximated sweep; dS uses current factors; the
    relative residual is evaluated after every sweep, approximated or not, and
    the stopping test |r - r_old| <= Delta is applied there too.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------------------
# Basic objects: Khatri-Rao rows, Gram, Hadamard chain, MTTKRP by definition
# --------------------------------------------------------------------------------------


def khatri_rao_rows(mats):
    """Rows of the Khatri-Rao product of `mats`, first matrix slowest (C order).

    Row (i_a, i_b, ...) = A_a(i_a, :) * A_b(i_b, :) * ...  (Sec. II-A defines the
    column-wise Kronecker product; only the row order differs from the paper's
    column-major notation, which does not change M's values.)
    """
    R = mats[0].shape[1]
    out = np.ones((1, R))
    for A in mats:
        out = (out[:, None, :] * A[None, :, :]).reshape(-1, R)
    return out


def unfold(T, n):
    """Mode-n matricization T_(n): s_n x prod(other dims), other modes in C order."""
    return np.moveaxis(T, n, 0).reshape(T.shape[n], -1)


def mttkrp(T, A, n):
    """MTTKRP by its definition M^(n) = T_(n) P^(n) (Sec. II-B).

    P^(n) is the Khatri-Rao product of all factors except A[n].
    """
    others = [A[k] for k in range(T.ndim) if k != n]
    return unfold(T, n) @ khatri_rao_rows(others)


def mttkrp_bruteforce(T, A, n):
    """Element-wise M^(n)(x,r) = sum over other indices of T * prod_k A[k](i_k, r).

    Pure-Python loops; only for tiny tensors.
    """
    R = A[0].shape[1]
    M = np.zeros((T.shape[n], R))
    for idx in np.ndindex(*T.shape):
        t = T[idx]
        for r in range(R):
            p = t
            for k, i in enumerate(idx):
                if k != n:
                    p *= A[k][i, r]
            M[idx[n], r] += p
    return M


def gram(A):
    """S = A^T A (Alg. 1)."""
    return A.T @ A


def hadamard_except(S, n):
    """Gamma^(n) = S^(1) * ... * S^(n-1) * S^(n+1) * ... * S^(N) (Eq. gram)."""
    G = np.ones_like(S[0])
    for k, Sk in enumerate(S):
        if k != n:
            G = G * Sk
    return G


def solve_normal(M, Gamma):
    """A = M Gamma^dagger: Cholesky solve, eigen pseudo-inverse if not SPD (Alg. 1)."""
    try:
        L = np.linalg.cholesky(Gamma)
    except np.linalg.LinAlgError:
        w, V = np.linalg.eigh(Gamma)
        cut = Gamma.shape[0] * 2.0 ** -52 * max(w.max(), 0.0)
        winv = np.where(w > cut, 1.0 / np.where(w > cut, w, 1.0), 0.0)
        return M @ (V * winv) @ V.T
    # Gamma X^T = M^T  <=>  L L^T X^T = M^T
    Y = np.linalg.solve(L, M.T)
    return np.linalg.solve(L.T, Y).T


def cp_full(A):
    """[[A(1), ..., A(N)]] = sum_r A(1)(:,r) o ... o A(N)(:,r) (Sec. II-B)."""
    N = len(A)
    R = A[0].shape[1]
    T = np.zeros([a.shape[0] for a in A])
    for r in range(R):
        t = A[0][:, r]
        for k in range(1, N):
            t = np.multiply.outer(t, A[k][:, r])
        T += t
    return T


def residual_direct(T, A):
    """r = ||T - [[A]]||_F / ||T||_F (Eq. residual-def)."""
    return float(np.linalg.norm((T - cp_full(A)).ravel()) / np.linalg.norm(T.ravel()))


def residual_formula(normT2, Gamma_N, A_N, M_N):
    """Eq. (residual) with ||T||_F^2 (see module header):
    r = sqrt(||T||^2 + <Gamma^(N), A^(N)T A^(N)> - 2 <M^(N), A^(N)>) / ||T||.
    """
    val = normT2 + float(np.sum(Gamma_N * gram(A_N))) - 2.0 * float(np.sum(M_N * A_N))
    return math.sqrt(max(val, 0.0)) / math.sqrt(normT2)


# --------------------------------------------------------------------------------------
# Dimension-tree contractions (Sec. II-C, Eq. tensors-cp)
# --------------------------------------------------------------------------------------


@dataclass
class Node:
    """An intermediate M^(modes) (or the input tensor when has_r is False)."""
    modes: tuple
    data: np.ndarray
    has_r: bool


@dataclass
class Counters:
    ttm: int = 0              # first-level contractions T x_m A (2 s^N R flops each)
    ttm_flops: float = 0.0
    mttv_flops: float = 0.0   # 2 x (entries of the parent read) per multi-TTV
    pp_approx_flops: float = 0.0
    ttm_modes: list = field(default_factory=list)
    edges: list = field(default_factory=list)   # (parent modes or "T", child modes)


def contract(node: Node, A, k: int, ctr: Counters | None = None) -> Node:
    """Contract mode k of `node` with factor A[k] (Sec. II-C).

    On the input tensor this is the first-level TTM T x_k A[k]; on an
    intermediate it is the multi-TTV Y(..., r) = sum_i X(..., i, ..., r) A[k](i, r).
    """
    pos = node.modes.index(k)
    new_modes = tuple(m for m in node.modes if m != k)
    if ctr is not None:
        ctr.edges.append((node.modes if node.has_r else "T", new_modes))
    if not node.has_r:
        Y = np.tensordot(node.data, A[k], axes=([pos], [0]))
        if ctr is not None:
            ctr.ttm += 1
            ctr.ttm_flops += 2.0 * node.data.size * A[k].shape[1]
            ctr.ttm_modes.append(k)
    else:
        X = np.moveaxis(node.data, pos, 0)
        Y = np.einsum("i...r,ir->...r", X, A[k])
        if ctr is not None:
            ctr.mttv_flops += 2.0 * node.data.size
    return Node(new_modes, Y, True)


def contract_many(node: Node, A, order, ctr=None) -> Node:
    for k in order:
        node = contract(node, A, k, ctr)
    return node


def tree_updates(node: Node, leaves, A, ctr=None):
    """Binary dimension tree over ordered `leaves` below `node` (which holds exactly them).

    Generator: yields (n, M^(n)) for each leaf in order; the caller updates A[n]
    in place before resuming, so later contractions see the new factor.
    """
    if len(leaves) == 1:
        n = leaves[0]
        yield n, node.data.reshape(node.data.shape[-2], node.data.shape[-1])
        return
    h = (len(leaves) + 1) // 2
    L1, L2 = list(leaves[:h]), list(leaves[h:])
    # first child: contract the later leaves (factors not yet updated), last one first
    c1 = contract_many(node, A, sorted(L2, key=leaves.index, reverse=True), ctr)
    yield from tree_updates(c1, L1, A, ctr)
    # second child: contract the earlier leaves (just updated), first one first
    c2 = contract_many(node, A, sorted(L1, key=leaves.index), ctr)
    yield from tree_updates(c2, L2, A, ctr)


def dt_updates(T, A, ctr=None):
    """One sweep of the standard dimension tree (Sec. II-C, Fig. 1a): yields (n, M^(n))."""
    N = T.ndim
    root = Node(tuple(range(N)), T, False)
    yield from tree_updates(root, list(range(N)), A, ctr)


def contract_combined(T, A, modes, ctr=None):
    """T contracted with the factors of several modes at once (the upper levels of a
    tree combined, Sec. IV): one product of T with the Khatri-Rao product of those
    factors, 2 s^N R flops; the result keeps the other modes and r."""
    N = T.ndim
    keep = [k for k in range(N) if k not in modes]
    order = sorted(modes)
    X = np.transpose(T, keep + order).reshape([T.shape[k] for k in keep] + [-1])
    Y = X @ khatri_rao_rows([A[k] for k in order])
    if ctr is not None:
        ctr.edges.append(("T", tuple(keep)))
        ctr.ttm += 1
        ctr.ttm_flops += 2.0 * T.size * A[0].shape[1]
        ctr.ttm_modes.append(tuple(order) if len(order) > 1 else order[0])
    return Node(tuple(keep), Y, True)


def msdt_updates(T, A, n_updates, ctr=None, levels=1):
    """Multi-sweep dimension tree (Sec. III, Fig. 2): yields (n, M^(n)) for n_updates updates.

    levels = 1: subtree j has root m_j = (N-1-j) mod N, built right after A[m_j]
    was last updated, and serves the N-1 updates m_j+1, ..., m_j+N-1 (mod N).

    levels = l (1 <= l <= N-2, the upper l levels combined, Sec. IV): update t
    (mode t mod N) belongs to subtree j = t // (N-l), whose root contracts, in one
    pass over T, the l modes updated just before its first update t0 = j (N-l),
    i.e. t0-1, ..., t0-l (mod N); it serves the N-l updates t0, ..., t0+N-l-1 with a
    binary dimension tree over those leaves.  Auxiliary memory s^(N-l) R instead
    of s^(N-1) R; first-level cost 2N/(N-l) s^N R per sweep.
    """
    N = T.ndim
    if not 1 <= levels <= max(1, N - 2):
        raise ValueError("levels must lie in 1..N-2")
    done = 0
    j = 0
    while done < n_updates:
        t0 = j * (N - levels)
        if levels == 1:
            m = (N - 1 - j) % N
            root = contract(Node(tuple(range(N)), T, False), A, m, ctr)
        else:
            root = contract_combined(T, A, [(t0 - 1 - i) % N for i in range(levels)], ctr)
        leaves = [(t0 + i) % N for i in range(N - levels)]
        for item in tree_updates(root, leaves, A, ctr):
            yield item
            done += 1
            if done == n_updates:
                return
        j += 1


# --------------------------------------------------------------------------------------
# CP-ALS (Alg. 1)
# --------------------------------------------------------------------------------------


@dataclass
class ALSResult:
    A: list
    resid: list                  # relative residual after each sweep, Eq. (residual)
    counters: Counters


def als_update(A, S, n, M):
    """One factor update of Alg. 1: Gamma^(n), A(n) = M Gamma^dagger, S(n) = A^T A."""
    G = hadamard_except(S, n)
    A[n] = solve_normal(M, G)
    S[n] = gram(A[n])
    return G


def cp_als(T, A0, n_sweeps, route="naive", delta=None, levels=1):
    """CP-ALS (Alg. 1) for a fixed sweep count (or until |r - r_old| <= delta).

    route: "naive" (MTTKRP by definition), "dt" (Fig. 1a) or "msdt" (Fig. 2, with
    `levels` upper levels combined, Sec. IV); in exact arithmetic all give the
    same factors.
    """
    T = np.asarray(T, dtype=np.float64)
    N = T.ndim
    A = [np.array(a, dtype=np.float64) for a in A0]
    S = [gram(a) for a in A]
    normT2 = float(np.sum(T * T))
    ctr = Counters()
    resid = []
    r_old = 0.0
    r = 1.0
    if route == "msdt":
        gen = msdt_updates(T, A, n_sweeps * N, ctr, levels)
    for sweep in range(n_sweeps):
        if route == "naive":
            items = ((n, None) for n in range(N))
        elif route == "dt":
            items = dt_updates(T, A, ctr)
        elif route == "msdt":
            items = (next(gen) for _ in range(N))
        else:
            raise ValueError(route)
        for n, M in items:
            if M is None:
                M = mttkrp(T, A, n)
            G = als_update(A, S, n, M)
        r_old, r = r, residual_formula(normT2, G, A[N - 1], M)
        resid.append(r)
        if delta is not None and abs(r - r_old) <= delta:
            break
    return ALSResult(A, resid, ctr)


# --------------------------------------------------------------------------------------
# Pairwise perturbation (Sec. II-D, Alg. 2, Eqs. tensors-cp, ppupdate, U_ni, V_nij, ds)
# --------------------------------------------------------------------------------------


def pp_pair_operator(T, Ap, i, j):
    """M_p^(i,j) (i < j): T contracted with A_p on every mode except i and j.

    Returned with axes (i, j, r).  Eq. (tensors-cp) with A_p in place of A.
    """
    N = T.ndim
    others = [k for k in range(N) if k not in (i, j)]
    X = np.transpose(T, [i, j] + others).reshape(T.shape[i], T.shape[j], -1)
    return X @ khatri_rao_rows([Ap[k] for k in others])


def pp_operators(T, Ap):
    """All M_p^(i,j), i < j, and M_p^(n) (Alg. 2, PP initialization step)."""
    N = T.ndim
    pairs = {(i, j): pp_pair_operator(T, Ap, i, j) for i in range(N) for j in range(i + 1, N)}
    Mp = [mttkrp(T, Ap, n) for n in range(N)]
    return pairs, Mp


def pp_pair_view(pairs, n, i):
    """M_p^(n,i) with axes (n, i, r); for n > i the transpose of M_p^(i,n)."""
    if n < i:
        return pairs[(n, i)]
    return np.transpose(pairs[(i, n)], (1, 0, 2))


def pp_mttkrp(pairs, Mp, A, dA, S, n, ctr=None):
    """Approximated MTTKRP (Eq. ppupdate): M~ = M_p^(n) + sum_{i!=n} U^(n,i) + V^(n).

    U^(n,i)(x,k) = sum_y M_p^(n,i)(x,y,k) dA(i)(y,k)                      (Eq. U_ni)
    V^(n) = A(n) ( sum_{i<j; i,j != n} dS(i) * dS(j) * (*_{k != i,j,n} S(k)) )  (Eq. V_nij)
    dS(i) = A(i)^T dA(i)                                                  (Eq. ds)
    """
    N = len(A)
    R = A[0].shape[1]
    Mt = Mp[n].copy()
    for i in range(N):
        if i == n:
            continue
        Op = pp_pair_view(pairs, n, i)
        Mt += np.einsum("xyk,yk->xk", Op, dA[i])
    dS = [A[i].T @ dA[i] for i in range(N)]
    W = np.zeros((R, R))
    for i in range(N):
        for j in range(i + 1, N):
            if n in (i, j):
                continue
            term = dS[i] * dS[j]
            for k in range(N):
                if k not in (i, j, n):
                    term = term * S[k]
            W += term
    Mt += A[n] @ W
    if ctr is not None:
        s = A[n].shape[0]
        ctr.pp_approx_flops += 2.0 * (N * s * s * R + N * R * R + s * R * R)
    return Mt


@dataclass
class PPResult:
    A: list
    resid: list                     # relative residual (Eq. residual) after every sweep
    kinds: list                     # "als" or "pp" per sweep
    n_pp_init: int
    counters: Counters


def pp_cp_als(T, A0, n_sweeps, eps, delta=None, max_sweeps=None):
    """PP-CP-ALS (Alg. 2) for n_sweeps sweeps (PP initializations are not sweeps).

    A sweep is either a regular ALS sweep (MTTKRP by definition; dA(i) = change
    of A(i) over that sweep) or an approximated sweep (Eq. ppupdate; dA(i) =
    A(i) - A_p(i)).  PP is entered when every ||dA(i)||_F < eps ||A(i)||_F and
    left as soon as one is not; a regular sweep follows leaving.
    """
    T = np.asarray(T, dtype=np.float64)
    N = T.ndim
    A = [np.array(a, dtype=np.float64) for a in A0]
    S = [gram(a) for a in A]
    dA = [a.copy() for a in A]                       # Alg. 2: dA <- A initially
    normT2 = float(np.sum(T * T))
    ctr = Counters()
    resid, kinds = [], []
    n_init = 0
    in_pp = False
    Ap = pairs = Mp = None
    r_old, r = 0.0, 1.0

    def small():
        return all(np.linalg.norm(dA[i]) < eps * np.linalg.norm(A[i]) for i in range(N))

    for sweep in range(n_sweeps):
        if not in_pp and small():
            Ap = [a.copy() for a in A]
            dA = [np.zeros_like(a) for a in A]
            pairs, Mp = pp_operators(T, Ap)
            n_init += 1
            in_pp = True
        if in_pp and small():
            for n in range(N):
                G = hadamard_except(S, n)
                M = pp_mttkrp(pairs, Mp, A, dA, S, n, ctr)
                A[n] = solve_normal(M, G)
                dA[n] = A[n] - Ap[n]
                S[n] = gram(A[n])
            kinds.append("pp")
        else:
            in_pp = False
            for n in range(N):
                before = A[n].copy()
                M = mttkrp(T, A, n)
                G = als_update(A, S, n, M)
                dA[n] = A[n] - before
            kinds.append("als")
        r_old, r = r, residual_formula(normT2, G, A[N - 1], M)
        resid.append(r)
        if delta is not None and abs(r - r_old) <= delta:
            break
    return PPResult(A, resid, kinds, n_init, ctr)
