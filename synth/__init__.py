"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and assembles input tensors; it holds no
step of CP-ALS (no MTTKRP, solve, tree or residual).  Both the CPU oracle and
the GPU path consume the bytes it produces, so neither side generates its own
inputs.

Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), written here from its published
definition: a 4x32-bit counter, a 2x32-bit key, ten rounds of two 32x32->64-bit
multiplies (multipliers 0xD2511F53 and 0xCD9E8D57) with the key bumped by the
Weyl constants 0x9E3779B9 / 0xBB67AE85 between rounds.

Stream layout (the GPU library's own Philox for default factor init follows the
same layout, independently written): key = (seed low 32 bits, seed high 32
bits); counter = (j low, j high, stream, 0) for block j.  Block j yields four
words w0..w3; uniform double 2j is ((w0<<32 | w1) >> 11) * 2^-53 and double
2j+1 is ((w2<<32 | w3) >> 11) * 2^-53, so values lie in [0, 1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "philox4x32_10", "uniform", "normal", "uniform_factors", "gaussian_factors",
    "collinear_factors", "cp_full", "add_noise", "make_problem",
]

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on uint64 arrays holding 32-bit words; returns 4 word arrays."""
    c0 = np.asarray(c0, np.uint64) & _MASK
    c1 = np.asarray(c1, np.uint64) & _MASK
    c2 = np.asarray(c2, np.uint64) & _MASK
    c3 = np.asarray(c3, np.uint64) & _MASK
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0,1) from (seed, stream), element i independent of n."""
    nblk = (n + 1) // 2
    j = np.arange(nblk, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32_10(j & _MASK, j >> _S32, np.uint64(stream), np.uint64(0),
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    a = ((w0 << _S32) | w1) >> np.uint64(11)
    b = ((w2 << _S32) | w3) >> np.uint64(11)
    out = np.empty(2 * nblk, dtype=np.float64)
    out[0::2] = a.astype(np.float64) * 2.0 ** -53
    out[1::2] = b.astype(np.float64) * 2.0 ** -53
    return out[:n]


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal doubles by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, stream, 2 * m)
    u1 = 1.0 - u[0::2]                      # (0, 1]: log is finite
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:n]


def uniform_factors(seed: int, dims, R: int, stream0: int = 0):
    """Factor matrices with U[0,1) entries: mode n uses stream stream0+n, row-major s_n x R."""
    return [uniform(seed, stream0 + n, s * R).reshape(s, R) for n, s in enumerate(dims)]


def gaussian_factors(seed: int, dims, R: int, stream0: int = 0):
    return [normal(seed, stream0 + n, s * R).reshape(s, R) for n, s in enumerate(dims)]


def collinear_factors(seed: int, dims, R: int, C: float, stream0: int = 0):
    """Factors whose columns have unit norm and pairwise cosine exactly C.

    Q (s x R, orthonormal columns) from a Householder QR of a seeded Gaussian
    matrix; K = (1-C) I + C 11^T = L L^T; A = Q L^T, so A^T A = K.  Needs s >= R.
    """
    K = (1.0 - C) * np.eye(R) + C * np.ones((R, R))
    L = np.linalg.cholesky(K)
    out = []
    for n, s in enumerate(dims):
        if s < R:
            raise ValueError("collinear factors need s >= R")
        G = normal(seed, stream0 + n, s * R).reshape(s, R)
        Q, _ = np.linalg.qr(G)
        out.append(Q @ L.T)
    return out


def cp_full(factors) -> np.ndarray:
    """Dense tensor sum_r a1_r o a2_r o ... (C order, last index fastest), FP64.

    Built as a product of the first N-1 factors' row-wise Khatri-Rao rows with the
    last factor; written here independently of the oracle.
    """
    R = factors[0].shape[1]
    rows = factors[0]
    for F in factors[1:-1]:
        rows = (rows[:, None, :] * F[None, :, :]).reshape(-1, R)
    full = rows @ factors[-1].T
    return full.reshape([F.shape[0] for F in factors])


def add_noise(T: np.ndarray, eta: float, seed: int, stream: int) -> np.ndarray:
    """T + E with E i.i.d. N(0,1) scaled so that ||E||_F = eta ||T||_F."""
    if eta == 0.0:
        return T.copy()
    E = normal(seed, stream, T.size).reshape(T.shape)
    E *= eta * np.linalg.norm(T.ravel()) / np.linalg.norm(E.ravel())
    return T + E


def make_problem(seed: int, dims, R: int, law: str = "uniform", eta: float = 0.0,
                 C: float | None = None, init_seed: int | None = None):
    """A seeded CP test problem: (T float64, true factors, initial factors U[0,1)).

    law: "uniform" (U[0,1) true factors), "gaussian" (N(0,1)) or "collinear"
    (pairwise column cosine C).  Streams 0..N-1 draw the true factors, stream 64
    the noise; the initial factors use init_seed (default seed+1) streams 0..N-1.
    """
    dims = list(dims)
    if law == "uniform":
        F = uniform_factors(seed, dims, R)
    elif law == "gaussian":
        F = gaussian_factors(seed, dims, R)
    elif law == "collinear":
        F = collinear_factors(seed, dims, R, C)
    else:
        raise ValueError(law)
    T = add_noise(cp_full(F), eta, seed, 64)
    A0 = uniform_factors(seed + 1 if init_seed is None else init_seed, dims, R)
    return T, F, A0


def make_problem_device(seed: int, dims, R: int, law: str = "uniform", eta: float = 0.0,
                        C: float | None = None, device="cuda", init_seed: int | None = None,
                        slab_elems: int = 1 << 27):
    """Large-tensor variant of make_problem, assembled with torch on `device`.

    Factors come from the same Philox streams as make_problem; the dense product
    is formed in FP64 with a torch matmul, the noise from torch's own seeded
    generator (N(0,1), scaled to eta ||T||_F), and the result is returned as a
    contiguous FP32 tensor.  Returns (T float32 on device, true factors, initial
    factors); the host oracle reads back exactly these FP32 bytes.  slab_elems bounds
    the FP64 Khatri-Rao rows formed at once (the product is built in mode-0 slices).
    """
    import torch

    dims = list(dims)
    if law == "uniform":
        F = uniform_factors(seed, dims, R)
    elif law == "gaussian":
        F = gaussian_factors(seed, dims, R)
    elif law == "collinear":
        F = collinear_factors(seed, dims, R, C)
    else:
        raise ValueError(law)
    Ft = [torch.from_numpy(f).to(device) for f in F]

    def slab(first):
        # rows of the Khatri-Rao product of modes 0..N-2 for the given mode-0 rows
        rows = first
        for f in Ft[1:-1]:
            rows = (rows[:, None, :] * f[None, :, :]).reshape(-1, R)
        return rows @ Ft[-1].T

    inner = 1
    for d in dims[1:-1]:
        inner *= d
    # slices of mode 0 keep the FP64 Khatri-Rao rows near 1 GB (uneven shapes
    # with a small last mode would otherwise need many times the tensor's size)
    step = max(1, int(slab_elems // max(1, inner * R)))
    if step >= dims[0]:
        T = slab(Ft[0])
    else:
        T = torch.cat([slab(Ft[0][i:i + step]) for i in range(0, dims[0], step)])
    if eta > 0.0:
        g = torch.Generator(device=device)
        g.manual_seed(int(seed))
        E = torch.randn(T.shape, generator=g, dtype=torch.float64, device=device)
        E *= eta * torch.linalg.vector_norm(T) / torch.linalg.vector_norm(E)
        T += E
        del E
    T32 = T.to(torch.float32).reshape(dims).contiguous()
    del T
    A0 = uniform_factors(seed + 1 if init_seed is None else init_seed, dims, R)
    return T32, F, A0
