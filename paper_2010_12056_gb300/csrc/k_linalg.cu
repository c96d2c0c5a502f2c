// Normal-equation side of every factor update (Alg. 1 lines 6, 8, 9; Alg. 2
// lines 10-12; Eq. gram, Eq. V_nij, Eq. ds) and the residual (Eq. residual,
// Eq. residual-def).  All R x R work is FP64: the Hadamard chain
// Gamma(n) = *_{k != n} S(k), its Cholesky factor, the two triangular solves per
// row of A(n) = M(n) Gamma(n)^{-1}, the Grams S(n) = A^T A and dS(n) = A^T dA,
// and the scalar terms of the residual.
#include <cuda_bf16.h>

#include "cpals_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// block-wide sum of one double; every thread gets the result
__device__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (lane < nw) ? sh[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) sh[0] = t;
    }
    __syncthreads();
    t = sh[0];
    __syncthreads();
    return t;
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// tf32 split of the factor operand: hi at [j][x], lo at Rpad*Kpad + [j][x]
__device__ __forceinline__ void tf32_store(float* bt, size_t lo_off, size_t e, float x) {
    const float h = tf32_rna(x);
    bt[e] = h;
    bt[lo_off + e] = tf32_rna(x - h);
}

__device__ __forceinline__ void bf16_split(float x, uint16_t& hi, uint16_t& lo) {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
}

// ------------------------------------------------------------------ Gamma + Cholesky
// One CTA.  work = Gamma with row stride ld (smem, ld = R + 1 so column reads
// hit distinct banks, when R <= 128; otherwise the Lt half of the output
// buffer with ld = R, rewritten at the end).  Right-looking factorisation in
// the LDL^T form, one barrier per column: at step j every thread updates
// work[i][k] -= work[i][j] work[k][j] / d_j for j < k <= i.  The pivot of the
// next column, d_{j+1} = work[j+1][j+1], is always updated by thread 0 as its
// first element of step j, so thread 0 alone tests it and forms 1/d_{j+1}
// while the other threads finish the step.  Finally L[i][k] = work[i][k] /
// sqrt(d_k), L[k][k] = sqrt(d_k).  If a pivot is not positive the
// factorisation restarts once on Gamma + 1e-12 * trace(Gamma)/R * I (flag 1);
// a second failure sets flag 2 and leaves L = I so that later kernels stay
// finite.  scal[SCAL_FLAGS] gets the flag and scal[SCAL_GS] is cleared for the
// Gram kernel's accumulation.
__global__ void __launch_bounds__(512) k_gamma_chol(double* const* __restrict__ S_list,
                                                    double* const* __restrict__ dS_list, int N,
                                                    int n, int R, int pp, double* __restrict__ G,
                                                    double* __restrict__ Lout,
                                                    double* __restrict__ invd,
                                                    double* __restrict__ W,
                                                    double* __restrict__ scal, int use_smem) {
    extern __shared__ double smw[];
    __shared__ double red[32];
    __shared__ double sinv[CP_MAXR];   // 1/d_j
    __shared__ double srs[CP_MAXR];    // 1/sqrt(d_j)
    __shared__ int sfail;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int RR = R * R;
    const int ld = use_smem ? R + 1 : R;
    double* L = Lout;            // lower, row-major
    double* Lt = Lout + RR;      // upper (transpose), row-major
    double* work = use_smem ? smw : Lt;
    const double* Sp[CP_MAXN];
    const double* dSp[CP_MAXN];
    for (int k = 0; k < N; ++k) {
        Sp[k] = S_list[k];
        dSp[k] = pp ? dS_list[k] : nullptr;
    }

    double tr = 0.0;
    for (int e = tid; e < RR; e += nt) {
        const int i = e / R, k = e % R;
        double g = 1.0;
        for (int m = 0; m < N; ++m)
            if (m != n) g *= Sp[m][e];
        G[e] = g;
        work[i * ld + k] = g;
        if (i == k) tr += g;
        if (pp) {
            double w = 0.0;
            for (int a = 0; a < N; ++a) {
                if (a == n) continue;
                for (int b = a + 1; b < N; ++b) {
                    if (b == n) continue;
                    double t = dSp[a][e] * dSp[b][e];
                    for (int m = 0; m < N; ++m)
                        if (m != a && m != b && m != n) t *= Sp[m][e];
                    w += t;
                }
            }
            W[e] = w;
        }
    }
    tr = block_sum(tr, red);  // also a barrier: work is complete
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    double flag = 0.0;
    bool bad = false;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (attempt == 1) {
            const double shift = 1e-12 * tr / R;
            for (int e = tid; e < RR; e += nt) {
                const int i = e / R, k = e % R;
                work[i * ld + k] = G[e] + ((i == k) ? shift : 0.0);
            }
            flag = 1.0;
            __syncthreads();
        }
        if (tid == 0) {
            const double d = work[0];
            sfail = (!(d > 0.0) || !isfinite(d)) ? 1 : 0;
            if (!sfail) sinv[0] = 1.0 / d;
        }
        __syncthreads();
        for (int j = 0; j < R && !sfail; ++j) {
            const double inv = sinv[j];
            for (int i = j + 1 + warp; i < R; i += nw) {
                double* wi = work + (size_t)i * ld;
                const double lij = wi[j] * inv;
                for (int k = j + 1 + lane; k <= i; k += 32) wi[k] = fma(-lij, work[k * ld + j], wi[k]);
            }
            if (tid == 0 && j + 1 < R) {
                const double d = work[(j + 1) * ld + j + 1];
                if (!(d > 0.0) || !isfinite(d)) sfail = 1;
                else sinv[j + 1] = 1.0 / d;
            }
            __syncthreads();
        }
        const bool failed = sfail != 0;
        __syncthreads();
        if (!failed) break;
        if (attempt == 1) {
            flag = 2.0;
            bad = true;
        }
    }
    for (int j = tid; j < R; j += nt) {
        const double v = bad ? 1.0 : 1.0 / sqrt(work[j * ld + j]);
        srs[j] = v;
        invd[j] = v;
    }
    __syncthreads();
    if (!use_smem) {
        // work aliases Lt: build L first, then its transpose
        for (int e = tid; e < RR; e += nt) {
            const int i = e / R, k = e % R;
            double v = 0.0;
            if (bad) v = (i == k) ? 1.0 : 0.0;
            else if (k < i) v = work[e] * srs[k];
            else if (k == i) v = 1.0 / srs[k];
            L[e] = v;
        }
        __syncthreads();
        for (int e = tid; e < RR; e += nt) {
            const int i = e / R, k = e % R;
            Lt[e] = L[k * R + i];
        }
    } else {
        for (int e = tid; e < RR; e += nt) {
            const int i = e / R, k = e % R;
            double v = 0.0;
            if (bad) v = (i == k) ? 1.0 : 0.0;
            else if (k < i) v = work[i * ld + k] * srs[k];
            else if (k == i) v = 1.0 / srs[k];
            L[e] = v;
            Lt[k * R + i] = v;
        }
    }
    if (tid == 0) {
        scal[SCAL_FLAGS] = flag;
        scal[SCAL_GS] = 0.0;
    }
}

// ------------------------------------------------------------------ row solves
// One warp per row x: m~ = M(x,:) [+ A_old(x,:) W]; forward substitution with L,
// back substitution with L^T (column-oriented, lane l owns entries l + 32t).
// With SMEM the block first stages L (row stride R+1, so that column reads are
// free of bank conflicts) and 1/L[j][j] in shared memory.
template <int RT, bool SMEM>
__global__ void __launch_bounds__(128) k_solve(const float* __restrict__ M,
                                               const double* __restrict__ W,
                                               const double* __restrict__ L,
                                               const double* __restrict__ invd, cpk::SolveOut o,
                                               int s, int R, double* __restrict__ scal_part) {
    extern __shared__ double sL[];
    __shared__ double red[4][CP_NSCAL];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwb = blockDim.x >> 5;
    const int x = blockIdx.x * nwb + wib;
    const int ld = SMEM ? R + 1 : R;
    const double* Lc;   // column access L[k][j] = Lc[j * ldc + k]... see below
    const double* Lr;   // row access    L[j][k] = Lr[j * ld + k]
    const double* iv;
    if (SMEM) {
        const int RR = R * R;
        int e = threadIdx.x;
        for (; e + 7 * (int)blockDim.x < RR; e += 8 * blockDim.x) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldg(L + e + u * blockDim.x);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int f = e + u * blockDim.x;
                sL[(f / R) * ld + (f % R)] = v[u];
            }
        }
        for (; e < RR; e += blockDim.x) sL[(e / R) * ld + (e % R)] = __ldg(L + e);
        for (int j = threadIdx.x; j < R; j += blockDim.x) sL[R * ld + j] = invd[j];
        __syncthreads();
        Lr = sL;
        Lc = sL;
        iv = sL + R * ld;
    } else {
        Lr = L;
        Lc = L + (size_t)R * R;  // Lt row-major: L[k][j] = Lt[j][k]
        iv = invd;
    }
    double sc[CP_NSCAL];
#pragma unroll
    for (int i = 0; i < CP_NSCAL; ++i) sc[i] = 0.0;
    if (x < s) {
        double aold[RT], acc[RT], mt[RT], z[RT], xs[RT];
#pragma unroll
        for (int t = 0; t < RT; ++t) {
            const int j = lane + 32 * t;
            aold[t] = (j < R) ? o.A64[(size_t)x * R + j] : 0.0;
            acc[t] = (j < R) ? (double)M[(size_t)x * R + j] : 0.0;
            z[t] = 0.0;
            xs[t] = 0.0;
        }
        if (W) {
            double vt[RT];
#pragma unroll
            for (int t = 0; t < RT; ++t) vt[t] = 0.0;
            for (int q = 0; q < R; ++q) {
                const double aq = o.A64[(size_t)x * R + q];
                const double* wr = W + (size_t)q * R;
#pragma unroll
                for (int t = 0; t < RT; ++t) {
                    const int j = lane + 32 * t;
                    if (j < R) vt[t] = fma(aq, wr[j], vt[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < RT; ++t) {
                acc[t] += vt[t];
                sc[SCAL_V2] += vt[t] * vt[t];
            }
        }
#pragma unroll
        for (int t = 0; t < RT; ++t) mt[t] = acc[t];
        // forward: z_j = (m_j - sum_{k<j} L[j][k] z_k) / L[j][j]
#pragma unroll
        for (int tt = 0; tt < RT; ++tt) {
            for (int jj = 0; jj < 32; ++jj) {
                const int j = tt * 32 + jj;
                if (j >= R) break;
                const double zj = __shfl_sync(FULL, acc[tt], jj) * iv[j];
                if (lane == jj) z[tt] = zj;
#pragma unroll
                for (int t2 = tt; t2 < RT; ++t2) {
                    const int k = lane + 32 * t2;
                    if (k > j && k < R) {
                        const double lkj = SMEM ? Lc[(size_t)k * ld + j] : Lc[(size_t)j * R + k];
                        acc[t2] = fma(-lkj, zj, acc[t2]);
                    }
                }
            }
        }
        // back: x_j = (z_j - sum_{k>j} L[k][j] x_k) / L[j][j]
#pragma unroll
        for (int t = 0; t < RT; ++t) acc[t] = z[t];
#pragma unroll
        for (int tt = RT - 1; tt >= 0; --tt) {
            for (int jj = 31; jj >= 0; --jj) {
                const int j = tt * 32 + jj;
                if (j >= R) continue;
                const double xj = __shfl_sync(FULL, acc[tt], jj) * iv[j];
                if (lane == jj) xs[tt] = xj;
                const double* lr = Lr + (size_t)j * ld;
#pragma unroll
                for (int t2 = 0; t2 <= tt; ++t2) {
                    const int k = lane + 32 * t2;
                    if (k < j) acc[t2] = fma(-lr[k], xj, acc[t2]);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < RT; ++t) {
            const int j = lane + 32 * t;
            if (j >= R) continue;
            const double a = xs[t];
            const size_t e = (size_t)x * R + j;
            o.A64[e] = a;
            const float af = (float)a;
            if (o.A32) o.A32[e] = af;
            if (o.bhi) {
                uint16_t hi, lo;
                bf16_split(af, hi, lo);
                o.bhi[(size_t)j * o.Kpad + x] = hi;
                o.blo[(size_t)j * o.Kpad + x] = lo;
            }
            if (o.bt32) tf32_store(o.bt32, (size_t)o.Rpad * o.Kpad, (size_t)j * o.Kpad + x, af);
            const double base = o.Ap ? o.Ap[e] : aold[t];
            const double d = a - base;
            if (o.dA32) o.dA32[e] = (float)d;
            if (o.dA64) o.dA64[e] = d;
            sc[SCAL_A2] += a * a;
            sc[SCAL_STEP2] += (a - aold[t]) * (a - aold[t]);
            if (o.Ap) sc[SCAL_DAP2] += d * d;
            sc[SCAL_MA] += mt[t] * a;
            sc[SCAL_M2] += mt[t] * mt[t];
        }
    }
#pragma unroll
    for (int i = 0; i < CP_NSCAL; ++i) {
        double v = warp_sum(sc[i]);
        if (lane == 0) red[wib][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < CP_NSCAL) {
        double v = 0.0;
        for (int w = 0; w < nwb; ++w) v += red[w][threadIdx.x];
        scal_part[(size_t)blockIdx.x * CP_NSCAL + threadIdx.x] = v;
    }
}

// ------------------------------------------------------------------ Gram partials
// grid (ceil(R/16), ceil(R/16), nchunk), block 16x16: part[c][0] = A_c^T A_c,
// part[c][1] = A_c^T dA_c over the rows of chunk c.
__global__ void __launch_bounds__(256) k_gram_part(const double* __restrict__ A,
                                                  const double* __restrict__ dA, int s, int R,
                                                  double* __restrict__ part, int rows_per) {
    __shared__ double a1[16][17], a2[16][17], d2[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r1 = blockIdx.x * 16 + ty, r2 = blockIdx.y * 16 + tx;
    const int c = blockIdx.z;
    const int x0 = c * rows_per, x1 = min(s, x0 + rows_per);
    double acc = 0.0, accd = 0.0;
    for (int xb = x0; xb < x1; xb += 16) {
        const int x = xb + ty;
        const int ca = blockIdx.x * 16 + tx, cb = blockIdx.y * 16 + tx;
        a1[ty][tx] = (x < x1 && ca < R) ? A[(size_t)x * R + ca] : 0.0;
        a2[ty][tx] = (x < x1 && cb < R) ? A[(size_t)x * R + cb] : 0.0;
        if (dA) d2[ty][tx] = (x < x1 && cb < R) ? dA[(size_t)x * R + cb] : 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            acc = fma(a1[k][ty], a2[k][tx], acc);
            if (dA) accd = fma(a1[k][ty], d2[k][tx], accd);
        }
        __syncthreads();
    }
    if (r1 < R && r2 < R) {
        const size_t RR = (size_t)R * R;
        part[(size_t)c * 2 * RR + (size_t)r1 * R + r2] = acc;
        if (dA) part[(size_t)c * 2 * RR + RR + (size_t)r1 * R + r2] = accd;
    }
}

// ------------------------------------------------------------------ finalize
// Grid over the R x R entries: S = sum of chunk partials (and dS); <Gamma, S>
// accumulates into scal[SCAL_GS] (cleared by the Cholesky kernel of the same
// update).  Block 0 also reduces the solve kernel's per-block scalars.
__global__ void __launch_bounds__(256) k_finalize(const double* __restrict__ part, int nchunk,
                                                  const double* __restrict__ scal_part, int nblk,
                                                  const double* __restrict__ Gamma, int R,
                                                  int want_dS, double* __restrict__ S,
                                                  double* __restrict__ dS,
                                                  double* __restrict__ scal_out) {
    __shared__ double red[32];
    const int tid = threadIdx.x;
    const size_t RR = (size_t)R * R;
    double gs = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + tid; e < RR; e += (size_t)gridDim.x * blockDim.x) {
        double v0 = 0.0, v1 = 0.0, d0 = 0.0, d1 = 0.0;
        int c = 0;
        for (; c + 1 < nchunk; c += 2) {
            v0 += part[(size_t)c * 2 * RR + e];
            v1 += part[(size_t)(c + 1) * 2 * RR + e];
            if (want_dS) {
                d0 += part[(size_t)c * 2 * RR + RR + e];
                d1 += part[(size_t)(c + 1) * 2 * RR + RR + e];
            }
        }
        if (c < nchunk) {
            v0 += part[(size_t)c * 2 * RR + e];
            if (want_dS) d0 += part[(size_t)c * 2 * RR + RR + e];
        }
        const double v = v0 + v1;
        S[e] = v;
        if (want_dS) dS[e] = d0 + d1;
        if (Gamma) gs += Gamma[e] * v;
    }
    if (Gamma) {
        gs = block_sum(gs, red);
        if (tid == 0) atomicAdd(scal_out + SCAL_GS, gs);
    }
    if (blockIdx.x != 0) return;
    for (int slot = 0; slot < CP_NSCAL; ++slot) {
        if (slot == SCAL_GS || slot == SCAL_FLAGS) continue;
        double v = 0.0;
        for (int b = tid; b < nblk; b += blockDim.x) v += scal_part[(size_t)b * CP_NSCAL + slot];
        v = block_sum(v, red);
        if (tid == 0) scal_out[slot] = v;
    }
}

// ------------------------------------------------------------------ factor copies
__global__ void k_factor_copies(const double* __restrict__ A64, float* __restrict__ A32,
                                uint16_t* __restrict__ bhi, uint16_t* __restrict__ blo,
                                float* __restrict__ bt32, int s, int R, int Rpad, int Kpad) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)s * R) return;
    const int x = (int)(e / R), j = (int)(e % R);
    const float af = (float)A64[e];
    if (A32) A32[e] = af;
    if (bhi) {
        uint16_t hi, lo;
        bf16_split(af, hi, lo);
        bhi[(size_t)j * Kpad + x] = hi;
        blo[(size_t)j * Kpad + x] = lo;
    }
    if (bt32) tf32_store(bt32, (size_t)Rpad * Kpad, (size_t)j * Kpad + x, af);
}

// ------------------------------------------------------------------ norms
// sum of squares: FP32 inside an 8-element chunk, FP64 across chunks
__global__ void __launch_bounds__(256) k_norm2(const float* __restrict__ x, int64_t n,
                                               double* __restrict__ partials) {
    __shared__ double red[32];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n8 = n / 8;
    const bool al = ((uintptr_t)x & 15) == 0;
    if (al) {
        const float4* x4 = reinterpret_cast<const float4*>(x);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += stride) {
            float4 a = __ldg(x4 + 2 * i), b = __ldg(x4 + 2 * i + 1);
            float s = a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w + b.x * b.x + b.y * b.y +
                      b.z * b.z + b.w * b.w;
            acc += (double)s;
        }
    }
    const int64_t start = al ? n8 * 8 : 0;
    for (int64_t i = start + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double v = x[i];
        acc += v * v;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void k_sum(const double* __restrict__ p, int n, double* __restrict__ out) {
    __shared__ double red[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += p[i];
    v = block_sum(v, red);
    if (threadIdx.x == 0) out[0] = v;
}

__global__ void k_f64_to_f32(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

// ------------------------------------------------------------------ direct residual
// ||T - [[A]]||^2 with T viewed as rows (modes 0..N-2) x cols (mode N-1): per
// 64 x 64 tile, t~ = KR(row) . A_last(col) over r in chunks of 16 (FP32), then
// (t - t~)^2 summed in FP32 per thread and FP64 across tiles.
__global__ void __launch_bounds__(256) k_resid_direct(cpk::ResidArgs a, int64_t nrows,
                                                      int64_t ncols, int64_t ntile_c,
                                                      double* __restrict__ partials,
                                                      int64_t ntiles) {
    __shared__ __align__(16) float KR[16][64];
    __shared__ __align__(16) float Bs[16][64];
    __shared__ int rowoff[64][CP_MAXN];
    __shared__ double red[32];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int N = a.N, R = a.R;
    const float* Alast = a.A32[N - 1];
    double total = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t row0 = (tile / ntile_c) * 64, col0 = (tile % ntile_c) * 64;
        __syncthreads();
        if (tid < 64) {
            int64_t row = row0 + tid;
            if (row >= nrows) row = 0;
            for (int k = N - 2; k >= 0; --k) {
                rowoff[tid][k] = (int)(row % a.dims[k]);
                row /= a.dims[k];
            }
        }
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        for (int r0 = 0; r0 < R; r0 += 16) {
            __syncthreads();
            for (int e = tid; e < 16 * 64; e += 256) {
                const int rr = e >> 6, m = e & 63;
                float v = 0.f, b = 0.f;
                if (r0 + rr < R) {
                    v = 1.f;
                    for (int k = 0; k < N - 1; ++k) v *= a.A32[k][(size_t)rowoff[m][k] * R + r0 + rr];
                    if (col0 + m < ncols) b = Alast[(size_t)(col0 + m) * R + r0 + rr];
                }
                KR[rr][m] = v;
                Bs[rr][m] = b;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float4 av = *reinterpret_cast<const float4*>(&KR[k][ty * 4]);
                float4 bv = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
                float aa[4] = {av.x, av.y, av.z, av.w}, bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(aa[i], bb[j], acc[i][j]);
            }
        }
        float part = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t row = row0 + ty * 4 + i;
            if (row >= nrows) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t col = col0 + tx * 4 + j;
                if (col < ncols) {
                    float d = __ldg(a.T + row * ncols + col) - acc[i][j];
                    part = fmaf(d, d, part);
                }
            }
        }
        total += (double)part;
    }
    total = block_sum(total, red);
    if (tid == 0) partials[blockIdx.x] = total;
}

// ------------------------------------------------------------------ PP first-order terms
struct PPArgs {
    cpk::PPTerm t[CP_MAXN];
    int nterms;
};

template <int VEC>
__global__ void __launch_bounds__(256) k_pp_u(const float* __restrict__ Mp, PPArgs a,
                                              float* __restrict__ Mt, int sx, int R, int TX,
                                              int KS) {
    extern __shared__ float4 red4[];
    const int RV = R / VEC;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int64_t nout = (int64_t)sx * RV;
    const int64_t o = (int64_t)blockIdx.x * TX + tx;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (o < nout) {
        const int x = (int)(o / RV), rv = (int)(o % RV);
        const int r = rv * VEC;
        for (int i = 0; i < a.nterms; ++i) {
            const float* op = a.t[i].op;
            const float* dA = a.t[i].dA;
            const int sy = a.t[i].sy;
            const bool tr = a.t[i].trans;
            for (int y = ty; y < sy; y += KS) {
                const size_t e = tr ? ((size_t)y * sx + x) * R + r : ((size_t)x * sy + y) * R + r;
                if (VEC == 4) {
                    float4 v = __ldg(reinterpret_cast<const float4*>(op + e));
                    float4 d = __ldg(reinterpret_cast<const float4*>(dA + (size_t)y * R + r));
                    acc.x = fmaf(v.x, d.x, acc.x); acc.y = fmaf(v.y, d.y, acc.y);
                    acc.z = fmaf(v.z, d.z, acc.z); acc.w = fmaf(v.w, d.w, acc.w);
                } else {
                    acc.x = fmaf(__ldg(op + e), __ldg(dA + (size_t)y * R + r), acc.x);
                }
            }
        }
    }
    red4[ty * TX + tx] = acc;
    __syncthreads();
    if (ty == 0 && o < nout) {
        for (int j = 1; j < KS; ++j) {
            float4 v = red4[j * TX + tx];
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
        }
        if (VEC == 4) {
            float4 m = __ldg(reinterpret_cast<const float4*>(Mp) + o);
            *reinterpret_cast<float4*>(Mt + o * 4) =
                make_float4(m.x + acc.x, m.y + acc.y, m.z + acc.z, m.w + acc.w);
        } else {
            Mt[o] = Mp[o] + acc.x;
        }
    }
}


// ------------------------------------------------------------------ PP helpers
// dA = A - A_p in FP64 and FP32
__global__ void k_pp_delta(const double* __restrict__ A, const double* __restrict__ Ap,
                           float* __restrict__ d32, double* __restrict__ d64, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double d = A[i] - Ap[i];
        d64[i] = d;
        d32[i] = (float)d;
    }
}

// out[x][j] = Mt[x][j] + sum_q A[x][q] W[q][j]   (second-order term V = A W, FP64)
__global__ void k_add_aw(const float* __restrict__ Mt, const double* __restrict__ A,
                         const double* __restrict__ W, int s, int R, float* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)s * R) return;
    const int x = (int)(e / R), j = (int)(e % R);
    double v = 0.0;
    for (int q = 0; q < R; ++q) v = fma(A[(size_t)x * R + q], W[(size_t)q * R + j], v);
    out[e] = (float)((double)Mt[e] + v);
}


// ------------------------------------------------------------------ Khatri-Rao operand
// out[r][k] (r < Rpad, k < Kpad; zero outside R x K): row k = ia * sb + ib of the
// Khatri-Rao product, A_a[ia][r] * A_b[ib][r], split into two parts.
template <int KIND>
__global__ void k_kr(const double* __restrict__ Aa, const double* __restrict__ Ab, int sa, int sb,
                     int R, int Rpad, int Kpad, void* __restrict__ hi, void* __restrict__ lo) {
    const int64_t K = (int64_t)sa * sb;
    const int64_t n = (int64_t)Rpad * Kpad;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / Kpad);
        const int64_t k = idx - (int64_t)r * Kpad;
        float v = 0.f;
        if (r < R && k < K) {
            const int ia = (int)(k / sb), ib = (int)(k - (int64_t)ia * sb);
            v = (float)(Aa[(size_t)ia * R + r] * Ab[(size_t)ib * R + r]);
        }
        if (KIND == 0) {
            uint16_t h, l;
            bf16_split(v, h, l);
            static_cast<uint16_t*>(hi)[idx] = h;
            static_cast<uint16_t*>(lo)[idx] = l;
        } else {
            const float h = tf32_rna(v);
            static_cast<float*>(hi)[idx] = h;
            static_cast<float*>(lo)[idx] = tf32_rna(v - h);
        }
    }
}

}  // namespace

namespace cpk {

cudaError_t kr_operand(const double* Aa, const double* Ab, int sa, int sb, int R, int Kpad,
                       int kind, void* hi, void* lo, cudaStream_t st) {
    const int Rpad = (R + 15) / 16 * 16;
    const int64_t n = (int64_t)Rpad * Kpad;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (kind == 0)
        k_kr<0><<<(unsigned)blocks, 256, 0, st>>>(Aa, Ab, sa, sb, R, Rpad, Kpad, hi, lo);
    else
        k_kr<1><<<(unsigned)blocks, 256, 0, st>>>(Aa, Ab, sa, sb, R, Rpad, Kpad, hi, lo);
    return cudaGetLastError();
}

cudaError_t pp_delta(const double* A, const double* Ap, float* d32, double* d64, int64_t n,
                     cudaStream_t st) {
    int64_t want = (n + 255) / 256;
    unsigned blocks = (unsigned)(want > 4096 ? 4096 : (want < 1 ? 1 : want));
    k_pp_delta<<<blocks, 256, 0, st>>>(A, Ap, d32, d64, n);
    return cudaGetLastError();
}

cudaError_t add_aw(const float* Mt, const double* A, const double* W, int s, int R, float* out,
                   cudaStream_t st) {
    const int64_t n = (int64_t)s * R;
    k_add_aw<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Mt, A, W, s, R, out);
    return cudaGetLastError();
}

cudaError_t gamma_chol(double* const* S_list, double* const* dS_list, int N, int n, int R,
                       int pp, double* Gamma, double* L, double* invdiag, double* W,
                       double* scal, cudaStream_t st) {
    const int use_smem = (R <= 128) ? 1 : 0;
    size_t smem = use_smem ? (size_t)R * (R + 1) * sizeof(double) : 0;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_gamma_chol, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             128 * 129 * sizeof(double));
        attr_set = true;
    }
    k_gamma_chol<<<1, 512, smem, st>>>(S_list, dS_list, N, n, R, pp, Gamma, L, invdiag, W, scal,
                                       use_smem);
    return cudaGetLastError();
}

template <int RT, bool SM>
static cudaError_t launch_solve(unsigned blocks, unsigned threads, const float* M, const double* W,
                                const double* L, const double* invdiag, const SolveOut& o, int s,
                                int R, double* scal_part, cudaStream_t st) {
    size_t smem = SM ? ((size_t)R * (R + 1) + R) * sizeof(double) : 0;
    static bool attr_set = false;
    if (SM && !attr_set) {
        cudaFuncSetAttribute(k_solve<RT, SM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(((size_t)128 * 129 + 128) * sizeof(double)));
        attr_set = true;
    }
    k_solve<RT, SM><<<blocks, threads, smem, st>>>(M, W, L, invdiag, o, s, R, scal_part);
    return cudaGetLastError();
}

cudaError_t solve_rows(const float* M, const double* W, const double* L, const double* invdiag,
                       const SolveOut& o, int s, int R, double* scal_part, int* nblk,
                       cudaStream_t st) {
    const int RT = (R + 31) / 32;
    // one row per warp; small factor matrices get one warp per block so that the
    // FP64 work spreads over as many SMs as there are rows
    const int wpb = (s <= 512) ? 1 : 4;
    const unsigned blocks = (unsigned)((s + wpb - 1) / wpb);
    const unsigned th = 32u * wpb;
    *nblk = (int)blocks;
    switch (RT) {
        case 1: return launch_solve<1, true>(blocks, th, M, W, L, invdiag, o, s, R, scal_part, st);
        case 2: return launch_solve<2, true>(blocks, th, M, W, L, invdiag, o, s, R, scal_part, st);
        case 3: return launch_solve<3, true>(blocks, th, M, W, L, invdiag, o, s, R, scal_part, st);
        case 4: return launch_solve<4, true>(blocks, th, M, W, L, invdiag, o, s, R, scal_part, st);
        case 5: return launch_solve<5, false>(blocks, th, M, W, L, invdiag, o, s, R, scal_part, st);
        case 6: return launch_solve<6, false>(blocks, th, M, W, L, invdiag, o, s, R, scal_part, st);
        case 7: return launch_solve<7, false>(blocks, th, M, W, L, invdiag, o, s, R, scal_part, st);
        case 8: return launch_solve<8, false>(blocks, th, M, W, L, invdiag, o, s, R, scal_part, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t gram_partials(const double* A, const double* dA, int s, int R, double* part,
                          int nchunk, cudaStream_t st) {
    const int rows_per = (s + nchunk - 1) / nchunk;
    dim3 grid((R + 15) / 16, (R + 15) / 16, nchunk);
    k_gram_part<<<grid, 256, 0, st>>>(A, dA, s, R, part, rows_per);
    return cudaGetLastError();
}

cudaError_t finalize_update(const double* gram_part, int nchunk, const double* scal_part,
                            int nblk, const double* Gamma, int R, int want_dS, double* S,
                            double* dS, double* scal_out, cudaStream_t st) {
    const size_t RR = (size_t)R * R;
    unsigned blocks = (unsigned)((RR + 255) / 256);
    if (blocks > 64) blocks = 64;
    k_finalize<<<blocks, 256, 0, st>>>(gram_part, nchunk, scal_part, nblk, Gamma, R, want_dS, S, dS,
                                       scal_out);
    return cudaGetLastError();
}

cudaError_t factor_copies(const double* A64, float* A32, uint16_t* bhi, uint16_t* blo,
                          float* bt32, int s, int R, int Rpad, int Kpad, cudaStream_t st) {
    const int64_t n = (int64_t)s * R;
    k_factor_copies<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(A64, A32, bhi, blo, bt32, s, R,
                                                                 Rpad, Kpad);
    return cudaGetLastError();
}

int norm2_partials(const float* x, int64_t n, double* partials, int max_blocks, cudaStream_t st) {
    int64_t want = (n / 8 + 255) / 256;
    int blocks = (int)(want < 1 ? 1 : (want > max_blocks ? max_blocks : want));
    k_norm2<<<blocks, 256, 0, st>>>(x, n, partials);
    return blocks;
}

cudaError_t sum_partials(const double* partials, int n, double* out, cudaStream_t st) {
    k_sum<<<1, 1024, 0, st>>>(partials, n, out);
    return cudaGetLastError();
}

cudaError_t f64_to_f32(const double* x, float* y, int64_t n, cudaStream_t st) {
    int64_t want = (n + 255) / 256;
    unsigned blocks = (unsigned)(want > 65535 * 4 ? 65535 * 4 : (want < 1 ? 1 : want));
    k_f64_to_f32<<<blocks, 256, 0, st>>>(x, y, n);
    return cudaGetLastError();
}

int resid_direct_partials(const ResidArgs& a, double* partials, int max_blocks, cudaStream_t st) {
    int64_t nrows = 1;
    for (int k = 0; k < a.N - 1; ++k) nrows *= a.dims[k];
    const int64_t ncols = a.dims[a.N - 1];
    const int64_t ntr = (nrows + 63) / 64, ntc = (ncols + 63) / 64;
    const int64_t ntiles = ntr * ntc;
    int blocks = (int)(ntiles < max_blocks ? ntiles : max_blocks);
    k_resid_direct<<<blocks, 256, 0, st>>>(a, nrows, ncols, ntc, partials, ntiles);
    return blocks;
}

cudaError_t pp_u(const float* Mp, const PPTerm* terms, int nterms, float* Mt, int sx, int R,
                 cudaStream_t st) {
    PPArgs a;
    a.nterms = nterms;
    bool al = ((uintptr_t)Mp | (uintptr_t)Mt) % 16 == 0;
    for (int i = 0; i < nterms; ++i) {
        a.t[i] = terms[i];
        al = al && (((uintptr_t)terms[i].op | (uintptr_t)terms[i].dA) % 16 == 0);
    }
    const bool v4 = (R % 4 == 0) && al;
    const int VEC = v4 ? 4 : 1;
    const int64_t nout = (int64_t)sx * (R / VEC);
    int maxs = 1;
    for (int i = 0; i < nterms; ++i) maxs = terms[i].sy > maxs ? terms[i].sy : maxs;
    int KS = 1;
    while (KS < 32 && KS < maxs && nout * KS < 152LL * 2 * 256) KS *= 2;
    const int TX = 256 / KS;
    const unsigned blocks = (unsigned)((nout + TX - 1) / TX);
    if (blocks == 0) return cudaSuccess;
    if (v4)
        k_pp_u<4><<<blocks, 256, 256 * sizeof(float4), st>>>(Mp, a, Mt, sx, R, TX, KS);
    else
        k_pp_u<1><<<blocks, 256, 256 * sizeof(float4), st>>>(Mp, a, Mt, sx, R, TX, KS);
    return cudaGetLastError();
}

}  // namespace cpk
