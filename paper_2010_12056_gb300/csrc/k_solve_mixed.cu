// Normal equations of one factor update, A(n) Gamma(n) = M(n) (Alg. 1 and
// Alg. 2, the solve step), solved to FP64 accuracy with FP32 factorisation plus FP64
// iterative refinement (Wilkinson; Moler, JACM 1967; Carson and Higham, SISC 2018).
//
// On this GPU an FP64 FMA has a 64-cycle dependent latency and 1/70 of the FP32
// throughput, so the sequential parts of a Cholesky factorisation and of
// triangular substitution are run in FP32, and FP64 is kept for work that is
// parallel across the R entries of a row:
//   k_gamma_form  Gamma = *_{k != n} S(k) and PP's W in FP64 (many blocks)
//   k_gj_inv      (one CTA) the FP32 inverse of the diagonally scaled Gamma by
//                 Gauss-Jordan elimination; if the scaled condition number is
//                 above 1e6 or a pivot is not positive, an FP64 LDL^T of Gamma
//                 instead, and the solve kernel substitutes in FP64.
//   k_solve_mixed (one block per row) m = M(x,:) [+ A_old(x,:) W];
//                 x0 = m G32;  repeat  r = m - x Gamma,  d = r G32,  x += d
//                 until the estimated remaining error ||d||_inf * rho is below
//                 2^-36 ||x||_inf (rho = contraction seen between iterations),
//                 four orders of magnitude below the FP32 rounding of M itself.
//                 For R <= 128 the residual (and V) is formed in double-float
//                 arithmetic on the FP32 pipe (about 2^-44 relative), with x and
//                 Gamma held as pairs of floats; above, in FP64.
#include <cuda_bf16.h>

#include <algorithm>

#include "cpals_internal.h"
#include "df_arith.h"
#include "pdl.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int MIXED_MAXR = 128;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
__device__ double block_sum_d(double v, double* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (lane < nw) ? sh[lane] : 0.0;
        t = warp_sum_d(t);
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

// ------------------------------------------------------------------ factorisation
// FP64 LDL^T of Gamma (global work, row stride R) into L (lower) / Lt (upper) and
// 1/L[j][j]: the fallback for ill-conditioned or indefinite Gamma.  Restarts once
// on Gamma + 1e-12 trace/R I.  Returns the flag (0, 1 shifted, 2 failed).
__device__ double chol_fp64(const double* G, int R, double tr, double* L, double* Lt, double* invd,
                            double* sinv, double* srs, int* sfail) {
    const int tid = threadIdx.x, nt = blockDim.x, RR = R * R;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    double* work = Lt;
    double flag = 0.0;
    bool bad = false;
    for (int attempt = 0; attempt < 2; ++attempt) {
        const double shift = attempt ? 1e-12 * tr / R : 0.0;
        for (int e = tid; e < RR; e += nt) work[e] = G[e] + ((e / R == e % R) ? shift : 0.0);
        if (attempt) flag = 1.0;
        __syncthreads();
        if (tid == 0) {
            const double d = work[0];
            *sfail = (!(d > 0.0) || !isfinite(d)) ? 1 : 0;
            if (!*sfail) sinv[0] = 1.0 / d;
        }
        __syncthreads();
        for (int j = 0; j < R && !*sfail; ++j) {
            const double inv = sinv[j];
            for (int i = j + 1 + warp; i < R; i += nw) {
                double* wi = work + (size_t)i * R;
                const double lij = wi[j] * inv;
                for (int k = j + 1 + lane; k <= i; k += 32) wi[k] = fma(-lij, work[k * R + j], wi[k]);
            }
            if (tid == 0 && j + 1 < R) {
                const double d = work[(j + 1) * R + j + 1];
                if (!(d > 0.0) || !isfinite(d)) *sfail = 1;
                else sinv[j + 1] = 1.0 / d;
            }
            __syncthreads();
        }
        const bool failed = *sfail != 0;
        __syncthreads();
        if (!failed) break;
        if (attempt == 1) {
            flag = 2.0;
            bad = true;
        }
    }
    for (int j = tid; j < R; j += nt) {
        const double v = bad ? 1.0 : 1.0 / sqrt(work[j * R + j]);
        srs[j] = v;
        invd[j] = v;
    }
    __syncthreads();
    for (int e = tid; e < RR; e += nt) {
        const int i = e / R, k = e % R;
        double v = 0.0;
        if (bad) v = (i == k) ? 1.0 : 0.0;
        else if (k < i) v = work[e] * srs[k];
        else if (k == i) v = 1.0 / srs[k];
        L[e] = v;
    }
    __syncthreads();
    for (int e = tid; e < RR; e += nt) Lt[e] = L[(e % R) * R + e / R];
    __syncthreads();
    return flag;
}

// Gamma (FP64) and PP's W for update n, element (i, j) = (row, column).
__device__ __forceinline__ double gamma_entry(const double* const* Sp, const double* const* dSp, int N,
                                              int n, int pp, size_t e, double* w_out) {
    double g = 1.0;
    for (int m = 0; m < N; ++m)
        if (m != n) g *= Sp[m][e];
    if (pp) {
        double acc = 0.0;
        for (int a = 0; a < N; ++a) {
            if (a == n) continue;
            for (int b = a + 1; b < N; ++b) {
                if (b == n) continue;
                double t = dSp[a][e] * dSp[b][e];
                for (int m = 0; m < N; ++m)
                    if (m != a && m != b && m != n) t *= Sp[m][e];
                acc += t;
            }
        }
        *w_out = acc;
    }
    return g;
}

// The same from the Grams' float pairs (R <= 128), in double-float arithmetic:
// the one formula for Gamma that every path of an update uses, so that a kernel
// that forms it (k_gamma_form, or the Gauss-Jordan kernel of an exact sweep)
// gives the same pairs.
__device__ __forceinline__ float2 gamma_entry_df(const float2* const* S2, const float2* const* dS2, int N, int n,
                                                 int pp, size_t e, float2* w_out) {
    float2 g = make_float2(1.f, 0.f);
    bool first = true;
    for (int m = 0; m < N; ++m) {
        if (m == n) continue;
        g = first ? S2[m][e] : cpdf::mul(g, S2[m][e]);
        first = false;
    }
    if (pp) {
        float ah = 0.f, al = 0.f;
        for (int a = 0; a < N; ++a) {
            if (a == n) continue;
            for (int b = a + 1; b < N; ++b) {
                if (b == n) continue;
                float2 t = cpdf::mul(dS2[a][e], dS2[b][e]);
                for (int m = 0; m < N; ++m)
                    if (m != a && m != b && m != n) t = cpdf::mul(t, S2[m][e]);
                cpdf::add(ah, al, t.x, t.y);
            }
        }
        *w_out = make_float2(ah, al);
    }
    return g;
}

// Gamma (FP64), its FP32 copy and PP's W, one entry per thread over many
// blocks: FP64 throughput per SM is low, so this work is spread over the GPU.
__global__ void __launch_bounds__(256) k_gamma_form(double* const* __restrict__ S_list,
                                                    double* const* __restrict__ dS_list, int N,
                                                    int n, int R, int pp, double* __restrict__ G,
                                                    float* __restrict__ G32, float* __restrict__ G2,
                                                    double* __restrict__ W, float* __restrict__ W2,
                                                    const float2* const* __restrict__ S2_list,
                                                    const float2* const* __restrict__ dS2_list) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= R * R) return;
    if (S2_list) {
        // R <= 128: from the Grams' float pairs
        float2 w = make_float2(0.f, 0.f);
        const float2 g = gamma_entry_df(S2_list, dS2_list, N, n, pp, (size_t)e, &w);
        G[e] = (double)g.x + (double)g.y;
        G32[e] = g.x;
        reinterpret_cast<float2*>(G2)[e] = g;
        if (pp) {
            W[e] = (double)w.x + (double)w.y;
            reinterpret_cast<float2*>(W2)[e] = w;
        }
        return;
    }
    const double* Sp[CP_MAXN];
    const double* dSp[CP_MAXN];
    for (int k = 0; k < N; ++k) {
        Sp[k] = S_list[k];
        dSp[k] = pp ? dS_list[k] : nullptr;
    }
    double w = 0.0;
    const double g = gamma_entry(Sp, dSp, N, n, pp, (size_t)e, &w);
    G[e] = g;
    const float gh = (float)g;
    G32[e] = gh;
    // float pairs (hi, lo) for the double-float refinement of the row solve
    G2[2 * e] = gh;
    G2[2 * e + 1] = (float)(g - (double)gh);
    if (pp) {
        W[e] = w;
        const float wh = (float)w;
        W2[2 * e] = wh;
        W2[2 * e + 1] = (float)(w - (double)wh);
    }
}

// R <= 128: explicit inverse of the diagonally scaled matrix
//   Gt = D Gamma D,  D = diag(Gamma)^(-1/2),   Ginv = D Gt^{-1} D,
// by Gauss-Jordan elimination without pivoting (Gt is SPD with unit diagonal, so
// its pivots are its LDL^T pivots) in FP32.  32 TY threads as a TY x 32 grid:
// thread (ty, tx) keeps rows ty IR + a (a < IR) of columns tx JC + b (b < JC) in
// registers.  Step k reads the pivot row and column of the matrix after step
// k - 1 from one of two shared buffers (their owners publish them after their
// own update, so each step has one barrier).  The step loop is unrolled by IR:
// the register slot of row k and of column k is then a compile-time constant.
// Row i != k: a_ij <- a_ij - (a_ik / p) a_kj for j != k, a_ik <- -a_ik / p;
// row k: a_kj <- a_kj / p, a_kk <- 1 / p.  Scaling removes the part of Gamma's
// condition number that comes from unequal column norms; if the scaled
// condition number ||Gt||_inf ||Gt^{-1}||_inf exceeds 1e6 (refinement would
// contract too slowly) or a pivot is not positive, Gamma is factored in FP64
// (LDL^T) instead.
// The R Gauss-Jordan steps on register tiles a (an n x n SPD matrix with unit
// diagonal, padded with zeros) with the layout described above.  Returns false
// if a pivot is not positive.  Ends with a barrier.
template <int TY, int IR, int JC>
__device__ __forceinline__ bool gj_steps(float (&a)[IR][JC], int n, float (*prow)[MIXED_MAXR],
                                         float (*pcol)[MIXED_MAXR]) {
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int r0 = ty * IR, c0 = tx * JC;
    // publish row 0 and column 0
    if (ty == 0)
#pragma unroll
        for (int j = 0; j < JC; ++j) prow[0][c0 + j] = a[0][j];
    if (tx == 0)
#pragma unroll
        for (int i = 0; i < IR; ++i) pcol[0][r0 + i] = a[i][0];
    __syncthreads();
    bool bad = false;
    for (int kb = 0; kb < n && !bad; kb += IR) {
        const bool own_rows = ty == kb / IR;  // this warp holds rows kb .. kb + IR - 1
#pragma unroll
        for (int kk = 0; kk < IR; ++kk) {
            const int k = kb + kk;
            if (k >= n) break;
            const int cur = k & 1;
            const float p = prow[cur][k];
            if (!(p > 0.f) || !isfinite(p)) {
                bad = true;
                break;
            }
            const float inv = __frcp_rn(p);
            const int jk = kk % JC;  // register slot of column k (constant once unrolled)
            const bool kcol = tx == k / JC;
            float rp[JC];
#pragma unroll
            for (int j = 0; j < JC; ++j) rp[j] = prow[cur][c0 + j];
            if (kcol) rp[jk] = 1.f;
            float f[IR];
#pragma unroll
            for (int i = 0; i < IR; i += 4) {
                const float4 v = *reinterpret_cast<const float4*>(&pcol[cur][r0 + i]);
                f[i] = v.x * inv;
                f[i + 1] = v.y * inv;
                f[i + 2] = v.z * inv;
                f[i + 3] = v.w * inv;
            }
#pragma unroll
            for (int i = 0; i < IR; ++i) {
                if (own_rows && i == kk) {
#pragma unroll
                    for (int j = 0; j < JC; ++j) a[i][j] = rp[j] * inv;
                } else {
#pragma unroll
                    for (int j = 0; j < JC; ++j) {
                        const float g = fmaf(-f[i], rp[j], a[i][j]);
                        a[i][j] = (j == jk && kcol) ? -f[i] : g;
                    }
                }
            }
            // owners of row / column k + 1 publish them for the next step
            const int k1 = k + 1;
            if (k1 < n) {
                const int nxt = cur ^ 1;
                const int i1 = (kk + 1) % IR, j1 = (kk + 1) % JC;
                if (ty == k1 / IR)
#pragma unroll
                    for (int j = 0; j < JC; ++j) prow[nxt][c0 + j] = a[i1][j];
                if (tx == k1 / JC)
#pragma unroll
                    for (int i = 0; i < IR; i += 4)
                        *reinterpret_cast<float4*>(&pcol[nxt][r0 + i]) =
                            make_float4(a[i][j1], a[i + 1][j1], a[i + 2][j1], a[i + 3][j1]);
            }
            __syncthreads();
        }
    }
    __syncthreads();
    return !bad;
}

template <int TY, int IR, int JC>
__global__ void __launch_bounds__(32 * TY, 1) k_gj_inv(float* __restrict__ G32, int R,
                                                       double* __restrict__ G,
                                                       float* __restrict__ Ginv,
                                                       double* __restrict__ L64,
                                                       double* __restrict__ invd64,
                                                       double* __restrict__ scal,
                                                       int* __restrict__ mode,
                                                       const float2* const* __restrict__ S2_list,
                                                       int N, int n, float2* __restrict__ G2) {
    constexpr int NT = 32 * TY, RMAX = TY * IR;
    static_assert(RMAX <= MIXED_MAXR && 32 * JC <= MIXED_MAXR && IR % JC == 0 && IR % 4 == 0,
                  "tile shape");
    __shared__ double red[32];
    __shared__ double sinv[CP_MAXR], srs[CP_MAXR];
    __shared__ __align__(16) float prow[2][MIXED_MAXR];
    __shared__ __align__(16) float pcol[2][MIXED_MAXR];
    __shared__ float dsc[MIXED_MAXR];
    __shared__ int sfail;
    __shared__ unsigned gmax_bits, imax_bits;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int r0 = ty * IR, c0 = tx * JC;
    if (tid == 0) {
        sfail = (R > RMAX || R > 32 * JC) ? 1 : 0;
        gmax_bits = 0u;
        imax_bits = 0u;
    }
    __syncthreads();
    // S2_list: an exact sweep's update with R <= 128 forms Gamma here from the
    // Grams' float pairs (the product order of k_gamma_form, so the same pairs),
    // writing its pairs and FP32 copy; its FP64 copy only if the FP64
    // factorisation is needed.  The thread's entries of each Gram are loaded at
    // once (IR rows x JC columns), one round of loads per Gram.
    float a[IR][JC];
    if (S2_list) {
        float2 acc[IR][JC];
        bool first = true;
        for (int m = 0; m < N; ++m) {
            if (m == n) continue;
            const float2* Sm = S2_list[m];
            float2 v[IR][JC];
#pragma unroll
            for (int i = 0; i < IR; ++i)
#pragma unroll
                for (int j = 0; j < JC; ++j) {
                    const int r = r0 + i, c = c0 + j;
                    v[i][j] = (r < R && c < R) ? Sm[(size_t)r * R + c] : make_float2(0.f, 0.f);
                }
#pragma unroll
            for (int i = 0; i < IR; ++i)
#pragma unroll
                for (int j = 0; j < JC; ++j) acc[i][j] = first ? v[i][j] : cpdf::mul(acc[i][j], v[i][j]);
            first = false;
        }
#pragma unroll
        for (int i = 0; i < IR; ++i)
#pragma unroll
            for (int j = 0; j < JC; ++j) {
                const int r = r0 + i, c = c0 + j;
                a[i][j] = acc[i][j].x;
                if (r < R && c < R) {
                    const size_t e = (size_t)r * R + c;
                    G2[e] = acc[i][j];
                    G32[e] = acc[i][j].x;
                    if (r == c) {
                        const float g = acc[i][j].x;
                        const float d = (g > 0.f && isfinite(g)) ? rsqrtf(g) : 0.f;
                        if (!(d > 0.f)) sfail = 1;
                        dsc[r] = d;
                    }
                }
            }
    } else {
        for (int r = tid; r < MIXED_MAXR; r += NT) {
            float d = 0.f;
            if (r < R) {
                const float g = G32[(size_t)r * R + r];
                d = (g > 0.f && isfinite(g)) ? rsqrtf(g) : 0.f;
                if (!(d > 0.f)) sfail = 1;
            }
            dsc[r] = d;
        }
#pragma unroll
        for (int i = 0; i < IR; ++i)
#pragma unroll
            for (int j = 0; j < JC; ++j) {
                const int r = r0 + i, c = c0 + j;
                a[i][j] = (r < R && c < R) ? G32[(size_t)r * R + c] : 0.f;
            }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IR; ++i)
#pragma unroll
        for (int j = 0; j < JC; ++j) {
            const int r = r0 + i, c = c0 + j;
            a[i][j] = (r < R && c < R) ? a[i][j] * (dsc[r] * dsc[c]) : 0.f;
        }
    // ||Gt||_inf: a warp holds whole rows
#pragma unroll
    for (int i = 0; i < IR; ++i) {
        float rs = 0.f;
#pragma unroll
        for (int j = 0; j < JC; ++j) rs += fabsf(a[i][j]);
#pragma unroll
        for (int o = 16; o; o >>= 1) rs += __shfl_xor_sync(FULL, rs, o);
        if (tx == 0 && r0 + i < R) atomicMax(&gmax_bits, __float_as_uint(rs));
    }
    bool use64 = sfail != 0;
    if (!use64) use64 = !gj_steps<TY, IR, JC>(a, R, prow, pcol);
    if (!use64) {
#pragma unroll
        for (int i = 0; i < IR; ++i) {
            float rs = 0.f;
#pragma unroll
            for (int j = 0; j < JC; ++j) rs += fabsf(a[i][j]);
#pragma unroll
            for (int o = 16; o; o >>= 1) rs += __shfl_xor_sync(FULL, rs, o);
            if (tx == 0 && r0 + i < R) atomicMax(&imax_bits, __float_as_uint(rs));
        }
        __syncthreads();
        const float kappa = __uint_as_float(gmax_bits) * __uint_as_float(imax_bits);
        use64 = !(kappa <= 1e6f);
    }
    if (use64) {
        if (S2_list) {
            // the FP64 copy of Gamma for the FP64 factorisation (its pairs, written
            // above by this CTA, are visible after the barrier)
            __syncthreads();
            for (int e = tid; e < R * R; e += NT) G[e] = (double)G2[e].x + (double)G2[e].y;
            __syncthreads();
        }
        double tr = 0.0;
        for (int j = tid; j < R; j += NT) tr += G[(size_t)j * R + j];
        tr = block_sum_d(tr, red);
        const double flag = chol_fp64(G, R, tr, L64, L64 + (size_t)R * R, invd64, sinv, srs, &sfail);
        if (tid == 0) {
            scal[SCAL_FLAGS] = 10.0 + flag;  // FP64 path: 10 ok, 11 shifted, 12 failed
            scal[SCAL_GS] = 0.0;
            *mode = 1;
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < IR; ++i) {
        const int r = r0 + i;
        if (r >= R) break;
#pragma unroll
        for (int j = 0; j < JC; ++j) {
            const int c = c0 + j;
            if (c < R) Ginv[(size_t)r * R + c] = a[i][j] * (dsc[r] * dsc[c]);
        }
    }
    if (tid == 0) {
        scal[SCAL_FLAGS] = 0.0;
        scal[SCAL_GS] = 0.0;
        *mode = 0;
    }
}

// ------------------------------------------------------------------ 128 < R <= 512
// Gt = D Gamma D is inverted in FP32 by block Gauss-Jordan elimination with
// blocks of b = 128 (the scalar elimination of the single-CTA kernel above,
// reordered by blocks): for each diagonal block K, P = Gt_KK^{-1} (Gauss-Jordan
// kernel), U = P Gt_K*, Gt_ij -= Gt_iK U_Kj and Gt_iK = -Gt_iK P for i, j not in
// K, Gt_K* = U, Gt_KK = P.  One Newton-Schulz step W <- 2W - W Gt W then squares
// the inverse's error.  (The recursive Schur-complement formula used before
// loses accuracy on collinear factors: measured rho(I - W Gt) = 1.002 at R = 400,
// against 0.027 for block elimination and 7e-4 after the Newton-Schulz step.)
// The accuracy is checked a posteriori: e = ||I - Gt W||_inf before the step
// bounds the refinement's contraction after it by about e^2; if e > 1/4, or a
// block pivot fails, the FP64 factorisation runs instead.

// Gt = D G32 D (FP32, row stride R) and ||Gt||_inf; flags[0] = 0
__global__ void __launch_bounds__(256) k_scale_big(const float* __restrict__ G32, int R, float* __restrict__ Gt,
                                                   float* __restrict__ dvec, unsigned* __restrict__ flags) {
    __shared__ float dsc[CP_MAXR];
    const int tid = threadIdx.x;
    for (int r = tid; r < R; r += blockDim.x) {
        const float g = G32[(size_t)r * R + r];
        const float d = (g > 0.f && isfinite(g)) ? rsqrtf(g) : 0.f;
        dsc[r] = d;
        dvec[r] = d;
        if (!(d > 0.f)) atomicOr(flags, 1u);
    }
    __syncthreads();
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
        float rs = 0.f;
        for (int c = tid; c < R; c += blockDim.x) {
            const float v = G32[(size_t)r * R + c] * (dsc[r] * dsc[c]);
            Gt[(size_t)r * R + c] = v;
            rs += fabsf(v);
        }
        for (int o = 16; o; o >>= 1) rs += __shfl_xor_sync(FULL, rs, o);
        __shared__ float wsum[8];
        if ((tid & 31) == 0) wsum[tid >> 5] = rs;
        __syncthreads();
        if (tid == 0) {
            float t = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
            atomicMax(flags + 1, __float_as_uint(t));
        }
        __syncthreads();
    }
}

// inverse of an n x n block (n <= 128) of an SPD matrix: src row stride lds,
// dst row stride ldd; flags[0] |= 2 if a pivot fails
template <int TY, int IR, int JC>
__global__ void __launch_bounds__(32 * TY, 1) k_gj_block(const float* __restrict__ src, int lds, int n,
                                                         float* __restrict__ dst, int ldd,
                                                         unsigned* __restrict__ flags) {
    __shared__ __align__(16) float prow[2][MIXED_MAXR];
    __shared__ __align__(16) float pcol[2][MIXED_MAXR];
    __shared__ float dsc[MIXED_MAXR];
    __shared__ int sfail;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int r0 = ty * IR, c0 = tx * JC;
    if (tid == 0) sfail = 0;
    __syncthreads();
    for (int r = tid; r < MIXED_MAXR; r += 32 * TY) {
        float d = 0.f;
        if (r < n) {
            const float g = src[(size_t)r * lds + r];
            d = (g > 0.f && isfinite(g)) ? rsqrtf(g) : 0.f;
            if (!(d > 0.f)) sfail = 1;
        }
        dsc[r] = d;
    }
    __syncthreads();
    float a[IR][JC];
#pragma unroll
    for (int i = 0; i < IR; ++i)
#pragma unroll
        for (int j = 0; j < JC; ++j) {
            const int r = r0 + i, c = c0 + j;
            a[i][j] = (r < n && c < n) ? src[(size_t)r * lds + c] * (dsc[r] * dsc[c]) : 0.f;
        }
    bool ok = sfail == 0;
    if (ok) ok = gj_steps<TY, IR, JC>(a, n, prow, pcol);
    if (!ok) {
        if (tid == 0) atomicOr(flags, 2u);
        return;
    }
#pragma unroll
    for (int i = 0; i < IR; ++i)
#pragma unroll
        for (int j = 0; j < JC; ++j) {
            const int r = r0 + i, c = c0 + j;
            if (r < n && c < n) dst[(size_t)r * ldd + c] = a[i][j] * (dsc[r] * dsc[c]);
        }
}

// C = beta Cin + alpha op(A) op(B) (FP32), op(X) = X or X^T; 32 x 32 output tile
// per block of 256 threads (2 x 2 per thread)
__global__ void __launch_bounds__(256) k_gemm_small(int M, int N, int K, float alpha, const float* __restrict__ A,
                                                    int lda, int ta, const float* __restrict__ B, int ldb, int tb,
                                                    float beta, const float* __restrict__ Cin, int ldci,
                                                    float* __restrict__ C, int ldc) {
    __shared__ float As[32][33], Bs[32][33];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int k0 = 0; k0 < K; k0 += 32) {
        for (int e = tid; e < 32 * 32; e += 256) {
            const int i = e >> 5, kk = e & 31;
            const int gm = m0 + i, gk = k0 + kk;
            As[i][kk] = (gm < M && gk < K) ? (ta ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : 0.f;
            const int gn = n0 + i;
            Bs[kk][i] = (gn < N && gk < K) ? (tb ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn]) : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const float a0 = As[ty][kk], a1 = As[ty + 16][kk];
            const float b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
            acc[0][0] = fmaf(a0, b0, acc[0][0]);
            acc[0][1] = fmaf(a0, b1, acc[0][1]);
            acc[1][0] = fmaf(a1, b0, acc[1][0]);
            acc[1][1] = fmaf(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
            if (gm < M && gn < N)
                C[(size_t)gm * ldc + gn] = alpha * acc[i][j] + (Cin ? beta * Cin[(size_t)gm * ldci + gn] : 0.f);
        }
}

// block elimination step on the whole matrix W (row stride R): rows of block K
// [k0, k1) become U (or P on the diagonal block); the rest of block K's columns
// become -C_K P; everything else gets W -= C_K U.  C_K is a copy of W's block
// columns taken before the step (R x bk), so every element is read and written by
// one thread only.  One thread per element, 256 threads per block.
__global__ void __launch_bounds__(256) k_bgj_update(float* __restrict__ W, int R, int k0, int bk,
                                                    const float* __restrict__ Ck, const float* __restrict__ U,
                                                    const float* __restrict__ P) {
    const int64_t n = (int64_t)R * R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / R), j = (int)(e % R);
        const bool ik = i >= k0 && i < k0 + bk, jk = j >= k0 && j < k0 + bk;
        float v;
        if (ik) {
            v = jk ? P[(size_t)(i - k0) * bk + (j - k0)] : U[(size_t)(i - k0) * R + j];
        } else if (jk) {
            float acc = 0.f;
            const float* c = Ck + (size_t)i * bk;
            for (int t = 0; t < bk; ++t) acc = fmaf(c[t], P[(size_t)t * bk + (j - k0)], acc);
            v = -acc;
        } else {
            float acc = W[e];
            const float* c = Ck + (size_t)i * bk;
            for (int t = 0; t < bk; ++t) acc = fmaf(-c[t], U[(size_t)t * R + j], acc);
            v = acc;
        }
        W[e] = v;
    }
}

// dst (R x bk, row stride bk) = W[:, k0 .. k0 + bk)
__global__ void __launch_bounds__(256) k_copy_cols(const float* __restrict__ W, int R, int k0, int bk,
                                                   float* __restrict__ dst) {
    const int64_t n = (int64_t)R * bk;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / bk), t = (int)(e % bk);
        dst[e] = W[(size_t)i * R + k0 + t];
    }
}

// Ginv = D W D from the inverse W of Gt (row stride R) after the Newton-Schulz
// step, with the path decision from Y = Gt W0 (W0 the inverse before the step):
// e = ||I - Y||_inf <= 1/4 and no failed pivot -> FP32 inverse + refinement
__global__ void __launch_bounds__(256) k_inv_finish(int R, const float* __restrict__ Wi, const float* __restrict__ Y,
                                                    const float* __restrict__ dvec, float* __restrict__ Ginv,
                                                    unsigned* __restrict__ flags, double* __restrict__ scal,
                                                    int* __restrict__ mode) {
    __shared__ float wsum[8];
    __shared__ unsigned emax_bits;
    const int tid = threadIdx.x;
    if (tid == 0) emax_bits = 0u;
    __syncthreads();
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
        float rs = 0.f;
        for (int c = tid; c < R; c += blockDim.x) {
            Ginv[(size_t)r * R + c] = Wi[(size_t)r * R + c] * (dvec[r] * dvec[c]);
            rs += fabsf((r == c ? 1.f : 0.f) - Y[(size_t)r * R + c]);
        }
        for (int o = 16; o; o >>= 1) rs += __shfl_xor_sync(FULL, rs, o);
        if ((tid & 31) == 0) wsum[tid >> 5] = rs;
        __syncthreads();
        if (tid == 0) {
            float t = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
            atomicMax(&emax_bits, __float_as_uint(isfinite(t) ? t : 1e30f));
        }
        __syncthreads();
    }
    if (tid == 0) atomicMax(flags + 2, emax_bits);
    // the last block decides (blocks count themselves in flags[3])
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned done = atomicAdd(flags + 3, 1u);
        if (done == gridDim.x - 1) {
            __threadfence();
            const float e = __uint_as_float(atomicOr(flags + 2, 0u));
            const bool ok = atomicOr(flags, 0u) == 0u && e <= 0.25f;
            *mode = ok ? 0 : 1;
            scal[SCAL_FLAGS] = 0.0;
            scal[SCAL_GS] = 0.0;
        }
    }
}

// the FP64 factorisation on request (every update)
__global__ void k_choose_fp64(int* __restrict__ mode) {
    if (threadIdx.x == 0) *mode = 1;
}

// FP64 LDL^T of Gamma when the blocked FP32 inverse was not usable (*mode == 1)
__global__ void __launch_bounds__(1024) k_chol_fp64_if(const double* __restrict__ G, int R,
                                                       double* __restrict__ L64, double* __restrict__ invd64,
                                                       double* __restrict__ scal, const int* __restrict__ mode) {
    __shared__ double red[32];
    __shared__ double sinv[CP_MAXR], srs[CP_MAXR];
    __shared__ int sfail;
    if (*mode == 0) return;
    double tr = 0.0;
    for (int j = threadIdx.x; j < R; j += blockDim.x) tr += G[(size_t)j * R + j];
    tr = block_sum_d(tr, red);
    const double flag = chol_fp64(G, R, tr, L64, L64 + (size_t)R * R, invd64, sinv, srs, &sfail);
    if (threadIdx.x == 0) scal[SCAL_FLAGS] = 10.0 + flag;
}

// ------------------------------------------------------------------ row solves
__device__ __forceinline__ void bf16_split(float x, uint16_t& hi, uint16_t& lo) {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
}

constexpr int SOLVE_THREADS = 64;

// shared layout of the solve kernel (doubles unless noted)
struct SolveSmem {
    size_t G, Gi, m, x, r, part, red, pk, total;
};
__host__ __device__ inline SolveSmem solve_smem(int R) {
    // R > 128 solves in FP64 straight from global memory: no staged matrices
    SolveSmem L;
    const bool staged = R <= MIXED_MAXR;
    const size_t RR = staged ? (size_t)R * R : 0;
    const size_t RRp = (RR + 1) & ~(size_t)1;
    L.G = 0;                                   // RR doubles (or padded R x (R+1) FP64 factor)
    L.Gi = staged ? (((size_t)R * (R + 1) + 1) & ~(size_t)1) : 0;  // RR floats
    L.m = L.Gi + (staged ? RRp / 2 + 2 : 0);
    L.x = L.m + R;
    L.r = L.x + R;                             // R floats
    L.part = L.r + (R + 1) / 2 + 1;            // SOLVE_THREADS doubles
    L.red = L.part + SOLVE_THREADS;            // 2 * SOLVE_THREADS / 32 doubles
    L.pk = L.red + 16;                         // k-split partials: 3 R doubles + 3 R floats
    L.total = L.pk + 5 * (size_t)R;
    return L;
}

using cpdf::fast_two_sum;
using cpdf::two_sum;
__device__ __forceinline__ void df_fma(float vh, float vl, float2 p, float& ah, float& al) {
    cpdf::fma_acc(vh, vl, p.x, p.y, ah, al);
}
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) { cpdf::add(ah, al, bh, bl); }

// h[c] + l[c] = sum_{k0 <= k < k1} (vh[k] + vl[k]) P[k][jj[c]]  (two chains per column)
template <int CT>
__device__ __forceinline__ void df_dot(const float* vh, const float* vl, const float2* __restrict__ P, int R,
                                       int k0, int k1, const int (&jj)[CT], float (&h)[CT], float (&l)[CT]) {
    float h2[CT], l2[CT];
#pragma unroll
    for (int c = 0; c < CT; ++c) h[c] = l[c] = h2[c] = l2[c] = 0.f;
    int k = k0;
    for (; k + 1 < k1; k += 2) {
        const float a0 = vh[k], b0 = vl[k], a1 = vh[k + 1], b1 = vl[k + 1];
        const float2* p0 = P + (size_t)k * R;
        const float2* p1 = p0 + R;
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            df_fma(a0, b0, p0[jj[c]], h[c], l[c]);
            df_fma(a1, b1, p1[jj[c]], h2[c], l2[c]);
        }
    }
    if (k < k1) {
        const float2* p0 = P + (size_t)k * R;
#pragma unroll
        for (int c = 0; c < CT; ++c) df_fma(vh[k], vl[k], p0[jj[c]], h[c], l[c]);
    }
#pragma unroll
    for (int c = 0; c < CT; ++c) df_add(h[c], l[c], h2[c], l2[c]);
}

// One row x per block of KS groups of 64 threads; thread t of a group owns the
// columns t + 64 c (c < CT), each group sums its 1/KS share of every dot product
// of those columns, and the shares meet in shared memory.  Per refinement step:
//   r = m - x Gamma   R <= 128: in double-float arithmetic on the FP32 pipe, x =
//                     xh + xl and Gamma = Gh + Gl (staged as float pairs), exact
//                     leading products, about 2^-44 relative accuracy;
//                     R > 128: FP64, Gamma read from L2
//   d = r G32         (FP32; r is small, so FP32 carries it to full accuracy)
//   x += d
// GB300's FP64 pipe retires about 1.6 FMAs per cycle per SM, so an FP64 residual
// of a 64-column row took about 5 us per step; the double-float one needs a
// tenth of the issue slots of the FP32 pipe.  The iteration stops once the error
// left after the step, estimated as rho ||d||_inf with rho the contraction seen
// between steps, is below 2^-36 ||x||_inf (far below the FP32 error of the
// MTTKRP that forms m), or once the steps stop contracting at the residual's
// rounding floor, if that floor is below 2^-20 ||x||_inf.
template <int RT, int KS>
__global__ void __launch_bounds__(SOLVE_THREADS * KS, 1) k_solve_mixed(
    const float* __restrict__ M, const double* __restrict__ W, const float2* __restrict__ W2,
    const double* __restrict__ G, const float2* __restrict__ G2, const float* __restrict__ Ginv,
    const double* __restrict__ L64, const double* __restrict__ invd64, const int* __restrict__ mode,
    cpk::SolveOut o, int s, int R, double* __restrict__ scal, double* __restrict__ scal_part,
    unsigned* __restrict__ dev_err) {
    constexpr bool DF = RT <= 4;       // R <= 128: staged matrices, double-float refinement
    constexpr int CT = (RT + 1) / 2;   // columns per thread in the refinement path
    extern __shared__ __align__(16) double sm[];
    __shared__ __align__(8) uint64_t bar;
    const SolveSmem lay = solve_smem(R);
    double* sG = sm + lay.G;
    const float2* sG2 = reinterpret_cast<const float2*>(sm + lay.G);
    float* sGi = reinterpret_cast<float*>(sm + lay.Gi);
    double* mv = sm + lay.m;
    double* xv = sm + lay.x;
    float* xh_s = reinterpret_cast<float*>(sm + lay.x);   // double-float x: hi then lo
    float* xl_s = xh_s + R;
    float* rv = reinterpret_cast<float*>(sm + lay.r);
    double* part = sm + lay.part;
    float* redf = reinterpret_cast<float*>(sm + lay.red);   // warp maxima of the step and of x
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // KS groups of 64 threads: group q sums its 1/KS share of every dot product of
    // the refinement; group 0 owns the columns (tcol + 64 c) and everything else
    const int q = tid / SOLVE_THREADS, tcol = tid % SOLVE_THREADS;
    double* pk = sm + lay.pk;                                      // (KS-1) x R FP64 partials
    float2* pk2 = reinterpret_cast<float2*>(sm + lay.pk);          // (KS-1) x R double-float partials
    float* pkf = reinterpret_cast<float*>(sm + lay.pk + 3 * (size_t)R);  // (KS-1) x R FP32 partials
    const int kq = (R + KS - 1) / KS, k0 = q * kq, k1 = min(R, k0 + kq);
    const int x = blockIdx.x;
    pdl::wait();
    pdl::trigger();
    const int path = *mode;
    const int RR = R * R;
    double sc[CP_NSCAL];
#pragma unroll
    for (int i = 0; i < CP_NSCAL; ++i) sc[i] = 0.0;
    double xj[CT], mj[CT], aold[CT];
    float mh[CT], ml[CT], xh[CT], xl[CT];
    int jj[CT];
#pragma unroll
    for (int c = 0; c < CT; ++c) {
        const int j = tcol + SOLVE_THREADS * c;
        jj[c] = j < R ? j : 0;  // idle columns read column 0 and are dropped
        xj[c] = 0.0;
        xh[c] = xl[c] = 0.f;
        aold[c] = (j < R) ? o.A64[(size_t)x * R + j] : 0.0;
        mh[c] = (j < R) ? M[(size_t)x * R + j] : 0.f;
        ml[c] = 0.f;
        mj[c] = 0.0;
        if constexpr (!DF) mj[c] = (double)mh[c];
    }
    float fv2 = 0.f;   // double-float path: ||V||^2 of this thread's columns

    if (path == 0) {
        // R <= 128: stage Gamma (as float pairs, or FP64 above) and G32 with two
        // bulk copies (sizes rounded up to 16 bytes; the sources have 16 spare bytes)
        const float* Gim = DF ? sGi : Ginv;
        const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
        const uint32_t bytesG = (uint32_t)((RR * 8 + 15) & ~15), bytesGi = (uint32_t)((RR * 4 + 15) & ~15);
        if (DF && tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytesG + bytesGi)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    (uint32_t)__cvta_generic_to_shared(sG)),
                "l"(G2), "r"(bytesG), "r"(b)
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    (uint32_t)__cvta_generic_to_shared(sGi)),
                "l"(Ginv), "r"(bytesGi), "r"(b)
                : "memory");
        }
        __syncthreads();  // the barrier is initialised before any thread waits on it
        if (W) {
            // V(x,:) = A_old(x,:) W (Eq. V_nij), added to m
            if constexpr (DF) {
#pragma unroll
                for (int c = 0; c < CT; ++c) {
                    const int j = tcol + SOLVE_THREADS * c;
                    if (q == 0 && j < R) {
                        const float ah = (float)aold[c];
                        xh_s[j] = ah;
                        xl_s[j] = (float)(aold[c] - (double)ah);
                    }
                }
                __syncthreads();
                float vh[CT], vl[CT];
                df_dot<CT>(xh_s, xl_s, W2, R, k0, k1, jj, vh, vl);
                if (KS > 1) {
                    if (q > 0)
#pragma unroll
                        for (int c = 0; c < CT; ++c) {
                            const int j = tcol + SOLVE_THREADS * c;
                            if (j < R) pk2[(size_t)(q - 1) * R + j] = make_float2(vh[c], vl[c]);
                        }
                    __syncthreads();
                    if (q == 0)
#pragma unroll
                        for (int c = 0; c < CT; ++c) {
                            const int j = tcol + SOLVE_THREADS * c;
                            if (j < R)
                                for (int g = 1; g < KS; ++g) {
                                    const float2 t = pk2[(size_t)(g - 1) * R + j];
                                    df_add(vh[c], vl[c], t.x, t.y);
                                }
                        }
                }
                if (q == 0)
#pragma unroll
                    for (int c = 0; c < CT; ++c) {
                        const int j = tcol + SOLVE_THREADS * c;
                        if (j >= R) continue;
                        const float vf = __fadd_rn(vh[c], vl[c]);
                        fv2 = fmaf(vf, vf, fv2);
                        float sh, sl;
                        two_sum(mh[c], vh[c], sh, sl);
                        sl = __fadd_rn(sl, vl[c]);
                        fast_two_sum(sh, sl, mh[c], ml[c]);
                    }
            } else {
#pragma unroll
                for (int c = 0; c < CT; ++c) {
                    const int j = tcol + SOLVE_THREADS * c;
                    if (q == 0 && j < R) xv[j] = aold[c];
                }
                __syncthreads();
                if (q == 0) {
#pragma unroll
                    for (int c = 0; c < CT; ++c) {
                        const int j = tcol + SOLVE_THREADS * c;
                        if (j >= R) continue;
                        double v0 = 0.0, v1 = 0.0;
                        int k = 0;
                        for (; k + 1 < R; k += 2) {
                            v0 = fma(xv[k], W[(size_t)k * R + j], v0);
                            v1 = fma(xv[k + 1], W[(size_t)(k + 1) * R + j], v1);
                        }
                        if (k < R) v0 = fma(xv[k], W[(size_t)k * R + j], v0);
                        const double v = v0 + v1;
                        mj[c] += v;
                        sc[SCAL_V2] += v * v;
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            const int j = tcol + SOLVE_THREADS * c;
            if (q == 0 && j < R) rv[j] = DF ? __fadd_rn(mh[c], ml[c]) : (float)mj[c];
        }
        // bounded wait for the staged matrices (about 1 s)
        if (DF) {
            const long long t0 = clock64();
            uint32_t ok = 0;
            int give_up = 0;
            while (!ok) {
                asm volatile(
                    "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                    "selp.u32 %0, 1, 0, p;\n\t}"
                    : "=r"(ok)
                    : "r"(b)
                    : "memory");
                if (!ok && clock64() - t0 > 2000000000LL) {
                    give_up = 1;
                    break;
                }
            }
            if (give_up) {
                if (tid == 0) atomicOr(dev_err, (unsigned)DEVERR_TIMEOUT);
                return;
            }
        }
        __syncthreads();
        // d = rv G32 for the owned columns (FP32, four partial sums over this
        // group's k share; the groups' shares meet in shared memory)
        auto apply_ginv = [&](float* d) {
#pragma unroll
            for (int c = 0; c < CT; ++c) {
                const int j = tcol + SOLVE_THREADS * c;
                float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
                if (j < R) {
                    int k = k0;
                    for (; k + 3 < k1; k += 4) {
                        a0 = fmaf(rv[k], Gim[k * R + j], a0);
                        a1 = fmaf(rv[k + 1], Gim[(k + 1) * R + j], a1);
                        a2 = fmaf(rv[k + 2], Gim[(k + 2) * R + j], a2);
                        a3 = fmaf(rv[k + 3], Gim[(k + 3) * R + j], a3);
                    }
                    for (; k < k1; ++k) a0 = fmaf(rv[k], Gim[k * R + j], a0);
                }
                d[c] = (a0 + a1) + (a2 + a3);
            }
            if (KS > 1) {
                if (q > 0)
#pragma unroll
                    for (int c = 0; c < CT; ++c) {
                        const int j = tcol + SOLVE_THREADS * c;
                        if (j < R) pkf[(size_t)(q - 1) * R + j] = d[c];
                    }
                __syncthreads();
                if (q == 0)
#pragma unroll
                    for (int c = 0; c < CT; ++c) {
                        const int j = tcol + SOLVE_THREADS * c;
                        if (j < R)
                            for (int g = 1; g < KS; ++g) d[c] += pkf[(size_t)(g - 1) * R + j];
                    }
            }
        };
        float d0[CT];
        apply_ginv(d0);
        float dmx = 0.f, xmx = 0.f;
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            const int j = tcol + SOLVE_THREADS * c;
            if constexpr (!DF) xj[c] = (double)d0[c];
            xh[c] = d0[c];
            xl[c] = 0.f;
            if (q == 0 && j < R) {
                if (DF) {
                    xh_s[j] = d0[c];
                    xl_s[j] = 0.f;
                } else {
                    xv[j] = xj[c];
                }
            }
        }
        __syncthreads();
        float prev = 0.f;
        bool conv = false;
        for (int itr = 0; itr < 30; ++itr) {
            if constexpr (DF) {
                // r = m - x Gamma in double-float arithmetic
                float th[CT], tl[CT];
                df_dot<CT>(xh_s, xl_s, sG2, R, k0, k1, jj, th, tl);
                if (KS > 1) {
                    if (q > 0)
#pragma unroll
                        for (int c = 0; c < CT; ++c) {
                            const int j = tcol + SOLVE_THREADS * c;
                            if (j < R) pk2[(size_t)(q - 1) * R + j] = make_float2(th[c], tl[c]);
                        }
                    __syncthreads();
                }
                if (q == 0)
#pragma unroll
                    for (int c = 0; c < CT; ++c) {
                        const int j = tcol + SOLVE_THREADS * c;
                        if (j < R) {
                            for (int g = 1; g < KS; ++g) {
                                const float2 t = pk2[(size_t)(g - 1) * R + j];
                                df_add(th[c], tl[c], t.x, t.y);
                            }
                            // m - S: the leading difference is exact when the two
                            // are close (Sterbenz), so r keeps its own 24 bits
                            rv[j] = __fadd_rn(__fsub_rn(mh[c], th[c]), __fsub_rn(ml[c], tl[c]));
                        }
                    }
            } else {
                // r = m - x Gamma (FP64).  NQ partial sums per column, the thread's
                // columns interleaved: NQ CT independent chains cover the FP64 FMA
                // latency (64 cycles) with the few warps a row has
                constexpr int NQ = CT <= 4 ? 8 : 4;
                double ra[CT][NQ];
#pragma unroll
                for (int c = 0; c < CT; ++c)
#pragma unroll
                    for (int u = 0; u < NQ; ++u) ra[c][u] = 0.0;
                int k = k0;
                for (; k + NQ - 1 < k1; k += NQ) {
#pragma unroll
                    for (int u = 0; u < NQ; ++u) {
                        const double xk = xv[k + u];
                        const double* grow = G + (size_t)(k + u) * R;
#pragma unroll
                        for (int c = 0; c < CT; ++c) ra[c][u] = fma(xk, grow[jj[c]], ra[c][u]);
                    }
                }
                for (; k < k1; ++k) {
#pragma unroll
                    for (int c = 0; c < CT; ++c) ra[c][0] = fma(xv[k], G[(size_t)k * R + jj[c]], ra[c][0]);
                }
                double tt[CT];
#pragma unroll
                for (int c = 0; c < CT; ++c) {
                    if (NQ == 8)
                        tt[c] = ((ra[c][0] + ra[c][1]) + (ra[c][2] + ra[c][3])) +
                                ((ra[c][4 % NQ] + ra[c][5 % NQ]) + (ra[c][6 % NQ] + ra[c][7 % NQ]));
                    else
                        tt[c] = (ra[c][0] + ra[c][1]) + (ra[c][2 % NQ] + ra[c][3 % NQ]);
                }
                if (KS > 1) {
                    if (q > 0)
#pragma unroll
                        for (int c = 0; c < CT; ++c) {
                            const int j = tcol + SOLVE_THREADS * c;
                            if (j < R) pk[(size_t)(q - 1) * R + j] = tt[c];
                        }
                    __syncthreads();
                }
                if (q == 0)
#pragma unroll
                    for (int c = 0; c < CT; ++c) {
                        const int j = tcol + SOLVE_THREADS * c;
                        if (j < R) {
                            double t = tt[c];
                            for (int g = 1; g < KS; ++g) t += pk[(size_t)(g - 1) * R + j];
                            rv[j] = (float)(mj[c] - t);
                        }
                    }
            }
            __syncthreads();
            float dd[CT];
            apply_ginv(dd);
            dmx = 0.f;
            xmx = 0.f;
            if (q == 0) {
#pragma unroll
                for (int c = 0; c < CT; ++c) {
                    const int j = tcol + SOLVE_THREADS * c;
                    dmx = fmaxf(dmx, fabsf(dd[c]));
                    if (DF) {
                        float s1, e1;
                        two_sum(xh[c], dd[c], s1, e1);
                        fast_two_sum(s1, __fadd_rn(e1, xl[c]), xh[c], xl[c]);
                        xmx = fmaxf(xmx, fabsf(xh[c]));
                        if (j < R) {
                            xh_s[j] = xh[c];
                            xl_s[j] = xl[c];
                        }
                    } else {
                        xj[c] += (double)dd[c];
                        xmx = fmaxf(xmx, fabsf((float)xj[c]));
                        if (j < R) xv[j] = xj[c];
                    }
                }
#pragma unroll
                for (int o2 = 16; o2; o2 >>= 1) {
                    dmx = fmaxf(dmx, __shfl_xor_sync(FULL, dmx, o2));
                    xmx = fmaxf(xmx, __shfl_xor_sync(FULL, xmx, o2));
                }
                if (lane == 0) {
                    redf[warp] = dmx;
                    redf[2 + warp] = xmx;
                }
            }
            __syncthreads();  // also publishes x for the next residual
            // in FP32: every thread evaluates the test, and each FP64 instruction
            // of a warp holds this GPU's FP64 pipe for tens of cycles
            const float dmax = fmaxf(redf[0], redf[1]), xmax = fmaxf(redf[2], redf[3]);
            // remaining error after this step is about rho * dmax, rho = dmax / prev
            const float rho = (itr > 0 && prev > 0.f) ? __fdiv_rn(dmax, prev) : 1.f;
            conv = rho * dmax <= 0x1.0p-36f * xmax || dmax == 0.f;
            // The residual's own rounding (about 2^-44 cond(Gamma) relative in
            // double-float, 2^-53 cond in FP64) is a floor the steps cannot go
            // below: once they stop contracting there (rho >= 0.9; a slower but
            // real contraction goes on to 2^-36), x is as accurate as this
            // residual can make it.  The floor is accepted up to 2^-20 ||x||: it is
            // above 2^-36 only for cond >= 2^8, and then the FP32-rounded m alone
            // moves the exact solution by about 2^-24 cond >= 2^-16.
            conv = conv || ((itr >= 2 && rho >= 0.9f) || itr == 29) && dmax <= 0x1.0p-20f * xmax;
            prev = dmax;
            if (conv) break;
            __syncthreads();  // redf[] is rewritten by the next step
        }
        if (tid == 0 && !conv) scal[SCAL_FLAGS] = 3.0;
        if constexpr (DF) {
            // outputs and scalar partials with FP64 only for what is stored in FP64:
            // the norms that steer the PP regime in FP32, <m, x> (Eq. residual, a
            // difference of nearly equal terms) in double-float
            float fs[5] = {0.f, 0.f, 0.f, 0.f, fv2};   // ||A||^2, ||dA_step||^2, ||A - A_p||^2, ||m||^2, ||V||^2
            float mah = 0.f, mal = 0.f;
            if (q == 0) {
#pragma unroll
                for (int c = 0; c < CT; ++c) {
                    const int j = tcol + SOLVE_THREADS * c;
                    if (j >= R) continue;
                    const size_t e = (size_t)x * R + j;
                    const double av = (double)xh[c] + (double)xl[c];
                    // every copy derives from the stored FP64 value, as after a restore
                    const float af = (float)av;
                    o.A64[e] = av;
                    if (o.A32) o.A32[e] = af;
                    if (o.bhi) {
                        uint16_t hi, lo;
                        bf16_split(af, hi, lo);
                        o.bhi[(size_t)j * o.Kpad + x] = hi;
                        o.blo[(size_t)j * o.Kpad + x] = lo;
                    }
                    if (o.bt32) {
                        const float h = tf32_rna(af);
                        const size_t f = (size_t)j * o.Kpad + x;
                        o.bt32[f] = h;
                        o.bt32[(size_t)o.Rpad * o.Kpad + f] = tf32_rna(af - h);
                    }
                    // the pair of the stored FP64 value, so that a Gram formed later
                    // from A64 (after a restore) sees the same pairs
                    if (o.A2) o.A2[e] = cpdf::split(av);
                    const double d = av - (o.Ap ? o.Ap[e] : aold[c]);
                    const float df = (float)d;
                    if (o.dA32) o.dA32[e] = df;
                    if (o.dA64) o.dA64[e] = d;
                    if (o.dA2) o.dA2[e] = cpdf::split(d);
                    const float step = o.Ap ? (float)(av - aold[c]) : df;
                    const float mf = __fadd_rn(mh[c], ml[c]);
                    fs[0] = fmaf(af, af, fs[0]);
                    fs[1] = fmaf(step, step, fs[1]);
                    if (o.Ap) fs[2] = fmaf(df, df, fs[2]);
                    fs[3] = fmaf(mf, mf, fs[3]);
                    // <m, x>: exact leading product, double-float sum
                    const float pm = __fmul_rn(mh[c], xh[c]);
                    float pe = __fmaf_rn(mh[c], xh[c], -pm);
                    pe = __fmaf_rn(mh[c], xl[c], __fmaf_rn(ml[c], xh[c], pe));
                    float s1, t1;
                    two_sum(mah, pm, s1, t1);
                    mah = s1;
                    mal = __fadd_rn(mal, __fadd_rn(t1, pe));
                }
#pragma unroll
                for (int o2 = 16; o2; o2 >>= 1) {
#pragma unroll
                    for (int i = 0; i < 5; ++i) fs[i] += __shfl_xor_sync(FULL, fs[i], o2);
                    const float bh = __shfl_xor_sync(FULL, mah, o2), bl = __shfl_xor_sync(FULL, mal, o2);
                    df_add(mah, mal, bh, bl);
                }
                if (lane == 0) {
                    float* pf = reinterpret_cast<float*>(part) + warp * 8;
#pragma unroll
                    for (int i = 0; i < 5; ++i) pf[i] = fs[i];
                    pf[5] = mah;
                    pf[6] = mal;
                }
            }
            __syncthreads();
            if (tid == 0) {
                // the two warps of group 0
                const float* p0 = reinterpret_cast<const float*>(part);
                const float* p1 = p0 + 8;
                float h = p0[5], l = p0[6];
                df_add(h, l, p1[5], p1[6]);
                double* out = scal_part + (size_t)blockIdx.x * CP_NSCAL;
                out[SCAL_A2] = (double)p0[0] + (double)p1[0];
                out[SCAL_STEP2] = (double)p0[1] + (double)p1[1];
                out[SCAL_DAP2] = (double)p0[2] + (double)p1[2];
                out[SCAL_MA] = (double)h + (double)l;
                out[SCAL_GS] = 0.0;
                out[SCAL_M2] = (double)p0[3] + (double)p1[3];
                out[SCAL_V2] = (double)p0[4] + (double)p1[4];
                out[SCAL_FLAGS] = 0.0;
            }
            return;
        }
    } else {
        // FP64 substitution with the fallback factor: warp 0, lane l owns l + 32 t
        if (warp == 0) {
            const bool stage = R <= MIXED_MAXR;
            const int ldl = stage ? R + 1 : R;
            if (stage)
                for (int e = lane; e < RR; e += 32) sG[(e / R) * (R + 1) + (e % R)] = __ldg(L64 + e);
            __syncwarp();
            const double* Lr = stage ? sG : L64;
            double acc[RT], z[RT], xs[RT];
#pragma unroll
            for (int t = 0; t < RT; ++t) {
                const int j = lane + 32 * t;
                acc[t] = (j < R) ? (double)M[(size_t)x * R + j] : 0.0;
                z[t] = 0.0;
                xs[t] = 0.0;
            }
            if (W) {
                // V term (FP64 path): lane-parallel over j
#pragma unroll
                for (int t = 0; t < RT; ++t) {
                    const int j = lane + 32 * t;
                    double v = 0.0;
                    if (j < R)
                        for (int q = 0; q < R; ++q) v = fma(o.A64[(size_t)x * R + q], W[(size_t)q * R + j], v);
                    acc[t] += v;
                    sc[SCAL_V2] += v * v;
                }
            }
#pragma unroll
            for (int t = 0; t < RT; ++t) {
                const int j = lane + 32 * t;
                if (j < R) mv[j] = acc[t];
            }
#pragma unroll
            for (int tt = 0; tt < RT; ++tt) {
                for (int jj = 0; jj < 32; ++jj) {
                    const int j = tt * 32 + jj;
                    if (j >= R) break;
                    const double zj = __shfl_sync(FULL, acc[tt], jj) * invd64[j];
                    if (lane == jj) z[tt] = zj;
#pragma unroll
                    for (int t2 = tt; t2 < RT; ++t2) {
                        const int k = lane + 32 * t2;
                        if (k > j && k < R) acc[t2] = fma(-Lr[(size_t)k * ldl + j], zj, acc[t2]);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < RT; ++t) acc[t] = z[t];
#pragma unroll
            for (int tt = RT - 1; tt >= 0; --tt) {
                for (int jj = 31; jj >= 0; --jj) {
                    const int j = tt * 32 + jj;
                    if (j >= R) continue;
                    const double xjj = __shfl_sync(FULL, acc[tt], jj) * invd64[j];
                    if (lane == jj) xs[tt] = xjj;
#pragma unroll
                    for (int t2 = 0; t2 <= tt; ++t2) {
                        const int k = lane + 32 * t2;
                        if (k < j) acc[t2] = fma(-Lr[(size_t)j * ldl + k], xjj, acc[t2]);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < RT; ++t) {
                const int j = lane + 32 * t;
                if (j < R) xv[j] = xs[t];
            }
        }
        __syncthreads();
        if (warp != 0) sc[SCAL_V2] = 0.0;
    }
    // outputs: FP64 master, FP32 copy, split operand copies, dA, scalar partials
    auto emit = [&](int j, double av, double mj, double ao) {
        const size_t e = (size_t)x * R + j;
        o.A64[e] = av;
        const float af = (float)av;
        if (o.A32) o.A32[e] = af;
        if (o.bhi) {
            uint16_t hi, lo;
            bf16_split(af, hi, lo);
            o.bhi[(size_t)j * o.Kpad + x] = hi;
            o.blo[(size_t)j * o.Kpad + x] = lo;
        }
        if (o.bt32) {
            const float h = tf32_rna(af);
            const size_t f = (size_t)j * o.Kpad + x;
            o.bt32[f] = h;
            o.bt32[(size_t)o.Rpad * o.Kpad + f] = tf32_rna(af - h);
        }
        if (o.A2) o.A2[e] = cpdf::split(av);
        const double base = o.Ap ? o.Ap[e] : ao;
        const double d = av - base;
        if (o.dA32) o.dA32[e] = (float)d;
        if (o.dA64) o.dA64[e] = d;
        if (o.dA2) o.dA2[e] = cpdf::split(d);
        sc[SCAL_A2] += av * av;
        sc[SCAL_STEP2] += (av - ao) * (av - ao);
        if (o.Ap) sc[SCAL_DAP2] += d * d;
        sc[SCAL_MA] += mj * av;
        sc[SCAL_M2] += mj * mj;
    };
    if (q == 0) {
        if (path == 0) {
#pragma unroll
            for (int c = 0; c < CT; ++c) {
                const int j = tcol + SOLVE_THREADS * c;
                if (j < R) emit(j, xj[c], mj[c], aold[c]);
            }
        } else {
            // the FP64 path covers any R: every thread takes columns tid, tid + 64, ...
            for (int j = tcol; j < R; j += SOLVE_THREADS) emit(j, xv[j], mv[j], o.A64[(size_t)x * R + j]);
        }
    }
    // block reduction of the 8 scalars.  Warp sums by a transposing butterfly:
    // after the exchanges at distance 16, 8 and 4, lane l holds scalar
    // 4 b4 + 2 b3 + b2 (bits of l) summed over 8 lanes, and two more exchanges
    // finish it: 9 FP64 additions per lane instead of 40
    double v4[4], v2[2], v1;
    {
        const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            v4[i] = (u16 ? sc[4 + i] : sc[i]) + __shfl_xor_sync(FULL, u16 ? sc[i] : sc[4 + i], 16);
#pragma unroll
        for (int i = 0; i < 2; ++i)
            v2[i] = (u8 ? v4[2 + i] : v4[i]) + __shfl_xor_sync(FULL, u8 ? v4[i] : v4[2 + i], 8);
        v1 = (u4 ? v2[1] : v2[0]) + __shfl_xor_sync(FULL, u4 ? v2[0] : v2[1], 4);
        v1 += __shfl_xor_sync(FULL, v1, 2);
        v1 += __shfl_xor_sync(FULL, v1, 1);
    }
    const int sidx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    __syncthreads();
    if (q == 0 && (lane & 3) == 0) part[warp * CP_NSCAL + sidx] = v1;
    __syncthreads();
    if (tid < CP_NSCAL) {
        double v = 0.0;
        for (int w = 0; w < SOLVE_THREADS / 32; ++w) v += part[w * CP_NSCAL + tid];
        scal_part[(size_t)blockIdx.x * CP_NSCAL + tid] = v;
    }
}

template <int RT>
cudaError_t launch_solve_mixed(const float* M, const double* W, const float2* W2, const double* G,
                               const float2* G2, const float* Ginv, const double* L64, const double* invd64,
                               const int* mode, const cpk::SolveOut& o, int s, int R, double* scal,
                               double* scal_part, unsigned* dev_err, cudaStream_t st) {
    // groups of 64 threads per row that split the refinement's dot products.
    // R <= 128 (double-float residual on the FP32 pipe): four groups, so that
    // every SM sub-partition issues; R > 128 (FP64 residual from L2): one group
    constexpr int KS = RT <= 4 ? 4 : 1;
    const size_t smem = solve_smem(R).total * sizeof(double) + 64;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_solve_mixed<RT, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(solve_smem(MIXED_MAXR).total * sizeof(double) + 64));
        attr = true;
    }
    return pdl::launch(k_solve_mixed<RT, KS>, (unsigned)s, SOLVE_THREADS * KS, smem, st, M, W, W2, G, G2, Ginv, L64,
                       invd64, mode, o, s, R, scal, scal_part, dev_err);
}

}  // namespace

namespace cpk {

size_t schur_ws_floats(int R) {
    // Gt, W, Y (= Gt W), the Newton-Schulz result, one column block copy, U, P,
    // dvec, 4 flag words
    return R <= MIXED_MAXR ? 0
                           : 4 * (size_t)R * R + 2 * (size_t)R * MIXED_MAXR + (size_t)MIXED_MAXR * MIXED_MAXR + R + 4;
}

cudaError_t chol_mixed(double* const* S_list, double* const* dS_list, const float2* const* S2_list,
                       const float2* const* dS2_list, int N, int n, int R, int pp, double* Gamma, float* G32,
                       float* G2, float* Ginv, double* L64, double* invd64, double* W, float* W2, double* scal,
                       int* mode, float* ws, cudaStream_t st, bool force64) {
    float2* g2 = reinterpret_cast<float2*>(G2);
    if (R <= MIXED_MAXR && S2_list && !pp && !force64) {
        // exact sweep: Gamma formed inside the one-CTA inverse (one launch, so
        // that the inverse takes its SM before the update's contraction fills the GPU)
        if (R <= 32)
            k_gj_inv<8, 4, 1><<<1, 256, 0, st>>>(G32, R, Gamma, Ginv, L64, invd64, scal, mode, S2_list, N, n, g2);
        else if (R <= 64)
            k_gj_inv<16, 4, 2><<<1, 512, 0, st>>>(G32, R, Gamma, Ginv, L64, invd64, scal, mode, S2_list, N, n, g2);
        else
            k_gj_inv<16, 8, 4><<<1, 512, 0, st>>>(G32, R, Gamma, Ginv, L64, invd64, scal, mode, S2_list, N, n, g2);
        return cudaGetLastError();
    }
    k_gamma_form<<<(R * R + 255) / 256, 256, 0, st>>>(S_list, dS_list, N, n, R, pp, Gamma, G32, G2, W, W2,
                                                      R <= MIXED_MAXR ? S2_list : nullptr,
                                                      R <= MIXED_MAXR ? dS2_list : nullptr);
    if (force64) {
        k_choose_fp64<<<1, 32, 0, st>>>(mode);
        k_chol_fp64_if<<<1, 1024, 0, st>>>(Gamma, R, L64, invd64, scal, mode);
        return cudaGetLastError();
    }
    if (R > MIXED_MAXR) {
        if (!ws) return cudaErrorInvalidValue;
        const size_t RR = (size_t)R * R;
        float* Gt = ws;
        float* Wb = Gt + RR;        // block elimination, in place
        float* Y = Wb + RR;         // Gt Wb
        float* Wn = Y + RR;         // after the Newton-Schulz step
        float* Ck = Wn + RR;        // R x 128
        float* U = Ck + (size_t)R * MIXED_MAXR;   // 128 x R
        float* P = U + (size_t)R * MIXED_MAXR;    // 128 x 128
        float* dvec = P + (size_t)MIXED_MAXR * MIXED_MAXR;
        unsigned* flags = reinterpret_cast<unsigned*>(dvec + R);
        cudaError_t e = cudaMemsetAsync(flags, 0, 4 * sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        k_scale_big<<<64, 256, 0, st>>>(G32, R, Gt, dvec, flags);
        e = cudaMemcpyAsync(Wb, Gt, RR * sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        auto grid = [](int M, int Nn) { return dim3((unsigned)((Nn + 31) / 32), (unsigned)((M + 31) / 32)); };
        const unsigned ug = (unsigned)std::min<int64_t>(2048, ((int64_t)R * R + 255) / 256);
        for (int k0 = 0; k0 < R; k0 += MIXED_MAXR) {
            const int bk = std::min(MIXED_MAXR, R - k0);
            k_gj_block<16, 8, 4><<<1, 512, 0, st>>>(Wb + (size_t)k0 * R + k0, R, bk, P, bk, flags);
            k_copy_cols<<<(unsigned)std::min<int64_t>(1024, ((int64_t)R * bk + 255) / 256), 256, 0, st>>>(Wb, R, k0,
                                                                                                       bk, Ck);
            k_gemm_small<<<grid(bk, R), 256, 0, st>>>(bk, R, bk, 1.f, P, bk, 0, Wb + (size_t)k0 * R, R, 0, 0.f,
                                                       nullptr, 0, U, R);
            k_bgj_update<<<ug, 256, 0, st>>>(Wb, R, k0, bk, Ck, U, P);
        }
        // Newton-Schulz: Y = Gt Wb, Wn = 2 Wb - Wb Y
        k_gemm_small<<<grid(R, R), 256, 0, st>>>(R, R, R, 1.f, Gt, R, 0, Wb, R, 0, 0.f, nullptr, 0, Y, R);
        k_gemm_small<<<grid(R, R), 256, 0, st>>>(R, R, R, -1.f, Wb, R, 0, Y, R, 0, 2.f, Wb, R, Wn, R);
        k_inv_finish<<<64, 256, 0, st>>>(R, Wn, Y, dvec, Ginv, flags, scal, mode);
        k_chol_fp64_if<<<1, 1024, 0, st>>>(Gamma, R, L64, invd64, scal, mode);
        return cudaGetLastError();
    }
    // (warps, rows per thread, columns per thread): TY x IR >= R, 32 JC >= R.
    // Sixteen warps hide the latency of each step's dependent chain.
    if (R <= 32)
        k_gj_inv<8, 4, 1><<<1, 256, 0, st>>>(G32, R, Gamma, Ginv, L64, invd64, scal, mode, nullptr, N, n, g2);
    else if (R <= 64)
        k_gj_inv<16, 4, 2><<<1, 512, 0, st>>>(G32, R, Gamma, Ginv, L64, invd64, scal, mode, nullptr, N, n, g2);
    else
        k_gj_inv<16, 8, 4><<<1, 512, 0, st>>>(G32, R, Gamma, Ginv, L64, invd64, scal, mode, nullptr, N, n, g2);
    return cudaGetLastError();
}

cudaError_t solve_mixed(const float* M, const double* W, const float* W2, const double* Gamma, const float* G2,
                        const float* Ginv, const double* L64, const double* invd64, const int* mode,
                        const SolveOut& o, int s, int R, double* scal, double* scal_part, int* nblk,
                        unsigned* dev_err, cudaStream_t st) {
    *nblk = s;
    const float2* w2 = reinterpret_cast<const float2*>(W2);
    const float2* g2 = reinterpret_cast<const float2*>(G2);
#define CP_SOLVE(RT) launch_solve_mixed<RT>(M, W, w2, Gamma, g2, Ginv, L64, invd64, mode, o, s, R, scal, scal_part, dev_err, st)
    switch ((R + 31) / 32) {
        case 1: return CP_SOLVE(1);
        case 2: return CP_SOLVE(2);
        case 3: return CP_SOLVE(3);
        case 4: return CP_SOLVE(4);
        case 5: return CP_SOLVE(5);
        case 6: return CP_SOLVE(6);
        case 7: return CP_SOLVE(7);
        case 8: return CP_SOLVE(8);
        case 9: case 10: return CP_SOLVE(10);
        case 11: case 12: return CP_SOLVE(12);
        case 13: case 14: return CP_SOLVE(14);
        case 15: case 16: return CP_SOLVE(16);
        default: return cudaErrorInvalidValue;
    }
#undef CP_SOLVE
}

}  // namespace cpk
