// Dense side kernels of the factor updates and the residual (Alg. 1 solve and Gram;
// Alg. 2 approximated update; Eq. ds, Eq. residual, Eq. residual-def): the Grams
// S(n) = A^T A and dS(n) = A^T dA (thread-block clusters; from the factor's float
// pairs in double-float arithmetic for R <= 128, FP64 above), the update's
// scalar terms, the operand copies of a factor for the tensor-core TTM (bf16 /
// tf32 / scaled fp16 parts), norms and maxima, the direct residual on the CUDA
// cores, the PP first-order terms (Eq. U_ni) and the Khatri-Rao operand of the
// fused standard-tree contraction.  The normal equations themselves (Hadamard
// chain, FP32 inverse with iterative refinement) are in k_solve_mixed.cu.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cpals_internal.h"
#include "df_arith.h"
#include "pdl.h"

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


// Gram of an updated factor: S = A^T A (and dS = A^T dA), grid (R/16, R/16, nc)
// with clusters of (1, 1, nc): the nc CTAs of a cluster each sum one row chunk
// of the same 16 x 16 tile; the partials meet in distributed shared memory and
// CTA 0 of the cluster adds them in chunk order, writes the tile and its share
// of <Gamma, S> (tile_gs).  No global fences or counters.
constexpr int GRAM_MAX_CHUNKS = 8;

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ double ld_cluster_f64(const double* local, unsigned rank) {
    uint32_t la = (uint32_t)__cvta_generic_to_shared(local), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
    return v;
}

__global__ void __launch_bounds__(256) k_gram_cl(const double* __restrict__ A,
                                                 const double* __restrict__ dA, int s, int R,
                                                 int rows_per, const double* __restrict__ Gamma,
                                                 double* __restrict__ S, double* __restrict__ dS,
                                                 double* __restrict__ tile_gs) {
    __shared__ double a1[16][17], a2[16][17], d2[16][17];
    __shared__ double ps[256], pd[256];
    __shared__ double red[32];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int r1 = blockIdx.x * 16 + ty, r2 = blockIdx.y * 16 + tx;
    const int c = blockIdx.z, nc = gridDim.z;
    const int x0 = c * rows_per, x1 = min(s, x0 + rows_per);
    double acc0 = 0.0, acc1 = 0.0, accd0 = 0.0, accd1 = 0.0;
    for (int xb = x0; xb < x1; xb += 16) {
        const int x = xb + ty;
        const int ca = blockIdx.x * 16 + tx, cb = blockIdx.y * 16 + tx;
        a1[ty][tx] = (x < x1 && ca < R) ? A[(size_t)x * R + ca] : 0.0;
        a2[ty][tx] = (x < x1 && cb < R) ? A[(size_t)x * R + cb] : 0.0;
        if (dA) d2[ty][tx] = (x < x1 && cb < R) ? dA[(size_t)x * R + cb] : 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k += 2) {
            acc0 = fma(a1[k][ty], a2[k][tx], acc0);
            acc1 = fma(a1[k + 1][ty], a2[k + 1][tx], acc1);
            if (dA) {
                accd0 = fma(a1[k][ty], d2[k][tx], accd0);
                accd1 = fma(a1[k + 1][ty], d2[k + 1][tx], accd1);
            }
        }
        __syncthreads();
    }
    ps[tid] = acc0 + acc1;
    pd[tid] = accd0 + accd1;
    cluster_sync_all();
    if (c == 0) {
        // cluster dims (1, 1, nc): the rank of a CTA in its cluster is blockIdx.z
        double pv[GRAM_MAX_CHUNKS], pq[GRAM_MAX_CHUNKS];
#pragma unroll
        for (int q = 0; q < GRAM_MAX_CHUNKS; ++q) {
            pv[q] = q < nc ? ld_cluster_f64(&ps[tid], (unsigned)q) : 0.0;
            pq[q] = (q < nc && dA) ? ld_cluster_f64(&pd[tid], (unsigned)q) : 0.0;
        }
        double v = 0.0, d = 0.0;
#pragma unroll
        for (int q = 0; q < GRAM_MAX_CHUNKS; ++q) {
            v += pv[q];
            d += pq[q];
        }
        double gs = 0.0;
        if (r1 < R && r2 < R) {
            const size_t e = (size_t)r1 * R + r2;
            S[e] = v;
            if (dA) dS[e] = d;
            if (Gamma) gs = Gamma[e] * v;
        }
        if (tile_gs) {
            gs = block_sum(gs, red);
            if (tid == 0) tile_gs[blockIdx.y * gridDim.x + blockIdx.x] = gs;
        }
    }
    cluster_sync_all();  // every CTA's partials stay readable until CTA 0 is done
}

__device__ __forceinline__ float2 ld_cluster_f2(const float2* local, unsigned rank) {
    uint32_t la = (uint32_t)__cvta_generic_to_shared(local), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(ra) : "memory");
    return v;
}

// The same Gram from the float-pair copy of the factor (hi + lo = its FP64 value,
// written by the row solve): the products in double-float arithmetic on the FP32
// pipe (exact leading products, about 2^-44 relative), the chunk partials added
// in chunk order by CTA 0 of the cluster, FP64 only for the stored entries.
// <Gamma, S> per tile from Gamma's float pairs, also in double-float.
__global__ void __launch_bounds__(256) k_gram_df(const float2* __restrict__ A, const float2* __restrict__ dA,
                                                 int s, int R, int rows_per, const float2* __restrict__ G2,
                                                 double* __restrict__ S, double* __restrict__ dS,
                                                 float2* __restrict__ S2, float2* __restrict__ dS2,
                                                 double* __restrict__ tile_gs) {
    __shared__ float2 a1[16][17], a2[16][17], d2[16][17];
    __shared__ float2 ps[256], pd[256];
    __shared__ float2 red[8];
    pdl::wait();
    pdl::trigger();
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31, warp = tid >> 5;
    const int r1 = blockIdx.x * 16 + ty, r2 = blockIdx.y * 16 + tx;
    const int c = blockIdx.z, nc = gridDim.z;
    const int x0 = c * rows_per, x1 = min(s, x0 + rows_per);
    const float2 z = make_float2(0.f, 0.f);
    float sh = 0.f, sl = 0.f, dh = 0.f, dl = 0.f;
    for (int xb = x0; xb < x1; xb += 16) {
        const int x = xb + ty;
        const int ca = blockIdx.x * 16 + tx, cb = blockIdx.y * 16 + tx;
        a1[ty][tx] = (x < x1 && ca < R) ? A[(size_t)x * R + ca] : z;
        a2[ty][tx] = (x < x1 && cb < R) ? A[(size_t)x * R + cb] : z;
        if (dA) d2[ty][tx] = (x < x1 && cb < R) ? dA[(size_t)x * R + cb] : z;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float2 u = a1[k][ty], v = a2[k][tx];
            cpdf::fma_acc(u.x, u.y, v.x, v.y, sh, sl);
            if (dA) {
                const float2 w = d2[k][tx];
                cpdf::fma_acc(u.x, u.y, w.x, w.y, dh, dl);
            }
        }
        __syncthreads();
    }
    ps[tid] = make_float2(sh, sl);
    pd[tid] = make_float2(dh, dl);
    cluster_sync_all();
    if (c == 0) {
        // cluster dims (1, 1, nc): the rank of a CTA in its cluster is blockIdx.z
        float2 pv[GRAM_MAX_CHUNKS], pq[GRAM_MAX_CHUNKS];
#pragma unroll
        for (int q = 0; q < GRAM_MAX_CHUNKS; ++q) {
            pv[q] = q < nc ? ld_cluster_f2(&ps[tid], (unsigned)q) : z;
            pq[q] = (q < nc && dA) ? ld_cluster_f2(&pd[tid], (unsigned)q) : z;
        }
        float vh = pv[0].x, vl = pv[0].y, wh = pq[0].x, wl = pq[0].y;
#pragma unroll
        for (int q = 1; q < GRAM_MAX_CHUNKS; ++q) {
            cpdf::add(vh, vl, pv[q].x, pv[q].y);
            if (dA) cpdf::add(wh, wl, pq[q].x, pq[q].y);
        }
        float gh = 0.f, gl = 0.f;
        if (r1 < R && r2 < R) {
            const size_t e = (size_t)r1 * R + r2;
            S[e] = (double)vh + (double)vl;
            S2[e] = make_float2(vh, vl);
            if (dA) {
                dS[e] = (double)wh + (double)wl;
                dS2[e] = make_float2(wh, wl);
            }
            if (G2) {
                const float2 g = G2[e];
                cpdf::fma_acc(g.x, g.y, vh, vl, gh, gl);
            }
        }
        if (tile_gs) {
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const float bh = __shfl_xor_sync(0xffffffffu, gh, o), bl = __shfl_xor_sync(0xffffffffu, gl, o);
                cpdf::add(gh, gl, bh, bl);
            }
            if (lane == 0) red[warp] = make_float2(gh, gl);
            __syncthreads();
            if (tid == 0) {
                float h = red[0].x, l = red[0].y;
                for (int w = 1; w < 8; ++w) cpdf::add(h, l, red[w].x, red[w].y);
                tile_gs[blockIdx.y * gridDim.x + blockIdx.x] = (double)h + (double)l;
            }
        }
    }
    cluster_sync_all();  // every CTA's partials stay readable until CTA 0 is done
}

// y = float pairs (hi, lo) of x, the same rounding the row solve uses
__global__ void __launch_bounds__(256) k_split_pairs(const double* __restrict__ x, float2* __restrict__ y,
                                                     int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = cpdf::split(x[i]);
}

// The update's scalars: the solve's per-block partials and the tile shares of
// <Gamma, S>, added in a fixed order.  Off the critical path (own stream).
__global__ void __launch_bounds__(256) k_scal_fin(const double* __restrict__ scal_part, int nblk,
                                                  const double* __restrict__ tile_gs, int ntiles,
                                                  double* __restrict__ scal_out) {
    __shared__ double red[32];
    const int tid = threadIdx.x;
    double v[CP_NSCAL];
#pragma unroll
    for (int slot = 0; slot < CP_NSCAL; ++slot) v[slot] = 0.0;
    for (int b = tid; b < nblk; b += blockDim.x) {
        double w[CP_NSCAL];
#pragma unroll
        for (int slot = 0; slot < CP_NSCAL; ++slot) w[slot] = scal_part[(size_t)b * CP_NSCAL + slot];
#pragma unroll
        for (int slot = 0; slot < CP_NSCAL; ++slot) v[slot] += w[slot];
    }
    double t = 0.0;
    for (int q = tid; q < ntiles; q += blockDim.x) t += tile_gs[q];
    t = block_sum(t, red);
    if (tid == 0) scal_out[SCAL_GS] = t;
#pragma unroll
    for (int slot = 0; slot < CP_NSCAL; ++slot) {
        if (slot == SCAL_GS || slot == SCAL_FLAGS) continue;
        const double r = block_sum(v[slot], red);
        if (tid == 0) scal_out[slot] = r;
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
// ||T - [[A]]||^2 (Eq. residual-def): T seen as rows (modes
// 0..N-2, C order) x columns (mode N-1); the model block of a 128 x 128 tile is
// KR(rows) A_{N-1}(cols)^T with the Khatri-Rao rows formed on the fly.  256
// threads, 8 x 8 model values per thread (FP32 FMAs over r, in order), the
// operands staged in shared memory 8 ranks at a time, double-buffered through
// registers.  Per block: FP64 sum of the per-tile FP32 sums of squares.
constexpr int RD_T = 128, RD_K = 8;

template <int NF>  // tensor order when fixed at compile time (3, 4), else 0
__global__ void __launch_bounds__(256, 2) k_resid_direct(cpk::ResidArgs a, int64_t nrows,
                                                      int64_t ncols, int64_t ntile_c,
                                                      double* __restrict__ partials,
                                                      int64_t ntiles) {
    __shared__ __align__(16) float KR[2][RD_K][RD_T];
    __shared__ __align__(16) float Bs[2][RD_K][RD_T];
    __shared__ double red[32];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int N = NF ? NF : a.N, R = a.R;
    constexpr int NMAX = NF ? NF : CP_MAXN;
    const float* Alast = a.A32[N - 1];
    // staging: thread loads ranks sr .. sr + 3 of row / column sm of the tile
    const int sm = tid & 127, sr = (tid >> 7) * 4;
    const bool r4 = (R & 3) == 0;  // rows of every factor are 16-byte aligned
    double total = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t row0 = (tile / ntile_c) * RD_T, col0 = (tile % ntile_c) * RD_T;
        // the factor rows of this thread's staging row (multi-index of modes 0..N-2)
        const float* frow[NMAX];
        {
            int64_t row = row0 + sm;
            if (row >= nrows) row = 0;
#pragma unroll
            for (int k = NMAX - 2; k >= 0; --k) {
                if (k > N - 2) continue;
                frow[k] = a.A32[k] + (size_t)(row % a.dims[k]) * R;
                row /= a.dims[k];
            }
        }
        const bool rok = row0 + sm < nrows, cok = col0 + sm < ncols;
        const float* brow = Alast + (size_t)(cok ? col0 + sm : 0) * R;
        auto stage = [&](int r0, float* kv, float* bv) {
            const int r = r0 + sr;
            if (r4 && r + 4 <= R) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f), b = v;
                if (rok) {
                    v = __ldg(reinterpret_cast<const float4*>(frow[0] + r));
#pragma unroll
                    for (int k = 1; k < NMAX - 1; ++k) {
                        if (k >= N - 1) break;
                        const float4 w = __ldg(reinterpret_cast<const float4*>(frow[k] + r));
                        v.x *= w.x; v.y *= w.y; v.z *= w.z; v.w *= w.w;
                    }
                }
                if (cok) b = __ldg(reinterpret_cast<const float4*>(brow + r));
                kv[0] = v.x; kv[1] = v.y; kv[2] = v.z; kv[3] = v.w;
                bv[0] = b.x; bv[1] = b.y; bv[2] = b.z; bv[3] = b.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float v = 0.f, b = 0.f;
                    if (r + q < R) {
                        if (rok) {
                            v = 1.f;
#pragma unroll
                            for (int k = 0; k < NMAX - 1; ++k)
                                if (k < N - 1) v *= __ldg(frow[k] + r + q);
                        }
                        if (cok) b = __ldg(brow + r + q);
                    }
                    kv[q] = v;
                    bv[q] = b;
                }
            }
        };
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        float kv[4], bv[4];
        stage(0, kv, bv);
        int buf = 0;
        for (int r0 = 0; r0 < R; r0 += RD_K) {
            __syncthreads();  // buffer `buf` is free (its last readers are two barriers back)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                KR[buf][sr + q][sm] = kv[q];
                Bs[buf][sr + q][sm] = bv[q];
            }
            __syncthreads();
            if (r0 + RD_K < R) stage(r0 + RD_K, kv, bv);  // next ranks in flight
            // rows ty*4 + {0..3} and 64 + ty*4 + {0..3}; columns likewise with tx:
            // a warp's 16 column groups are contiguous 16-byte words (no bank conflicts)
#pragma unroll
            for (int k = 0; k < RD_K; ++k) {
                const float4 a0 = *reinterpret_cast<const float4*>(&KR[buf][k][ty * 4]);
                const float4 a1 = *reinterpret_cast<const float4*>(&KR[buf][k][64 + ty * 4]);
                const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
                const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bw[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bw[j], acc[i][j]);
            }
            buf ^= 1;
        }
        float part = 0.f;
        const bool al = (((uintptr_t)a.T & 15) == 0) && ((ncols & 3) == 0);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t row = row0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
            if (row >= nrows) continue;
            const float* trow = a.T + row * ncols;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t c0 = col0 + h * 64 + tx * 4;
                if (al && c0 + 4 <= ncols) {
                    const float4 t = __ldg(reinterpret_cast<const float4*>(trow + c0));
                    const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float d = tv[j] - acc[i][h * 4 + j];
                        part = fmaf(d, d, part);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (c0 + j < ncols) {
                            const float d = __ldg(trow + c0 + j) - acc[i][h * 4 + j];
                            part = fmaf(d, d, part);
                        }
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

// VEC consecutive floats (4, 2 or 1) as the low lanes of a float4
template <int VEC>
__device__ __forceinline__ float4 ldv_pp(const float* p) {
    if (VEC == 4) return __ldg(reinterpret_cast<const float4*>(p));
    if (VEC == 2) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        return make_float4(v.x, v.y, 0.f, 0.f);
    }
    return make_float4(__ldg(p), 0.f, 0.f, 0.f);
}

// U operator rows in flight per thread (the operators are read once per update)
constexpr int PPU_U = 8;

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
            // element (x, y, r) of the operator: [y][x][r] (trans) or [x][y][r]
            const size_t ystep = tr ? (size_t)sx * R : (size_t)R;
            const float* opx = op + (tr ? (size_t)x * R : (size_t)x * sy * R) + r;
            int y = ty;
            for (; y + (PPU_U - 1) * KS < sy; y += PPU_U * KS) {
                float4 v[PPU_U], d[PPU_U];
#pragma unroll
                for (int u = 0; u < PPU_U; ++u) {
                    v[u] = ldv_pp<VEC>(opx + (size_t)(y + u * KS) * ystep);
                    d[u] = ldv_pp<VEC>(dA + (size_t)(y + u * KS) * R + r);
                }
#pragma unroll
                for (int u = 0; u < PPU_U; ++u) {
                    acc.x = fmaf(v[u].x, d[u].x, acc.x);
                    if (VEC > 1) acc.y = fmaf(v[u].y, d[u].y, acc.y);
                    if (VEC > 2) { acc.z = fmaf(v[u].z, d[u].z, acc.z); acc.w = fmaf(v[u].w, d[u].w, acc.w); }
                }
            }
            for (; y < sy; y += KS) {
                const float4 v = ldv_pp<VEC>(opx + (size_t)y * ystep);
                const float4 d = ldv_pp<VEC>(dA + (size_t)y * R + r);
                acc.x = fmaf(v.x, d.x, acc.x);
                if (VEC > 1) acc.y = fmaf(v.y, d.y, acc.y);
                if (VEC > 2) { acc.z = fmaf(v.z, d.z, acc.z); acc.w = fmaf(v.w, d.w, acc.w); }
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
        } else if (VEC == 2) {
            float2 m = __ldg(reinterpret_cast<const float2*>(Mp) + o);
            *reinterpret_cast<float2*>(Mt + o * 2) = make_float2(m.x + acc.x, m.y + acc.y);
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


// ------------------------------------------------------------------ scaled fp16 operands
// Power-of-two exponent that brings a maximum magnitude m into [2^14, 2^15)
// (the top binade below the fp16 maximum 65504); 0 for m = 0 or non-finite m.
__device__ __forceinline__ int f16_exp_for(float m) {
    if (!(m > 0.f) || !isfinite(m)) return 0;
    const int e = 14 - ilogbf(m);
    return e < -126 ? -126 : (e > 127 ? 127 : e);
}

// Factor operand of the fp16 tensor-core TTM: for each column c of the s x R
// FP32 factor, e_c = f16_exp_for(max_x |A(x, c)|); A(x, c) 2^e_c split into fp16
// hi = rn(y), lo = rn(y - hi), written transposed ([c][x], x contiguous, row
// stride Kpad); colinv[c] = 2^-(e_c + eT) for c < Rpad (0 past R).  One block of
// 32 x 32 threads per 32 columns: the column maxima, then 32 x 32 tiles through
// shared memory so that reads (along c) and writes (along x) are coalesced.
__global__ void __launch_bounds__(1024) k_f16_operand(const float* __restrict__ A, int s, int R, int Rpad,
                                                      int Kpad, int eT, uint16_t* __restrict__ hi,
                                                      uint16_t* __restrict__ lo, float* __restrict__ colinv) {
    __shared__ float red[32][33];
    __shared__ uint16_t th[32][33], tl[32][33];
    __shared__ float scl[32];
    pdl::wait();
    pdl::trigger();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + tx;
    float m = 0.f;
    if (c < R)
        for (int x = ty; x < s; x += 32) m = fmaxf(m, fabsf(A[(size_t)x * R + c]));
    red[ty][tx] = m;
    __syncthreads();
    if (ty == 0) {
        float mm = 0.f;
        for (int k = 0; k < 32; ++k) mm = fmaxf(mm, red[k][tx]);
        const int e = c < R ? f16_exp_for(mm) : 0;
        scl[tx] = ldexpf(1.f, e);
        if (c < Rpad) colinv[c] = c < R ? ldexpf(1.f, -(e + eT)) : 0.f;
    }
    __syncthreads();
    const float sc = scl[tx];
    for (int x0 = 0; x0 < s; x0 += 32) {
        const int x = x0 + ty;
        const float y = (c < R && x < s) ? A[(size_t)x * R + c] * sc : 0.f;
        const __half h = __float2half_rn(y);
        const __half l = __float2half_rn(y - __half2float(h));
        th[tx][ty] = __half_as_ushort(h);
        tl[tx][ty] = __half_as_ushort(l);
        __syncthreads();
        // thread (ty, tx) writes column blockIdx.x * 32 + ty, row x0 + tx
        const int cw = blockIdx.x * 32 + ty, xw = x0 + tx;
        if (cw < R && xw < s) {
            hi[(size_t)cw * Kpad + xw] = th[ty][tx];
            lo[(size_t)cw * Kpad + xw] = tl[ty][tx];
        }
        __syncthreads();
    }
}

// Column powers of two of the Khatri-Rao operand of modes a, a+1: the largest
// entry of column c is max|A_a(:, c)| * max|A_b(:, c)|.
__global__ void __launch_bounds__(256) k_kr_scale(const double* __restrict__ Aa, const double* __restrict__ Ab,
                                                  int sa, int sb, int R, int Rpad, int eT,
                                                  float* __restrict__ scale, float* __restrict__ colinv) {
    for (int c = blockIdx.x * 8 + (threadIdx.x >> 5); c < Rpad; c += gridDim.x * 8) {
        const int lane = threadIdx.x & 31;
        double ma = 0.0, mb = 0.0;
        if (c < R) {
            for (int i = lane; i < sa; i += 32) ma = fmax(ma, fabs(Aa[(size_t)i * R + c]));
            for (int i = lane; i < sb; i += 32) mb = fmax(mb, fabs(Ab[(size_t)i * R + c]));
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            ma = fmax(ma, __shfl_xor_sync(FULL, ma, o));
            mb = fmax(mb, __shfl_xor_sync(FULL, mb, o));
        }
        if (lane == 0) {
            const int e = c < R ? f16_exp_for((float)(ma * mb)) : 0;
            scale[c] = ldexpf(1.f, e);
            colinv[c] = c < R ? ldexpf(1.f, -(e + eT)) : 0.f;
        }
    }
}

// max |x| over n floats -> one partial per block
__global__ void __launch_bounds__(256) k_absmax(const float* __restrict__ x, int64_t n, float* __restrict__ part) {
    __shared__ float red[8];
    float m = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool al = ((uintptr_t)x & 15) == 0;
    const int64_t n4 = al ? n / 4 : 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(x) + i);
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        m = fmaxf(m, fabsf(x[i]));
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        part[blockIdx.x] = m;
    }
}

__global__ void k_absmax_fin(const float* __restrict__ part, int n, float* __restrict__ out) {
    __shared__ float red[32];
    float m = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, part[i]);
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        out[0] = m;
    }
}

// ------------------------------------------------------------------ Khatri-Rao operand
// out[r][k] (r < Rpad, k < Kpad; zero outside R x K): row k = ia * sb + ib of the
// Khatri-Rao product, A_a[ia][r] * A_b[ib][r], split into two parts (KIND 2:
// fp16 parts of the product times scale[r], a power of two from k_kr_scale).
template <int KIND>
__global__ void k_kr(const double* __restrict__ Aa, const double* __restrict__ Ab, int sa, int sb,
                     int R, int Rpad, int Kpad, void* __restrict__ hi, void* __restrict__ lo,
                     const float* __restrict__ scale) {
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
        } else if (KIND == 2) {
            const float y = v * scale[r];
            const __half h = __float2half_rn(y);
            static_cast<uint16_t*>(hi)[idx] = __half_as_ushort(h);
            static_cast<uint16_t*>(lo)[idx] = __half_as_ushort(__float2half_rn(y - __half2float(h)));
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
                       int kind, void* hi, void* lo, cudaStream_t st, int eT, float* scale, float* colinv) {
    const int Rpad = (R + 15) / 16 * 16;
    const int64_t n = (int64_t)Rpad * Kpad;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (kind == 0) {
        k_kr<0><<<(unsigned)blocks, 256, 0, st>>>(Aa, Ab, sa, sb, R, Rpad, Kpad, hi, lo, nullptr);
    } else if (kind == 1) {
        k_kr<1><<<(unsigned)blocks, 256, 0, st>>>(Aa, Ab, sa, sb, R, Rpad, Kpad, hi, lo, nullptr);
    } else {
        if (!scale || !colinv) return cudaErrorInvalidValue;
        k_kr_scale<<<(Rpad + 7) / 8, 256, 0, st>>>(Aa, Ab, sa, sb, R, Rpad, eT, scale, colinv);
        k_kr<2><<<(unsigned)blocks, 256, 0, st>>>(Aa, Ab, sa, sb, R, Rpad, Kpad, hi, lo, scale);
    }
    return cudaGetLastError();
}

cudaError_t f16_operand(const float* A32, int s, int R, int Rpad, int Kpad, int eT, uint16_t* hi, uint16_t* lo,
                        float* colinv, cudaStream_t st) {
    cudaError_t e = pdl::launch(k_f16_operand, (unsigned)((R + 31) / 32), 1024, 0, st, A32, s, R, Rpad, Kpad, eT,
                                hi, lo, colinv);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t absmax(const float* x, int64_t n, float* part, int max_blocks, float* out, cudaStream_t st) {
    int64_t want = (n / 4 + 255) / 256;
    const int blocks = (int)(want < 1 ? 1 : (want > max_blocks ? max_blocks : want));
    k_absmax<<<blocks, 256, 0, st>>>(x, n, part);
    k_absmax_fin<<<1, 1024, 0, st>>>(part, blocks, out);
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

int gram_tiles(int R) { return ((R + 15) / 16) * ((R + 15) / 16); }

cudaError_t gram(const double* A, const double* dA, int s, int R, const double* Gamma, double* S,
                 double* dS, double* tile_gs, cudaStream_t st) {

    int nc = (s + 31) / 32;  // about 32 rows per chunk
    if (nc > GRAM_MAX_CHUNKS) nc = GRAM_MAX_CHUNKS;
    if (nc < 1) nc = 1;
    const int rows_per = (s + nc - 1) / nc;
    nc = (s + rows_per - 1) / rows_per;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((R + 15) / 16, (R + 15) / 16, nc);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = nc;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_gram_cl, A, dA, s, R, rows_per, Gamma, S, dS, tile_gs);
}

cudaError_t split_pairs(const double* x, float2* y, int64_t n, cudaStream_t st) {
    int64_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want > 4096 ? 4096 : (want < 1 ? 1 : want));
    k_split_pairs<<<blocks, 256, 0, st>>>(x, y, n);
    return cudaGetLastError();
}

cudaError_t gram_df(const float2* A2, const float2* dA2, int s, int R, const float2* G2, double* S,
                    double* dS, float2* S2, float2* dS2, double* tile_gs, cudaStream_t st) {
    // about 32 rows per chunk, at most GRAM_MAX_CHUNKS chunks (one cluster)
    int nc = (s + 31) / 32;
    if (nc > GRAM_MAX_CHUNKS) nc = GRAM_MAX_CHUNKS;
    if (nc < 1) nc = 1;
    const int rows_per = (s + nc - 1) / nc;
    nc = (s + rows_per - 1) / rows_per;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((R + 15) / 16, (R + 15) / 16, nc);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = nc;
    pdl::set_attr(attr[1]);
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k_gram_df, A2, dA2, s, R, rows_per, G2, S, dS, S2, dS2, tile_gs);
}

cudaError_t scal_fin(const double* scal_part, int nblk, const double* tile_gs, int ntiles, double* scal_out,
                     cudaStream_t st) {
    k_scal_fin<<<1, 256, 0, st>>>(scal_part, nblk, tile_gs, ntiles, scal_out);
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
    const int64_t ntr = (nrows + RD_T - 1) / RD_T, ntc = (ncols + RD_T - 1) / RD_T;
    const int64_t ntiles = ntr * ntc;
    int blocks = (int)(ntiles < max_blocks ? ntiles : max_blocks);
    if (a.N == 3) k_resid_direct<3><<<blocks, 256, 0, st>>>(a, nrows, ncols, ntc, partials, ntiles);
    else if (a.N == 4) k_resid_direct<4><<<blocks, 256, 0, st>>>(a, nrows, ncols, ntc, partials, ntiles);
    else k_resid_direct<0><<<blocks, 256, 0, st>>>(a, nrows, ncols, ntc, partials, ntiles);
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
    bool al8 = ((uintptr_t)Mp | (uintptr_t)Mt) % 8 == 0;
    for (int i = 0; i < nterms; ++i) al8 = al8 && (((uintptr_t)terms[i].op | (uintptr_t)terms[i].dA) % 8 == 0);
    const int VEC = (R % 4 == 0 && al) ? 4 : (R % 2 == 0 && al8) ? 2 : 1;
    const int64_t nout = (int64_t)sx * (R / VEC);
    int maxs = 1;
    for (int i = 0; i < nterms; ++i) maxs = terms[i].sy > maxs ? terms[i].sy : maxs;
    int KS = 1;
    while (KS < 32 && KS < maxs && nout * KS < 152LL * 2 * 256) KS *= 2;
    const int TX = 256 / KS;
    const unsigned blocks = (unsigned)((nout + TX - 1) / TX);
    if (blocks == 0) return cudaSuccess;
    if (VEC == 4)
        k_pp_u<4><<<blocks, 256, 256 * sizeof(float4), st>>>(Mp, a, Mt, sx, R, TX, KS);
    else if (VEC == 2)
        k_pp_u<2><<<blocks, 256, 256 * sizeof(float4), st>>>(Mp, a, Mt, sx, R, TX, KS);
    else
        k_pp_u<1><<<blocks, 256, 256 * sizeof(float4), st>>>(Mp, a, Mt, sx, R, TX, KS);
    return cudaGetLastError();
}

}  // namespace cpk
