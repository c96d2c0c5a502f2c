// Direct residual ||T - [[A(0), ..., A(N-1)]]||_F^2 (Sec. II-B, Eq. residual-def)
// on the 5th-generation tensor cores.
//
// T is viewed as a matrix [rows][cols]: rows = multi-index of modes 0..N-2 (mode
// N-2 fastest), cols = the last mode (contiguous).  For a tile of 128 rows and a
// block of 128 columns the model values are the contraction over r of
//   KR[i][r] = prod_{k < N-1} A(k)[i_k][r]      (the Khatri-Rao rows of the tile)
// with A(N-1)[j][r]:  M = KR A(N-1)^T, an M = 128, N = 128, K = R tcgen05 product
// in tf32x3 (hi*hi into one accumulator, hi*lo + lo*hi into another; tf32 has
// FP32's exponent range, so no scaling is needed), FP32 accumulation.
//
// One persistent CTA per SM keeps one column block (its A(N-1) block is split
// into tf32 parts once) and walks row tiles:
//   warp 0      TMA loads of T in chunks of 128 rows x 32 columns into a ring
//   warps 4-11  two groups of 128 threads, thread = tile row, taking turns over
//               the 32-k chunks of the tiles: the row's KR values (FP32 products
//               of factor rows), split into tf32 hi / lo in the K-major
//               128-byte-swizzled operand layout
//   warp 1      one thread issues tcgen05.mma into two TMEM accumulator sets
//   warps 12-15 thread = TMEM lane = tile row: model values, the T chunk from the
//               ring, sum of (T - M)^2 in FP32 per 16 columns, accumulated in
//               double-float arithmetic; one FP64 partial per CTA
// Rows past the tensor read zeros from the TMA unit and have zero KR rows; columns
// past it read zeros and have zero A(N-1) rows: their terms are exactly zero.
// Every mbarrier wait is bounded; on expiry the CTA sets DEVERR_TIMEOUT, drains
// what it issued (bounded), frees its tensor memory and returns.
#include <cuda.h>

#include "cpals_internal.h"
#include "df_arith.h"
#include "tc_ptx.h"

namespace {

using namespace tcx;

constexpr int RM = 128;            // rows per tile (TMEM lanes)
constexpr int RN = 128;            // columns per block (MMA N)
constexpr int TSTG = 4;            // T chunk stages of 32 columns (one tile's worth)
constexpr uint32_t CHUNK = RM * 128;   // 128 rows x 128 bytes: one T chunk, one operand k-chunk
constexpr int RES_MAXR = 64;
constexpr int RES_THREADS = 512;   // warp 0 TMA, 1 MMA, 2-3 idle, 4-11 KR rows, 12-15 epilogue
constexpr long long RES_WAIT = 2000000000LL;

struct ResArgs {
    const float* A[CP_MAXN];
    int64_t dims[CP_MAXN];
    int N, R, nkc;        // nkc: chunks of 32 k covering R (zero-padded)
    int64_t nrows, ncols;
    int ncb;              // column blocks of 128
    int64_t nrt;          // row tiles of 128
    int S_c;              // KR operand stages, one 32-k chunk (hi and lo) each
    double* partials;     // one per CTA
    unsigned* dev_err;
    long long wait_limit;
};

template <int NF>   // tensor order when fixed at compile time (3, 4), else 0
__global__ void __launch_bounds__(RES_THREADS, 1)
    k_resid_tc(const __grid_constant__ CUtensorMap tmT, const ResArgs a) {
    constexpr int NMAX = NF ? NF - 1 : CP_MAXN - 1;   // factor rows of a KR row
    const int NV = NF ? NF : a.N;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t apart = (uint32_t)a.nkc * CHUNK;                  // one tf32 part of the A(N-1) block
    const uint32_t t0 = base;                                        // T ring
    const uint32_t a0 = t0 + TSTG * CHUNK;                           // KR ring: [stage][hi, lo] of one chunk
    const uint32_t b0 = a0 + (uint32_t)a.S_c * 2u * CHUNK;           // A(N-1) block: [hi, lo][chunk]
    const uint32_t bar0 = b0 + 2u * apart;
    auto t_full = [&](int s) { return bar0 + 8u * s; };
    auto t_empty = [&](int s) { return bar0 + 8u * (4 + s); };
    auto a_full = [&](int j) { return bar0 + 8u * (8 + j); };
    auto a_empty = [&](int j) { return bar0 + 8u * (12 + j); };
    auto acc_full = [&](int b) { return bar0 + 8u * (16 + b); };
    auto acc_empty = [&](int b) { return bar0 + 8u * (18 + b); };
    const uint32_t b_ready = bar0 + 8u * 20, drain_bar = bar0 + 8u * 21;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + (bar0 - base) + 8 * 22);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + (bar0 - base) + 8 * 23);
    float2* red = reinterpret_cast<float2*>(gbase + (bar0 - base) + 8 * 24);   // 4 epilogue warps
    const int tpc = 128;   // threads that form one KR chunk

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cb = blockIdx.x % a.ncb;                 // this CTA's column block
    const int64_t rt0 = blockIdx.x / a.ncb, rstep = gridDim.x / a.ncb;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TSTG; ++s) {
            mbar_init(t_full(s), 1);
            mbar_init(t_empty(s), 128);
        }
        for (int j = 0; j < a.S_c; ++j) {
            mbar_init(a_full(j), tpc);
            mbar_init(a_empty(j), 1);
        }
        for (int j = 0; j < 2; ++j) {
            mbar_init(acc_full(j), 1);
            mbar_init(acc_empty(j), 128);
        }
        mbar_init(b_ready, 256);
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    float eh = 0.f, el = 0.f;   // epilogue: this row's sum of squares (double-float)

    if (warp == 0) {
        // ------------------------------------------------ TMA producer of T chunks
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmT) : "memory");
            int64_t it = 0;
            bool ok = true;
            for (int64_t rt = rt0; rt < a.nrt && ok; rt += rstep) {
                for (int c = 0; c < 4 && ok; ++c, ++it) {
                    const int s = (int)(it % TSTG);
                    const uint32_t u = (uint32_t)(it / TSTG);
                    if (!(ok = mbar_wait(t_empty(s), (u & 1u) ^ 1u, abort_flag, a.wait_limit))) break;
                    mbar_expect_tx(t_full(s), CHUNK);
                    tma_load_2d(t0 + (uint32_t)s * CHUNK, &tmT, cb * RN + 32 * c, (int)(rt * RM), t_full(s));
                }
            }
            if (!ok) {
                volatile int never = 0;
                for (int64_t k = (it > TSTG ? it - TSTG : 0); k < it; ++k)
                    mbar_wait(t_full((int)(k % TSTG)), (uint32_t)((k / TSTG) & 1), &never, RES_WAIT);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            // kind::tf32, FP32 accumulation, K-major A and B, N = 128, M = 128
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(RN >> 3) << 17) |
                                   ((uint32_t)(RM >> 4) << 24);
            bool ok = mbar_wait(b_ready, 0u, abort_flag, a.wait_limit);
            int lt = 0;
            for (int64_t rt = rt0; rt < a.nrt && ok; rt += rstep, ++lt) {
                const int buf = lt & 1;
                if (!(ok = mbar_wait(acc_empty(buf), (uint32_t)(((lt >> 1) & 1) ^ 1), abort_flag, a.wait_limit)))
                    break;
                const uint32_t dm = tmem_base + (uint32_t)(buf * 256), dc = dm + 128;
                for (int kc = 0; kc < a.nkc && ok; ++kc) {
                    const int64_t ci = (int64_t)lt * a.nkc + kc;     // chunk sequence number
                    const int cs = (int)(ci % a.S_c);
                    if (!(ok = mbar_wait(a_full(cs), (uint32_t)((ci / a.S_c) & 1), abort_flag, a.wait_limit))) break;
                    tc_fence_after();
                    const uint32_t ahi = a0 + (uint32_t)cs * 2u * CHUNK, alo = ahi + CHUNK;
                    const uint32_t bhi = b0 + (uint32_t)kc * CHUNK, blo = bhi + apart;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {   // tf32: K = 8 per MMA, 32 bytes of the 128-byte row
                        const uint32_t off = (uint32_t)kk * 32u;
                        const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
                        tc_mma<1>(dm, sw128_desc(ahi + off), sw128_desc(bhi + off), idesc, acc);
                        tc_mma<1>(dc, sw128_desc(ahi + off), sw128_desc(blo + off), idesc, acc);
                        tc_mma<1>(dc, sw128_desc(alo + off), sw128_desc(bhi + off), idesc, 1u);
                    }
                    tc_commit(a_empty(cs));
                }
                if (!ok) break;
                tc_commit(acc_full(buf));
            }
            if (!ok) {
                tc_commit(drain_bar);
                volatile int never = 0;
                mbar_wait(drain_bar, 0u, &never, RES_WAIT);
            }
        }
    } else if (warp >= 4 && warp < 12) {
        // ------------------------------------------------ KR rows and the A(N-1) block
        // two groups of 128 threads (thread = tile row): group h forms the KR chunks
        // ci = h, h + 2, ... of the chunk sequence (chunk ci = k range 32 (ci mod nkc)
        // of tile ci / nkc), so every use of a ring stage has one writer group; the
        // A(N-1) block is split between the groups by k (KP / 2, a multiple of 16)
        const int ct = threadIdx.x - 128;
        const int m = ct & (RM - 1), half = ct >> 7;
        const int R = a.R, KP = a.nkc * 32;
        const int kb = half * (KP / 2), ke = kb + KP / 2;   // this group's k range of the A(N-1) block
        const bool vec = (R & 3) == 0;
        // k = r .. r+3 of row p (zeros past R): float4 when the rows are 16-byte aligned
        auto load4 = [&](const float* p, int r) {
            if (vec) return r < R ? __ldg(reinterpret_cast<const float4*>(p + r)) : make_float4(0.f, 0.f, 0.f, 0.f);
            return make_float4(r < R ? __ldg(p + r) : 0.f, r + 1 < R ? __ldg(p + r + 1) : 0.f,
                               r + 2 < R ? __ldg(p + r + 2) : 0.f, r + 3 < R ? __ldg(p + r + 3) : 0.f);
        };
        // tf32 hi / lo of k = r .. r+3 of row m: chunk r / 32, 16-byte piece (r % 32) / 4 at piece ^ (m mod 8)
        // (ph, pl: the chunk holding k = r, for the A(N-1) block the part base plus r / 32 chunks)
        auto store4 = [&](uint8_t* ph, uint8_t* pl, int r, float4 v) {
            const float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
            const float4 l = make_float4(tf32_rna(v.x - h.x), tf32_rna(v.y - h.y), tf32_rna(v.z - h.z),
                                         tf32_rna(v.w - h.w));
            const int q = (r & 31) >> 2;
            const size_t off = (size_t)m * 128 + (size_t)((q ^ (m & 7)) << 4);
            *reinterpret_cast<float4*>(ph + off) = h;
            *reinterpret_cast<float4*>(pl + off) = l;
        };
        {
            uint8_t* bh = gbase + (b0 - base);
            const int64_t col = (int64_t)cb * RN + m;
            const float* brow = a.A[NV - 1] + (size_t)(col < a.ncols ? col : 0) * R;
            for (int r = kb; r < ke; r += 4)
                store4(bh + (size_t)(r >> 5) * CHUNK, bh + apart + (size_t)(r >> 5) * CHUNK, r,
                       col < a.ncols ? load4(brow, r) : make_float4(0.f, 0.f, 0.f, 0.f));
            fence_proxy_async();
            mbar_arrive(b_ready);
        }
        bool ok = true;
        for (int64_t ci = half; ok; ci += 2) {
            const int64_t rt = rt0 + (ci / a.nkc) * rstep;
            if (rt >= a.nrt) break;
            const int k0 = 32 * (int)(ci % a.nkc);
            const int cs = (int)(ci % a.S_c);
            if (!(ok = mbar_wait(a_empty(cs), (uint32_t)(((ci / a.S_c) & 1) ^ 1), abort_flag, a.wait_limit))) break;
            uint8_t* ph = gbase + (a0 - base) + (size_t)cs * 2 * CHUNK;
            const int64_t row = rt * RM + m;
            const bool rok = row < a.nrows;
            const float* frow[NMAX];
            {
                int64_t q = rok ? row : 0;
#pragma unroll
                for (int k = NMAX - 1; k >= 0; --k) {
                    if (k > NV - 2) continue;
                    frow[k] = a.A[k] + (size_t)(q % a.dims[k]) * R;
                    q /= a.dims[k];
                }
            }
            // two groups of four per step, their loads issued before the products
            for (int r = k0; r < k0 + 32; r += 8) {
                float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
                if (rok) {
                    v0 = load4(frow[0], r);
                    v1 = load4(frow[0], r + 4);
#pragma unroll
                    for (int k = 1; k < NMAX; ++k) {
                        if (k > NV - 2) break;
                        const float4 w0 = load4(frow[k], r), w1 = load4(frow[k], r + 4);
                        v0.x *= w0.x; v0.y *= w0.y; v0.z *= w0.z; v0.w *= w0.w;
                        v1.x *= w1.x; v1.y *= w1.y; v1.z *= w1.z; v1.w *= w1.w;
                    }
                }
                store4(ph, ph + CHUNK, r, v0);
                store4(ph, ph + CHUNK, r + 4, v1);
            }
            fence_proxy_async();
            mbar_arrive(a_full(cs));
        }
    } else if (warp >= 12) {
        // ------------------------------------------------ epilogue: (T - M)^2
        const int quad = warp & 3;
        const int m = quad * 32 + lane;                 // tile row = TMEM lane
        const uint8_t* tr = gbase + (t0 - base) + (size_t)m * 128;
        int lt = 0;
        int64_t it = 0;
        bool ok = true;
        for (int64_t rt = rt0; rt < a.nrt && ok; rt += rstep, ++lt) {
            const int buf = lt & 1;
            if (!(ok = mbar_wait(acc_full(buf), (uint32_t)((lt >> 1) & 1), abort_flag, a.wait_limit))) break;
            tc_fence_after();
            const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * 256);
            for (int g = 0; g < 8; ++g) {
                const int s = (int)(it % TSTG);
                if ((g & 1) == 0 &&
                    !(ok = mbar_wait(t_full(s), (uint32_t)((it / TSTG) & 1), abort_flag, a.wait_limit)))
                    break;
                float mv[16], cv[16];
                tmem_ld16x2(taddr + (uint32_t)(16 * g), taddr + 128u + (uint32_t)(16 * g), mv, cv);
                const uint8_t* rowp = tr + (size_t)s * CHUNK;
                float ss = 0.f;
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    const int q = 4 * (g & 1) + q4;    // 16-byte piece of the 128-byte row
                    const float4 t = *reinterpret_cast<const float4*>(rowp + ((q ^ (m & 7)) << 4));
                    const float e0 = t.x - (mv[4 * q4] + cv[4 * q4]);
                    const float e1 = t.y - (mv[4 * q4 + 1] + cv[4 * q4 + 1]);
                    const float e2 = t.z - (mv[4 * q4 + 2] + cv[4 * q4 + 2]);
                    const float e3 = t.w - (mv[4 * q4 + 3] + cv[4 * q4 + 3]);
                    ss = fmaf(e0, e0, ss);
                    ss = fmaf(e1, e1, ss);
                    ss = fmaf(e2, e2, ss);
                    ss = fmaf(e3, e3, ss);
                }
                cpdf::add(eh, el, ss, 0.f);
                if (g & 1) {
                    // the stage's next fill is a TMA write (async proxy) after these
                    // generic reads: order them across the proxies before the release
                    fence_proxy_async();
                    mbar_arrive(t_empty(s));
                    ++it;
                }
            }
            if (!ok) break;
            tc_fence_before();
            mbar_arrive(acc_empty(buf));
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float bh = __shfl_xor_sync(0xffffffffu, eh, o), bl = __shfl_xor_sync(0xffffffffu, el, o);
            cpdf::add(eh, el, bh, bl);
        }
        if (lane == 0) red[quad] = make_float2(eh, el);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512)
                     : "memory");
    }
    if (threadIdx.x == 0) {
        float h = red[0].x, l = red[0].y;
        for (int q = 1; q < 4; ++q) cpdf::add(h, l, red[q].x, red[q].y);
        a.partials[blockIdx.x] = (double)h + (double)l;
        if (*abort_flag) atomicOr(a.dev_err, (unsigned)DEVERR_TIMEOUT);
    }
}

}  // namespace

namespace cpk {

int resid_tc_partials(const ResidArgs& ra, double* partials, int max_blocks, int num_sms, unsigned* dev_err,
                      long long wait_limit, cudaStream_t st) {
    const int N = ra.N, R = ra.R;
    if (N < 3 || N > CP_MAXN || R < 1 || R > RES_MAXR) return 0;
    int64_t nrows = 1;
    for (int k = 0; k < N - 1; ++k) nrows *= ra.dims[k];
    const int64_t ncols = ra.dims[N - 1];
    if (nrows < 1 || ncols < 1 || ncols % 4 != 0 || ((uintptr_t)ra.T & 15)) return 0;
    if (nrows > ((int64_t)1 << 31) - RM) return 0;   // TMA row coordinate is a 32-bit int
    const int64_t ncb = (ncols + RN - 1) / RN;
    const int cap = num_sms < max_blocks ? num_sms : max_blocks;
    if (ncb > cap) return 0;
    if ((R & 3) == 0)
        for (int k = 0; k < N; ++k)
            if ((uintptr_t)ra.A32[k] & 15) return 0;
    EncodeTiledFn enc = encoder();
    if (!enc) return 0;
    ResArgs a;
    for (int k = 0; k < N; ++k) {
        a.A[k] = ra.A32[k];
        a.dims[k] = ra.dims[k];
    }
    a.N = N;
    a.R = R;
    a.nkc = (R + 31) / 32;
    a.nrows = nrows;
    a.ncols = ncols;
    a.ncb = (int)ncb;
    a.nrt = (nrows + RM - 1) / RM;
    a.S_c = a.nkc == 1 ? 4 : 3;
    a.partials = partials;
    a.dev_err = dev_err;
    a.wait_limit = wait_limit > 0 ? wait_limit : RES_WAIT;
    CUtensorMap tmT;
    const cuuint64_t dims[2] = {(cuuint64_t)ncols, (cuuint64_t)nrows};
    const cuuint64_t strides[1] = {(cuuint64_t)ncols * 4};
    const cuuint32_t box[2] = {32, RM};
    const cuuint32_t es[2] = {1, 1};
    if (enc(&tmT, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ra.T, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return 0;
    // whole column-block groups of CTAs, no more than there are (row tile, block) units
    int64_t grid = (cap / ncb) * ncb;
    if (grid > a.nrt * ncb) grid = a.nrt * ncb;
    const uint32_t apart = (uint32_t)a.nkc * CHUNK;
    const size_t smem = 1024 + (size_t)TSTG * CHUNK + (size_t)a.S_c * 2 * CHUNK + 2 * (size_t)apart + 256;
    auto kern = N == 3 ? k_resid_tc<3> : N == 4 ? k_resid_tc<4> : k_resid_tc<0>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<(unsigned)grid, RES_THREADS, smem, st>>>(tmT, a);
    return cudaGetLastError() == cudaSuccess ? (int)grid : -1;
}

}  // namespace cpk
