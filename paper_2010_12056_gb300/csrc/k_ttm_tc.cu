// First-level TTM on the 5th-generation tensor cores (Sec. II-C: T x_m A(m),
// the dominant 2 s^N R-flop contraction of every dimension tree).
//
//   X[g][r] = sum_k T(g, k) A(m)[k][r],   g = (p, q) over the modes kept.
//
// One persistent CTA per SM streams 128-row tiles of T exactly once:
//   warp 0      TMA producer: FP32 tensor chunks (128 rows x BK k) into a staging
//               ring; the factor operand (stored [r][k], K-major, split in two
//               parts) either once for the whole kernel (when all of K fits) or
//               one chunk per k-step.
//   warps 4-7   converters, thread = tile row: split every FP32 value into two
//               parts in the canonical K-major 128-byte-swizzled layout (rows of
//               128 B, 16-byte chunk c of row m at c ^ (m mod 8)):
//                 bf16 family (BK = 64): hi = rn_bf16(x), lo = rn_bf16(x - hi)
//                 tf32 family (BK = 32): hi = rna_tf32(x), lo = rna_tf32(x - hi)
//                 fp16 (BK = 64): y = x * 2^eT, hi = rn_f16(y), lo = rn_f16(y - hi),
//                   with the power of two 2^eT chosen once per tensor so that
//                   max |y| lies in [2^14, 2^15); the factor operand carries a
//                   power of two per column the same way, and the epilogue
//                   multiplies column r by 2^-(eT + e_r) (exact).  Two 11-bit
//                   parts keep about 22 bits of every value (tf32x3 accuracy at
//                   the bf16 rate); values below 2^-24 of max |T| lose their low
//                   part, an error far below the FP32 rounding of the result.
//               For the last mode the chunk is K-contiguous (TMA SWIZZLE_128B keeps
//               row reads conflict-free); for other modes it is q-contiguous
//               (BK k x 128 q) and the converter transposes while splitting.
//   warp 1      one thread issues tcgen05.mma (M=128, N=Rpad): x3 = hi*hi +
//               hi*lo + lo*hi, single = hi*hi.  The tensor core rounds its FP32
//               accumulation towards zero once per instruction, so the hi*hi
//               products of k-chunk kc go to accumulator kc mod nsplit and the
//               (2^-8 or 2^-11 smaller) corrections to one more; the epilogue
//               adds them with round-to-nearest.  Two sets of accumulators let
//               the epilogue overlap the next tile.
//   epilogue    (the last EW warps) tcgen05.ld 32x32b -> registers -> a warp-private smem
//               transpose -> full-sector coalesced stores of X.  Optionally (the
//               multi-sweep tree's first child, Fig. 2) it also forms
//                 Y[y][r] = sum_{j < sc} X[y sc + j][r] Ac[j][r]
//               (X's innermost kept mode contracted) from the accumulators.
//               sc a multiple of 32: each warp's 32 rows lie in one segment; the
//               warp writes its column sums and a second kernel adds the sc / 32
//               pieces of each segment in order.  Other sc: segmented warp sums,
//               boundary pieces combined per tile by the first epilogue warp, pieces of segments
//               that cross tiles added by a second kernel in a fixed order.
// Every mbarrier wait is bounded; on expiry the CTA sets DEVERR_TIMEOUT, drains
// what it issued (bounded), frees TMEM and exits.
#include <atomic>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cpals_internal.h"
#include "tc_ptx.h"
#include "pdl.h"

namespace {

constexpr int BM = 128;
// warps 0 producer, 1 MMA, 2-3 idle, 4.. converters, then the epilogue: EW = 4
// epilogue warps (one per TMEM lane quarter), or 8 (two per quarter, alternate
// 16-column groups) for passes of 128 columns, where the epilogue is the slowest
// stage (measured on 128^4: R = 128 0.73 -> 0.81-0.87 of HBM; R <= 64 slower with
// 8, whose extra warps take issue slots from the converters)
// four converter warps (one per SM sub-partition; measured: eight are slower,
// 0.290 vs 0.272 ms at 128^4 R = 64, their issue slots are the epilogue's)
__host__ __device__ constexpr int conv_warps(int, int) { return 4; }
__host__ __device__ constexpr int nthreads(int ew, int child) { return 128 + 32 * conv_warps(ew, child) + 32 * ew; }
// (scaled fp16 parts also at 64 columns: their epilogue multiplies every value by
// its column scale; measured 0.301 -> 0.281 ms at 128^4 R = 64, bf16 0.272 -> 0.277)
inline int epi_warps_for(int Rpad, int kind) { return (Rpad >= 128 || (kind == 2 && Rpad >= 64)) ? 8 : 4; }
constexpr int EPI_STRIDE = 20;             // floats per row of the epilogue transpose buffer
constexpr int EPI_WARP_BYTES = 32 * EPI_STRIDE * 4;   // one epilogue warp's transpose buffer
constexpr int BAR_BYTES = 512;
// first-child pieces: [2 tiles in flight][4 warps][2 pieces][128 columns] floats + keys
constexpr int CHILD_BYTES = 2 * 4 * 2 * 128 * 4 + 2 * 4 * 2 * 8;
constexpr int MAX_STG = 8, MAX_OP = 4;
// bounded waits: the pipeline's waits give up after TcArgs::wait_limit cycles
// (default about 1 s; a test may shorten it to make a wait run out), the drain
// after an abort always waits up to DRAIN_LIMIT for the copies and MMAs in flight
constexpr long long DEFAULT_WAIT_LIMIT = 2000000000LL;
constexpr long long DRAIN_LIMIT = 2000000000LL;
constexpr size_t SMEM_LIMIT = 232448;

struct TcArgs {
    float* X;
    int64_t PQ;       // rows of X
    int64_t Q;        // rows per p-slice (mode != last)
    int64_t ntiles;
    int64_t tiles_per_p;
    int R, Rpad, nk, S_stg, S_op, tmem_cols, x3, b_resident, nsplit, nacc;
    int nsk;          // split-K factor: work item w = (tile w / nsk, k-slice w % nsk)
    int64_t slice;    // floats between split-K output slices
    int ldx;          // row stride of X in floats (R of the whole factor)
    // column passes (R > 128): work item w = (tile, k-slice, pass) with the pass
    // innermost, so a tile's second pass finds its T chunks in L2.  R / Rpad above
    // are the largest pass's (they size the shared-memory slots and TMEM sets).
    int npass;
    int Rp[4], Rpadp[4];   // columns of pass p (written at column 128 p of X), padded
    uint32_t idescp[4];    // MMA instruction descriptor of pass p (N = Rpadp[p])
    int set_cols;          // TMEM columns of one accumulator set
    uint32_t idesc;
    unsigned* dev_err;
    // first child (NULL Yc: off): Yc[(g / sc)][r] += X[g][r] Ac[g % sc][r].  Pieces:
    // sc % 32 == 0 (sc > 32): cws[(g0 / 32) * R + r] per warp of rows g0..g0+31;
    // else segments that cross a tile: cws[(tile * 2 + piece) * R + r]
    float* Yc;
    const float* Ac;
    float* cws;
    int sc;
    int ac_bytes;   // > 0: Ac (sc x R floats) is copied to shared memory once per CTA
    // fp16 parts (KIND 2): T is multiplied by tscale before splitting; column c of
    // X is multiplied by colinv[c] = 1 / (tscale * factor column scale)
    float tscale;
    const float* colinv;
    long long wait_limit;   // cycles a pipeline wait may take before the CTA aborts
};

using namespace tcx;

// 8 floats -> one 16-byte chunk of bf16 hi and one of bf16 lo
__device__ __forceinline__ void split8_bf16(const float* f, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 hb = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
        float2 hf = __bfloat1622float2(hb);
        __nv_bfloat162 lb = __floats2bfloat162_rn(f[2 * i] - hf.x, f[2 * i + 1] - hf.y);
        h[i] = *reinterpret_cast<uint32_t*>(&hb);
        l[i] = *reinterpret_cast<uint32_t*>(&lb);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}
// 8 floats -> one 16-byte chunk of fp16 hi and one of fp16 lo of y = x * sc
__device__ __forceinline__ void split8_f16(const float* f, float sc, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float y0 = f[2 * i] * sc, y1 = f[2 * i + 1] * sc;
        __half2 hh = __floats2half2_rn(y0, y1);
        float2 hf = __half22float2(hh);
        __half2 lh = __floats2half2_rn(y0 - hf.x, y1 - hf.y);
        h[i] = *reinterpret_cast<uint32_t*>(&hh);
        l[i] = *reinterpret_cast<uint32_t*>(&lh);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}
// 4 floats -> one 16-byte chunk of tf32 hi and one of tf32 lo
__device__ __forceinline__ void split4_tf32(float4 v, float4& hi, float4& lo) {
    hi.x = tf32_rna(v.x); hi.y = tf32_rna(v.y); hi.z = tf32_rna(v.z); hi.w = tf32_rna(v.w);
    lo.x = tf32_rna(v.x - hi.x); lo.y = tf32_rna(v.y - hi.y);
    lo.z = tf32_rna(v.z - hi.z); lo.w = tf32_rna(v.w - hi.w);
}

struct Layout {
    uint32_t stg0, op0, b0, epi0, bar0;
    uint32_t stg_bytes, op_bytes, bchunk_bytes;
};

// scaled fp16 parts: the per-column output scales of both passes in shared memory
constexpr int CS_BYTES = 512 * 4;

__host__ __device__ inline size_t layout_bytes(int S_stg, int S_op, int Rpad, int nk, int b_resident,
                                               int BK, int ew, int kind, bool child = false, int ac_bytes = 0,
                                               bool wide = false) {
    // operand rows: 128 bytes (64 16-bit or 32 tf32 k), or 64 bytes in wide mode
    const size_t rowb = wide ? 64 : 128;
    const size_t stg = (size_t)BM * BK * 4;
    const size_t bchunk = 2 * (size_t)Rpad * rowb;
    const size_t nb = b_resident ? (size_t)nk : (size_t)S_op;
    return 1024 + (size_t)S_stg * stg + (size_t)S_op * 2 * BM * rowb + nb * bchunk +
           (size_t)ew * EPI_WARP_BYTES +
           (child ? CHILD_BYTES + (size_t)ac_bytes : 0) + (kind == 2 ? CS_BYTES : 0) + BAR_BYTES;
}

// ------------------------------------------------------------------ kernel
// MODE 0: last mode, T rows K-contiguous (2-D map {K, PQ}, boxes {32, 128}, SWIZZLE_128B)
// MODE 1: other modes, T[p][k][q] with Q % 4 == 0 (3-D map {Q, K, P}, box {128, BK, 1}; the
//         last q-tile of each p is zero-filled past Q by the TMA unit and written up to Q)
// KIND 0: bf16 parts, BK = 64, kind::f16;  KIND 1: tf32 parts, BK = 32, kind::tf32;
// KIND 2: scaled fp16 parts, BK = 64, kind::f16
// CHILD: 0 plain; 1 the epilogue also forms the first child (a.Yc) for sc a
// multiple of 32; 2 for other sc.  Separate instantiations keep each kernel's
// code, registers and shared memory to what it runs.
// WIDE (16-bit parts, R > 128): column passes of up to 256 (one MMA N = 256, so T
// is split once per tile and read once), 32-k chunks in the 64-byte swizzle so that
// three operand stages fit, and one TMEM accumulator set (hi*hi and corrections,
// 2 x 256 columns): the epilogue does not overlap the next tile's MMAs.
// PRE (wide only): T was stored once as fp16 / bf16 parts with the contracted mode
// innermost ([rows][K], rows = the kept modes in order): the TMA loads the A
// operand directly (two 2-D maps, hi and lo), with no staging ring and no
// converter warps; rows are the flattened kept modes (MODE 0 addressing).
template <int MODE, int KIND, int CHILD, int EW, int WIDE = 0, int PRE = 0>
__global__ void __launch_bounds__(nthreads(EW, CHILD), 1)
    k_ttm_tc(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmBhi,
             const __grid_constant__ CUtensorMap tmBlo, const __grid_constant__ CUtensorMap tmBhi1,
             const __grid_constant__ CUtensorMap tmBlo1, const __grid_constant__ CUtensorMap tmBhi2,
             const __grid_constant__ CUtensorMap tmBlo2, const __grid_constant__ CUtensorMap tmBhi3,
             const __grid_constant__ CUtensorMap tmBlo3, const __grid_constant__ CUtensorMap tmTlo,
             const TcArgs a) {
    static_assert(!WIDE || (KIND != 1 && CHILD == 0), "wide passes use 16-bit parts and no first child");
    static_assert(!PRE || MODE == 0, "stored parts: flattened rows");
    constexpr int BK = (KIND == 1 || WIDE) ? 32 : 64;
    constexpr uint32_t STG = BM * BK * 4;
    constexpr uint32_t ROWB = WIDE ? 64u : 128u;     // bytes of one operand row (k-chunk)
    constexpr uint32_t OPA = BM * ROWB;               // one split part of a 128-row chunk
    constexpr int KSTEPS = ROWB / 32;                 // MMAs of K = 16 (32 bytes) per chunk
    constexpr int PW = WIDE ? 256 : 128;              // columns per pass
    constexpr int NSETS = WIDE ? 1 : 2;               // TMEM accumulator sets
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    const int S_stg = a.S_stg, S_op = a.S_op;
    const uint32_t bchunk = 2u * (uint32_t)a.Rpad * ROWB;   // hi + lo of one k-chunk
    const uint32_t stg0 = base;
    const uint32_t op0 = stg0 + (uint32_t)S_stg * STG;
    const uint32_t b0 = op0 + (uint32_t)S_op * 2u * OPA;
    const uint32_t epi0 = b0 + (uint32_t)(a.b_resident ? a.nk : S_op) * bchunk;
    static_assert(EW == 4 || (EW == 8 && CHILD == 0), "first-child epilogues use four warps");
    constexpr int NEPI = EW;
    constexpr int NCONV = conv_warps(EW, CHILD);
    constexpr int EPI0 = 4 + NCONV;   // first epilogue warp (a multiple of 4: TMEM lane quarters)
    const uint32_t child0 = epi0 + NEPI * EPI_WARP_BYTES;
    const uint32_t ac0 = child0 + (CHILD ? CHILD_BYTES : 0);
    const uint32_t cs0 = ac0 + (CHILD ? (uint32_t)a.ac_bytes : 0u);
    const uint32_t bar0 = cs0 + (KIND == 2 ? (uint32_t)CS_BYTES : 0u);
    auto stg_full = [&](int s) { return bar0 + 8u * s; };
    auto stg_empty = [&](int s) { return bar0 + 8u * (MAX_STG + s); };
    auto op_full = [&](int j) { return bar0 + 8u * (2 * MAX_STG + j); };
    auto op_empty = [&](int j) { return bar0 + 8u * (2 * MAX_STG + MAX_OP + j); };
    auto acc_full = [&](int b) { return bar0 + 8u * (2 * MAX_STG + 2 * MAX_OP + b); };
    auto acc_empty = [&](int b) { return bar0 + 8u * (2 * MAX_STG + 2 * MAX_OP + 2 + b); };
    const uint32_t b_full = bar0 + 8u * (2 * MAX_STG + 2 * MAX_OP + 4);
    const uint32_t drain_bar = bar0 + 8u * (2 * MAX_STG + 2 * MAX_OP + 5);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + (bar0 - base) + 8 * 30);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + (bar0 - base) + 8 * 31);
    auto epi_bar = [&](int b) { return bar0 + 8u * (32 + b); };  // first child: the 4 epilogue warps

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S_stg; ++s) {
            mbar_init(stg_full(s), 1);
            mbar_init(stg_empty(s), 32 * NCONV);
        }
        for (int j = 0; j < S_op; ++j) {
            // converted A (NCONV warps) and the factor chunk (one expect_tx), or with
            // stored parts both by the producer's one expect_tx
            mbar_init(op_full(j), PRE ? 1 : (a.b_resident ? 32 * NCONV : 32 * NCONV + 1));
            mbar_init(op_empty(j), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full(b), 1);
            mbar_init(acc_empty(b), 32 * NEPI);
        }
        mbar_init(b_full, 1);
        mbar_init(drain_bar, 1);
        mbar_init(epi_bar(0), 128);
        mbar_init(epi_bar(1), 128);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // everything above touched only this CTA's shared memory and TMEM: the kernel
    // before this one on the stream may still be running until here.  No early
    // signal to the next kernel: its blocks (a multi-TTV of many blocks) would
    // take the SM this grid leaves to the next update's normal-equation inverse.
    pdl::wait();
    if (KIND == 2) {
        // per-column output scales, read by the epilogue for every tile
        float* sCs = reinterpret_cast<float*>(gbase + (cs0 - base));
        const int n = PW * (a.npass - 1) + a.Rpadp[a.npass - 1];
        for (int i = threadIdx.x; i < n; i += nthreads(EW, CHILD)) sCs[i] = __ldg(a.colinv + i);
    }
    if (CHILD && a.ac_bytes > 0) {
        // the contracted factor, read by the epilogue for every tile
        float* sAc = reinterpret_cast<float*>(gbase + (ac0 - base));
        const int n = a.sc * a.R;
        for (int i = threadIdx.x; i < n; i += nthreads(EW, CHILD)) sAc[i] = __ldg(a.Ac + i);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint32_t bpart = (uint32_t)a.Rpad * ROWB;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmT) : "memory");
            if (PRE) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmTlo) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmBhi) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmBlo) : "memory");
            if (a.npass > 1) {
                asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmBhi1) : "memory");
                asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmBlo1) : "memory");
            }
            if (a.npass > 2) {
                asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmBhi2) : "memory");
                asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmBlo2) : "memory");
            }
            if (a.npass > 3) {
                asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmBhi3) : "memory");
                asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmBlo3) : "memory");
            }
            if (a.b_resident) {
                mbar_expect_tx(b_full, (uint32_t)a.nk * bchunk);
                for (int kc = 0; kc < a.nk; ++kc) {
                    const uint32_t d = b0 + (uint32_t)kc * bchunk;
                    tma_load_2d(d, &tmBhi, kc * BK, 0, b_full);
                    tma_load_2d(d + bpart, &tmBlo, kc * BK, 0, b_full);
                }
            }
            int64_t it = 0;
            bool ok = true;
            const int64_t nwork = a.ntiles * a.nsk * a.npass;
            for (int64_t w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
                const int64_t tile = w / ((int64_t)a.nsk * a.npass);
                const int ks = (int)((w / a.npass) % a.nsk);
                const int pass = (int)(w % a.npass);
                const CUtensorMap* mhi = pass == 0 ? &tmBhi : pass == 1 ? &tmBhi1 : pass == 2 ? &tmBhi2 : &tmBhi3;
                const CUtensorMap* mlo = pass == 0 ? &tmBlo : pass == 1 ? &tmBlo1 : pass == 2 ? &tmBlo2 : &tmBlo3;
                const int kc0 = ks * a.nk / a.nsk, kc1 = (ks + 1) * a.nk / a.nsk;
                if (PRE) {
                    // the A chunk's hi and lo parts and the factor chunk into one stage
                    for (int kc = kc0; kc < kc1 && ok; ++kc, ++it) {
                        const int j = (int)(it % S_op);
                        const uint32_t uj = (uint32_t)(it / S_op);
                        if (!(ok = mbar_wait(op_empty(j), (uj & 1u) ^ 1u, abort_flag, a.wait_limit))) break;
                        const uint32_t bbytes = a.b_resident ? 0u : 2u * (uint32_t)a.Rpadp[pass] * ROWB;
                        mbar_expect_tx(op_full(j), 2u * OPA + bbytes);
                        const uint32_t adst = op0 + (uint32_t)j * 2u * OPA;
                        tma_load_2d(adst, &tmT, kc * BK, (int)(tile * BM), op_full(j));
                        tma_load_2d(adst + OPA, &tmTlo, kc * BK, (int)(tile * BM), op_full(j));
                        if (!a.b_resident) {
                            const uint32_t bdst = b0 + (uint32_t)j * bchunk;
                            tma_load_2d(bdst, mhi, kc * BK, 0, op_full(j));
                            tma_load_2d(bdst + bpart, mlo, kc * BK, 0, op_full(j));
                        }
                    }
                    continue;
                }
                for (int kc = kc0; kc < kc1 && ok; ++kc, ++it) {
                    const int s = (int)(it % S_stg);
                    const uint32_t us = (uint32_t)(it / S_stg);
                    if (!(ok = mbar_wait(stg_empty(s), (us & 1u) ^ 1u, abort_flag, a.wait_limit))) break;
                    mbar_expect_tx(stg_full(s), STG);
                    const uint32_t dst = stg0 + (uint32_t)s * STG;
                    if (MODE == 0) {
                        const int row0 = (int)(tile * BM);
#pragma unroll
                        for (int bx = 0; bx < BK / 32; ++bx)
                            tma_load_2d(dst + bx * (BM * 128), &tmT, kc * BK + 32 * bx, row0, stg_full(s));
                    } else {
                        const int p = (int)(tile / a.tiles_per_p);
                        const int q0 = (int)((tile % a.tiles_per_p) * BM);
                        tma_load_3d(dst, &tmT, q0, kc * BK, p, stg_full(s));
                    }
                    if (!a.b_resident) {
                        const int j = (int)(it % S_op);
                        const uint32_t uj = (uint32_t)(it / S_op);
                        if (!(ok = mbar_wait(op_empty(j), (uj & 1u) ^ 1u, abort_flag, a.wait_limit))) break;
                        // this pass's operand rows only (a smaller last pass leaves the
                        // rest of the slot unused)
                        mbar_expect_tx(op_full(j), 2u * (uint32_t)a.Rpadp[pass] * ROWB);
                        const uint32_t bdst = b0 + (uint32_t)j * bchunk;
                        tma_load_2d(bdst, mhi, kc * BK, 0, op_full(j));
                        tma_load_2d(bdst + bpart, mlo, kc * BK, 0, op_full(j));
                    }
                }
            }
            if (!ok) {
                // drain: wait (bounded) for the copies issued into the last stages
                volatile int never = 0;
                if (PRE) {
                    for (int64_t k = (it > S_op ? it - S_op : 0); k < it; ++k)
                        mbar_wait(op_full((int)(k % S_op)), (uint32_t)((k / S_op) & 1), &never, DRAIN_LIMIT);
                } else {
                    for (int64_t k = (it > S_stg ? it - S_stg : 0); k <= it; ++k)
                        mbar_wait(stg_full((int)(k % S_stg)), (uint32_t)((k / S_stg) & 1), &never, DRAIN_LIMIT);
                }
                if (a.b_resident) mbar_wait(b_full, 0u, &never, DRAIN_LIMIT);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            int64_t it = 0;
            int lt = 0;
            bool ok = true;
            if (a.b_resident) ok = mbar_wait(b_full, 0u, abort_flag, a.wait_limit);
            const int64_t nwork = a.ntiles * a.nsk * a.npass;
            for (int64_t w = blockIdx.x; w < nwork && ok; w += gridDim.x, ++lt) {
                const int ks = (int)((w / a.npass) % a.nsk);
                const int pass = (int)(w % a.npass);
                const uint32_t idesc = a.idescp[pass];
                const int kc0 = ks * a.nk / a.nsk, kc1 = (ks + 1) * a.nk / a.nsk;
                const int buf = lt % NSETS;
                const uint32_t ub = (uint32_t)(lt / NSETS);
                if (!(ok = mbar_wait(acc_empty(buf), (ub & 1u) ^ 1u, abort_flag, a.wait_limit))) break;
                tc_fence_after();
                const uint32_t dt = tmem_base + (uint32_t)(buf * a.set_cols);
                const uint32_t dcorr = dt + (uint32_t)(a.nsplit * a.Rpad);
                for (int kc = kc0; kc < kc1; ++kc, ++it) {
                    const int rc = kc - kc0;  // chunk index within this work item
                    const uint32_t dmain = dt + (uint32_t)((rc % a.nsplit) * a.Rpad);
                    const int j = (int)(it % S_op);
                    if (!(ok = mbar_wait(op_full(j), (uint32_t)((it / S_op) & 1), abort_flag, a.wait_limit))) break;
                    tc_fence_after();
                    const uint32_t ahi = op0 + (uint32_t)j * 2u * OPA, alo = ahi + OPA;
                    const uint32_t bhi = b0 + (uint32_t)(a.b_resident ? kc : j) * bchunk, blo = bhi + bpart;
                    auto desc = [](uint32_t addr) { return WIDE ? sw64_desc(addr) : sw128_desc(addr); };
#pragma unroll
                    for (int kk = 0; kk < KSTEPS; ++kk) {  // k-steps of 32 bytes per operand row
                        const uint32_t off = (uint32_t)kk * 32u;
                        const uint32_t accm = (rc >= a.nsplit || kk > 0) ? 1u : 0u;
                        tc_mma<KIND>(dmain, desc(ahi + off), desc(bhi + off), idesc, accm);
                        if (a.x3) {
                            const uint32_t accc = (rc > 0 || kk > 0) ? 1u : 0u;
                            tc_mma<KIND>(dcorr, desc(ahi + off), desc(blo + off), idesc, accc);
                            tc_mma<KIND>(dcorr, desc(alo + off), desc(bhi + off), idesc, 1u);
                        }
                    }
                    tc_commit(op_empty(j));
                }
                if (!ok) break;
                tc_commit(acc_full(buf));
            }
            if (!ok) {
                // let every MMA issued so far finish before TMEM is released
                tc_commit(drain_bar);
                volatile int never = 0;
                mbar_wait(drain_bar, 0u, &never, DRAIN_LIMIT);
            }
        }
    } else if (!PRE && warp >= 4 && warp < EPI0) {
        // ------------------------------------------------ converters (thread = tile row)
        // the 8 output chunks of a row are handled four at a time, with all their
        // shared-memory loads issued before the first store (the compiler may not
        // move a load above a store to a buffer it cannot tell apart; measured
        // 0.290 -> 0.272 ms at 128^4 R = 64)
        const int m = threadIdx.x - 128;
        constexpr int cbeg = 0;
        constexpr int CPT = WIDE ? 4 : 8;   // output chunks per thread
        const int sw = m & 7;
        int64_t it = 0;
        bool ok = true;
        const int64_t nwork = a.ntiles * a.nsk * a.npass;
        for (int64_t w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
            const int ks = (int)((w / a.npass) % a.nsk);
            const int kc0 = ks * a.nk / a.nsk, kc1 = (ks + 1) * a.nk / a.nsk;
            for (int kc = kc0; kc < kc1; ++kc, ++it) {
                const int s = (int)(it % S_stg);
                const int j = (int)(it % S_op);
                if (!(ok = mbar_wait(stg_full(s), (uint32_t)((it / S_stg) & 1), abort_flag, a.wait_limit))) break;
                if (!(ok = mbar_wait(op_empty(j), (uint32_t)(((it / S_op) & 1) ^ 1), abort_flag, a.wait_limit))) break;
                const uint8_t* stg = gbase + (stg0 - base) + (size_t)s * STG;
                uint8_t* ophi = gbase + (op0 - base) + (size_t)j * 2 * OPA;
                uint8_t* oplo = ophi + OPA;
#pragma unroll
                for (int g = 0; g < CPT; g += 4) {
                    if (KIND != 1) {
                        float f[4][8];   // output chunk c: k = 8c .. 8c+7
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) {
                            const int c = cbeg + g + cc;
                            if (MODE == 0) {
                                // box c/4 holds k = 32(c/4)..; row m, 16-byte chunk q at q ^ (m & 7)
                                const uint8_t* rowp = stg + (c >> 2) * (BM * 128) + m * 128;
                                const int q0 = (2 * c) & 7;
                                const float4 v0 = *reinterpret_cast<const float4*>(rowp + ((q0 ^ sw) << 4));
                                const float4 v1 = *reinterpret_cast<const float4*>(rowp + (((q0 + 1) ^ sw) << 4));
                                f[cc][0] = v0.x; f[cc][1] = v0.y; f[cc][2] = v0.z; f[cc][3] = v0.w;
                                f[cc][4] = v1.x; f[cc][5] = v1.y; f[cc][6] = v1.z; f[cc][7] = v1.w;
                            } else {
                                const float* col = reinterpret_cast<const float*>(stg) + m;  // [BK][128]
#pragma unroll
                                for (int i = 0; i < 8; ++i) f[cc][i] = col[(8 * c + i) * BM];
                            }
                        }
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) {
                            const int c = cbeg + g + cc;
                            uint4 hi, lo;
                            if (KIND == 2)
                                split8_f16(f[cc], a.tscale, hi, lo);
                            else
                                split8_bf16(f[cc], hi, lo);
                            // 16-byte chunk c of row m: 128-byte rows, chunk at c ^ (m mod 8);
                            // wide: 64-byte rows, chunk at c ^ ((m / 2) mod 4)
                            const int pos = WIDE ? ((c ^ ((m >> 1) & 3)) << 4) + m * 64 : ((c ^ sw) << 4) + m * 128;
                            *reinterpret_cast<uint4*>(ophi + pos) = hi;
                            *reinterpret_cast<uint4*>(oplo + pos) = lo;
                        }
                    } else {
                        float4 v[4];     // output chunk c: k = 4c .. 4c+3
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) {
                            const int c = cbeg + g + cc;
                            if (MODE == 0) {
                                v[cc] = *reinterpret_cast<const float4*>(stg + m * 128 + ((c ^ sw) << 4));
                            } else {
                                const float* col = reinterpret_cast<const float*>(stg) + m;
                                v[cc] = make_float4(col[(4 * c) * BM], col[(4 * c + 1) * BM],
                                                    col[(4 * c + 2) * BM], col[(4 * c + 3) * BM]);
                            }
                        }
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) {
                            const int c = cbeg + g + cc;
                            float4 hi, lo;
                            split4_tf32(v[cc], hi, lo);
                            const int pos = ((c ^ sw) << 4) + m * 128;
                            *reinterpret_cast<float4*>(ophi + pos) = hi;
                            *reinterpret_cast<float4*>(oplo + pos) = lo;
                        }
                    }
                }
                fence_proxy_async();
                mbar_arrive(stg_empty(s));
                mbar_arrive(op_full(j));
            }
        }
    } else if (warp >= EPI0) {
        // ------------------------------------------------ epilogue (thread = TMEM lane = row)
        const int quad = warp & 3;             // TMEM lane quarter (warp id mod 4)
        const int half = (warp - EPI0) >> 2;  // which alternate 16-column groups
        constexpr int NHALF = NEPI / 4;
        float* tb = reinterpret_cast<float*>(gbase + (epi0 - base)) + (warp - EPI0) * 32 * EPI_STRIDE;
        // first-child pieces and their segment keys (-1: none), double-buffered by tile
        float* cpart = reinterpret_cast<float*>(gbase + (child0 - base));           // [2][4][2][128]
        long long* ckey = reinterpret_cast<long long*>(gbase + (child0 - base) + 2 * 4 * 2 * 128 * 4);
        const int sc = CHILD ? a.sc : 1;
        // sc a multiple of 32: every warp's 32 rows lie in one segment (tiles and
        // warps start at multiples of 32), so a warp's share is a plain column sum
        constexpr bool aligned = CHILD == 1;
        const int qq = lane & 3, rr = lane >> 2;  // transposed layout: rows rr + 8i, columns 4qq..4qq+3
        const bool avec = CHILD && (a.R % 4 == 0);
        int lt = 0;
        bool ok = true;
        const int64_t nwork = a.ntiles * a.nsk * a.npass;
        for (int64_t w = blockIdx.x; w < nwork && ok; w += gridDim.x, ++lt) {
            const int64_t tile = w / ((int64_t)a.nsk * a.npass);
            const int pass = (int)(w % a.npass);
            const int Rw = a.Rp[pass], Rpw = a.Rpadp[pass];
            float* Xs = a.X + (int64_t)((w / a.npass) % a.nsk) * a.slice + PW * pass;
            const int buf = lt % NSETS;
            if (!(ok = mbar_wait(acc_full(buf), (uint32_t)((lt / NSETS) & 1), abort_flag, a.wait_limit))) break;
            tc_fence_after();
            int64_t g0;       // global row of this warp's first row
            int64_t gend;     // rows g0 + r < gend belong to this tile
            if (MODE == 0) {
                g0 = tile * BM + quad * 32;
                gend = a.PQ;
            } else {
                const int64_t p = tile / a.tiles_per_p;
                const int64_t qb = (tile % a.tiles_per_p) * BM;
                g0 = p * a.Q + qb + quad * 32;
                gend = p * a.Q + a.Q;  // the last tile of a p is ragged when BM does not divide Q
            }
            // first child: rows of the transposed layout and their factor rows
            int jt[4] = {0, 0, 0, 0};
            long long key = -1;           // general path: this lane's row segment
            bool head = false, head_complete = false;
            int piece = 0;
            int64_t glast = g0;
            if (CHILD) {
                if (aligned) {
                    // g0 % 32 == 0 and sc % 32 == 0: the warp's rows are consecutive in one segment
                    const int j0 = (int)(g0 % sc);
#pragma unroll
                    for (int i = 0; i < 4; ++i) jt[i] = j0 + rr + 8 * i;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) jt[i] = (int)((g0 + rr + 8 * i) % sc);
                }
                glast = (gend - 1 < g0 + 31) ? gend - 1 : g0 + 31;
                if (!aligned) {
                    const int64_t gme = g0 + lane;
                    const bool vme = gme < gend;
                    key = vme ? (long long)(gme / sc) : -1ll;
                    const long long kprev = __shfl_up_sync(0xffffffffu, key, 1);
                    head = vme && (lane == 0 || kprev != key);
                    if (head) {
                        const int64_t S = (int64_t)key * sc, E = S + sc - 1;
                        head_complete = S >= g0 && E <= glast;
                        piece = lane == 0 ? 0 : 1;
                    }
                }
            }
            float* cpart = reinterpret_cast<float*>(gbase + (child0 - base));           // [2][4][2][128]
            long long* ckey = reinterpret_cast<long long*>(gbase + (child0 - base) + 2 * 4 * 2 * 128 * 4);
            float* mypart = cpart + (((lt & 1) * 4 + quad) * 2 + piece) * 128;
            const uint32_t taddr =
                tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * a.set_cols);
            for (int c0 = 16 * half; c0 < Rpw; c0 += 16 * NHALF) {
                float v[16];
                // scaled fp16 parts: this lane's four output columns' scales, read
                // before the accumulator loads so that their latency overlaps
                float4 cs4 = make_float4(1.f, 1.f, 1.f, 1.f);
                if (KIND == 2)
                    cs4 = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(gbase + (cs0 - base)) +
                                                           PW * pass + c0 + 4 * qq);
                // corrections first (last accumulator), then the hi*hi partial sums;
                // up to three accumulators per TMEM round trip
                const uint32_t tcol = taddr + (uint32_t)c0;
                const uint32_t rp = (uint32_t)a.Rpad;
                int ac = a.nacc - 1;
                if (ac >= 2) {
                    float w1[16], w2[16];
                    tmem_ld16x3(tcol + ac * rp, tcol + (ac - 1) * rp, tcol + (ac - 2) * rp, v, w1, w2);
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += w1[i];
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += w2[i];
                    ac -= 3;
                } else if (ac == 1) {
                    float w1[16];
                    tmem_ld16x2(tcol + rp, tcol, v, w1);
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += w1[i];
                    ac = -1;
                } else {
                    tmem_ld16(tcol, v);
                    ac = -1;
                }
                for (; ac >= 0; --ac) {
                    float w[16];
                    tmem_ld16(tcol + ac * rp, w);
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += w[i];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    *reinterpret_cast<float4*>(tb + lane * EPI_STRIDE + 4 * q) =
                        make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                __syncwarp();
                // lanes 4i..4i+3 write the 64 bytes of row i (+8, +16, +24): full sectors
                const int q = qq;
                const int col = c0 + 4 * q;
                float4 csum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = rr + 8 * i;
                    const int64_t g = g0 + r;
                    if (g < gend && col < Rw) {
                        float4 w = *reinterpret_cast<const float4*>(tb + r * EPI_STRIDE + 4 * q);
                        if (KIND == 2) {
                            // undo the powers of two of T and of the factor's columns (exact)
                            w.x *= cs4.x; w.y *= cs4.y; w.z *= cs4.z; w.w *= cs4.w;
                        }
                        float* dst = Xs + g * (int64_t)a.ldx + col;
                        if (((Rw | a.ldx) & 3) == 0) {
                            *reinterpret_cast<float4*>(dst) = w;
                        } else {
                            dst[0] = w.x;
                            if (col + 1 < Rw) dst[1] = w.y;
                            if (col + 2 < Rw) dst[2] = w.z;
                            if (col + 3 < Rw) dst[3] = w.w;
                        }
                        if (CHILD) {
                            // weight by the contracted factor's row (coalesced: 4 lanes
                            // read one 64-byte piece of it)
                            const int64_t ao = (int64_t)jt[i] * a.R + col;
                            float4 f;
                            if (a.ac_bytes > 0) {
                                const float* ap = reinterpret_cast<const float*>(gbase + (ac0 - base)) + ao;
                                if (avec) {
                                    f = *reinterpret_cast<const float4*>(ap);
                                } else {
                                    f.x = ap[0];
                                    f.y = col + 1 < Rw ? ap[1] : 0.f;
                                    f.z = col + 2 < Rw ? ap[2] : 0.f;
                                    f.w = col + 3 < Rw ? ap[3] : 0.f;
                                }
                            } else {
                                const float* ap = a.Ac + ao;
                                if (avec) {
                                    f = __ldg(reinterpret_cast<const float4*>(ap));
                                } else {
                                    f.x = __ldg(ap);
                                    f.y = col + 1 < Rw ? __ldg(ap + 1) : 0.f;
                                    f.z = col + 2 < Rw ? __ldg(ap + 2) : 0.f;
                                    f.w = col + 3 < Rw ? __ldg(ap + 3) : 0.f;
                                }
                            }
                            if (aligned) {
                                csum.x = fmaf(w.x, f.x, csum.x); csum.y = fmaf(w.y, f.y, csum.y);
                                csum.z = fmaf(w.z, f.z, csum.z); csum.w = fmaf(w.w, f.w, csum.w);
                            } else {
                                *reinterpret_cast<float4*>(tb + r * EPI_STRIDE + 4 * q) =
                                    make_float4(w.x * f.x, w.y * f.y, w.z * f.z, w.w * f.w);
                            }
                        }
                    } else if (CHILD && !aligned) {
                        *reinterpret_cast<float4*>(tb + r * EPI_STRIDE + 4 * q) = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
                __syncwarp();
                if (CHILD && aligned) {
                    // the 8 lanes of each column quad hold 4 rows each: add them up
#pragma unroll
                    for (int off = 4; off < 32; off <<= 1) {
                        csum.x += __shfl_xor_sync(0xffffffffu, csum.x, off);
                        csum.y += __shfl_xor_sync(0xffffffffu, csum.y, off);
                        csum.z += __shfl_xor_sync(0xffffffffu, csum.z, off);
                        csum.w += __shfl_xor_sync(0xffffffffu, csum.w, off);
                    }
                    if (rr == 0 && g0 < gend && col < Rw) {
                        // sc == 32: the warp is the whole segment; else its piece
                        float* dst = (sc == 32 ? a.Yc : a.cws) + (g0 >> 5) * (int64_t)a.ldx + col;
                        if (((Rw | a.ldx) & 3) == 0) {
                            *reinterpret_cast<float4*>(dst) = csum;
                        } else {
                            dst[0] = csum.x;
                            if (col + 1 < Rw) dst[1] = csum.y;
                            if (col + 2 < Rw) dst[2] = csum.z;
                            if (col + 3 < Rw) dst[3] = csum.w;
                        }
                    }
                } else if (CHILD) {
                    // general segments: this lane's row of weighted values back from
                    // the buffer, then segmented suffix sums over the lanes; the first
                    // lane of every segment ends with the warp's part of it
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const float4 t4 = *reinterpret_cast<const float4*>(tb + lane * EPI_STRIDE + 4 * q4);
                        v[4 * q4] = t4.x; v[4 * q4 + 1] = t4.y; v[4 * q4 + 2] = t4.z; v[4 * q4 + 3] = t4.w;
                    }
                    __syncwarp();
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const long long kp = __shfl_down_sync(0xffffffffu, key, off);
                        const bool take = lane + off < 32 && kp == key;
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const float t = __shfl_down_sync(0xffffffffu, v[i], off);
                            if (take) v[i] += t;
                        }
                    }
                    if (head) {
                        if (head_complete) {
                            float* yrow = a.Yc + (int64_t)key * a.ldx + c0;
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if (c0 + i < Rw) yrow[i] = v[i];
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; ++i) mypart[c0 + i] = v[i];
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acc_empty(buf));
            if (CHILD && !aligned) {
                // keys of this warp's two boundary pieces: 0 = the segment of its first
                // row, 1 = a later segment that runs past its last row
                if (lane == 0) {
                    long long k0 = -1, k1 = -1;
                    if (g0 < gend) {
                        const int64_t a0 = g0 / sc;
                        if (!(a0 * sc >= g0 && a0 * sc + sc - 1 <= glast)) k0 = a0;
                        const int64_t al = glast / sc;
                        if (al * sc > g0 && al * sc + sc - 1 > glast) k1 = al;
                    }
                    ckey[((lt & 1) * 4 + quad) * 2 + 0] = k0;
                    ckey[((lt & 1) * 4 + quad) * 2 + 1] = k1;
                }
                __syncwarp();
                mbar_arrive(epi_bar(lt & 1));
                if (!(ok = mbar_wait(epi_bar(lt & 1), (uint32_t)((lt >> 1) & 1), abort_flag, a.wait_limit))) break;
                if (quad == 0) {
                    // warp 8 adds the pieces of each segment in row order; a segment
                    // inside the tile is final, one that crosses the tile's first row
                    // (piece 0) or last row (piece 1) waits for the cross-tile sum
                    const int64_t t0 = g0;
                    const int64_t tl = (gend - 1 < t0 + 127) ? gend - 1 : t0 + 127;
                    const float* pb = cpart + (lt & 1) * 4 * 2 * 128;
                    const long long* kb = ckey + (lt & 1) * 4 * 2;
                    for (int col = lane; col < Rw; col += 32) {
                        long long ck = -1;
                        float acc = 0.f;
                        for (int e = 0; e <= 8; ++e) {
                            const long long k = e < 8 ? kb[e] : -2ll;
                            if (e < 8 && k < 0) continue;
                            if (e < 8 && k == ck) {
                                acc += pb[e * 128 + col];
                                continue;
                            }
                            if (ck >= 0) {
                                const int64_t S = (int64_t)ck * sc, E = S + sc - 1;
                                if (S >= t0 && E <= tl)
                                    a.Yc[(int64_t)ck * a.ldx + col] = acc;
                                else
                                    a.cws[(tile * 2 + (S <= t0 ? 0 : 1)) * (int64_t)a.ldx + col] = acc;
                            }
                            if (e < 8) {
                                ck = k;
                                acc = pb[e * 128 + col];
                            }
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(a.tmem_cols)
                     : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicOr(a.dev_err, (unsigned)DEVERR_TIMEOUT);
}

// ------------------------------------------------------------------ host helpers
}  // namespace

namespace cpk {

// R > 128 runs as column passes: of at most 256 for the 16-bit parts (wide
// kernel: one MMA N = 256, one TMEM accumulator set), of at most 128 for tf32
// parts; pass p multiplies by factor rows (pass width) p .. and writes those columns.
constexpr int MAX_PASS = 4, PASS_COLS = 128, PASS_COLS_WIDE = 256;

struct TcPass {
    CUtensorMap tmBhi, tmBlo;
    int R, Rpad, S_stg, b_resident;
};

struct TcPlan {
    CUtensorMap tmT;
    CUtensorMap tmTlo;   // stored parts: the lo map (tmT holds the hi map)
    TcPass pass[MAX_PASS];
    int npass;
    int mode;   // kernel MODE
    int kind;   // kernel KIND
    int64_t P, Q, PQ;
    int K, R, nk, S_op;
    float tscale = 1.f;              // fp16 parts: power of two applied to T
    const float* colinv = nullptr;   // fp16 parts: per-column output scale (Rpad floats)
    bool depth_bound = false;        // split K so that no accumulator sums more than 64 MMAs
    bool wide = false;               // R > 128 with 16-bit parts: the wide kernel
    bool pre = false;                // the A operand from T's stored 16-bit parts
};

bool ttm_tc_supported(int64_t P, int K, int64_t Q, int R) {
    const int Rpad = (R + 15) / 16 * 16;
    if (Rpad > MAX_PASS * PASS_COLS || K < 1 || P * Q < 1) return false;
    if (Q == 1) return K % 4 == 0 && P <= ((int64_t)1 << 31);
    // ragged Q: the last tile of each p reads past Q (TMA fills zeros) and
    // writes only its rows q < Q; the row stride Q * 4 bytes must be 16-byte aligned
    return Q % 4 == 0 && Q <= ((int64_t)1 << 31) && P <= ((int64_t)1 << 31);
}

TcPlan* ttm_tc_plan(const float* T, int64_t P, int K, int64_t Q, int R, int kind, const void* bhi,
                    const void* blo, int Rpad, int Kpad, float tscale, const float* colinv, const void* pre_hi,
                    const void* pre_lo, bool pre_narrow) {
    if (!ttm_tc_supported(P, K, Q, R) || ((uintptr_t)T & 15)) return nullptr;
    if (kind == 2 && (!colinv || ((uintptr_t)colinv & 15))) return nullptr;
    EncodeTiledFn enc = encoder();
    if (!enc) return nullptr;
    // stored parts: rows of K 16-bit values must be 16-byte aligned for the TMA
    const bool pre = kind != 1 && R > PASS_COLS && pre_hi && pre_lo && K % 8 == 0 &&
                     P * Q <= ((int64_t)1 << 31) && (((uintptr_t)pre_hi | (uintptr_t)pre_lo) & 15) == 0;
    // R > 128 with 16-bit parts: one pass of up to 256 columns (one accumulator
    // set), or with stored parts on request passes of 128 with two sets (the
    // epilogue overlaps the next work item; A is read once per pass)
    const bool wide = kind != 1 && R > PASS_COLS && !(pre && pre_narrow);
    const int BK = (kind == 1 || wide) ? 32 : 64;
    const int pcols = wide ? PASS_COLS_WIDE : PASS_COLS;
    const size_t rowb = wide ? 64 : 128;
    TcPlan* pl = new TcPlan();
    pl->wide = wide;
    pl->pre = pre;
    pl->kind = kind;
    pl->P = P;
    pl->Q = Q;
    pl->PQ = P * Q;
    pl->K = K;
    pl->R = R;
    pl->nk = (K + BK - 1) / BK;
    pl->S_op = pre ? (wide ? 4 : 3) : (wide ? 3 : 2);   // wide: 32-k chunks, a deeper operand ring
    pl->npass = (R + pcols - 1) / pcols;
    pl->tscale = tscale;
    pl->colinv = colinv;
    const int esz = kind == 1 ? 4 : 2;
    const CUtensorMapDataType bt = kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const cuuint32_t es[3] = {1, 1, 1};
    for (int q = 0; q < pl->npass; ++q) {
        TcPass& ps = pl->pass[q];
        ps.R = std::min(pcols, R - q * pcols);
        ps.Rpad = pl->npass == 1 ? Rpad : (ps.R + 15) / 16 * 16;
        // with two passes the operand slots are refilled per work item
        ps.b_resident = (pl->npass == 1 && (size_t)pl->nk * 2 * ps.Rpad * rowb <= 64 * 1024) ? 1 : 0;
        ps.S_stg = 0;
        bool fits = false;
        if (pre) {
            // no staging ring
            fits = layout_bytes(0, pl->S_op, ps.Rpad, pl->nk, ps.b_resident, BK, 8, kind, false, 0, wide) <= SMEM_LIMIT;
        } else {
            for (int st = MAX_STG; st >= 2 && !fits; --st)
                if (layout_bytes(st, pl->S_op, ps.Rpad, pl->nk, ps.b_resident, BK, epi_warps_for(ps.Rpad, kind), kind,
                                 false, 0, wide) <= SMEM_LIMIT) {
                    ps.S_stg = st;
                    fits = true;
                }
        }
        if (!fits) {
            delete pl;
            return nullptr;
        }
        // rows pcols q .. pcols q + Rpad_q - 1 of the [Rpad][Kpad] operand copies
        const size_t off = (size_t)q * pcols * Kpad * esz;
        const CUtensorMapSwizzle bsw = wide ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
        const cuuint64_t bd[2] = {(cuuint64_t)Kpad, (cuuint64_t)ps.Rpad};
        const cuuint64_t bs[1] = {(cuuint64_t)Kpad * esz};
        const cuuint32_t bb[2] = {(cuuint32_t)BK, (cuuint32_t)ps.Rpad};
        CUresult r2 = enc(&ps.tmBhi, bt, 2, (void*)((const char*)bhi + off), bd, bs, bb, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, bsw,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        CUresult r3 = enc(&ps.tmBlo, bt, 2, (void*)((const char*)blo + off), bd, bs, bb, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, bsw,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r2 != CUDA_SUCCESS || r3 != CUDA_SUCCESS) {
            delete pl;
            return nullptr;
        }
    }
    CUresult r1;
    if (pre) {
        // rows = the kept modes flattened, K contiguous: the last-mode addressing
        pl->mode = 0;
        const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)(P * Q)};
        const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
        // one operand row per tile row: BK 16-bit values (64 bytes wide, 128 narrow)
        const cuuint32_t box[2] = {(cuuint32_t)BK, BM};
        const CUtensorMapSwizzle asw = wide ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
        const CUtensorMapDataType pt = kind == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
        r1 = enc(&pl->tmT, pt, 2, (void*)pre_hi, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, asw,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r1 == CUDA_SUCCESS)
            r1 = enc(&pl->tmTlo, pt, 2, (void*)pre_lo, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, asw,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else if (Q == 1) {
        pl->mode = 0;
        const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)P};
        const cuuint64_t strides[1] = {(cuuint64_t)K * 4};
        const cuuint32_t box[2] = {32, BM};
        r1 = enc(&pl->tmT, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)T, dims, strides, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        pl->mode = 1;
        const cuuint64_t dims[3] = {(cuuint64_t)Q, (cuuint64_t)K, (cuuint64_t)P};
        const cuuint64_t strides[2] = {(cuuint64_t)Q * 4, (cuuint64_t)Q * K * 4};
        const cuuint32_t box[3] = {BM, (cuuint32_t)BK, 1};
        r1 = enc(&pl->tmT, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)T, dims, strides, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r1 != CUDA_SUCCESS) {
        delete pl;
        return nullptr;
    }
    return pl;
}

void ttm_tc_plan_free(TcPlan* p) { delete p; }

void ttm_tc_set_tscale(TcPlan* p, float tscale) {
    if (p) p->tscale = tscale;
}

int ttm_tc_kind(const TcPlan* p) { return p ? p->kind : -1; }

static int64_t plan_tiles(const TcPlan* pl) {
    return pl->mode == 1 ? pl->P * ((pl->Q + BM - 1) / BM) : (pl->PQ + BM - 1) / BM;
}

// hi*hi accumulators of one tile with three products per term (the corrections
// take one more of the 256 TMEM columns a set may hold); single-product
// precisions have one more, so the bound derived from this is conservative
static int plan_nsplit(const TcPlan* pl) {
    int nsplit = 256 / pl->pass[0].Rpad - 1;
    if (nsplit > 4) nsplit = 4;
    return nsplit < 1 ? 1 : nsplit;
}

bool ttm_tc_stored_parts(const TcPlan* pl) { return pl && pl->pre; }

int ttm_tc_splitk(const TcPlan* pl, int num_sms) {
    // split K when the row tiles alone cannot fill the GPU and K is long enough
    const int64_t nt = plan_tiles(pl);
    int nsk = 1;
    if (!pl->pass[0].b_resident && nt < 2 * (int64_t)num_sms && pl->nk >= 8) {
        nsk = (int)((4 * (int64_t)num_sms + nt - 1) / nt);
        if (nsk > pl->nk / 4) nsk = pl->nk / 4;
        if (nsk > 16) nsk = 16;
    }
    if (pl->depth_bound) {
        // the tensor core truncates its FP32 accumulation once per instruction
        // (16 k): at most 64 instructions per accumulator keep that bias near 2^-19
        // of the sum; longer contractions (the fused two-mode operand, K = s_a s_b)
        // are split, and their slices added with round-to-nearest
        const int64_t kslice = (int64_t)64 * 16 * plan_nsplit(pl);
        const int64_t need = ((int64_t)pl->K + kslice - 1) / kslice;
        if (need > nsk) nsk = (int)std::min<int64_t>(need, pl->nk);
    }
    return nsk < 1 ? 1 : nsk;
}

int ttm_tc_depth_slices(const TcPlan* pl) {
    const int64_t kslice = (int64_t)64 * 16 * plan_nsplit(pl);
    return (int)(((int64_t)pl->K + kslice - 1) / kslice);
}

void ttm_tc_set_depth_bound(TcPlan* p, bool on) {
    if (p) p->depth_bound = on;
}

int64_t ttm_tc_rows(const TcPlan* pl) { return pl->PQ; }

template <int MODE, int KIND, int CHILD, int EW, int WIDE = 0, int PRE = 0>
static cudaError_t launch(const TcPlan* pl, const TcArgs& a, size_t smem, unsigned grid,
                          cudaStream_t st) {
    // the shared-memory limit once per device (every layout stays below it)
    static std::atomic<unsigned> set_on{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned bit = 1u << (dev & 31);
    if (!(set_on.load() & bit)) {
        e = cudaFuncSetAttribute(k_ttm_tc<MODE, KIND, CHILD, EW, WIDE, PRE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_LIMIT);
        if (e != cudaSuccess) return e;
        set_on.fetch_or(bit);
    }
    if (smem > SMEM_LIMIT) return cudaErrorInvalidValue;
    // passes beyond npass repeat pass 0's maps (never read)
    auto ps = [&](int q) -> const TcPass& { return pl->pass[q < pl->npass ? q : 0]; };
    // tmTlo is read only with stored parts (PRE)
    return pdl::launch(k_ttm_tc<MODE, KIND, CHILD, EW, WIDE, PRE>, grid, nthreads(EW, CHILD), smem, st, pl->tmT,
                       ps(0).tmBhi, ps(0).tmBlo, ps(1).tmBhi, ps(1).tmBlo, ps(2).tmBhi, ps(2).tmBlo, ps(3).tmBhi,
                       ps(3).tmBlo, PRE ? pl->tmTlo : pl->tmT, a);
}

namespace {
__global__ void k_splitk_sum(const float* __restrict__ ws, int nsk, int64_t n, float* __restrict__ out) {
    // float4 only when every slice and the output start on 16-byte boundaries
    const bool vec = (n % 4 == 0) && (((uintptr_t)ws | (uintptr_t)out) % 16 == 0);
    const int64_t n4 = vec ? n / 4 : 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        float4 acc = __ldg(reinterpret_cast<const float4*>(ws) + i);
        for (int s = 1; s < nsk; ++s) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(ws + (int64_t)s * n) + i);
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
        }
        reinterpret_cast<float4*>(out)[i] = acc;
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float acc = ws[i];
        for (int s = 1; s < nsk; ++s) acc += ws[(int64_t)s * n + i];
        out[i] = acc;
    }
}
}  // namespace

namespace {
// one value's 16-bit parts, as the converter warps split it: fp16 of y = x tscale
// (KIND 2) or bf16 of x (KIND 0); hi = rn(y), lo = rn(y - hi)
template <int KIND>
__device__ __forceinline__ void split_one(float x, float tscale, uint16_t& h, uint16_t& l) {
    if (KIND == 2) {
        const float y = x * tscale;
        const __half hh = __float2half_rn(y);
        h = __half_as_ushort(hh);
        l = __half_as_ushort(__float2half_rn(y - __half2float(hh)));
    } else {
        const __nv_bfloat16 hb = __float2bfloat16_rn(x);
        h = __bfloat16_as_ushort(hb);
        l = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(hb)));
    }
}
// T viewed as [P][K][Q] -> parts [P][Q][K] (the contracted mode innermost), in
// 32 x 32 tiles through shared memory; Q == 1 needs no transpose
template <int KIND>
__global__ void __launch_bounds__(256) k_presplit(const float* __restrict__ T, int64_t P, int K, int64_t Q,
                                                  float tscale, uint16_t* __restrict__ hi, uint16_t* __restrict__ lo) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t q0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 32;
    for (int64_t p = blockIdx.z; p < P; p += gridDim.z) {
        const float* Tp = T + (size_t)p * K * Q;
        for (int i = ty; i < 32; i += 8) {
            const int k = k0 + i;
            const int64_t q = q0 + tx;
            tile[i][tx] = (k < K && q < Q) ? Tp[(size_t)k * Q + q] : 0.f;
        }
        __syncthreads();
        for (int i = ty; i < 32; i += 8) {
            const int64_t q = q0 + i;
            const int k = k0 + tx;
            if (q < Q && k < K) {
                uint16_t h, l;
                split_one<KIND>(tile[tx][i], tscale, h, l);
                const size_t o = ((size_t)p * Q + q) * K + k;
                hi[o] = h;
                lo[o] = l;
            }
        }
        __syncthreads();
    }
}
template <int KIND>
__global__ void __launch_bounds__(256) k_presplit_flat(const float* __restrict__ T, int64_t n, float tscale,
                                                       uint16_t* __restrict__ hi, uint16_t* __restrict__ lo) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint16_t h, l;
        split_one<KIND>(T[i], tscale, h, l);
        hi[i] = h;
        lo[i] = l;
    }
}
}  // namespace

cudaError_t ttm_presplit(const float* T, int64_t P, int K, int64_t Q, int kind, float tscale, uint16_t* hi,
                         uint16_t* lo, int num_sms, cudaStream_t st) {
    if (kind != 0 && kind != 2) return cudaErrorInvalidValue;
    if (Q == 1) {
        const int64_t n = P * (int64_t)K;
        int64_t blocks = (n + 255) / 256;
        if (blocks > 16 * (int64_t)num_sms) blocks = 16 * (int64_t)num_sms;
        if (kind == 2) k_presplit_flat<2><<<(unsigned)blocks, 256, 0, st>>>(T, n, tscale, hi, lo);
        else k_presplit_flat<0><<<(unsigned)blocks, 256, 0, st>>>(T, n, tscale, hi, lo);
    } else {
        const int64_t gx = (Q + 31) / 32;
        if (gx > 0x7fffffff) return cudaErrorInvalidValue;
        const dim3 grid((unsigned)gx, (unsigned)((K + 31) / 32), (unsigned)(P < 65535 ? P : 65535));
        if (kind == 2) k_presplit<2><<<grid, 256, 0, st>>>(T, P, K, Q, tscale, hi, lo);
        else k_presplit<0><<<grid, 256, 0, st>>>(T, P, K, Q, tscale, hi, lo);
    }
    return cudaGetLastError();
}

bool ttm_tc_child_ok(const TcPlan* pl, int sc) {
    // one column pass, rows = one run of X's row index (last mode, or first mode
    // with nothing before it), and the contracted mode innermost in that index
    if (!pl || pl->npass != 1 || pl->wide || sc < 1) return false;
    if (!(pl->mode == 0 || pl->P == 1)) return false;
    return pl->PQ % sc == 0;
}

int64_t ttm_tc_child_ws_floats(const TcPlan* pl, int sc) {
    if (!ttm_tc_child_ok(pl, sc)) return 0;
    if (sc % 32 == 0) return sc == 32 ? 0 : (pl->PQ / 32) * (int64_t)pl->R;  // one piece per warp
    if (BM % sc == 0) return 0;  // no segment crosses a tile
    return plan_tiles(pl) * 2 * (int64_t)pl->R;
}

namespace {
// sc % 32 == 0: Y[y] = sum of the sc / 32 warp pieces of segment y, in row order.
__global__ void k_child_warpsum(const float* __restrict__ ws, float* __restrict__ Y, int64_t nseg, int nw, int R) {
    const int64_t n = nseg * R;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = i / R;
        const int col = (int)(i - y * R);
        const float* p = ws + (y * nw) * R + col;
        float acc = p[0];
        for (int k = 1; k < nw; ++k) acc += p[(int64_t)k * R];
        Y[i] = acc;
    }
}
// Segments of the first child that cross tiles: piece 0 of every tile they cover
// (piece 1 of the tile where they start, unless they start on its first row),
// added in tile order.
__global__ void k_child_cross(const float* __restrict__ ws, float* __restrict__ Y, int64_t nseg, int sc, int R) {
    const int64_t n = nseg * R;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = i / R;
        const int col = (int)(i - y * R);
        const int64_t S = y * sc, E = S + sc - 1;
        const int64_t tf = S / BM, tl = E / BM;
        if (tf == tl) continue;
        float acc = ws[(tf * 2 + (S == tf * BM ? 0 : 1)) * R + col];
        for (int64_t t = tf + 1; t <= tl; ++t) acc += ws[(t * 2) * R + col];
        Y[y * R + col] = acc;
    }
}
}  // namespace

cudaError_t ttm_tc_run(const TcPlan* pl, float* X, int prec, int num_sms, unsigned* dev_err,
                       cudaStream_t st, float* splitk_ws, const TcChild* child, long long wait_limit) {
    if (!pl) return cudaErrorInvalidValue;
    if (child) {
        if (!ttm_tc_child_ok(pl, child->sc) || !child->Y || !child->Ac) return cudaErrorInvalidValue;
        if (ttm_tc_child_ws_floats(pl, child->sc) > 0 && !child->ws) return cudaErrorInvalidValue;
        splitk_ws = nullptr;  // the epilogue needs complete sums
    }
    const bool bf = (prec == CP_BF16X3 || prec == CP_BF16);
    const bool tf = (prec == CP_TF32X3 || prec == CP_TF32);
    const bool hf = prec == CP_F16X3;
    if ((pl->kind == 0 && !bf) || (pl->kind == 1 && !tf) || (pl->kind == 2 && !hf)) return cudaErrorInvalidValue;
    if (((uintptr_t)X & 15) && (pl->R & 3) == 0) return cudaErrorMisalignedAddress;
    const int nsk = splitk_ws ? ttm_tc_splitk(pl, num_sms) : 1;
    const int BK = (pl->kind == 1 || pl->wide) ? 32 : 64;
    const TcPass& p0 = pl->pass[0];  // the widest pass: it sizes the slots and TMEM sets
    TcArgs a;
    a.X = nsk > 1 ? splitk_ws : X;
    a.ldx = pl->R;
    a.PQ = pl->PQ;
    a.Q = pl->Q;
    a.tiles_per_p = pl->mode == 1 ? (pl->Q + BM - 1) / BM : 1;
    a.ntiles = pl->mode == 1 ? pl->P * a.tiles_per_p : (pl->PQ + BM - 1) / BM;
    a.R = p0.R;
    a.Rpad = p0.Rpad;
    a.nk = pl->nk;
    // the first child's buffers, and its factor in shared memory when that fits
    // with at least two staging stages (else the epilogue reads it from L2), may
    // cost staging stages
    int S_stg = p0.S_stg;
    int ac_bytes = 0;
    if (child) {
        auto fit = [&](int acb) {
            int st2 = p0.S_stg;
            while (st2 > 2 && layout_bytes(st2, pl->S_op, p0.Rpad, pl->nk, p0.b_resident, BK, 4, pl->kind, true, acb) > SMEM_LIMIT)
                --st2;
            return layout_bytes(st2, pl->S_op, p0.Rpad, pl->nk, p0.b_resident, BK, 4, pl->kind, true, acb) <= SMEM_LIMIT ? st2 : 0;
        };
        const int acb = (child->sc * pl->R * 4 + 15) / 16 * 16;
        if (int st2 = fit(acb)) {
            S_stg = st2;
            ac_bytes = acb;
        } else if (int st3 = fit(0)) {
            S_stg = st3;
        } else {
            return cudaErrorInvalidValue;
        }
    }
    a.S_stg = S_stg;
    a.S_op = pl->S_op;
    a.b_resident = p0.b_resident;
    a.x3 = (prec == CP_BF16X3 || prec == CP_TF32X3 || prec == CP_F16X3) ? 1 : 0;
    // accumulators per tile: nsplit for hi*hi (by k-chunk) + 1 for the corrections;
    // two sets must fit the 512 TMEM columns (one set in the wide kernel)
    const int nsets = pl->wide ? 1 : 2;   // the kernel's NSETS
    const int per_set = (512 / nsets) / p0.Rpad;
    int nsplit = per_set - a.x3;
    if (nsplit > 4) nsplit = 4;
    if (nsplit > pl->nk) nsplit = pl->nk;
    if (nsplit < 1) nsplit = 1;
    a.nsplit = nsplit;
    a.nacc = nsplit + a.x3;
    a.set_cols = a.nacc * p0.Rpad;
    int cols = 32;
    while (cols < nsets * a.set_cols) cols *= 2;
    a.tmem_cols = cols;
    // instruction-descriptor operand format: F16 = 0, BF16 = 1 (kind::f16); TF32 = 2 (kind::tf32)
    const uint32_t fmt = pl->kind == 0 ? 1u : (pl->kind == 1 ? 2u : 0u);
    a.npass = pl->npass;
    for (int q = 0; q < MAX_PASS; ++q) {
        const TcPass& ps = pl->pass[q < pl->npass ? q : 0];
        a.Rp[q] = ps.R;
        a.Rpadp[q] = ps.Rpad;
        a.idescp[q] = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(ps.Rpad >> 3) << 17) |
                      ((uint32_t)(BM >> 4) << 24);
    }
    a.idesc = a.idescp[0];
    a.dev_err = dev_err;
    a.nsk = nsk;
    a.slice = pl->PQ * (int64_t)pl->R;
    a.Yc = child ? child->Y : nullptr;
    a.Ac = child ? child->Ac : nullptr;
    a.cws = child ? child->ws : nullptr;
    a.sc = child ? child->sc : 1;
    a.ac_bytes = ac_bytes;
    a.tscale = pl->tscale;
    a.colinv = pl->colinv;
    a.wait_limit = wait_limit > 0 ? wait_limit : DEFAULT_WAIT_LIMIT;
    // first-child epilogues use four warps; plain ones eight for wide passes
    const int ew = child ? 4 : epi_warps_for(p0.Rpad, pl->kind);
    const size_t smem = layout_bytes(S_stg, pl->S_op, p0.Rpad, pl->nk, p0.b_resident, BK, ew, pl->kind, child != nullptr,
                                     ac_bytes, pl->wide);
    const int64_t nwork = a.ntiles * a.nsk * a.npass;
    const unsigned grid = (unsigned)(nwork < num_sms ? nwork : num_sms);
    if (grid == 0) return cudaSuccess;
    cudaError_t e;
    const int ck = child ? (child->sc % 32 == 0 ? 1 : 2) : 0;
#define CP_TTM_LAUNCH(C, W)                                                                               \
    (pl->mode == 0 ? (pl->kind == 0   ? launch<0, 0, C, W>(pl, a, smem, grid, st)                   \
                      : pl->kind == 1 ? launch<0, 1, C, W>(pl, a, smem, grid, st)                   \
                                      : launch<0, 2, C, W>(pl, a, smem, grid, st))                  \
                   : (pl->kind == 0   ? launch<1, 0, C, W>(pl, a, smem, grid, st)                   \
                      : pl->kind == 1 ? launch<1, 1, C, W>(pl, a, smem, grid, st)                   \
                                      : launch<1, 2, C, W>(pl, a, smem, grid, st)))
    if (pl->pre && pl->wide)
        e = pl->kind == 0 ? launch<0, 0, 0, 8, 1, 1>(pl, a, smem, grid, st) : launch<0, 2, 0, 8, 1, 1>(pl, a, smem, grid, st);
    else if (pl->pre)
        e = pl->kind == 0 ? launch<0, 0, 0, 8, 0, 1>(pl, a, smem, grid, st) : launch<0, 2, 0, 8, 0, 1>(pl, a, smem, grid, st);
    else if (pl->wide)
        e = pl->mode == 0 ? (pl->kind == 0 ? launch<0, 0, 0, 8, 1>(pl, a, smem, grid, st)
                                           : launch<0, 2, 0, 8, 1>(pl, a, smem, grid, st))
                          : (pl->kind == 0 ? launch<1, 0, 0, 8, 1>(pl, a, smem, grid, st)
                                           : launch<1, 2, 0, 8, 1>(pl, a, smem, grid, st));
    else if (ck == 1)
        e = CP_TTM_LAUNCH(1, 4);
    else if (ck == 2)
        e = CP_TTM_LAUNCH(2, 4);
    else if (ew == 8)
        e = CP_TTM_LAUNCH(0, 8);
    else
        e = CP_TTM_LAUNCH(0, 4);
#undef CP_TTM_LAUNCH
    if (e != cudaSuccess) return e;
    if (child && ttm_tc_child_ws_floats(pl, child->sc) > 0) {
        const int64_t nseg = pl->PQ / child->sc;
        int64_t blocks = (nseg * pl->R + 255) / 256;
        if (blocks > 4 * num_sms) blocks = 4 * num_sms;
        if (child->sc % 32 == 0)
            k_child_warpsum<<<(unsigned)blocks, 256, 0, st>>>(child->ws, child->Y, nseg, child->sc / 32, pl->R);
        else
            k_child_cross<<<(unsigned)blocks, 256, 0, st>>>(child->ws, child->Y, nseg, child->sc, pl->R);
        return cudaGetLastError();
    }
    if (nsk == 1) return cudaSuccess;
    const int64_t n = pl->PQ * (int64_t)pl->R;
    int64_t blocks = (n / 4 + 255) / 256;
    if (blocks > 4 * num_sms) blocks = 4 * num_sms;
    if (blocks < 1) blocks = 1;
    k_splitk_sum<<<(unsigned)blocks, 256, 0, st>>>(splitk_ws, nsk, n, X);
    return cudaGetLastError();
}

}  // namespace cpk
