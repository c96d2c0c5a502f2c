// Multi-TTV (Sec. II-C): every dimension-tree contraction below the first level.
// An intermediate keeps its modes in increasing order with the rank index r
// fastest, so contracting one of its modes is
//     Y[p][q][r] = sum_k X[p][k][q][r] * A[k][r]
// (p: kept modes before the contracted one, q: those after it).  Reads of X are
// contiguous along (q, r) for every k; the factor is tiny and stays in L1/L2.
// The kernel is bandwidth-bound: one pass over X, 2 flops per element read.
#include "cpals_internal.h"
#include "pdl.h"

namespace {

// VEC consecutive floats (VEC = 4, 2 or 1) as the low lanes of a float4
template <int VEC>
__device__ __forceinline__ float4 ldv(const float* p) {
    if (VEC == 4) return __ldg(reinterpret_cast<const float4*>(p));
    if (VEC == 2) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        return make_float4(v.x, v.y, 0.f, 0.f);
    }
    return make_float4(__ldg(p), 0.f, 0.f, 0.f);
}

// Block = TX outputs (vectors of VEC along r) x KS partial sums over k.  Each
// thread keeps U loads of X in flight: the kernel is bound by how many bytes the
// SMs have outstanding (measured on 128^4 R = 64 roots: 4 in flight gave
// 3.2-3.6 TB/s, 16 in flight with a 4-way k-split 5.4-5.5 TB/s).  R not a multiple
// of 4 uses float2 or float vectors with the same unrolling.
// STRIDE: blocks loop over the chunks of TX outputs (a capped grid); else one
// chunk per block.
template <int VEC, int U, bool STRIDE>
__global__ void __launch_bounds__(256) k_mttv(const float* __restrict__ X,
                                              const float* __restrict__ A,
                                              float* __restrict__ Y, int64_t P, int K, int64_t Q,
                                              int R, int TX, int KS) {
    extern __shared__ float4 red[];  // TX * KS
    pdl::wait();
    pdl::trigger();
    const int RV = R / VEC;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int64_t nout = P * Q * RV;
    const int64_t nchunks = (nout + TX - 1) / TX;
    // grid-stride over chunks of TX outputs: a launch may use fewer blocks than
    // chunks to leave room on every SM for concurrent kernels
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += (STRIDE ? gridDim.x : nchunks)) {
        const int64_t o = ch * TX + tx;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (o < nout) {
            const int64_t pq = o / RV;
            const int rv = (int)(o - pq * RV);
            const int64_t p = pq / Q, q = pq - p * Q;
            const int64_t strideK = Q * R;
            const float* xp = X + (p * K) * strideK + q * R + rv * VEC;
            const float* ap = A + rv * VEC;
            int k = ty;
            for (; k + (U - 1) * KS < K; k += U * KS) {
                float4 x[U], a[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    x[u] = ldv<VEC>(xp + (int64_t)(k + u * KS) * strideK);
                    a[u] = ldv<VEC>(ap + (int64_t)(k + u * KS) * R);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    acc.x = fmaf(x[u].x, a[u].x, acc.x);
                    if (VEC > 1) acc.y = fmaf(x[u].y, a[u].y, acc.y);
                    if (VEC > 2) { acc.z = fmaf(x[u].z, a[u].z, acc.z); acc.w = fmaf(x[u].w, a[u].w, acc.w); }
                }
            }
            for (; k < K; k += KS) {
                const float4 x0 = ldv<VEC>(xp + (int64_t)k * strideK);
                const float4 a0 = ldv<VEC>(ap + (int64_t)k * R);
                acc.x = fmaf(x0.x, a0.x, acc.x);
                if (VEC > 1) acc.y = fmaf(x0.y, a0.y, acc.y);
                if (VEC > 2) { acc.z = fmaf(x0.z, a0.z, acc.z); acc.w = fmaf(x0.w, a0.w, acc.w); }
            }
        }
        red[ty * TX + tx] = acc;
        __syncthreads();
        if (ty == 0 && o < nout) {
            for (int j = 1; j < KS; ++j) {
                float4 v = red[j * TX + tx];
                acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
            }
            if (VEC == 4)
                *reinterpret_cast<float4*>(Y + o * 4) = acc;
            else if (VEC == 2)
                *reinterpret_cast<float2*>(Y + o * 2) = make_float2(acc.x, acc.y);
            else
                Y[o] = acc.x;
        }
        if (STRIDE) __syncthreads();  // red is rewritten by the next chunk
    }
}

}  // namespace

namespace cpk {

cudaError_t mttv(const float* X, const float* A, float* Y, int64_t P, int K, int64_t Q, int R,
                 int num_sms, cudaStream_t st, int max_blocks_per_sm) {
    const uintptr_t al = (uintptr_t)X | (uintptr_t)A | (uintptr_t)Y;
    const int VEC = (R % 4 == 0 && al % 16 == 0) ? 4 : (R % 2 == 0 && al % 8 == 0) ? 2 : 1;
    const int64_t nout = P * Q * (R / VEC);
    // k-split: enough blocks to cover the GPU twice, and at least two rounds of 16
    // loads per thread where K allows a split
    int KS = 1;
    while (KS < 32 && KS < K && (nout * KS) < (int64_t)num_sms * 2 * 256) KS *= 2;
    while (KS < 8 && K / (2 * KS) >= 32) KS *= 2;
    int TX = 256 / KS;
    int64_t nchunks = (nout + TX - 1) / TX;
    const bool stride = max_blocks_per_sm > 0 && nchunks > (int64_t)max_blocks_per_sm * num_sms;
    if (stride) nchunks = (int64_t)max_blocks_per_sm * num_sms;
    const unsigned nblk = (unsigned)nchunks;
    const size_t smem = sizeof(float4) * 256;
#define CP_MTTV_LAUNCH(V)                                                                               \
    (stride ? pdl::launch(k_mttv<V, 16, true>, nblk, 256, smem, st, X, A, Y, P, K, Q, R, TX, KS)        \
            : pdl::launch(k_mttv<V, 16, false>, nblk, 256, smem, st, X, A, Y, P, K, Q, R, TX, KS))
    cudaError_t e;
    if (VEC == 4)
        e = CP_MTTV_LAUNCH(4);
    else if (VEC == 2)
        e = CP_MTTV_LAUNCH(2);
    else
        e = CP_MTTV_LAUNCH(1);
#undef CP_MTTV_LAUNCH
    return e;
}

}  // namespace cpk
