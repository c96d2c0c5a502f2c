// First-level TTM on the CUDA cores in FP32 (Sec. II-C: the contraction of the
// input tensor with one factor matrix, 2 s^N R flops).
//
// The tensor is viewed as T[p][k][q] (p: modes before the contracted mode m,
// k: mode m, q: modes after it); the output keeps the remaining modes in order
// with the rank index fastest: X[p][q][r] = sum_k T[p][k][q] A[k][r].  That is a
// GEMM with M = P*Q rows, inner dimension K = s_m and N = R columns; for m = N-1
// (Q = 1) the tensor rows are K-contiguous, otherwise each p-slice is a K x Q
// matrix with q contiguous, so no transposed copy of T is ever made.
#include "cpals_internal.h"

namespace {

constexpr int BM = 128, BN = 64, BK = 16, TM = 8, TN = 4;  // 16 x 16 threads
constexpr int APAD = 4;                                     // As row padding (floats)

// Tile loaders fill As[BK][BM + APAD] with As[k][m] = T(row g0 + m, k0 + k).
enum { LOAD_QTILE = 0, LOAD_ROWK = 1, LOAD_GENERIC = 2 };

// rowoff (LOAD_GENERIC): offset of T[p][0][q] for this thread's row m = tid & 127
// (fixed for the whole tile), or -1 past the last row
template <int MODE>
__device__ __forceinline__ void load_a(float (*As)[BM + APAD], const float* __restrict__ T,
                                       int64_t g0, int k0, int64_t P, int K, int64_t Q, int tid,
                                       int64_t rowoff) {
    const int64_t PQ = P * Q;
    if (MODE == LOAD_QTILE) {
        // whole tile inside one p-slice, contiguous along m; Q % BM == 0, Q % 4 == 0
        const int64_t p = g0 / Q, q0 = g0 % Q;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            int idx = tid + 256 * j;  // 512 float4
            int k = idx >> 5, m4 = idx & 31;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k0 + k < K)
                v = __ldg(reinterpret_cast<const float4*>(T + (p * K + k0 + k) * Q + q0) + m4);
            *reinterpret_cast<float4*>(&As[k][4 * m4]) = v;
        }
    } else if (MODE == LOAD_ROWK) {
        // Q == 1, K % 4 == 0: row g is T[g*K .. g*K+K)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            int idx = tid + 256 * j;
            int m = idx >> 2, k4 = idx & 3;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            int64_t g = g0 + m;
            if (g < PQ && k0 + 4 * k4 < K)
                v = __ldg(reinterpret_cast<const float4*>(T + g * K + k0) + k4);
            As[4 * k4 + 0][m] = v.x;
            As[4 * k4 + 1][m] = v.y;
            As[4 * k4 + 2][m] = v.z;
            As[4 * k4 + 3][m] = v.w;
        }
    } else {
        // row m = tid & 127 for every j; k = (tid >> 7) + 2 j
        const int m = tid & 127;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = (tid >> 7) + 2 * j;
            v[j] = (rowoff >= 0 && k0 + k < K) ? __ldg(T + rowoff + (int64_t)(k0 + k) * Q) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) As[(tid >> 7) + 2 * j][m] = v[j];
    }
}

template <int MODE>
__global__ void __launch_bounds__(256) k_ttm_simt(const float* __restrict__ T,
                                                  const float* __restrict__ A,
                                                  float* __restrict__ X, int64_t P, int K,
                                                  int64_t Q, int R, int xvec) {
    __shared__ __align__(16) float As[BK][BM + APAD];
    __shared__ __align__(16) float Bs[BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t g0 = (int64_t)blockIdx.x * BM;
    const int r0 = blockIdx.y * BN;
    const int64_t PQ = P * Q;

    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

    int64_t rowoff = -1;
    if (MODE == LOAD_GENERIC) {
        const int64_t g = g0 + (tid & 127);
        if (g < PQ) {
            const int64_t p = g / Q, q = g - p * Q;
            rowoff = p * K * Q + q;
        }
    }
    for (int k0 = 0; k0 < K; k0 += BK) {
        load_a<MODE>(As, T, g0, k0, P, K, Q, tid, rowoff);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int idx = tid + 256 * j;
            int k = idx >> 6, n = idx & 63;
            float v = 0.f;
            if (k0 + k < K && r0 + n < R) v = __ldg(A + (int64_t)(k0 + k) * R + r0 + n);
            Bs[k][n] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            float4 a0 = *reinterpret_cast<const float4*>(&As[k][ty * TM]);
            float4 a1 = *reinterpret_cast<const float4*>(&As[k][ty * TM + 4]);
            float4 b = *reinterpret_cast<const float4*>(&Bs[k][tx * TN]);
            float av[TM] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float bv[TN] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }

    const int c0 = r0 + tx * TN;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int64_t g = g0 + ty * TM + i;
        if (g >= PQ) break;
        float* dst = X + g * R + c0;
        // xvec: widest store every row start allows (R and the base address)
        if (xvec == 4 && c0 + 3 < R) {
            *reinterpret_cast<float4*>(dst) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        } else if (xvec == 2 && c0 + 3 < R) {
            *reinterpret_cast<float2*>(dst) = make_float2(acc[i][0], acc[i][1]);
            *reinterpret_cast<float2*>(dst + 2) = make_float2(acc[i][2], acc[i][3]);
        } else {
#pragma unroll
            for (int j = 0; j < TN; ++j)
                if (c0 + j < R) dst[j] = acc[i][j];
        }
    }
}

}  // namespace

namespace cpk {

cudaError_t ttm_simt(const float* T, const float* A, float* X, int64_t P, int K, int64_t Q,
                     int R, cudaStream_t st) {
    const int64_t PQ = P * Q;
    dim3 grid((unsigned)((PQ + BM - 1) / BM), (unsigned)((R + BN - 1) / BN));
    bool al16 = ((uintptr_t)T & 15) == 0;
    const int xvec = ((R & 3) == 0 && ((uintptr_t)X & 15) == 0) ? 4 : ((R & 1) == 0 && ((uintptr_t)X & 7) == 0) ? 2 : 1;
    if (Q > 1 && Q % BM == 0 && al16)
        k_ttm_simt<LOAD_QTILE><<<grid, 256, 0, st>>>(T, A, X, P, K, Q, R, xvec);
    else if (Q == 1 && K % 4 == 0 && al16)
        k_ttm_simt<LOAD_ROWK><<<grid, 256, 0, st>>>(T, A, X, P, K, Q, R, xvec);
    else
        k_ttm_simt<LOAD_GENERIC><<<grid, 256, 0, st>>>(T, A, X, P, K, Q, R, xvec);
    return cudaGetLastError();
}

}  // namespace cpk
