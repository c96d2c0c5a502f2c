// Policy network 8 -> 64 -> 64 -> 1 (tanh, tanh, sigmoid) used to steer the PP
// regime; the paper's Alg. 2 threshold rule is the fallback.  Parameter order:
// W1 (64x8), b1 (64), W2 (64x64), b2 (64), w3 (64), b3 (1) = 4801 floats.
// Training loss: mean binary cross-entropy softplus(z) - y z; optimiser Adam
// (Kingma and Ba, ICLR 2015) with bias correction.  One warp per sample; lane l
// owns hidden units l and l + 32.
#include "cpals_internal.h"

namespace {

constexpr int DIN = 8, H = 64, NP = 4801;
constexpr int OW1 = 0, OB1 = 512, OW2 = 576, OB2 = 4672, OW3 = 4736, OB3 = 4800;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ float softplus(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }

// forward for one sample by one warp; h1/h2 in per-warp smem; returns z
__device__ float fwd(const float* th, const float* x, float* h1, float* h2, int lane) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int j = lane + 32 * u;
        float a = th[OB1 + j];
#pragma unroll
        for (int i = 0; i < DIN; ++i) a = fmaf(th[OW1 + j * DIN + i], x[i], a);
        h1[j] = tanhf(a);
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int j = lane + 32 * u;
        float a = th[OB2 + j];
        for (int k = 0; k < H; ++k) a = fmaf(th[OW2 + j * H + k], h1[k], a);
        h2[j] = tanhf(a);
    }
    __syncwarp();
    float z = th[OW3 + lane] * h2[lane] + th[OW3 + lane + 32] * h2[lane + 32];
    return wsum(z) + th[OB3];
}

__global__ void __launch_bounds__(256) k_mlp_fwd(const float* __restrict__ theta,
                                                 const float* __restrict__ X, int B,
                                                 float* __restrict__ prob) {
    __shared__ float th[NP];
    __shared__ float hs[8][2 * H];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) th[i] = theta[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b = blockIdx.x * 8 + w; b < B; b += gridDim.x * 8) {
        float x[DIN];
#pragma unroll
        for (int i = 0; i < DIN; ++i) x[i] = X[(size_t)b * DIN + i];
        const float z = fwd(th, x, hs[w], hs[w] + H, lane);
        if (lane == 0) prob[b] = 1.f / (1.f + expf(-z));
        __syncwarp();
    }
}

// per-block gradient accumulation in smem, written to part[blockIdx][NP+1] (last = loss sum)
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ theta,
                                                  const float* __restrict__ X,
                                                  const float* __restrict__ y, int B,
                                                  float* __restrict__ part) {
    __shared__ float th[NP];
    __shared__ float g[NP + 1];
    __shared__ float hs[8][4 * H];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) {
        th[i] = theta[i];
        g[i] = 0.f;
    }
    if (threadIdx.x == 0) g[NP] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float* h1 = hs[w];
    float* h2 = hs[w] + H;
    float* d2 = hs[w] + 2 * H;
    const float invB = 1.f / (float)B;
    for (int b = blockIdx.x * 8 + w; b < B; b += gridDim.x * 8) {
        float x[DIN];
#pragma unroll
        for (int i = 0; i < DIN; ++i) x[i] = X[(size_t)b * DIN + i];
        const float z = fwd(th, x, h1, h2, lane);
        const float yb = y[b];
        const float p = 1.f / (1.f + expf(-z));
        const float dz = (p - yb) * invB;
        if (lane == 0) {
            atomicAdd(&g[NP], softplus(z) - yb * z);
            atomicAdd(&g[OB3], dz);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int j = lane + 32 * u;
            atomicAdd(&g[OW3 + j], dz * h2[j]);
            const float da2 = dz * th[OW3 + j] * (1.f - h2[j] * h2[j]);
            d2[j] = da2;
            atomicAdd(&g[OB2 + j], da2);
            for (int k = 0; k < H; ++k) atomicAdd(&g[OW2 + j * H + k], da2 * h1[k]);
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int k = lane + 32 * u;
            float s = 0.f;
            for (int j = 0; j < H; ++j) s = fmaf(th[OW2 + j * H + k], d2[j], s);
            const float da1 = s * (1.f - h1[k] * h1[k]);
            atomicAdd(&g[OB1 + k], da1);
#pragma unroll
            for (int i = 0; i < DIN; ++i) atomicAdd(&g[OW1 + k * DIN + i], da1 * x[i]);
        }
        __syncwarp();
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= NP; i += blockDim.x) part[(size_t)blockIdx.x * (NP + 1) + i] = g[i];
}

__global__ void k_mlp_reduce(const float* __restrict__ part, int nb, int B, float* __restrict__ grad,
                             float* __restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > NP) return;
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * (NP + 1) + i];
    if (i < NP) grad[i] = s;
    else if (loss) loss[0] = s / (float)B;
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

constexpr int kMaxGradBlocks = 64;

}  // namespace

namespace cpk {

int mlp_nparams() { return NP; }
size_t mlp_scratch_floats() { return (size_t)kMaxGradBlocks * (NP + 1); }

cudaError_t mlp_forward(const float* theta, const float* X, int B, float* prob, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    int nb = (B + 7) / 8;
    if (nb > 1024) nb = 1024;
    k_mlp_fwd<<<nb, 256, 0, st>>>(theta, X, B, prob);
    return cudaGetLastError();
}

cudaError_t mlp_grad(const float* theta, const float* X, const float* y, int B, float* loss,
                     float* grad, float* scratch, cudaStream_t st) {
    if (B <= 0) return cudaErrorInvalidValue;
    int nb = (B + 7) / 8;
    if (nb > kMaxGradBlocks) nb = kMaxGradBlocks;
    k_mlp_grad<<<nb, 256, 0, st>>>(theta, X, y, B, scratch);
    k_mlp_reduce<<<(NP + 1 + 255) / 256, 256, 0, st>>>(scratch, nb, B, grad, loss);
    return cudaGetLastError();
}

cudaError_t mlp_adam(float* theta, const float* grad, float* m, float* v, int n, int t, float lr,
                     cudaStream_t st) {
    const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
    k_adam<<<(n + 255) / 256, 256, 0, st>>>(theta, grad, m, v, n, lr, c1, c2);
    return cudaGetLastError();
}

}  // namespace cpk
