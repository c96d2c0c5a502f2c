// Direct residual without any device allocation (cp_resid_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a fit:
// applications whose own memory pool has reserved the whole GPU (a raw
// cudaMalloc would then fail or fragment that pool), and latency-critical loops
// in which cudaMalloc/cudaFree would synchronise the device.  This entry point
// keeps its scratch - one partial sum per 64 x 64 tile of the tensor - in a
// file-scope device array of fixed size that every GPU loading the library
// holds until the process exits.
//
// Computed: out[0] = ||T - [[A]]||_F^2 and out[1] = ||T||_F^2 (FP64 sums of FP32
// terms), so the relative residual of Eq. (residual-def) is sqrt(out[0]/out[1]).
// Same arithmetic as the residual kernel behind cp_fit(exact = 1): T is viewed
// as rows (modes 0..N-2) x columns (mode N-1); a tile's model values are the
// FP32 dot products of Khatri-Rao rows with rows of the last factor.
#include <mutex>

#include "cpals_internal.h"

namespace {

constexpr int64_t NOALLOC_MAX_TILES = 65536;
constexpr int NOALLOC_MAXR = 256;   // the rank limit this entry point documents

// [0, MAX): per-tile sum of (t - t~)^2;  [MAX, 2 MAX): per-tile sum of t^2.
// Every slot a call reads is written earlier in the same call, so nothing has
// to be cleared between calls.
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_TILES];

struct Args {
    const float* T;
    const float* A[CP_MAXN];
    int64_t dims[CP_MAXN];
    int N, R;
};

__device__ double blk_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// one 64 x 64 tile per block (256 threads, 4 x 4 values per thread)
__global__ void __launch_bounds__(256) k_resid_tiles(Args a, int64_t nrows, int64_t ncols, int64_t ntile_c,
                                                     double* __restrict__ part, int64_t max_tiles) {
    __shared__ __align__(16) float KR[16][64];
    __shared__ __align__(16) float Bs[16][64];
    __shared__ int rowoff[64][CP_MAXN];
    __shared__ double sh[32];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int N = a.N, R = a.R;
    const float* Alast = a.A[N - 1];
    const int64_t tile = blockIdx.x;
    const int64_t row0 = (tile / ntile_c) * 64, col0 = (tile % ntile_c) * 64;
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
                for (int k = 0; k < N - 1; ++k) v *= a.A[k][(size_t)rowoff[m][k] * R + r0 + rr];
                if (col0 + m < ncols) b = Alast[(size_t)(col0 + m) * R + r0 + rr];
            }
            KR[rr][m] = v;
            Bs[rr][m] = b;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float4 av = *reinterpret_cast<const float4*>(&KR[k][ty * 4]);
            const float4 bv = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
            const float aa[4] = {av.x, av.y, av.z, av.w}, bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(aa[i], bb[j], acc[i][j]);
        }
    }
    float pd = 0.f, pt = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t row = row0 + ty * 4 + i;
        if (row >= nrows) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t col = col0 + tx * 4 + j;
            if (col < ncols) {
                const float t = __ldg(a.T + row * ncols + col);
                const float d = t - acc[i][j];
                pd = fmaf(d, d, pd);
                pt = fmaf(t, t, pt);
            }
        }
    }
    const double sd = blk_sum((double)pd, sh);
    __syncthreads();
    const double st = blk_sum((double)pt, sh);
    if (tid == 0) {
        part[tile] = sd;
        part[max_tiles + tile] = st;
    }
}

__global__ void __launch_bounds__(1024) k_resid_total(const double* __restrict__ part, int64_t ntiles,
                                                      int64_t max_tiles, double* __restrict__ out) {
    __shared__ double sh[32];
    double d = 0.0, t = 0.0;
    for (int64_t i = threadIdx.x; i < ntiles; i += blockDim.x) {
        d += part[i];
        t += part[max_tiles + i];
    }
    const double sd = blk_sum(d, sh);
    __syncthreads();
    const double st = blk_sum(t, sh);
    if (threadIdx.x == 0) {
        out[0] = sd;
        out[1] = st;
    }
}

// device address of the scratch array, looked up once per device
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(double** p) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* q = nullptr;
        e = cudaGetSymbolAddress(&q, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = static_cast<double*>(q);
    }
    *p = g_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" cp_status cp_resid_noalloc(int N, const int64_t* dims, int R, const float* T_dev,
                                      const float* const* A_dev, double* out_dev, void* stream) {
    if (N < 3 || N > CP_MAXN || !dims || R < 1 || R > NOALLOC_MAXR || !T_dev || !A_dev || !out_dev)
        return CP_EINVAL;
    Args a;
    a.T = T_dev;
    a.N = N;
    a.R = R;
    int64_t nrows = 1;
    for (int k = 0; k < N; ++k) {
        if (dims[k] < 1 || !A_dev[k]) return CP_EINVAL;
        a.dims[k] = dims[k];
        a.A[k] = A_dev[k];
        if (k < N - 1) {
            if (nrows > ((int64_t)1 << 40) / dims[k]) return CP_EINVAL;
            nrows *= dims[k];
        }
    }
    const int64_t ncols = dims[N - 1];
    const int64_t ntc = (ncols + 63) / 64;
    const int64_t ntr = (nrows + 63) / 64;
    // the scratch holds 65536 tiles; both factors are bounded before their
    // product is formed, so a huge last mode cannot wrap it around
    if (ntc > NOALLOC_MAX_TILES || ntr > NOALLOC_MAX_TILES / ntc) return CP_EINVAL;
    const int64_t ntiles = ntr * ntc;
    double* part = nullptr;
    if (scratch_for_current_device(&part) != cudaSuccess) {
        cudaGetLastError();
        return CP_ECUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    k_resid_tiles<<<(unsigned)ntiles, 256, 0, st>>>(a, nrows, ncols, ntc, part, NOALLOC_MAX_TILES);
    k_resid_total<<<1, 1024, 0, st>>>(part, ntiles, NOALLOC_MAX_TILES, out_dev);
    return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
