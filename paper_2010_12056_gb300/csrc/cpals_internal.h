// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cpals.h"

#define CP_MAXN 8
#define CP_MAXR 512
#define CP_NSCAL 8  // per-update scalar slots, see SCAL_* below

// Per-update scalar reductions written by the solve kernel (partials per block,
// finalised by k_finalize into ctx->scal_mode[mode * CP_NSCAL + slot]).
enum {
    SCAL_A2 = 0,      // ||A_new||_F^2
    SCAL_STEP2 = 1,   // ||A_new - A_old||_F^2   (change made by this update)
    SCAL_DAP2 = 2,    // ||A_new - A_p||_F^2     (PP: accumulated change)
    SCAL_MA = 3,      // <M, A_new>              (Eq. residual)
    SCAL_GS = 4,      // <Gamma, S_new>          (Eq. residual)
    SCAL_M2 = 5,      // ||M~||_F^2              (PP: size of the MTTKRP)
    SCAL_V2 = 6,      // ||V||_F^2               (PP: size of the second-order term)
    SCAL_FLAGS = 7    // Cholesky flags: 1 = shifted, 2 = failed
};

// ----------------------------------------------------------------------- device status
// One device word per context; kernels OR error bits into it, host reads it at
// synchronisation points.
enum { DEVERR_TIMEOUT = 1, DEVERR_NOTSPD = 2, DEVERR_BADARG = 4 };

// ----------------------------------------------------------------------- launchers
// Each returns cudaGetLastError() after the launch.
namespace cpk {

// first-level TTM: X[p][q][r] = sum_k T[p][k][q] * A[k][r]   (A is K x R row-major)
cudaError_t ttm_simt(const float* T, const float* A, float* X, int64_t P, int K, int64_t Q,
                     int R, cudaStream_t st);

// tensor-core first-level TTM (k_ttm_tc.cu).  A plan holds the TMA descriptors
// of one contraction (tensor T viewed as [P][K][Q], factor operand bhi/blo stored
// [Rpad][Kpad] K-contiguous); NULL when the shape is not supported (the caller
// then uses the SIMT kernel).
struct TcPlan;
bool ttm_tc_supported(int64_t P, int K, int64_t Q, int R);
// kind 0: bf16 parts (bhi/blo uint16 [Rpad][Kpad]); kind 1: tf32 parts (fp32 [Rpad][Kpad]);
// kind 2: fp16 parts of the scaled factor (uint16 [Rpad][Kpad]); T is multiplied
// by tscale (a power of two) before its split and column c of the result by
// colinv[c] (device, Rpad floats, 16-byte aligned).
// pre_hi / pre_lo: T's 16-bit parts stored with the contracted mode innermost
// ([P][Q][K], from ttm_presplit with the same kind and tscale): for R > 128 the
// kernel then loads its A operand directly (no converter warps).
TcPlan* ttm_tc_plan(const float* T, int64_t P, int K, int64_t Q, int R, int kind, const void* bhi,
                    const void* blo, int Rpad, int Kpad, float tscale = 1.f, const float* colinv = nullptr,
                    const void* pre_hi = nullptr, const void* pre_lo = nullptr, bool pre_narrow = false);
// T viewed as [P][K][Q] -> its 16-bit parts [P][Q][K] (kind 2: fp16 of T tscale; kind 0: bf16),
// split exactly as the kernel's converter warps split it
cudaError_t ttm_presplit(const float* T, int64_t P, int K, int64_t Q, int kind, float tscale, uint16_t* hi,
                         uint16_t* lo, int num_sms, cudaStream_t st);
int ttm_tc_kind(const TcPlan* p);
void ttm_tc_set_tscale(TcPlan* p, float tscale);
void ttm_tc_plan_free(TcPlan* p);
// splitk_ws: NULL, or a workspace of ttm_tc_splitk() * rows * R floats that lets
// the kernel split K across CTAs when the row tiles alone cannot fill the GPU
// (partial sums are then added in a fixed order by a second kernel).
// child: NULL, or the first child of a multi-sweep root formed in the epilogue:
//   Y[y][r] = sum_{j < sc} X[y sc + j][r] Ac[j][r]   (X's innermost kept mode, size sc)
// Needs ttm_tc_child_ok(); ws holds ttm_tc_child_ws_floats() floats (NULL if 0).
struct TcChild {
    float* Y;
    const float* Ac;   // FP32 factor of the contracted mode, sc x R row-major
    int sc;
    float* ws;
};
bool ttm_tc_child_ok(const TcPlan* p, int sc);
int64_t ttm_tc_child_ws_floats(const TcPlan* p, int sc);
// wait_limit: cycles a pipeline wait may take before the kernel gives up and
// reports DEVERR_TIMEOUT (<= 0: the default, about 1 s)
cudaError_t ttm_tc_run(const TcPlan* p, float* X, int prec, int num_sms, unsigned* dev_err,
                       cudaStream_t st, float* splitk_ws, const TcChild* child = nullptr,
                       long long wait_limit = 0);
int ttm_tc_splitk(const TcPlan* p, int num_sms);
// the plan reads T's stored 16-bit parts
bool ttm_tc_stored_parts(const TcPlan* p);
// long contractions (the fused two-mode operand): split K so that no TMEM
// accumulator sums more than 64 MMAs; depth_slices is the split that needs
void ttm_tc_set_depth_bound(TcPlan* p, bool on);
int ttm_tc_depth_slices(const TcPlan* p);
int64_t ttm_tc_rows(const TcPlan* p);
// Khatri-Rao operand of two adjacent modes a, a+1 for a fused two-mode contraction:
// row k = i_a * s_b + i_b holds A_a[i_a][r] * A_b[i_b][r]; written transposed
// ([Rpad][Kpad], k contiguous) as bf16 hi/lo (kind 0) or tf32 hi/lo (kind 1).
// kind 2: fp16 parts of the product scaled per column by powers of two (scale,
// Rpad floats, written here with colinv = 2^-(column exponent + eT)).
cudaError_t kr_operand(const double* Aa, const double* Ab, int sa, int sb, int R, int Kpad,
                       int kind, void* hi, void* lo, cudaStream_t st, int eT = 0, float* scale = nullptr,
                       float* colinv = nullptr);
// fp16 factor operand of the tensor-core TTM (kind 2) from the FP32 factor: per
// column a power of two 2^e_c bringing max |A(:, c)| into [2^14, 2^15), parts
// written transposed [Rpad][Kpad]; colinv[c] = 2^-(e_c + eT) (Rpad floats).
cudaError_t f16_operand(const float* A32, int s, int R, int Rpad, int Kpad, int eT, uint16_t* hi, uint16_t* lo,
                        float* colinv, cudaStream_t st);
// max |x| over n floats into out[0] (device); part holds max_blocks floats
cudaError_t absmax(const float* x, int64_t n, float* part, int max_blocks, float* out, cudaStream_t st);

// multi-TTV: Y[p][q][r] = sum_k X[p][k][q][r] * A[k][r]
// max_blocks_per_sm > 0 caps the grid (blocks loop over the outputs) so that the
// whole launch is resident at once and leaves room for kernels of other streams.
cudaError_t mttv(const float* X, const float* A, float* Y, int64_t P, int K, int64_t Q, int R,
                 int num_sms, cudaStream_t st, int max_blocks_per_sm = 0);

// PP first-order corrections for one mode n (Eq. U_ni):
//   Mt[x][r] = Mp[x][r] + sum_i sum_y Op_i(x, y, r) dA_i[y][r]
// where operator i is stored [x][y][r] (trans=0) or [y][x][r] (trans=1).
struct PPTerm {
    const float* op;
    const float* dA;
    int sy;
    int trans;
};
cudaError_t pp_u(const float* Mp, const PPTerm* terms, int nterms, float* Mt, int sx, int R,
                 cudaStream_t st);

// ||x||^2 over n floats -> partials (nblocks doubles), returns nblocks used
int norm2_partials(const float* x, int64_t n, double* partials, int max_blocks, cudaStream_t st);
cudaError_t sum_partials(const double* partials, int n, double* out, cudaStream_t st);

// Outputs of the row solve A_new = (M + A_old W) Gamma^{-1}: every operand copy
// of the new factor and, in PP, its difference from the base factor.
struct SolveOut {
    double* A64;        // in: A_old, out: A_new (s x R)
    float* A32;         // FP32 copy
    uint16_t* bhi;      // bf16 hi, transposed [Rpad][Kpad]
    uint16_t* blo;      // bf16 lo
    float* bt32;        // tf32 parts, transposed: hi [Rpad][Kpad] then lo [Rpad][Kpad]
    int Rpad, Kpad;
    const double* Ap;   // PP base factor (NULL outside PP)
    float* dA32;        // A_new - A_p (or - A_old outside PP), FP32
    double* dA64;       // same in FP64
    float2* A2;         // A_new as float pairs (hi, lo) for gram_df (NULL: not written)
    float2* dA2;        // dA as float pairs (NULL: not written)
};
// Mixed-precision normal-equation solve (k_solve_mixed.cu): chol_mixed forms
// Gamma (FP64, written to Gamma; its FP32 copy G32 and float pairs hi, lo in
// G2), PP's W (FP64 and pairs W2), and either Ginv ~ Gamma^{-1} in FP32 from the
// diagonally scaled matrix (*mode = 0) or the FP64 factor L64 ([L | L^T], 2 R^2)
// and invd64 (*mode = 1);
// solve_mixed then solves every row to FP64 accuracy (refinement or FP64
// substitution).  Gamma, G2 and Ginv must have 16 spare bytes after their R*R entries.
// force64: skip the FP32 inverse and factor Gamma in FP64 (LDL^T) for this update.
// S2_list / dS2_list (device arrays of N pointers, R <= 128): the Grams as float
// pairs, from which Gamma and W are formed in double-float arithmetic (else from
// the FP64 Grams); an exact sweep's update then forms Gamma inside the inverse.
cudaError_t chol_mixed(double* const* S_list, double* const* dS_list, const float2* const* S2_list,
                       const float2* const* dS2_list, int N, int n, int R, int pp, double* Gamma, float* G32,
                       float* G2, float* Ginv, double* L64, double* invd64, double* W, float* W2, double* scal,
                       int* mode, float* ws, cudaStream_t st, bool force64 = false);
// floats of the workspace chol_mixed needs for R > 128 (blocked inverse), else 0
size_t schur_ws_floats(int R);
cudaError_t solve_mixed(const float* M, const double* W, const float* W2, const double* Gamma, const float* G2,
                        const float* Ginv, const double* L64, const double* invd64, const int* mode,
                        const SolveOut& o, int s, int R, double* scal, double* scal_part, int* nblk,
                        unsigned* dev_err, cudaStream_t st);

// S = A^T A (and dS = A^T dA when dA != NULL), one cluster launch over row
// chunks; with Gamma and tile_gs (gram_tiles(R) doubles) also the tile shares of
// <Gamma, S>.  scal_fin adds the solve's nblk per-block scalars and those shares
// into scal_out (every slot but SCAL_FLAGS).
int gram_tiles(int R);
cudaError_t gram(const double* A, const double* dA, int s, int R, const double* Gamma, double* S,
                 double* dS, double* tile_gs, cudaStream_t st);
// Same from the float-pair copies the solve writes (A2, dA2 = hi + lo of the FP64
// values), in double-float arithmetic; Gamma for <Gamma, S> as float pairs (G2);
// S and dS also written as float pairs (S2, dS2).
cudaError_t gram_df(const float2* A2, const float2* dA2, int s, int R, const float2* G2, double* S,
                    double* dS, float2* S2, float2* dS2, double* tile_gs, cudaStream_t st);
// y[i] = float pair (hi, lo) of x[i] (hi = x rounded to float, lo = the rest rounded)
cudaError_t split_pairs(const double* x, float2* y, int64_t n, cudaStream_t st);
cudaError_t scal_fin(const double* scal_part, int nblk, const double* tile_gs, int ntiles, double* scal_out,
                     cudaStream_t st);

// refresh all operand copies of a factor from its FP64 master (after set_factor / init)
cudaError_t factor_copies(const double* A64, float* A32, uint16_t* bhi, uint16_t* blo,
                          float* bt32, int s, int R, int Rpad, int Kpad, cudaStream_t st);

// direct residual partials: sum (T - [[A]])^2 over the tensor, FP64 partials per block
struct ResidArgs {
    const float* T;
    const float* A32[CP_MAXN];
    int64_t dims[CP_MAXN];
    int N, R;
};
int resid_direct_partials(const ResidArgs& a, double* partials, int max_blocks, cudaStream_t st);
// The same on the tensor cores (k_resid_tc.cu; tf32x3 model values, double-float
// sums): R <= 64, last mode a multiple of 4 and at most num_sms column blocks of
// 128.  Returns the number of partials written, 0 if the shape is not supported
// (nothing launched), -1 on a launch error.
int resid_tc_partials(const ResidArgs& a, double* partials, int max_blocks, int num_sms, unsigned* dev_err,
                      long long wait_limit, cudaStream_t st);

// PP: dA = A - A_p (FP64 and FP32); out = Mt + A W (the V term of Eq. ppupdate)
cudaError_t pp_delta(const double* A, const double* Ap, float* d32, double* d64, int64_t n,
                     cudaStream_t st);
cudaError_t add_aw(const float* Mt, const double* A, const double* W, int s, int R, float* out,
                   cudaStream_t st);
// FP64 -> FP32 conversion
cudaError_t f64_to_f32(const double* x, float* y, int64_t n, cudaStream_t st);
// MLP kernels
int mlp_nparams();
size_t mlp_scratch_floats();
cudaError_t mlp_forward(const float* theta, const float* X, int B, float* prob, cudaStream_t st);
cudaError_t mlp_grad(const float* theta, const float* X, const float* y, int B, float* loss,
                     float* grad, float* scratch, cudaStream_t st);
cudaError_t mlp_adam(float* theta, const float* grad, float* m, float* v, int n, int t, float lr,
                     cudaStream_t st);

}  // namespace cpk
