/*
 * cpals.h - C ABI of the GB300 CP-ALS engine (dimension tree, multi-sweep
 * dimension tree, pairwise perturbation) for dense order-N tensors.
 *
 * Problem (Sec. II-B, Alg. 1): given a dense tensor T of size s_1 x ... x s_N
 * and a rank R, find factors A(n) (s_n x R) minimising
 * 1/2 ||T - [[A(1), ..., A(N)]]||_F^2 by alternating least squares: each update
 * solves A(n) Gamma(n) = M(n) with the MTTKRP M(n) = T_(n) P(n) and
 * Gamma(n) = *_{k != n} A(k)^T A(k) (Eq. gram).
 *
 * Conventions shared by every call:
 *  - Modes are 0-based (the paper's mode n is n-1 here).
 *  - The tensor is C order (last index fastest), contiguous, on the device.
 *  - Factors are s_n x R row-major (r fastest), FP64 on the host side of the
 *    ABI; the library keeps FP64 masters plus FP32 / split-bf16 operand copies.
 *  - Every call is enqueued on the CUDA stream given to cp_init (a
 *    cudaStream_t passed as void*; NULL = legacy default stream).  Calls that
 *    return host values (cp_fit, cp_get_*, cp_sweep_pp's regime tests)
 *    synchronise that stream.
 *  - Errors are returned, never raised by abort().  After CP_ECUDA or
 *    CP_ETIMEOUT the context is poisoned and every later call returns
 *    CP_ESTATE; cp_last_error() describes the first failure.
 *  - The library owns every buffer it allocates (factors, tree intermediates,
 *    PP operators, traces) and frees them in cp_free.  It never writes T.
 */
#ifndef CPALS_H
#define CPALS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cp_ctx cp_ctx; /* opaque; owned by the library */

typedef enum {
    CP_OK = 0,
    CP_EINVAL = 1,    /* bad argument (sizes, mode, eps, NULL pointer)          */
    CP_ENOMEM = 2,    /* device or host allocation failed                       */
    CP_ECUDA = 3,     /* a CUDA call failed; context poisoned                   */
    CP_ENOTSPD = 4,   /* Gamma(n) not positive definite even after the shift    */
    CP_ENUMERIC = 5,  /* NaN or Inf in a factor or in the fit                   */
    CP_ETIMEOUT = 6,  /* a bounded device wait ran out; context poisoned        */
    CP_ESTATE = 7     /* context poisoned by an earlier failure, or wrong state */
} cp_status;

/* Arithmetic of the first-level TTM T x_m A(m) (Sec. II-C), the dominant
 * contraction.  All variants accumulate in FP32; mTTVs run in FP32 and the
 * Gram / Hadamard / Cholesky / residual terms in FP64 whatever is chosen. */
typedef enum {
    CP_FP32_SIMT = 0, /* FP32 FMA on the CUDA cores                              */
    CP_TF32 = 1,      /* tcgen05 kind::tf32 on rna_tf32(x) only (reported, 10-bit mantissa) */
    CP_BF16X3 = 2,    /* tcgen05 kind::f16: x = hi + lo in bf16, hi*hi+hi*lo+lo*hi */
    CP_BF16 = 3,      /* tcgen05 kind::f16 on bf16(x) only (reported, low accuracy) */
    CP_TF32X3 = 4,    /* tcgen05 kind::tf32: x = hi + lo in tf32 (round to nearest),
                         hi*hi+hi*lo+lo*hi; about FP32 accuracy at half bf16x3's rate */
    CP_F16X3 = 5      /* tcgen05 kind::f16 on fp16 parts: T scaled by one power of two
                         (max |T| to [2^14, 2^15)), each factor column by its own, then
                         x = hi + lo in fp16, hi*hi+hi*lo+lo*hi, the powers of two
                         removed exactly from the FP32 result.  About 22 bits per
                         value (tf32x3 accuracy) at bf16x3's rate.  Accuracy is
                         relative to max |T|: entries below 2^-24 max |T| keep only
                         part of their bits (negligible in any Frobenius norm; use
                         another precision for tensors whose MTTKRP rows differ in
                         magnitude by more than about 1e6) */
} cp_prec;

typedef struct {
    int prec;         /* cp_prec of the first-level TTM                           */
    double pp_eps;    /* PP tolerance epsilon of Alg. 2 (0 < eps < 1)             */
    double delta;     /* stopping tolerance on |r - r_old| (Alg. 1); <= 0: never  */
    int max_sweeps;   /* sweep cap of cp_run (<= 0: no cap)                       */
    int judge_every;  /* policy mode: direct residual every k sweeps (0 = off)    */
    int policy_gate;  /* 1: consult the policy only when approximating pays (see
                         cp_sweep_pp); 0: before every sweep                  */
    uint64_t seed;    /* Philox4x32-10 seed of the default U[0,1) initial factors */
} cp_config;

/* Fill *cfg with defaults: f16x3 TTM, eps 0.1, delta 0, judge every 5 sweeps,
 * policy gate on. */
void cp_config_default(cp_config *cfg);

/*
 * cp_init - create a decomposition context (Alg. 1 and Alg. 2, set-up).
 *   N        tensor order, 3 <= N <= 8
 *   dims     N mode sizes, each >= 1; host array, copied
 *   R        rank, 1 <= R <= 512 (the tensor-core TTM runs in column passes of
 *            128, the normal equations' FP32 inverse in blocks of 128)
 *   T_dev    pointer to the tensor, C order, contiguous.  dtype 0: FP32 on the
 *            device, borrowed (must outlive the context, never written); dtype 1:
 *            FP64 on the device, converted once into a library-owned FP32 copy;
 *            dtype 2: FP32 in HOST memory (pinned memory gives the full copy
 *            bandwidth), copied once into a library-owned device buffer.
 *   A0_host  NULL, or N host blocks (s_n x R row-major FP64, concatenated in mode
 *            order) of initial factors.  NULL draws U[0,1) entries (Alg. 1) from
 *            Philox4x32-10 with key = cfg->seed, counter = (j, 0, n, 0) for
 *            mode n, two doubles per block j, ((w0<<32|w1)>>11)*2^-53.
 *   cfg      NULL for defaults; copied.
 *   stream   cudaStream_t (as void*) every later call is enqueued on.
 * Computes ||T||_F^2 and the Grams S(n) = A(n)^T A(n).  Sets dA(n) = A(n), so the
 * first PP test fails and the first sweep is a regular one (Alg. 2 starts from dA = A).
 * Returns CP_EINVAL on bad sizes, CP_ENOMEM if the factor and normal-equation
 * workspace does not fit, CP_ECUDA on a CUDA failure.  *out is NULL on failure.
 * Tree intermediates (at most prod(dims)/min(dims) * R * 4 bytes per tree level)
 * and PP operators are allocated on first use, so a sweep call can also return
 * CP_ENOMEM; a schedule that never forms a level never allocates it.
 */
cp_status cp_init(cp_ctx **out, int N, const int64_t *dims, int R, const void *T_dev,
                  int dtype, const double *A0_host, const cp_config *cfg, void *stream);

/*
 * cp_load_tensor - a new tensor of the same sizes for an existing context (the
 * paper has no counterpart; it lets one context serve a stream of tensors).
 *   T        NULL: the tensor's contents changed in place (borrowed or owned
 *            buffer) and only the derived state is refreshed.  Otherwise FP32 data
 *            copied into the context's own tensor buffer, which exists for contexts
 *            created from an FP64 (dtype 1) or a host (dtype 2) tensor; a context
 *            that borrows its tensor returns CP_ESTATE.
 *   on_host  1: T is host memory (pinned for full bandwidth); 0: device memory.
 * Drops every cached tree intermediate (the multi-sweep root included) and the PP
 * operators, recomputes ||T||_F^2 (and, for f16x3, the tensor's power of two);
 * the factors are kept, so the next sweep starts from them.  Enqueued on the
 * context's stream behind earlier work; synchronises it (the norm is read back).
 */
cp_status cp_load_tensor(cp_ctx *ctx, const float *T, int on_host);

/*
 * cp_mttkrp - exact MTTKRP M(mode) = T_(mode) P(mode) with the current factors
 * (Sec. II-B), built down a dimension tree (first-level TTM, then mTTVs).
 *   M_dev  device buffer of s_mode x R floats, row-major; written.
 */
cp_status cp_mttkrp(cp_ctx *ctx, int mode, float *M_dev);

/*
 * cp_ttm - first-level contraction X = T x_mode A(mode) (Sec. II-C) with the
 * current factor.  X_dev: device buffer of prod_{k != mode} s_k x R floats, laid
 * out with the remaining modes in increasing order then r fastest.
 */
cp_status cp_ttm(cp_ctx *ctx, int mode, float *X_dev);

/*
 * cp_sweep_dt - nsweeps CP-ALS sweeps (Alg. 1), each updating A(0..N-1) in order
 * with MTTKRPs from the standard binary dimension tree (Sec. II-C, Fig. 1a): two
 * first-level TTMs per sweep.  After each sweep the relative residual is
 * evaluated with Eq. (residual) and recorded in the trace.
 */
cp_status cp_sweep_dt(cp_ctx *ctx, int nsweeps);

/*
 * cp_sweep_msdt - nsweeps sweeps with the multi-sweep dimension tree (Sec. III,
 * Fig. 2): root T x_m A(m) right after A(m) is updated, serving the next N-1
 * updates; roots cycle m = N-1, N-2, ..., 0.  The root persists across calls
 * (the cross-sweep cache) while its factor is unchanged.
 */
cp_status cp_sweep_msdt(cp_ctx *ctx, int nsweeps);

/*
 * cp_sweep_pp - nsweeps sweeps of PP-CP-ALS (Alg. 2).  While every
 * ||dA(i)||_F < eps ||A(i)||_F the sweep is approximated (Eq. ppupdate) from PP
 * operators M_p(i,j), M_p(n) built at the PP initialization (not counted as a
 * sweep); otherwise a regular MSDT sweep runs and dA(i) is that sweep's change.
 *   eps     PP tolerance, 0 < eps < 1.
 *   policy  NULL: the rule above.  Otherwise a cp_policy from cp_policy_create
 *           (no counterpart in the paper): before each sweep its network scores
 *           two choices from the features of cp_policy_features - an
 *           approximated sweep with the current operators (p_cur) and one with
 *           operators rebuilt now (p_new).  The sweep is approximated with the
 *           current operators if they exist and p_cur >= 0.5, else rebuilt and
 *           approximated if p_new >= 0.5, else regular (MSDT).  The network
 *           is consulted only while approximated sweeps are measured to cost,
 *           all in (operator builds, judge and queries included), less than 0.9
 *           of the cheapest regular sweep seen on this problem (a safe
 *           approximated sweep keeps at least 90% of a regular sweep's
 *           progress); before three have been measured, only while the MTTKRP
 *           traffic an approximated sweep avoids (at about 6 TB/s) covers its
 *           share of the query and the judge.  The first two policy-driven sweeps of a
 *           context are regular.  cfg.policy_gate = 0 consults the network
 *           before every sweep instead.  The judge (judge_every
 *           > 0): before a run of approximated sweeps the state and its direct
 *           residual are kept as the rollback point; after judge_every
 *           approximated sweeps, or when a regular sweep is chosen after some,
 *           the direct residual is computed again.  If it exceeds (1 + 1e-5)
 *           times the rollback point's (1e-5: above the rounding noise of the
 *           FP32 model values), the factors return to the rollback point, the
 *           operators are dropped, the undone sweeps stay in the trace with
 *           rolled_back = 1, and the next judge_every sweeps are regular
 *           (twice as many after each further rollback in a row, up to 64
 *           judge_every).  An approximated sweep whose normal equations break
 *           down (CP_ENOTSPD) is rolled back the same way, and a judged run
 *           that lowered the residual by less than 1e-7 relative is followed
 *           by judge_every regular sweeps.  If the network's output is not a
 *           probability, the rule above decides.  Query and judge time are
 *           added to the sweep's trace ms.
 */
typedef struct cp_policy cp_policy;
cp_status cp_sweep_pp(cp_ctx *ctx, int nsweeps, double eps, cp_policy *policy);

/*
 * cp_run - the outer loop of Alg. 1 (route 0 DT, 1 MSDT) or Alg. 2 (route 2: PP
 * with cfg.pp_eps and `policy`, which may be NULL): sweeps until the relative
 * residual of Eq. (residual) changes by at most cfg.delta between consecutive
 * sweeps (the first sweep of a context compares with r = 1), or cfg.max_sweeps
 * sweeps have run in this call.  At least one of the two must be set (delta > 0
 * or max_sweeps > 0), else CP_EINVAL.  *nsweeps (may be NULL) returns the sweeps
 * run.  Synchronises after every sweep.
 */
cp_status cp_run(cp_ctx *ctx, int route, cp_policy *policy, int *nsweeps);

/*
 * cp_policy_features - the 8 inputs of the PP policy network for the current
 * state (no counterpart in the paper), twice: f16[0..7] for an approximated
 * sweep with the current operators, f16[8..15] as if the operators were
 * rebuilt now.  L(x) = log10(clamp(x, 1e-12, 1)) / 6 + 1 maps [1e-12, 1] to
 * [-1, 1]; "last" is the newest trace record, r its residual, r' the one before.
 *   f0  min(3, sweeps done / 100)
 *   f1  L(last max_rel_step)                  (1 before any sweep)
 *   f2  L(max_i ||A(i) - A_p(i)|| / ||A(i)||) with operators; -1 without
 *       operators and in the rebuilt query
 *   f3  L(|r - r'| / r)
 *   f4  L(r)
 *   f5  min(3, approximated sweeps since the operators were built / 10);
 *       3 without operators, 0 in the rebuilt query
 *   f6  1 if the last sweep was approximated, else 0
 *   f7  L(last v_share) if the last sweep was approximated and not in the
 *       rebuilt query, else -1
 */
cp_status cp_policy_features(cp_ctx *ctx, float *f16);

/*
 * cp_pp_probe - one sweep step that also labels the PP choices (no counterpart
 * in the paper; it produces the policy's training data).  From the current
 * state it runs, each from the same starting factors: an approximated sweep
 * with the current operators (if any), a regular MSDT sweep, and an operator
 * rebuild followed by an approximated sweep, and evaluates the direct residual
 * (Eq. residual-def) before and after each.  An approximated choice is labelled
 * safe when r_pp - r_exact <= 0.1 max(0, r0 - r_exact) + 1e-9 r0, i.e. it
 * keeps at least 90% of the regular sweep's decrease.  The context then
 * continues along `follow`: 0 regular, 1 current operators (CP_EINVAL without
 * operators), 2 rebuilt, -1 the cheapest safe choice (current, else rebuilt,
 * else regular).  The trace gets one record (decided_by 3).  A second operator
 * set is allocated on first use.
 */
typedef struct {
    float feat_cur[8], feat_new[8];  /* cp_policy_features before the step     */
    double r0;                       /* direct residual before                  */
    double r_exact, r_cur, r_new;    /* after each branch (r_cur NaN w/o ops)   */
    double ms_exact, ms_cur, ms_new; /* device time of each branch              */
    int32_t has_ops, label_cur, label_new, followed;
} cp_probe_rec;
cp_status cp_pp_probe(cp_ctx *ctx, int follow, cp_probe_rec *out);

/*
 * cp_pp_init / cp_pp_mttkrp - the two PP steps exposed separately.  cp_pp_init
 * sets A_p = A, dA = 0 and builds every M_p(i,j) (i < j) and M_p(n) with the PP
 * dimension tree (Fig. 1b).  cp_pp_mttkrp writes the approximated MTTKRP of Eq.
 * ppupdate for `mode` with the current A, dA = A - A_p and S (s_mode x R floats,
 * device) without updating anything.  CP_ESTATE if no operators were built.
 */
cp_status cp_pp_init(cp_ctx *ctx);
cp_status cp_pp_mttkrp(cp_ctx *ctx, int mode, float *M_dev);

/*
 * cp_fit - relative residual r and fitness f = 1 - r (Sec. V-C).
 *   exact 0: Eq. (residual) from the amortized terms of the last update
 *            (||T||^2 + <Gamma(N), S(N)> - 2 <M(N), A(N)>, radicand clamped at 0)
 *   exact 1: directly, ||T - [[A]]||_F / ||T||_F (Eq. residual-def), one
 *            streaming pass over T.
 * Either output pointer may be NULL.  Synchronises the stream.
 */
cp_status cp_fit(cp_ctx *ctx, int exact, double *fit, double *resid);

/* Copy factor `mode` out (host, s_mode x R FP64) or replace it (and its Gram). */
cp_status cp_get_factor(cp_ctx *ctx, int mode, double *A_host);
cp_status cp_set_factor(cp_ctx *ctx, int mode, const double *A_host);

/* Per-sweep trace record, appended by every sweep call. */
typedef struct {
    int32_t sweep;        /* 0-based sweep index since cp_init                    */
    int32_t kind;         /* 0 DT, 1 MSDT, 2 PP approximated, 3 PP regular (MSDT) */
    int32_t pp_init;      /* 1 if PP operators were (re)built before this sweep   */
    int32_t rolled_back;  /* 1 if the policy's judge undid this sweep             */
    double resid;         /* Eq. (residual) after the sweep                       */
    double max_rel_step;  /* max_i ||A(i)_after - A(i)_before||_F / ||A(i)||_F    */
    double max_rel_dAp;   /* max_i ||A(i) - A_p(i)||_F / ||A(i)||_F (0 if no ops)  */
    double v_share;       /* ||V(N-1)||_F / ||M~(N-1)||_F in PP sweeps, else 0    */
    double ms;            /* device time of the sweep (CUDA events), including
                             its operator build and, with a policy, the network
                             query and the judge                               */
    float p_cur, p_new;   /* policy scores before the sweep (-1: not queried)     */
    int32_t decided_by;   /* 0 eps rule, 1 policy network, 2 regular sweep after
                             a rollback or a stalled run, 3 cp_pp_probe, 4 eps
                             rule because the network's output was invalid    */
    int32_t reserved;
} cp_trace_rec;

/* Copy up to *len records into buf (may be NULL); *len returns the total count. */
cp_status cp_get_trace(cp_ctx *ctx, cp_trace_rec *buf, size_t *len);

/* Work counters since cp_init. */
typedef struct {
    int64_t ttm;            /* first-level TTMs (2 s^N R flops each)          */
    int64_t mttv;           /* multi-TTV launches                             */
    int64_t pp_init;        /* PP operator builds                             */
    int64_t sweeps_exact;   /* DT/MSDT/regular sweeps                         */
    int64_t sweeps_pp;      /* approximated sweeps                            */
    int64_t launches;       /* kernel launches issued by the library          */
    double ttm_flops;       /* algorithmic flops of the first-level TTMs      */
    double mttv_flops;      /* 2 x entries read, summed over mTTVs            */
    double pp_flops;        /* U + V flops of approximated MTTKRPs            */
    double ttm_bytes;       /* algorithmic HBM bytes of the TTMs (read+write) */
    double mttv_bytes;      /* algorithmic bytes of the mTTVs                 */
    int64_t ttm_tensor_core;/* first-level TTMs that ran on tcgen05           */
    int64_t ttm_fused;      /* of those, two-level contractions T x_{a,a+1} with
                               the Khatri-Rao operand (standard tree)         */
    int64_t solves_fp64;    /* updates whose normal equations needed the FP64
                               factorisation (ill-conditioned Gamma)          */
    int64_t rollbacks;      /* policy judge rollbacks                         */
    int64_t lookahead;      /* multi-sweep nodes contracted ahead, overlapped
                               with the next update (cp_set_option)           */
    int64_t ttm_child;      /* first-level TTMs whose epilogue also produced
                               the first child node (cp_set_option)           */
    int64_t ttm_stored_parts;/* first-level TTMs that read T's stored 16-bit
                               parts (CP_OPT_TTM_PRESPLIT)                    */
} cp_stats;
cp_status cp_get_stats(cp_ctx *ctx, cp_stats *st);

/*
 * cp_set_option - schedule switches that change the order or fusion of the
 * tree's contractions, never which nodes are formed from which factor values
 * (Fig. 1a, Fig. 2): results agree to FP32 rounding.
 *   CP_OPT_FUSE_DT    (default 1) standard tree: contract a half's first two
 *                     modes from T in one pass with their Khatri-Rao product (no
 *                     s^(N-1) R node); 0 runs Fig. 1a literally (first-level TTM,
 *                     then one multi-TTV per level).
 *   CP_OPT_LOOKAHEAD  (default 0) multi-sweep tree, N >= 4: contract the level-2
 *                     node of the update after next on a second stream while the
 *                     next update runs; value 1..8 = blocks per SM that
 *                     contraction may hold (the rest is left to the next update's
 *                     kernels); results are bit-identical to 0.
 *   CP_OPT_FUSE_CHILD (default 0) multi-sweep tree: when the first child of a
 *                     root contracts the root's innermost mode (roots T x_0 and
 *                     T x_{N-1}), the tensor-core TTM's epilogue forms it too and
 *                     the root is read once instead of twice.
 *   CP_OPT_WAIT_LIMIT (default 0) the bounded waits of the tensor-core TTM
 *                     pipeline give up after `value` SM clock cycles (0: about
 *                     one second).  A wait that runs out makes the kernel drain
 *                     its copies in flight, free its tensor memory and return;
 *                     the next call that synchronises reports CP_ETIMEOUT and the
 *                     context is poisoned.  A tiny value exists for tests of that
 *                     path (no GPU fault, no hang).
 *   CP_OPT_MSDT_LEVELS (default 1) multi-sweep tree with its upper l levels
 *                     combined (Sec. IV, the memory / cost trade-off), 1 <= l <= N-2:
 *                     update t belongs to subtree t / (N-l), whose root contracts the
 *                     l modes updated just before its first update t0 = (t/(N-l))(N-l),
 *                     i.e. t0-1, ..., t0-l (mod N), and serves the next N-l updates.
 *                     Intermediates need s^(N-l) R entries instead of s^(N-1) R; the
 *                     first-level work becomes 2N/(N-l) s^N R per sweep.  For l = 2
 *                     and adjacent modes the root is one tensor-core pass over T with
 *                     the two factors' Khatri-Rao product.  The look-ahead applies to
 *                     l = 1 only; results agree with l = 1 to FP32 rounding.
 *   CP_OPT_SOLVE_FP64 (default 0) 1: solve every update's normal equations with
 *                     the FP64 LDL^T factorisation and FP64 substitution (Alg. 1,
 *                     solve step, as a Cholesky-type solve in FP64) instead of the FP32
 *                     inverse with FP64 refinement; slower, for inputs whose Gamma
 *                     is too ill-conditioned for the refinement.  The library also
 *                     falls back to it by itself per update when its a-posteriori
 *                     check of the FP32 inverse fails (cp_stats.solves_fp64).
 *   CP_OPT_TTM_PRESPLIT (default 1) R > 128 with CP_F16X3 / CP_BF16X3: keep T's
 *                     two 16-bit parts per mode in device memory, the contracted
 *                     mode innermost (2 x 2 bytes per entry and mode, written at
 *                     cp_init and cp_load_tensor), so that the first-level TTM
 *                     loads its operand with TMA instead of converting T; a mode
 *                     whose copy does not fit, or whose size is not a multiple
 *                     of 8, converts T as with 0.  1: column passes of up to 256
 *                     (results bit-identical to 0); 2: passes of 128 with two
 *                     accumulator sets (results equal to FP32 rounding; faster
 *                     only for small tensors).
 * CP_EINVAL for an unknown option or value.  Takes effect at the next call.
 */
enum { CP_OPT_FUSE_DT = 1, CP_OPT_LOOKAHEAD = 2, CP_OPT_FUSE_CHILD = 3, CP_OPT_WAIT_LIMIT = 4,
       CP_OPT_MSDT_LEVELS = 5, CP_OPT_SOLVE_FP64 = 6, CP_OPT_TTM_PRESPLIT = 7 };
cp_status cp_set_option(cp_ctx *ctx, int option, int value);

/*
 * cp_resid_noalloc - the direct residual of cp_fit(exact = 1) for callers that
 * cannot allocate device memory when they need it: programs whose own memory
 * pool has reserved the GPU (a raw cudaMalloc would fail or fragment it) and
 * latency-critical loops where cudaMalloc/cudaFree would synchronise the device.
 * The paper has no counterpart; this is a library convenience.
 *   N, dims, R  as in cp_init (3 <= N <= 8, 1 <= R <= 256).
 *   T_dev       FP32 tensor, C order, device.
 *   A_dev       host array of N device pointers to FP32 factors (s_n x R,
 *               row-major).
 *   out_dev     device buffer of 2 doubles: out[0] = ||T - [[A]]||_F^2,
 *               out[1] = ||T||_F^2; the relative residual is sqrt(out[0]/out[1]).
 *   stream      cudaStream_t (as void*) the two kernels are enqueued on; the
 *               call does not synchronise.
 * It allocates nothing: its scratch (one partial sum per 64 x 64 tile of T seen
 * as (modes 0..N-2) x mode N-1) is a fixed array of 2 x 65536 doubles (1 MiB) in
 * the library's device memory, held by every GPU that loads the library until
 * the process exits.  Tensors needing more than 65536 tiles are rejected with
 * CP_EINVAL (for example 128^4 fits exactly, 1024^3 does not).  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current, so make that first call before any stream capture.  All
 * calls share the array, and it keeps the last call's contents (each call writes
 * every slot it reads, so nothing needs clearing): calls that overlap on the GPU,
 * on different streams or devices' threads sharing a context, race and must be
 * serialised by the caller.  Returns CP_EINVAL on bad arguments, CP_ECUDA if a
 * CUDA call fails.
 */
cp_status cp_resid_noalloc(int N, const int64_t *dims, int R, const float *T_dev,
                           const float *const *A_dev, double *out_dev, void *stream);

/* Description of the first failure of this context ("" if none); never NULL. */
const char *cp_last_error(const cp_ctx *ctx);

/* Release everything the context owns.  NULL-safe; T is not freed. */
void cp_free(cp_ctx *ctx);

/*
 * Learned PP policy (no counterpart in the paper; Alg. 2's eps rule is the
 * fallback).  A small MLP 8 -> 64 -> 64 -> 1 (tanh, tanh, sigmoid; 4801 FP32
 * parameters, order W1, b1, W2, b2, w3, b3) scores from 8 trace features how
 * safe an approximated sweep is.  Training and inference run in the library's
 * own CUDA kernels on the stream given here.
 */
cp_status cp_policy_create(cp_policy **out, const float *theta_host, void *stream);
cp_status cp_policy_get(cp_policy *p, float *theta_host);
/* Forward pass: X_dev (B x 8 floats) -> prob_dev (B floats). */
cp_status cp_policy_forward(cp_policy *p, const float *X_dev, int B, float *prob_dev);
/* Mean binary cross-entropy and its gradient (4801 floats) on a batch. */
cp_status cp_policy_grad(cp_policy *p, const float *X_dev, const float *y_dev, int B,
                         float *loss_dev, float *grad_dev);
/* `steps` Adam steps (Kingma and Ba 2015) over one batch, lr given. */
cp_status cp_policy_train(cp_policy *p, const float *X_dev, const float *y_dev, int B,
                          int steps, float lr);
void cp_policy_free(cp_policy *p);

#ifdef __cplusplus
}
#endif
#endif /* CPALS_H */
