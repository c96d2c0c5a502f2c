// Host driver and C ABI of the CP-ALS engine.
//
// Schedules (Sec. II-C, III, Alg. 1-2) are expressed as contraction paths: the
// MTTKRP of mode u is reached from T by contracting the other modes one at a
// time, and each prefix of that sequence is a dimension-tree intermediate
// M^(kept modes) (Eq. tensors-cp).  Intermediates live in one device buffer per
// number of kept modes ("slot") and carry the version of every factor they were
// contracted with, so a node is reused exactly when its contents would be
// identical.  With the standard tree's paths this executes the dimension tree of
// Fig. 1a (two first-level TTMs per sweep); with the multi-sweep paths it
// executes Fig. 2, whose root survives across sweep and call boundaries.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>
#include <vector>

#include "cpals_internal.h"

namespace {

struct Slot {
    float* buf = nullptr;
    size_t cap = 0;            // floats
    bool valid = false;
    uint32_t contracted = 0;   // bitmask of contracted modes
    int ver[CP_MAXN] = {0};
};

}  // namespace

struct cp_policy {
    float* theta = nullptr;  // device, 4801
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    float* scratch = nullptr;
    float* loss = nullptr;
    int t = 0;
    cudaStream_t st = nullptr;
};

struct cp_ctx {
    int N = 0, R = 0, Rpad = 0;
    int64_t dims[CP_MAXN] = {0};
    int Kpad[CP_MAXN] = {0};
    int64_t numel = 0;
    int smax = 0;
    const float* T = nullptr;
    float* T_owned = nullptr;
    cudaStream_t st = nullptr;
    cp_config cfg;
    int num_sms = 148;

    double* A64[CP_MAXN] = {0};
    float* A32[CP_MAXN] = {0};
    uint16_t* bhi[CP_MAXN] = {0};   // bf16 parts, or fp16 parts of the scaled factor (f16x3)
    uint16_t* blo[CP_MAXN] = {0};
    float* bt32[CP_MAXN] = {0};
    // f16x3: per-column output scales of each factor operand, and the factor
    // version the fp16 parts were converted from (converted lazily, before a TTM)
    float* colinv[CP_MAXN] = {0};
    int f16_ver[CP_MAXN] = {-1, -1, -1, -1, -1, -1, -1, -1};
    int eT = 0;                     // f16x3: T is multiplied by 2^eT before its split
    // R > 128, f16x3 / bf16x3: T's 16-bit parts per mode, contracted mode
    // innermost ([P][Q][K]), read by that mode's first-level TTM instead of T
    uint16_t* Tp_hi[CP_MAXN] = {0};
    uint16_t* Tp_lo[CP_MAXN] = {0};
    int presplit = 1;   // 0 off, 1 on (256-column passes), 2 on with 128-column passes
    double* S[CP_MAXN] = {0};
    double* dS[CP_MAXN] = {0};
    double* Ap64[CP_MAXN] = {0};
    float* dA32[CP_MAXN] = {0};
    double* dA64[CP_MAXN] = {0};
    // R <= 128: the factor and its change as float pairs (hi + lo = the FP64
    // value), written by the row solve for the double-float Gram
    float2* A2[CP_MAXN] = {0};
    float2* dA2[CP_MAXN] = {0};
    float2* S2[CP_MAXN] = {0};      // the Grams as float pairs (R <= 128)
    float2* dS2[CP_MAXN] = {0};
    float2** d_S2list = nullptr;
    float2** d_dS2list = nullptr;
    int ver[CP_MAXN] = {0};
    double** d_Slist = nullptr;
    double** d_dSlist = nullptr;

    double *Gamma = nullptr, *L = nullptr, *invd = nullptr, *W = nullptr;
    float* Ginv = nullptr;      // FP32 Gamma^{-1} for iterative refinement
    float* G32 = nullptr;       // FP32 copy of Gamma (input of the inverse)
    float* G2 = nullptr;        // Gamma as float pairs (hi, lo): the double-float refinement
    float* W2 = nullptr;        // PP's W as float pairs
    float* schur_ws = nullptr;  // blocked inverse workspace (R > 128)
    cudaStream_t side = nullptr;            // normal-equation factorisation runs here,
    cudaEvent_t ev_ready = nullptr, ev_chol = nullptr;  // overlapped with the MTTKRP
    bool chol_pending = false;
    int chol_mode = -1;         // mode whose factorisation is pending
    int* d_mode = nullptr;      // 0: refinement path, 1: FP64 substitution path
    double* tile_gs = nullptr;     // per mode: tile shares of <Gamma, S>
    int ntiles = 1;
    double* scal_part = nullptr;   // per mode: the solve's per-block scalars
    // the update's scalars are reduced on their own stream, off the critical path
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_g = nullptr, ev_scal[CP_MAXN] = {0};
    int aux_last = -1;   // mode whose scalars the aux stream finished last (ev_scal)
    double* scal_hist = nullptr;   // [cap][N][CP_NSCAL]
    int scal_hist_cap = 0;
    double* red_part = nullptr;
    double* d_red_out = nullptr;
    unsigned* dev_err = nullptr;
    double normT2 = 0.0;

    Slot slot[CP_MAXN + 1];
    // Multi-sweep look-ahead: a node of the update after next whose inputs are
    // already final is contracted on `ahead` into alt[k] while the next update's
    // MTTKRP and normal equations run on the main stream (same nodes, same
    // arithmetic as Fig. 2; only the order of independent work changes).
    Slot alt[CP_MAXN + 1];
    int64_t alt_busy[CP_MAXN + 1] = {0};  // update index that still reads alt[k]
    cudaStream_t ahead = nullptr;
    cudaEvent_t ev_x = nullptr, ev_ahead = nullptr;
    bool ahead_pending = false;
    int64_t ahead_target = -1;
    bool lookahead = false;
    int ahead_blocks_per_sm = 3;  // leaves every SM room for the normal-equation kernels
    cpk::TcPlan* tc_plan[CP_MAXN] = {0};   // tensor-core TTM per mode (NULL: SIMT)
    // fused two-mode contraction T x_{a,a+1} KR(A_a, A_{a+1}) per adjacent pair a
    cpk::TcPlan* kr_plan[CP_MAXN] = {0};
    int kr_Kpad[CP_MAXN] = {0};
    void* kr_hi = nullptr;
    void* kr_lo = nullptr;
    float* kr_scale = nullptr;   // f16x3: column powers of two of the Khatri-Rao operand
    float* kr_colinv = nullptr;
    float* splitk_ws = nullptr;
    bool fuse_dt = true;
    bool fuse_child = false;
    int msdt_levels = 1;       // upper levels of the multi-sweep tree combined (Sec. IV)
    bool solve_fp64 = false;   // normal equations always by the FP64 factorisation
    long long wait_limit = 0;  // tensor-core TTM's bounded waits (cycles; 0: about 1 s)  // TTM epilogue forms the first child (multi-sweep tree)
    float* child_ws = nullptr;  // pieces of first-child segments that cross TTM tiles
    size_t child_ws_cap = 0;

    // PP state.  An operator set is A_p with the M_p(i,j) and M_p(n) built from
    // it; pair/Mp/Ap64 point into the current set.  A second set is allocated
    // only for branch probing, where a rebuild writes the idle set so that the
    // operators of the starting state survive.
    bool pp_alloc = false, pp_valid = false, ops2 = false;
    int ops = 0;
    float* pairset[2][CP_MAXN][CP_MAXN] = {{{0}}};
    float* Mpset[2][CP_MAXN] = {{0}};
    double* Apset[2][CP_MAXN] = {{0}};
    float* pair[CP_MAXN][CP_MAXN] = {{0}};
    float* Mp[CP_MAXN] = {0};
    float* Mt = nullptr;
    double dA_rel[CP_MAXN];  // ||dA(i)|| / ||A(i)|| as Alg. 2 tests it
    int since_init = 0;      // approximated sweeps since the operators were built

    int64_t t_msdt = 0;
    int sweeps_done = 0;
    bool have_last = false;
    double last_resid = 1.0;
    // factor versions come from one clock, so a version number names one factor
    // value for the life of the context (restored snapshots keep cache keys sound)
    int vclock = 0;

    // state snapshots: [0] branch probing, [1] the policy judge's rollback point
    struct Snap {
        bool have = false;
        double* A64[CP_MAXN] = {0};
        int ver[CP_MAXN] = {0};
        bool pp_valid = false;
        int ops = 0, since_init = 0, sweeps_done = 0;
        double dA_rel[CP_MAXN] = {0};
        int64_t t_msdt = 0;
        bool have_last = false;
        double last_resid = 1.0;
        size_t trace_len = 0;
    } snap[2];
    float* pol_io = nullptr;   // device: 16 policy features + 2 scores
    double judge_r = -1.0;     // direct residual at the judge's rollback point
    int since_judge = 0;       // approximated sweeps since the rollback point
    int fallback_left = 0;
    int rollbacks_in_row = 0;  // consecutive rollbacks (the fallback doubles each time)
    double pending_ms = 0.0;   // policy query / rollback-point time of the coming sweep
    // measured device time of the choices (exponential averages; < 0: not yet seen)
    double cost_exact = -1.0, cost_pp = -1.0, cost_init = -1.0, cost_judge = -1.0, cost_query = -1.0;
    int n_exact_seen = 0;
    double pp_ms_total = 0.0;   // all-in time of the approximated sweeps (builds, judge, queries)
    int pp_n = 0;
    double sweep_mttkrp_bytes = -1.0;  // MTTKRP bytes of the last regular sweep
    bool snap_current = false;  // the rollback point is the present state

    std::vector<cp_trace_rec> trace;
    std::vector<double> last_hist;   // host copy of the last harvested scalars
    std::vector<cudaEvent_t> events;
    cp_stats stats;
    std::string err;
    bool poisoned = false;
};

namespace {

// ------------------------------------------------------------------ errors
cp_status fail(cp_ctx* c, cp_status s, const std::string& msg) {
    if (c && c->err.empty()) c->err = msg;
    if (c && (s == CP_ECUDA || s == CP_ETIMEOUT)) c->poisoned = true;
    return s;
}

#define CKCUDA(ctx, expr)                                                                  \
    do {                                                                                   \
        cudaError_t e__ = (expr);                                                          \
        if (e__ != cudaSuccess)                                                            \
            return fail(ctx, CP_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e__)); \
    } while (0)

#define CKST(expr)                     \
    do {                               \
        cp_status s__ = (expr);        \
        if (s__ != CP_OK) return s__;  \
    } while (0)

#define LAUNCH(ctx, expr)          \
    do {                           \
        (ctx)->stats.launches++;   \
        CKCUDA(ctx, (expr));       \
    } while (0)

// which operand copies of a factor the chosen TTM precision reads
bool uses_bf16(const cp_ctx* c) { return c->cfg.prec == CP_BF16X3 || c->cfg.prec == CP_BF16; }
bool uses_tf32(const cp_ctx* c) { return c->cfg.prec == CP_TF32X3 || c->cfg.prec == CP_TF32; }

template <class Tp>
cp_status dalloc(cp_ctx* c, Tp** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(Tp));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, CP_ENOMEM, "cudaMalloc of " + std::to_string(n * sizeof(Tp)) + " bytes failed");
    }
    return CP_OK;
}

// ------------------------------------------------------------------ Philox4x32-10 (host)
// Salmon et al., SC'11: ten rounds; multipliers 0xD2511F53, 0xCD9E8D57; key
// increments 0x9E3779B9, 0xBB67AE85 between rounds.
void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        const uint32_t n1 = (uint32_t)p1;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        const uint32_t n3 = (uint32_t)p0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
}

void philox_uniform(uint64_t seed, uint32_t stream, size_t n, double* out) {
    for (size_t j = 0; 2 * j < n; ++j) {
        uint32_t c[4] = {(uint32_t)j, (uint32_t)((uint64_t)j >> 32), stream, 0u};
        philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        const uint64_t a = (((uint64_t)c[0] << 32) | c[1]) >> 11;
        const uint64_t b = (((uint64_t)c[2] << 32) | c[3]) >> 11;
        out[2 * j] = (double)a * 0x1.0p-53;
        if (2 * j + 1 < n) out[2 * j + 1] = (double)b * 0x1.0p-53;
    }
}

// ------------------------------------------------------------------ contraction helpers
// kept modes of a node = all modes minus `contracted`, in increasing order
void contract_dims(const cp_ctx* c, uint32_t contracted, int mode, int64_t* P, int64_t* Q) {
    int64_t p = 1, q = 1;
    for (int k = 0; k < c->N; ++k) {
        if (contracted & (1u << k)) continue;
        if (k < mode) p *= c->dims[k];
        if (k > mode) q *= c->dims[k];
    }
    *P = p;
    *Q = q;
}

// f16x3: the fp16 parts of factor `mode` (and its column scales) from its FP32
// copy, unless they already hold the current version
cp_status ensure_f16(cp_ctx* c, int mode) {
    if (c->cfg.prec != CP_F16X3 || c->f16_ver[mode] == c->ver[mode]) return CP_OK;
    LAUNCH(c, cpk::f16_operand(c->A32[mode], (int)c->dims[mode], c->R, c->Rpad, c->Kpad[mode], c->eT,
                               c->bhi[mode], c->blo[mode], c->colinv[mode], c->st));
    c->f16_ver[mode] = c->ver[mode];
    return CP_OK;
}

// SMs for a persistent tensor-core TTM: one fewer while the one-CTA
// factorisation of the side stream is in flight, so that no TTM CTA waits for its
// SM (the tiles are assigned statically; a late CTA would delay the whole TTM)
int tc_sms(const cp_ctx* c) { return c->chol_pending && c->num_sms > 1 ? c->num_sms - 1 : c->num_sms; }

cp_status launch_ttm(cp_ctx* c, int mode, float* X) {
    int64_t P, Q;
    contract_dims(c, 0u, mode, &P, &Q);
    const int K = (int)c->dims[mode];
    const int prec = c->cfg.prec;
    if (prec != CP_FP32_SIMT && c->tc_plan[mode]) {
        CKST(ensure_f16(c, mode));
        LAUNCH(c, cpk::ttm_tc_run(c->tc_plan[mode], X, prec, tc_sms(c), c->dev_err, c->st, c->splitk_ws, nullptr,
                                  c->wait_limit));
        if (c->splitk_ws && cpk::ttm_tc_splitk(c->tc_plan[mode], c->num_sms) > 1) c->stats.launches++;  // partial-sum kernel
        c->stats.ttm_tensor_core++;
        if (cpk::ttm_tc_stored_parts(c->tc_plan[mode])) c->stats.ttm_stored_parts++;
    } else {
        LAUNCH(c, cpk::ttm_simt(c->T, c->A32[mode], X, P, K, Q, c->R, c->st));
    }
    c->stats.ttm++;
    c->stats.ttm_flops += 2.0 * (double)c->numel * c->R;
    c->stats.ttm_bytes += 4.0 * ((double)c->numel + (double)(c->numel / K) * c->R);
    return CP_OK;
}

cp_status launch_mttv(cp_ctx* c, const float* X, uint32_t contracted, int mode, float* Y,
                      cudaStream_t st = nullptr, int max_blocks_per_sm = 0) {
    int64_t P, Q;
    contract_dims(c, contracted, mode, &P, &Q);
    const int K = (int)c->dims[mode];
    if (P * Q == 0) return CP_OK;
    LAUNCH(c, cpk::mttv(X, c->A32[mode], Y, P, K, Q, c->R, c->num_sms, st ? st : c->st, max_blocks_per_sm));
    const double nin = (double)P * K * Q * c->R;
    c->stats.mttv++;
    c->stats.mttv_flops += 2.0 * nin;
    c->stats.mttv_bytes += 4.0 * (nin + (double)P * Q * c->R);
    return CP_OK;
}

// Level-2 node straight from T: contract the adjacent modes a, a+1 at once with
// their Khatri-Rao product (two dimension-tree levels in one pass over T).
cp_status launch_fused2(cp_ctx* c, int a, float* X) {
    const int kind = cpk::ttm_tc_kind(c->kr_plan[a]);
    const int R = c->R, sa = (int)c->dims[a], sb = (int)c->dims[a + 1];
    LAUNCH(c, cpk::kr_operand(c->A64[a], c->A64[a + 1], sa, sb, R, c->kr_Kpad[a], kind, c->kr_hi, c->kr_lo,
                              c->st, c->eT, c->kr_scale, c->kr_colinv));
    LAUNCH(c, cpk::ttm_tc_run(c->kr_plan[a], X, c->cfg.prec, tc_sms(c), c->dev_err, c->st, c->splitk_ws, nullptr,
                              c->wait_limit));
    if (c->splitk_ws && cpk::ttm_tc_splitk(c->kr_plan[a], c->num_sms) > 1) c->stats.launches++;  // partial-sum kernel
    const double rows = (double)c->numel / ((double)sa * sb);
    c->stats.ttm++;
    c->stats.ttm_tensor_core++;
    c->stats.ttm_fused++;
    c->stats.ttm_flops += 2.0 * (double)c->numel * R;
    c->stats.ttm_bytes += 4.0 * ((double)c->numel + rows * R);
    return CP_OK;
}

// A cached node equal to the contraction of `mask` with the current factors:
// the slot of its level or the look-ahead slot, else NULL.
Slot* find_node(cp_ctx* c, uint32_t mask) {
    const int k = c->N - __builtin_popcount(mask);
    for (Slot* s : {&c->slot[k], &c->alt[k]}) {
        if (!s->buf || !s->valid || s->contracted != mask) continue;
        bool ok = true;
        for (int m = 0; ok && m < c->N; ++m)
            if ((mask >> m & 1u) && s->ver[m] != c->ver[m]) ok = false;
        if (ok) return s;
    }
    return nullptr;
}

// Tree intermediates are allocated on first use: a schedule that never forms a
// level (the fused standard tree, the multi-sweep tree with combined upper
// levels) never holds its memory.
cp_status slot_buf(cp_ctx* c, Slot& s) {
    if (!s.buf && s.cap) CKST(dalloc(c, &s.buf, s.cap));
    return CP_OK;
}

// The main stream waits for the look-ahead contraction in flight, if any.
cp_status ahead_join(cp_ctx* c) {
    if (!c->ahead_pending) return CP_OK;
    CKCUDA(c, cudaStreamWaitEvent(c->st, c->ev_ahead, 0));
    c->ahead_pending = false;
    return CP_OK;
}

// Multi-sweep root T x_m A(m) whose first child contracts cm: the TTM epilogue
// can form the child too when cm is the root's innermost kept mode.
bool child_fusable(const cp_ctx* c, int m, int cm) {
    if (!c->fuse_child || c->cfg.prec == CP_FP32_SIMT || !c->tc_plan[m]) return false;
    const int N = c->N;
    const int inner = (m == N - 1) ? N - 2 : N - 1;
    if (cm != inner || !(m == 0 || m == N - 1)) return false;
    const int sc = (int)c->dims[cm];
    if (!cpk::ttm_tc_child_ok(c->tc_plan[m], sc)) return false;
    return (size_t)cpk::ttm_tc_child_ws_floats(c->tc_plan[m], sc) <= c->child_ws_cap;
}

// Root X = T x_m A(m) and its first child Y = X x_cm A(cm) in one pass over T.
cp_status launch_ttm_child(cp_ctx* c, int m, int cm, float* X, float* Y) {
    cpk::TcChild ch;
    ch.Y = Y;
    ch.Ac = c->A32[cm];
    ch.sc = (int)c->dims[cm];
    ch.ws = c->child_ws;
    CKST(ensure_f16(c, m));
    LAUNCH(c, cpk::ttm_tc_run(c->tc_plan[m], X, c->cfg.prec, c->num_sms, c->dev_err, c->st, nullptr, &ch,
                              c->wait_limit));
    if (cpk::ttm_tc_child_ws_floats(c->tc_plan[m], ch.sc) > 0) c->stats.launches++;  // cross-tile segments
    const int64_t rows = c->numel / c->dims[m];
    c->stats.ttm++;
    c->stats.ttm_tensor_core++;
    c->stats.ttm_child++;
    c->stats.ttm_flops += 2.0 * (double)c->numel * c->R;
    c->stats.ttm_bytes += 4.0 * ((double)c->numel + (double)rows * c->R);
    // the child is the multi-TTV the epilogue replaced (its input is not re-read)
    c->stats.mttv_flops += 2.0 * (double)rows * c->R;
    c->stats.mttv_bytes += 4.0 * (double)(rows / ch.sc) * c->R;
    return CP_OK;
}

// Ensure the node reached by contracting path[0..d-1] is in its slot; returns it.
// fuse2: the level-1 node of this path has no other use, so the level-2 node may
// be computed from T directly when its two modes are adjacent.
// child: multi-sweep path; a level-2 node whose root is missing may come from
// the root's TTM epilogue (child_fusable).
cp_status ensure_node(cp_ctx* c, const int* path, int d, float** out, bool fuse2 = false,
                      bool child = false) {
    uint32_t mask = 0;
    for (int i = 0; i < d; ++i) mask |= 1u << path[i];
    if (Slot* h = find_node(c, mask)) {
        *out = h->buf;
        return CP_OK;
    }
    Slot& s = c->slot[c->N - d];
    CKST(slot_buf(c, s));
    s.valid = false;
    const int lo_m = d >= 2 ? std::min(path[0], path[1]) : -1;
    if (d == 2 && child && !find_node(c, 1u << path[0]) && child_fusable(c, path[0], path[1])) {
        Slot& root = c->slot[c->N - 1];
        CKST(slot_buf(c, root));
        root.valid = false;
        CKST(launch_ttm_child(c, path[0], path[1], root.buf, s.buf));
        root.valid = true;
        root.contracted = 1u << path[0];
        for (int k = 0; k < c->N; ++k) root.ver[k] = c->ver[k];
    } else if (d == 1) {
        CKST(launch_ttm(c, path[0], s.buf));
    } else if (d == 2 && fuse2 && std::abs(path[0] - path[1]) == 1 && c->kr_plan[lo_m]) {
        CKST(launch_fused2(c, lo_m, s.buf));
    } else {
        float* parent = nullptr;
        CKST(ensure_node(c, path, d - 1, &parent, fuse2, child));
        CKST(launch_mttv(c, parent, mask & ~(1u << path[d - 1]), path[d - 1], s.buf));
    }
    s.valid = true;
    s.contracted = mask;
    for (int k = 0; k < c->N; ++k) s.ver[k] = c->ver[k];
    *out = s.buf;
    return CP_OK;
}

// Binary dimension tree over ordered leaves: append the contractions that lead
// from the node holding `leaves` to leaf u.  First child: contract the later
// half starting from its last leaf; second child: the earlier half in order.
void tree_path(std::vector<int> leaves, int u, std::vector<int>& seq) {
    while (leaves.size() > 1) {
        const size_t h = (leaves.size() + 1) / 2;
        std::vector<int> L1(leaves.begin(), leaves.begin() + h), L2(leaves.begin() + h, leaves.end());
        if (std::find(L1.begin(), L1.end(), u) != L1.end()) {
            for (size_t i = L2.size(); i-- > 0;) seq.push_back(L2[i]);
            leaves = L1;
        } else {
            for (int m : L1) seq.push_back(m);
            leaves = L2;
        }
    }
}

// Standard tree (Fig. 1a).  *fuse2 is set when the first two contractions from T
// belong to one chain (the first half's other modes), i.e. the level-1 node
// serves a single child.
std::vector<int> dt_path(int N, int u, bool* fuse2 = nullptr) {
    std::vector<int> leaves(N), seq;
    for (int i = 0; i < N; ++i) leaves[i] = i;
    tree_path(leaves, u, seq);
    if (fuse2) {
        const int h = (N + 1) / 2;
        const bool left = u < h;
        *fuse2 = (left ? N - h : h) >= 2;
    }
    return seq;
}

// MSDT (Sec. III): update t belongs to subtree j = t / (N-1) with root mode
// m = (N-1-j) mod N serving leaves m+1, ..., m+N-1 (mod N).  With the upper
// `levels` = l levels combined (Sec. IV: the memory / cost trade-off), subtree
// j = t / (N-l) starts at update t0 = j (N-l); its root contracts the l modes
// updated just before, t0-1, ..., t0-l (mod N), in one pass over T when l = 2 and
// they are adjacent (Khatri-Rao operand), and serves leaves t0, ..., t0+N-l-1.
// For l = 1 both descriptions give the same tree.
std::vector<int> msdt_path(int N, int64_t t, int* u_out, int levels = 1) {
    const int l = levels;
    const int64_t j = t / (N - l);
    const int64_t t0 = j * (N - l);
    std::vector<int> leaves(N - l), seq;
    for (int i = 0; i < N - l; ++i) leaves[i] = (int)((t0 + i) % N);
    const int u = leaves[(size_t)(t - t0)];
    for (int i = 0; i < l; ++i) seq.push_back((int)(((t0 - 1 - i) % N + N) % N));
    tree_path(leaves, u, seq);
    *u_out = u;
    return seq;
}

cp_status mttkrp_leaf(cp_ctx* c, const std::vector<int>& path, float** M, bool fuse2 = false,
                      bool child = false) {
    return ensure_node(c, path.data(), (int)path.size(), M, fuse2, child);
}

double* scal_slot(cp_ctx* c, int k, int mode) {
    return c->scal_hist + ((size_t)k * c->N + mode) * CP_NSCAL;
}

cp_status grow_hist(cp_ctx* c, int nsweeps) {
    if (nsweeps <= c->scal_hist_cap) return CP_OK;
    if (c->scal_hist) cudaFree(c->scal_hist);
    c->scal_hist = nullptr;
    c->scal_hist_cap = 0;
    CKST(dalloc(c, &c->scal_hist, (size_t)nsweeps * c->N * CP_NSCAL));
    c->scal_hist_cap = nsweeps;
    return CP_OK;
}

// Hadamard chain and factorisation of Gamma(u) (Alg. 1, the Hadamard product of the Grams) on the side
// stream: Gamma(u) needs only the Grams of the other modes, so it is enqueued
// before the MTTKRP of update u and runs concurrently with it.
cp_status launch_chol(cp_ctx* c, int u, bool pp, double* scal) {
    CKCUDA(c, cudaEventRecord(c->ev_ready, c->st));
    CKCUDA(c, cudaStreamWaitEvent(c->side, c->ev_ready, 0));
    LAUNCH(c, cpk::chol_mixed(c->d_Slist, c->d_dSlist, c->d_S2list, c->d_dS2list, c->N, u, c->R, pp ? 1 : 0,
                              c->Gamma, c->G32, c->G2, c->Ginv, c->L, c->invd, c->W, c->W2, scal, c->d_mode,
                              c->schur_ws, c->side, c->solve_fp64));
    CKCUDA(c, cudaEventRecord(c->ev_chol, c->side));
    c->chol_pending = true;
    c->chol_mode = u;
    return CP_OK;
}

// One factor update (Alg. 1: Gamma, MTTKRP, solve, Gram; in PP mode Alg. 2's approximated update with V).
// launch_chol(u) must have been called for this update.
cp_status update_mode(cp_ctx* c, int u, const float* M, bool pp, double* scal) {
    const int R = c->R, s = (int)c->dims[u];
    if (!c->chol_pending) CKST(launch_chol(c, u, pp, scal));
    CKCUDA(c, cudaStreamWaitEvent(c->st, c->ev_chol, 0));
    c->chol_pending = false;
    cpk::SolveOut o;
    o.A64 = c->A64[u];
    o.A32 = c->A32[u];
    o.bhi = uses_bf16(c) ? c->bhi[u] : nullptr;
    o.blo = uses_bf16(c) ? c->blo[u] : nullptr;
    o.bt32 = uses_tf32(c) ? c->bt32[u] : nullptr;
    o.Rpad = c->Rpad;
    o.Kpad = c->Kpad[u];
    o.Ap = pp ? c->Ap64[u] : nullptr;
    o.dA32 = pp ? c->dA32[u] : nullptr;
    o.dA64 = pp ? c->dA64[u] : nullptr;
    o.A2 = c->A2[u];
    o.dA2 = pp ? c->dA2[u] : nullptr;
    int nblk = 0;
    double* sp = c->scal_part + (size_t)u * c->smax * CP_NSCAL;
    double* tg = c->tile_gs + (size_t)u * c->ntiles;
    CKCUDA(c, cudaStreamWaitEvent(c->st, c->ev_scal[u], 0));  // sp / tg of mode u are free
    LAUNCH(c, cpk::solve_mixed(M, pp ? c->W : nullptr, pp ? c->W2 : nullptr, c->Gamma, c->G2, c->Ginv, c->L,
                               c->invd, c->d_mode, o, s, R, scal,
                               sp, &nblk, c->dev_err, c->st));
    if (c->A2[u])
        LAUNCH(c, cpk::gram_df(c->A2[u], pp ? c->dA2[u] : nullptr, s, R, reinterpret_cast<const float2*>(c->G2),
                               c->S[u], c->dS[u], c->S2[u], c->dS2[u], tg, c->st));
    else
        LAUNCH(c, cpk::gram(c->A64[u], pp ? c->dA64[u] : nullptr, s, R, c->Gamma, c->S[u], c->dS[u], tg, c->st));
    CKCUDA(c, cudaEventRecord(c->ev_g, c->st));
    CKCUDA(c, cudaStreamWaitEvent(c->aux, c->ev_g, 0));
    LAUNCH(c, cpk::scal_fin(sp, nblk, tg, c->ntiles, scal, c->aux));
    CKCUDA(c, cudaEventRecord(c->ev_scal[u], c->aux));
    c->aux_last = u;
    c->ver[u] = ++c->vclock;
    return CP_OK;
}

cp_status check_dev_err(cp_ctx* c) {
    unsigned e = 0;
    CKCUDA(c, cudaMemcpyAsync(&e, c->dev_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
    CKCUDA(c, cudaStreamSynchronize(c->st));
    if (e & DEVERR_TIMEOUT) return fail(c, CP_ETIMEOUT, "a bounded device wait ran out");
    if (e & DEVERR_BADARG) return fail(c, CP_ECUDA, "a kernel rejected its launch arguments");
    return CP_OK;
}

// After `k` sweeps recorded in scal_hist: read them, append trace records.
cp_status harvest(cp_ctx* c, int k, const int* kinds, const int* inits, int first_event) {
    std::vector<double>& h = c->last_hist;
    h.assign((size_t)k * c->N * CP_NSCAL, 0.0);
    if (c->aux_last >= 0) CKCUDA(c, cudaStreamWaitEvent(c->st, c->ev_scal[c->aux_last], 0));  // the last scalars
    CKCUDA(c, cudaMemcpyAsync(h.data(), c->scal_hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CKST(check_dev_err(c));
    for (int i = 0; i < k; ++i) {
        const double* last = &h[((size_t)i * c->N + (c->N - 1)) * CP_NSCAL];
        cp_trace_rec rec;
        memset(&rec, 0, sizeof(rec));
        rec.sweep = c->sweeps_done + i;
        rec.kind = kinds[i];
        rec.pp_init = inits ? inits[i] : 0;
        rec.p_cur = rec.p_new = -1.f;
        const double r2 = c->normT2 + last[SCAL_GS] - 2.0 * last[SCAL_MA];
        rec.resid = sqrt(r2 > 0 ? r2 : 0.0) / sqrt(c->normT2);
        double mx = 0.0, mxp = 0.0;
        bool bad = false;
        // a NaN or Inf in a factor reaches every later Gamma; report it as such
        // before any factorisation failure it causes
        for (int n = 0; n < c->N; ++n) {
            const double* sc = &h[((size_t)i * c->N + n) * CP_NSCAL];
            if (!isfinite(sc[SCAL_A2]) || !isfinite(sc[SCAL_MA]) || !isfinite(sc[SCAL_GS])) bad = true;
        }
        if (bad) {
            c->sweeps_done += i + 1;
            return fail(c, CP_ENUMERIC, "non-finite factor or residual");
        }
        for (int n = 0; n < c->N; ++n) {
            const double* sc = &h[((size_t)i * c->N + n) * CP_NSCAL];
            const double a = sqrt(sc[SCAL_A2]);
            // flags: 0 refinement path, 3 refinement did not converge; 10 + (0 ok,
            // 1 shifted, 2 failed) for the FP64 factorisation path
            const double fl = sc[SCAL_FLAGS];
            if (fl >= 10.0) c->stats.solves_fp64++;
            if (fl == 3.0 || fl >= 12.0) {
                c->sweeps_done += i;
                return fail(c, CP_ENOTSPD, "Gamma(" + std::to_string(n) + ") not positive definite");
            }
            if (a > 0) {
                mx = std::max(mx, sqrt(sc[SCAL_STEP2]) / a);
                mxp = std::max(mxp, sqrt(sc[SCAL_DAP2]) / a);
            }
        }
        rec.max_rel_step = mx;
        rec.max_rel_dAp = mxp;
        if (kinds[i] == 2 && last[SCAL_M2] > 0) rec.v_share = sqrt(last[SCAL_V2] / last[SCAL_M2]);
        float ms = 0.f;
        if (first_event >= 0 && (size_t)(first_event + i + 1) < c->events.size())
            cudaEventElapsedTime(&ms, c->events[first_event + i], c->events[first_event + i + 1]);
        rec.ms = ms;
        c->trace.push_back(rec);
        c->last_resid = rec.resid;
        c->have_last = true;
        if (bad || !isfinite(rec.resid)) {
            c->sweeps_done += i + 1;
            return fail(c, CP_ENUMERIC, "non-finite factor or residual");
        }
    }
    c->sweeps_done += k;
    return CP_OK;
}

cp_status ensure_events(cp_ctx* c, size_t n) {
    while (c->events.size() < n) {
        cudaEvent_t e;
        CKCUDA(c, cudaEventCreate(&e));
        c->events.push_back(e);
    }
    return CP_OK;
}

cp_status entry_check(cp_ctx* c) {
    if (!c) return CP_EINVAL;
    if (c->poisoned) return CP_ESTATE;
    return CP_OK;
}

// After update t of the multi-sweep tree (Sec. III), when update t+2 belongs to
// the same subtree: the level-2 node on its path (root with one more mode
// contracted) is final once it contracts no factor that update t+1 changes.  If
// it is not on update t+1's path and not cached, contract it now on the `ahead`
// stream, on a capped grid, so that it overlaps update t+1.  For N = 4 this is
// the second child X x_a A(a) of Fig. 2 (root mode m, leaves a, b, c), computed
// while b is updated.
cp_status msdt_lookahead(cp_ctx* c, int64_t t) {
    const int N = c->N;
    if (!c->lookahead || N < 4 || !c->ahead || c->msdt_levels != 1) return CP_OK;
    if (t / (N - 1) != (t + 2) / (N - 1)) return CP_OK;
    int u1 = 0, u2 = 0;
    const std::vector<int> p1 = msdt_path(N, t + 1, &u1), p2 = msdt_path(N, t + 2, &u2);
    if (p2.size() < 3) return CP_OK;
    const uint32_t root = 1u << p2[0];
    const uint32_t mask = root | (1u << p2[1]);
    if (mask & (1u << u1)) return CP_OK;                               // changes at t+1
    if (p1.size() >= 2 && ((1u << p1[0]) | (1u << p1[1])) == mask) return CP_OK;  // next update builds it
    if (find_node(c, mask)) return CP_OK;
    Slot* parent = find_node(c, root);
    const int k = N - 2;
    if (!parent || parent == &c->alt[N - 1] || !c->alt[k].cap || c->alt_busy[k] > t) return CP_OK;
    Slot& s = c->alt[k];
    CKST(slot_buf(c, s));
    s.valid = false;
    CKCUDA(c, cudaEventRecord(c->ev_x, c->st));
    CKCUDA(c, cudaStreamWaitEvent(c->ahead, c->ev_x, 0));
    CKST(launch_mttv(c, parent->buf, root, p2[1], s.buf, c->ahead, c->ahead_blocks_per_sm));
    CKCUDA(c, cudaEventRecord(c->ev_ahead, c->ahead));
    s.valid = true;
    s.contracted = mask;
    for (int m = 0; m < N; ++m) s.ver[m] = c->ver[m];
    c->alt_busy[k] = t + 2;
    c->ahead_pending = true;
    c->ahead_target = t + 2;
    c->stats.lookahead++;
    return CP_OK;
}

// One exact sweep: DT (kind 0) or MSDT (kind 1/3).  Records into scal_hist[k].
// keep_ahead: the caller continues with another MSDT sweep, so a look-ahead
// contraction may stay in flight across the sweep boundary.
cp_status exact_sweep(cp_ctx* c, bool msdt, int k, bool keep_ahead = false) {
    for (int u0 = 0; u0 < c->N; ++u0) {
        int u = u0;
        std::vector<int> path;
        bool fuse2 = false;
        const int64_t t = c->t_msdt;
        if (msdt) {
            path = msdt_path(c->N, t, &u, c->msdt_levels);
            c->t_msdt++;
            if (c->ahead_pending && t >= c->ahead_target) CKST(ahead_join(c));
            // combined levels: the root's two contracted modes in one pass over T
            fuse2 = c->msdt_levels >= 2;
        } else {
            CKST(ahead_join(c));
            path = dt_path(c->N, u0, &fuse2);
            fuse2 = fuse2 && c->fuse_dt;
        }
        if (!(c->chol_pending && c->chol_mode == u)) CKST(launch_chol(c, u, false, scal_slot(c, k, u)));
        float* M = nullptr;
        CKST(mttkrp_leaf(c, path, &M, fuse2, msdt && c->msdt_levels == 1));
        CKST(update_mode(c, u, M, false, scal_slot(c, k, u)));
        if (msdt && c->lookahead && u0 + 1 < c->N) {
            // the next update's factorisation goes first, so that its one-CTA inverse
            // finds an SM before the look-ahead contraction fills them
            int un = 0;
            msdt_path(c->N, c->t_msdt, &un, c->msdt_levels);
            CKST(launch_chol(c, un, false, scal_slot(c, k, un)));
        }
        if (msdt) CKST(msdt_lookahead(c, t));
    }
    if (!keep_ahead) CKST(ahead_join(c));
    c->stats.sweeps_exact++;
    return CP_OK;
}

// ------------------------------------------------------------------ PP
void use_ops(cp_ctx* c, int k) {
    c->ops = k;
    for (int i = 0; i < CP_MAXN; ++i) {
        c->Ap64[i] = c->Apset[k][i];
        c->Mp[i] = c->Mpset[k][i];
        for (int j = 0; j < CP_MAXN; ++j) c->pair[i][j] = c->pairset[k][i][j];
    }
}

cp_status alloc_ops(cp_ctx* c, int k) {
    const int N = c->N, R = c->R;
    for (int i = 0; i < N; ++i) {
        CKST(dalloc(c, &c->Apset[k][i], (size_t)c->dims[i] * R));
        CKST(dalloc(c, &c->Mpset[k][i], (size_t)c->dims[i] * R));
        for (int j = i + 1; j < N; ++j)
            CKST(dalloc(c, &c->pairset[k][i][j], (size_t)c->dims[i] * c->dims[j] * R));
    }
    return CP_OK;
}

cp_status pp_alloc(cp_ctx* c) {
    if (c->pp_alloc) return CP_OK;
    const int N = c->N, R = c->R;
    CKST(alloc_ops(c, 0));
    use_ops(c, 0);
    for (int i = 0; i < N; ++i) {
        CKST(dalloc(c, &c->dA32[i], (size_t)c->dims[i] * R));
        CKST(dalloc(c, &c->dA64[i], (size_t)c->dims[i] * R));
    }
    CKST(dalloc(c, &c->Mt, (size_t)c->smax * R));
    c->pp_alloc = true;
    return CP_OK;
}

// second operator set, for probing (a rebuild then writes the idle set)
cp_status pp_alloc2(cp_ctx* c) {
    CKST(pp_alloc(c));
    if (c->ops2) return CP_OK;
    CKST(alloc_ops(c, 1));
    c->ops2 = true;
    return CP_OK;
}

// PP dimension tree (Fig. 1b).  1-based level-l nodes are (i, j, j+1, ..., j+N-l-1),
// i < j <= l+1 (Sec. II-D); level 2 nodes are first-level TTM results.  Parent
// rule: j <= l -> (i, j, ..., j+N-l); j = l+1, i < l -> (i, l, ..., N);
// j = l+1, i = l -> (1, l, ..., N).  Returns the contraction sequence from T to
// the 0-based pair (a, b).
std::vector<int> pp_pair_path(int N, int a, int b) {
    // walk up from the pair (level N-1) to level 2, recording kept-mode sets (1-based)
    std::vector<std::vector<int>> chain;
    int i = a + 1, j = b + 1;
    std::vector<int> node = {i, j};
    chain.push_back(node);
    for (int l = N - 1; l > 2; --l) {
        // node at level l is (i, j, j+1, ..., j+N-l-1)
        std::vector<int> parent;
        if (j <= l) {
            parent.push_back(i);
            for (int m = j; m <= j + N - l; ++m) parent.push_back(m);
        } else if (i < l) {
            parent.push_back(i);
            for (int m = l; m <= N; ++m) parent.push_back(m);
            j = l;
        } else {
            parent.push_back(1);
            for (int m = l; m <= N; ++m) parent.push_back(m);
            i = 1;
            j = l;
        }
        chain.push_back(parent);
    }
    // chain.back() is a level-2 node (N-1 modes); contractions from T downward
    std::vector<int> seq;
    std::vector<int> prev;
    for (int m = 1; m <= N; ++m) prev.push_back(m);
    for (size_t t = chain.size(); t-- > 0;) {
        const std::vector<int>& cur = chain[t];
        for (int m : prev)
            if (std::find(cur.begin(), cur.end(), m) == cur.end()) seq.push_back(m - 1);
        prev = cur;
    }
    return seq;
}

cp_status pp_init_impl(cp_ctx* c) {
    CKST(pp_alloc(c));
    if (c->ops2) use_ops(c, c->ops ^ 1);
    const int N = c->N, R = c->R;
    for (int i = 0; i < N; ++i) {
        CKCUDA(c, cudaMemcpyAsync(c->Ap64[i], c->A64[i], sizeof(double) * c->dims[i] * R, cudaMemcpyDeviceToDevice, c->st));
        CKCUDA(c, cudaMemsetAsync(c->dA32[i], 0, sizeof(float) * c->dims[i] * R, c->st));
        CKCUDA(c, cudaMemsetAsync(c->dA64[i], 0, sizeof(double) * c->dims[i] * R, c->st));
        CKCUDA(c, cudaMemsetAsync(c->dS[i], 0, sizeof(double) * R * R, c->st));
        if (c->dS2[i]) CKCUDA(c, cudaMemsetAsync(c->dS2[i], 0, sizeof(float2) * R * R, c->st));
    }
    // pairs ordered by their contraction sequence so shared ancestors stay cached
    struct PP { std::vector<int> seq; int a, b; };
    std::vector<PP> items;
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b) items.push_back({pp_pair_path(N, a, b), a, b});
    // the first-level node still cached from the last exact sweep is reused
    // (the amortized root of Sec. II-D): its pairs go first
    int cached = -1;
    {
        const Slot& r = c->slot[N - 1];
        if (r.valid && __builtin_popcount(r.contracted) == 1) {
            const int m = __builtin_ctz(r.contracted);
            if (r.ver[m] == c->ver[m]) cached = m;
        }
    }
    std::sort(items.begin(), items.end(), [cached](const PP& x, const PP& y) {
        const bool cx = x.seq[0] == cached, cy = y.seq[0] == cached;
        if (cx != cy) return cx;
        return x.seq < y.seq;
    });
    for (const PP& it : items) {
        const int d = (int)it.seq.size();  // N-2 contractions
        uint32_t mask = 0;
        for (int m : it.seq) mask |= 1u << m;
        if (d == 1) {
            if (it.seq[0] == cached)
                CKCUDA(c, cudaMemcpyAsync(c->pair[it.a][it.b], c->slot[N - 1].buf,
                                          sizeof(float) * c->dims[it.a] * c->dims[it.b] * R,
                                          cudaMemcpyDeviceToDevice, c->st));
            else
                CKST(launch_ttm(c, it.seq[0], c->pair[it.a][it.b]));
        } else {
            float* parent = nullptr;
            CKST(ensure_node(c, it.seq.data(), d - 1, &parent));
            CKST(launch_mttv(c, parent, mask & ~(1u << it.seq[d - 1]), it.seq[d - 1], c->pair[it.a][it.b]));
        }
    }
    // M_p(n) = M_p(n,i) x_i A_p(i)
    for (int n = 0; n < N; ++n) {
        const int i = (n == 0) ? 1 : 0;
        const int a = std::min(n, i), b = std::max(n, i);
        uint32_t mask = 0;
        for (int k = 0; k < N; ++k)
            if (k != a && k != b) mask |= 1u << k;
        CKST(launch_mttv(c, c->pair[a][b], mask, i, c->Mp[n]));
    }
    c->pp_valid = true;
    c->since_init = 0;
    c->stats.pp_init++;
    for (int i = 0; i < N; ++i) c->dA_rel[i] = 0.0;
    return CP_OK;
}

cp_status pp_mttkrp_impl(cp_ctx* c, int n, float* Mt) {
    std::vector<cpk::PPTerm> terms;
    for (int i = 0; i < c->N; ++i) {
        if (i == n) continue;
        cpk::PPTerm t;
        t.op = c->pair[std::min(n, i)][std::max(n, i)];
        t.dA = c->dA32[i];
        t.sy = (int)c->dims[i];
        t.trans = (i < n) ? 1 : 0;
        terms.push_back(t);
    }
    LAUNCH(c, cpk::pp_u(c->Mp[n], terms.data(), (int)terms.size(), Mt, (int)c->dims[n], c->R, c->st));
    double s = (double)c->dims[n], R = c->R, N = c->N;
    c->stats.pp_flops += 2.0 * (N * s * s * R + N * R * R + s * R * R);
    return CP_OK;
}

cp_status pp_sweep(cp_ctx* c, int k) {
    for (int n = 0; n < c->N; ++n) {
        CKST(launch_chol(c, n, true, scal_slot(c, k, n)));
        CKST(pp_mttkrp_impl(c, n, c->Mt));
        CKST(update_mode(c, n, c->Mt, true, scal_slot(c, k, n)));
    }
    c->stats.sweeps_pp++;
    return CP_OK;
}

cp_status regram(cp_ctx* c, int i, bool pp);

cp_status init_grams(cp_ctx* c) {
    for (int n = 0; n < c->N; ++n) {
        const int s = (int)c->dims[n];
        LAUNCH(c, cpk::factor_copies(c->A64[n], c->A32[n], uses_bf16(c) ? c->bhi[n] : nullptr,
                                     uses_bf16(c) ? c->blo[n] : nullptr, uses_tf32(c) ? c->bt32[n] : nullptr, s,
                                     c->R, c->Rpad, c->Kpad[n], c->st));
        CKST(regram(c, n, false));
    }
    return CP_OK;
}

// ||T - [[A]]||_F / ||T||_F (Eq. residual-def), one streaming pass over T
cp_status direct_resid(cp_ctx* c, double* r) {
    cpk::ResidArgs a;
    memset(&a, 0, sizeof(a));
    a.T = c->T;
    a.N = c->N;
    a.R = c->R;
    for (int i = 0; i < c->N; ++i) {
        a.A32[i] = c->A32[i];
        a.dims[i] = c->dims[i];
    }
    c->stats.launches += 2;
    // tensor cores where the shape allows it, else the FP32 SIMT kernel
    int nb = cpk::resid_tc_partials(a, c->red_part, 4096, c->num_sms, c->dev_err, c->wait_limit, c->st);
    if (nb < 0) CKCUDA(c, cudaGetLastError());
    if (nb == 0) nb = cpk::resid_direct_partials(a, c->red_part, 4096, c->st);
    CKCUDA(c, cudaGetLastError());
    CKCUDA(c, cpk::sum_partials(c->red_part, nb, c->d_red_out, c->st));
    double s2 = 0.0;
    CKCUDA(c, cudaMemcpyAsync(&s2, c->d_red_out, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CKCUDA(c, cudaStreamSynchronize(c->st));
    CKST(check_dev_err(c));
    // a NaN must not be clamped away with the rounding-level negatives
    if (!std::isfinite(s2)) return fail(c, CP_ENUMERIC, "non-finite residual");
    *r = sqrt(s2 > 0 ? s2 : 0.0) / sqrt(c->normT2);
    if (!isfinite(*r)) return fail(c, CP_ENUMERIC, "non-finite residual");
    return CP_OK;
}

// S(i) (and dS(i) when `pp`) from the factors now in A64 (and dA64).  For R <= 128
// through the float pairs the row solve also writes, so that a Gram formed here
// equals the one an update forms from the same factor.
cp_status regram(cp_ctx* c, int i, bool pp) {
    const int s = (int)c->dims[i];
    if (c->A2[i]) {
        LAUNCH(c, cpk::split_pairs(c->A64[i], c->A2[i], (int64_t)s * c->R, c->st));
        if (pp) LAUNCH(c, cpk::split_pairs(c->dA64[i], c->dA2[i], (int64_t)s * c->R, c->st));
        LAUNCH(c, cpk::gram_df(c->A2[i], pp ? c->dA2[i] : nullptr, s, c->R, nullptr, c->S[i], c->dS[i], c->S2[i],
                               c->dS2[i], nullptr, c->st));
    } else {
        LAUNCH(c, cpk::gram(c->A64[i], pp ? c->dA64[i] : nullptr, s, c->R, nullptr, c->S[i], c->dS[i], nullptr,
                            c->st));
    }
    return CP_OK;
}

// Snapshot of the iteration state at a sweep boundary: factors (device copies)
// and the host-side schedule state.  Intermediates are not copied: their cache
// keys are factor versions, restored with the factors.
cp_status snap_take(cp_ctx* c, cp_ctx::Snap& sn) {
    for (int i = 0; i < c->N; ++i) {
        if (!sn.A64[i]) CKST(dalloc(c, &sn.A64[i], (size_t)c->dims[i] * c->R));
        CKCUDA(c, cudaMemcpyAsync(sn.A64[i], c->A64[i], sizeof(double) * c->dims[i] * c->R,
                                  cudaMemcpyDeviceToDevice, c->st));
        sn.ver[i] = c->ver[i];
        sn.dA_rel[i] = c->dA_rel[i];
    }
    sn.pp_valid = c->pp_valid;
    sn.ops = c->ops;
    sn.since_init = c->since_init;
    sn.sweeps_done = c->sweeps_done;
    sn.t_msdt = c->t_msdt;
    sn.have_last = c->have_last;
    sn.last_resid = c->last_resid;
    sn.trace_len = c->trace.size();
    sn.have = true;
    return CP_OK;
}

// Back to a snapshot.  keep_ops: the snapshot's operator set is still intact
// (probing); otherwise the operators are dropped and the next sweep is regular.
// truncate: forget the trace records written since the snapshot.
cp_status snap_restore(cp_ctx* c, const cp_ctx::Snap& sn, bool keep_ops, bool truncate) {
    if (!sn.have) return fail(c, CP_ESTATE, "no snapshot to restore");
    const bool pp = keep_ops && sn.pp_valid;
    if (pp) use_ops(c, sn.ops);
    c->pp_valid = pp;
    for (int i = 0; i < c->N; ++i) {
        const int s = (int)c->dims[i];
        CKCUDA(c, cudaMemcpyAsync(c->A64[i], sn.A64[i], sizeof(double) * s * c->R, cudaMemcpyDeviceToDevice,
                                  c->st));
        LAUNCH(c, cpk::factor_copies(c->A64[i], c->A32[i], uses_bf16(c) ? c->bhi[i] : nullptr,
                                     uses_bf16(c) ? c->blo[i] : nullptr, uses_tf32(c) ? c->bt32[i] : nullptr, s,
                                     c->R, c->Rpad, c->Kpad[i], c->st));
        if (pp)
            LAUNCH(c, cpk::pp_delta(c->A64[i], c->Ap64[i], c->dA32[i], c->dA64[i], (int64_t)s * c->R, c->st));
        CKST(regram(c, i, pp));
        c->ver[i] = sn.ver[i];
        c->dA_rel[i] = (sn.pp_valid && !pp) ? 1.0 : sn.dA_rel[i];
    }
    c->since_init = sn.since_init;
    c->sweeps_done = sn.sweeps_done;
    c->t_msdt = sn.t_msdt;
    c->have_last = sn.have_last;
    c->last_resid = sn.last_resid;
    if (truncate && c->trace.size() > sn.trace_len) c->trace.resize(sn.trace_len);
    c->chol_pending = false;
    return CP_OK;
}

// Alg. 2's inputs to the regime test after a sweep: dA = A - A_p inside PP,
// the sweep's own change after a regular sweep.
void note_sweep(cp_ctx* c, int kind) {
    const std::vector<double>& h = c->last_hist;
    for (int i = 0; i < c->N; ++i) {
        const double* sc = &h[(size_t)i * CP_NSCAL];
        const double a = sqrt(sc[SCAL_A2]);
        const double d = (kind == 2) ? sqrt(sc[SCAL_DAP2]) : sqrt(sc[SCAL_STEP2]);
        c->dA_rel[i] = a > 0 ? d / a : 1.0;
    }
    if (kind == 2) c->since_init++;
}

// log10 of x clamped to [1e-12, 1], mapped to [-1, 1]
float logfeat(double x) {
    const double l = log10(std::min(1.0, std::max(x, 1e-12)));
    return (float)(l / 6.0 + 1.0);
}

// The policy's 8 inputs (see cp_policy_features in cpals.h).  rebuilt: as if
// the operators were built now (A_p = A).
void features(const cp_ctx* c, bool rebuilt, float f[8]) {
    const size_t n = c->trace.size();
    const cp_trace_rec* last = n ? &c->trace[n - 1] : nullptr;
    const double r1 = last ? last->resid : 1.0;
    const double r0 = n > 1 ? c->trace[n - 2].resid : 1.0;
    const bool in_pp = last && last->kind == 2;
    double dap = 0.0;
    for (int i = 0; i < c->N; ++i) dap = std::max(dap, c->dA_rel[i]);
    f[0] = (float)std::min(3.0, c->sweeps_done / 100.0);
    f[1] = logfeat(last ? last->max_rel_step : 1.0);
    f[2] = (rebuilt || !c->pp_valid) ? -1.f : logfeat(dap);
    f[3] = logfeat(n ? fabs(r1 - r0) / std::max(r1, 1e-300) : 1.0);
    f[4] = logfeat(r1);
    f[5] = rebuilt ? 0.f : (c->pp_valid ? (float)std::min(3.0, c->since_init / 10.0) : 3.f);
    f[6] = in_pp ? 1.f : 0.f;
    f[7] = (!rebuilt && in_pp) ? logfeat(last->v_share) : -1.f;
}

// network scores of the two choices: [0] current operators, [1] rebuilt ones
cp_status policy_scores(cp_ctx* c, cp_policy* p, float sc[2], bool* valid) {
    if (!c->pol_io) CKST(dalloc(c, &c->pol_io, 32));
    float f[16];
    features(c, false, f);
    features(c, true, f + 8);
    CKCUDA(c, cudaMemcpyAsync(c->pol_io, f, sizeof(f), cudaMemcpyHostToDevice, c->st));
    LAUNCH(c, cpk::mlp_forward(p->theta, c->pol_io, 2, c->pol_io + 16, c->st));
    CKCUDA(c, cudaMemcpyAsync(sc, c->pol_io + 16, 2 * sizeof(float), cudaMemcpyDeviceToHost, c->st));
    CKCUDA(c, cudaStreamSynchronize(c->st));
    *valid = true;
    for (int k = 0; k < 2; ++k)
        if (!(sc[k] >= 0.f && sc[k] <= 1.f)) *valid = false;  // NaN or garbage
    return CP_OK;
}

enum { CH_EXACT = 0, CH_CUR = 1, CH_NEW = 2 };

// bytes an approximated sweep reads: for every mode n the N-1 pair operators
// M_p(n,i) (s_n s_i R) plus M_p(n) and writes M~(n) (FP32)
double pp_sweep_bytes(const cp_ctx* c) {
    double b = 0.0;
    for (int n = 0; n < c->N; ++n) {
        for (int i = 0; i < c->N; ++i)
            if (i != n) b += (double)c->dims[n] * c->dims[i] * c->R;
        b += 2.0 * c->dims[n] * c->R;
    }
    return 4.0 * b;
}

// the policy judge's rollback point no longer describes a predecessor state
void drop_judge(cp_ctx* c) {
    c->snap[1].have = false;
    c->snap_current = false;
    c->rollbacks_in_row = 0;
    c->since_judge = 0;
    c->fallback_left = 0;
}

// One PP-mode sweep of the given choice, timed from events[0] (recorded by the
// caller) to events[1]; appends its trace record.
cp_status run_choice(cp_ctx* c, int choice) {
    int init = 0, kind;
    if (choice == CH_NEW) {
        CKST(pp_init_impl(c));
        init = 1;
    }
    if (choice != CH_EXACT && c->pp_valid) {
        CKST(pp_sweep(c, 0));
        kind = 2;
    } else {
        c->pp_valid = false;
        const double b0 = c->stats.ttm_bytes + c->stats.mttv_bytes;
        CKST(exact_sweep(c, true, 0));
        c->sweep_mttkrp_bytes = c->stats.ttm_bytes + c->stats.mttv_bytes - b0;
        kind = 3;
    }
    CKCUDA(c, cudaEventRecord(c->events[1], c->st));
    CKST(harvest(c, 1, &kind, &init, 0));
    note_sweep(c, kind);
    return CP_OK;
}

// ||T||_F^2 (one streaming pass), read back to the host
cp_status tensor_norm(cp_ctx* c) {
    c->stats.launches += 2;
    int nb = cpk::norm2_partials(c->T, c->numel, c->red_part, 4096, c->st);
    CKCUDA(c, cudaGetLastError());
    CKCUDA(c, cpk::sum_partials(c->red_part, nb, c->d_red_out, c->st));
    CKCUDA(c, cudaMemcpyAsync(&c->normT2, c->d_red_out, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CKCUDA(c, cudaStreamSynchronize(c->st));
    return CP_OK;
}

// f16x3: the power of two 2^eT that brings max |T| into [2^14, 2^15) (0 for an
// all-zero or non-finite tensor), and the plans' copy of it
cp_status tensor_exponent(cp_ctx* c) {
    float* part = reinterpret_cast<float*>(c->red_part);  // 4096 doubles hold the 4096 block maxima
    float* out = reinterpret_cast<float*>(c->d_red_out);
    LAUNCH(c, cpk::absmax(c->T, c->numel, part, 4096, out, c->st));
    c->stats.launches++;
    float m = 0.f;
    CKCUDA(c, cudaMemcpyAsync(&m, out, sizeof(float), cudaMemcpyDeviceToHost, c->st));
    CKCUDA(c, cudaStreamSynchronize(c->st));
    int e = 0;
    if (m > 0.f && std::isfinite(m)) e = std::min(127, std::max(-126, 14 - std::ilogb(m)));
    c->eT = e;
    for (int i = 0; i < CP_MAXN; ++i) {
        cpk::ttm_tc_set_tscale(c->tc_plan[i], ldexpf(1.f, e));
        cpk::ttm_tc_set_tscale(c->kr_plan[i], ldexpf(1.f, e));
        c->f16_ver[i] = -1;  // column scales include 2^-eT
    }
    return CP_OK;
}

void free_all(cp_ctx* c) {
    auto F = [](void* p) { if (p) cudaFree(p); };
    F(c->T_owned);
    for (int i = 0; i < CP_MAXN; ++i) {
        F(c->A64[i]); F(c->A32[i]); F(c->bhi[i]); F(c->blo[i]); F(c->bt32[i]);
        F(c->S[i]); F(c->dS[i]); F(c->dA32[i]); F(c->dA64[i]);
        for (int k = 0; k < 2; ++k) {
            F(c->Apset[k][i]); F(c->Mpset[k][i]);
            for (int j = 0; j < CP_MAXN; ++j) F(c->pairset[k][i][j]);
            F(c->snap[k].A64[i]);
        }
    }
    F(c->pol_io);
    for (int k = 0; k <= CP_MAXN; ++k) F(c->slot[k].buf);
    for (int k = 0; k <= CP_MAXN; ++k) F(c->alt[k].buf);
    if (c->ahead) { cudaStreamSynchronize(c->ahead); cudaStreamDestroy(c->ahead); c->ahead = nullptr; }
    for (cudaEvent_t* e : {&c->ev_x, &c->ev_ahead})
        if (*e) { cudaEventDestroy(*e); *e = nullptr; }
    for (int i = 0; i < CP_MAXN; ++i) {
        cpk::ttm_tc_plan_free(c->tc_plan[i]);
        c->tc_plan[i] = nullptr;
        cpk::ttm_tc_plan_free(c->kr_plan[i]);
        c->kr_plan[i] = nullptr;
    }
    F(c->kr_hi); F(c->kr_lo); F(c->kr_scale); F(c->kr_colinv); F(c->splitk_ws); F(c->child_ws);
    for (int i = 0; i < CP_MAXN; ++i) {
        F(c->colinv[i]);
        F(c->Tp_hi[i]);
        F(c->Tp_lo[i]);
        F(c->A2[i]);
        F(c->dA2[i]);
        F(c->S2[i]);
        F(c->dS2[i]);
    }
    F(c->d_S2list); F(c->d_dS2list);
    F(c->Ginv); F(c->G32); F(c->G2); F(c->W2); F(c->schur_ws); F(c->d_mode);
    if (c->side) { cudaStreamSynchronize(c->side); cudaStreamDestroy(c->side); c->side = nullptr; }
    if (c->ev_ready) { cudaEventDestroy(c->ev_ready); c->ev_ready = nullptr; }
    if (c->ev_chol) { cudaEventDestroy(c->ev_chol); c->ev_chol = nullptr; }
    F(c->Mt); F(c->d_Slist); F(c->d_dSlist); F(c->Gamma); F(c->L); F(c->invd); F(c->W);
    if (c->aux) { cudaStreamSynchronize(c->aux); cudaStreamDestroy(c->aux); c->aux = nullptr; }
    F(c->tile_gs); F(c->scal_part);
    for (cudaEvent_t* e : {&c->ev_g})
        if (*e) { cudaEventDestroy(*e); *e = nullptr; }
    for (int i = 0; i < CP_MAXN; ++i)
        if (c->ev_scal[i]) { cudaEventDestroy(c->ev_scal[i]); c->ev_scal[i] = nullptr; } F(c->scal_hist); F(c->red_part); F(c->d_red_out); F(c->dev_err);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    c->events.clear();
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void cp_config_default(cp_config* cfg) {
    if (!cfg) return;
    cfg->prec = CP_F16X3;
    cfg->pp_eps = 0.1;
    cfg->delta = 0.0;
    cfg->max_sweeps = 0;
    cfg->judge_every = 5;
    cfg->policy_gate = 1;
    cfg->seed = 20101205ull;
}

// tensor-core TTM plan of every mode's first-level contraction T x_m A(m)
// (NULL where the shape needs the SIMT kernel)
static void make_mode_plans(cp_ctx* c) {
    const bool bf = uses_bf16(c), hf = c->cfg.prec == CP_F16X3;
    const int kind = bf ? 0 : (hf ? 2 : 1);
    const float tscale = ldexpf(1.f, c->eT);
    for (int m = 0; m < c->N; ++m) {
        cpk::ttm_tc_plan_free(c->tc_plan[m]);
        int64_t P, Q;
        contract_dims(c, 0u, m, &P, &Q);
        const void* hi = (bf || hf) ? (const void*)c->bhi[m] : (const void*)c->bt32[m];
        const void* lo = (bf || hf) ? (const void*)c->blo[m]
                                    : (const void*)(c->bt32[m] + (size_t)c->Rpad * c->Kpad[m]);
        c->tc_plan[m] = cpk::ttm_tc_plan(c->T, P, (int)c->dims[m], Q, c->R, kind, hi, lo, c->Rpad, c->Kpad[m],
                                         tscale, c->colinv[m], c->Tp_hi[m], c->Tp_lo[m], c->presplit == 2);
    }
}

// T's stored 16-bit parts (one copy per mode whose TTM takes R > 128 columns):
// allocated where memory allows (a mode without them converts T in its TTM),
// refilled whenever T or its f16x3 scale changes
static bool presplit_wanted(const cp_ctx* c, int m) {
    if (!(c->presplit && c->R > 128 && (c->cfg.prec == CP_F16X3 || c->cfg.prec == CP_BF16X3) &&
          c->dims[m] % 8 == 0 && c->numel <= ((int64_t)1 << 31)))
        return false;
    // only for a mode whose first-level TTM runs on the tensor cores at all
    int64_t P, Q;
    contract_dims(c, 0u, m, &P, &Q);
    return cpk::ttm_tc_supported(P, (int)c->dims[m], Q, c->R);
}

static void free_presplit(cp_ctx* c) {
    for (int m = 0; m < CP_MAXN; ++m) {
        if (c->Tp_hi[m]) cudaFree(c->Tp_hi[m]);
        if (c->Tp_lo[m]) cudaFree(c->Tp_lo[m]);
        c->Tp_hi[m] = c->Tp_lo[m] = nullptr;
    }
}

static cp_status fill_presplit(cp_ctx* c) {
    const int kind = c->cfg.prec == CP_F16X3 ? 2 : 0;
    const float tscale = ldexpf(1.f, c->eT);
    for (int m = 0; m < c->N; ++m) {
        if (!c->Tp_hi[m]) continue;
        int64_t P, Q;
        contract_dims(c, 0u, m, &P, &Q);
        LAUNCH(c, cpk::ttm_presplit(c->T, P, (int)c->dims[m], Q, kind, tscale, c->Tp_hi[m], c->Tp_lo[m],
                                    c->num_sms, c->st));
        c->stats.launches++;
    }
    return CP_OK;
}

static cp_status alloc_presplit(cp_ctx* c) {
    for (int m = 0; m < c->N; ++m) {
        if (!presplit_wanted(c, m) || c->Tp_hi[m]) continue;
        const size_t bytes = sizeof(uint16_t) * (size_t)c->numel;
        void* hi = nullptr;
        void* lo = nullptr;
        if (cudaMalloc(&hi, bytes) == cudaSuccess && cudaMalloc(&lo, bytes) == cudaSuccess) {
            c->Tp_hi[m] = static_cast<uint16_t*>(hi);
            c->Tp_lo[m] = static_cast<uint16_t*>(lo);
        } else {
            // out of memory (not a sticky error): this mode splits T in its TTM
            (void)cudaGetLastError();
            if (hi) cudaFree(hi);
        }
    }
    return fill_presplit(c);
}

cp_status cp_init(cp_ctx** out, int N, const int64_t* dims, int R, const void* T_dev, int dtype,
                  const double* A0_host, const cp_config* cfg, void* stream) {
    if (!out) return CP_EINVAL;
    *out = nullptr;
    if (N < 3 || N > CP_MAXN || !dims || R < 1 || R > CP_MAXR || !T_dev || dtype < 0 || dtype > 2)
        return CP_EINVAL;
    int64_t numel = 1;
    for (int i = 0; i < N; ++i) {
        if (dims[i] < 1 || dims[i] > (1 << 30)) return CP_EINVAL;
        if (numel > ((int64_t)1 << 40) / dims[i]) return CP_EINVAL;
        numel *= dims[i];
    }
    cp_ctx* c = new cp_ctx();
    c->N = N;
    c->R = R;
    c->Rpad = (R + 15) / 16 * 16;
    c->numel = numel;
    c->st = (cudaStream_t)stream;
    if (cfg) c->cfg = *cfg; else cp_config_default(&c->cfg);
    if (c->cfg.prec < CP_FP32_SIMT || c->cfg.prec > CP_F16X3) { delete c; return CP_EINVAL; }
    memset(&c->stats, 0, sizeof(c->stats));
    for (int i = 0; i < N; ++i) {
        c->dims[i] = dims[i];
        c->Kpad[i] = (int)((dims[i] + 63) / 64 * 64);
        c->smax = std::max<int>(c->smax, (int)dims[i]);
        c->dA_rel[i] = 1.0;  // Alg. 2 starts from dA = A
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);

#define TRY(expr)                       \
    do {                                \
        cp_status s__ = (expr);         \
        if (s__ != CP_OK) {             \
            free_all(c);                \
            delete c;                   \
            return s__;                 \
        }                               \
    } while (0)
#define TRYC(expr)                                  \
    do {                                            \
        if ((expr) != cudaSuccess) {                \
            cudaGetLastError();                     \
            free_all(c);                            \
            delete c;                               \
            return CP_ECUDA;                        \
        }                                           \
    } while (0)

    if (dtype == 1) {
        TRY(dalloc(c, &c->T_owned, (size_t)numel));
        TRYC(cpk::f64_to_f32((const double*)T_dev, c->T_owned, numel, c->st));
        c->T = c->T_owned;
    } else if (dtype == 2) {
        TRY(dalloc(c, &c->T_owned, (size_t)numel));
        TRYC(cudaMemcpyAsync(c->T_owned, T_dev, sizeof(float) * numel, cudaMemcpyHostToDevice, c->st));
        c->T = c->T_owned;
    } else {
        c->T = (const float*)T_dev;
    }
    const int RR = R * R;
    for (int i = 0; i < N; ++i) {
        const size_t sR = (size_t)dims[i] * R;
        TRY(dalloc(c, &c->A64[i], sR));
        TRY(dalloc(c, &c->A32[i], sR));
        if (R <= 128) {
            TRY(dalloc(c, &c->A2[i], sR));
            TRY(dalloc(c, &c->dA2[i], sR));
            TRY(dalloc(c, &c->S2[i], RR));
            TRY(dalloc(c, &c->dS2[i], RR));
            TRYC(cudaMemsetAsync(c->dS2[i], 0, sizeof(float2) * RR, c->st));
        }
        TRY(dalloc(c, &c->S[i], RR));
        TRY(dalloc(c, &c->dS[i], RR));
        TRYC(cudaMemsetAsync(c->dS[i], 0, sizeof(double) * RR, c->st));
        const size_t op = (size_t)c->Rpad * c->Kpad[i];
        TRY(dalloc(c, &c->bhi[i], op));
        TRY(dalloc(c, &c->blo[i], op));
        TRY(dalloc(c, &c->bt32[i], 2 * op));
        TRYC(cudaMemsetAsync(c->bhi[i], 0, op * sizeof(uint16_t), c->st));
        TRYC(cudaMemsetAsync(c->blo[i], 0, op * sizeof(uint16_t), c->st));
        TRYC(cudaMemsetAsync(c->bt32[i], 0, 2 * op * sizeof(float), c->st));
        TRY(dalloc(c, &c->colinv[i], (size_t)c->Rpad));
        TRYC(cudaMemsetAsync(c->colinv[i], 0, c->Rpad * sizeof(float), c->st));
    }
    // one slot per number of kept modes k = 1..N-1: capacity = largest k-mode product x R
    std::vector<int64_t> sd(dims, dims + N);
    std::sort(sd.begin(), sd.end(), std::greater<int64_t>());
    for (int k = 1; k < N; ++k) {
        int64_t cap = R;
        for (int i = 0; i < k; ++i) cap *= sd[i];
        c->slot[k].cap = (size_t)cap;           // allocated on first use
        if (N >= 4 && k == N - 2) c->alt[k].cap = (size_t)cap;  // look-ahead slot of the multi-sweep tree
    }
    TRYC(cudaStreamCreateWithFlags(&c->ahead, cudaStreamNonBlocking));
    TRYC(cudaEventCreateWithFlags(&c->ev_x, cudaEventDisableTiming));
    TRYC(cudaEventCreateWithFlags(&c->ev_ahead, cudaEventDisableTiming));
    TRY(dalloc(c, &c->d_Slist, N));
    TRY(dalloc(c, &c->d_dSlist, N));
    TRYC(cudaMemcpyAsync(c->d_Slist, c->S, sizeof(double*) * N, cudaMemcpyHostToDevice, c->st));
    TRYC(cudaMemcpyAsync(c->d_dSlist, c->dS, sizeof(double*) * N, cudaMemcpyHostToDevice, c->st));
    if (R <= 128) {
        TRY(dalloc(c, &c->d_S2list, N));
        TRY(dalloc(c, &c->d_dS2list, N));
        TRYC(cudaMemcpyAsync(c->d_S2list, c->S2, sizeof(float2*) * N, cudaMemcpyHostToDevice, c->st));
        TRYC(cudaMemcpyAsync(c->d_dS2list, c->dS2, sizeof(float2*) * N, cudaMemcpyHostToDevice, c->st));
    }
    TRY(dalloc(c, &c->Gamma, RR + 2));
    TRY(dalloc(c, &c->Ginv, RR + 4));
    TRY(dalloc(c, &c->G32, RR + 4));
    TRY(dalloc(c, &c->G2, 2 * RR + 4));
    TRY(dalloc(c, &c->W2, 2 * RR + 4));
    if (cpk::schur_ws_floats(R)) TRY(dalloc(c, &c->schur_ws, cpk::schur_ws_floats(R)));
    TRYC(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    TRYC(cudaEventCreateWithFlags(&c->ev_ready, cudaEventDisableTiming));
    TRYC(cudaEventCreateWithFlags(&c->ev_chol, cudaEventDisableTiming));
    TRY(dalloc(c, &c->d_mode, 1));
    TRY(dalloc(c, &c->W, RR));
    TRY(dalloc(c, &c->L, 2 * (size_t)RR));
    TRY(dalloc(c, &c->invd, R));
    c->ntiles = cpk::gram_tiles(R);
    TRY(dalloc(c, &c->tile_gs, (size_t)N * c->ntiles));
    TRY(dalloc(c, &c->scal_part, (size_t)N * c->smax * CP_NSCAL));
    TRYC(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
    TRYC(cudaEventCreateWithFlags(&c->ev_g, cudaEventDisableTiming));
    for (int i = 0; i < N; ++i) TRYC(cudaEventCreateWithFlags(&c->ev_scal[i], cudaEventDisableTiming));
    TRY(dalloc(c, &c->red_part, 4096));
    TRY(dalloc(c, &c->d_red_out, 16));
    TRY(dalloc(c, &c->dev_err, 1));
    TRYC(cudaMemsetAsync(c->dev_err, 0, sizeof(unsigned), c->st));
    TRY(grow_hist(c, 8));

    // initial factors (Alg. 1)
    std::vector<double> h;
    for (int i = 0; i < N; ++i) {
        const size_t sR = (size_t)dims[i] * R;
        h.resize(sR);
        if (A0_host) {
            size_t off = 0;
            for (int k = 0; k < i; ++k) off += (size_t)dims[k] * R;
            memcpy(h.data(), A0_host + off, sR * sizeof(double));
        } else {
            philox_uniform(c->cfg.seed, (uint32_t)i, sR, h.data());
        }
        TRYC(cudaMemcpyAsync(c->A64[i], h.data(), sR * sizeof(double), cudaMemcpyHostToDevice, c->st));
        TRYC(cudaStreamSynchronize(c->st));
    }
    TRY(init_grams(c));
    if (c->cfg.prec == CP_F16X3) TRY(tensor_exponent(c));
    // tensor-core TTM plans (TMA descriptors of T and of each factor operand)
    if (c->cfg.prec != CP_FP32_SIMT) {
        const bool bf = uses_bf16(c), hf = c->cfg.prec == CP_F16X3;
        const int kind = bf ? 0 : (hf ? 2 : 1);
        const float tscale = ldexpf(1.f, c->eT);
        TRY(alloc_presplit(c));
        make_mode_plans(c);
        // fused two-mode contractions of adjacent pairs (standard tree, N >= 3)
        size_t kr_elems = 0;
        for (int a = 0; a + 1 < N; ++a) {
            const int64_t K = dims[a] * dims[a + 1];
            if (K > (1 << 30)) continue;
            c->kr_Kpad[a] = (int)((K + 63) / 64 * 64);
            kr_elems = std::max(kr_elems, (size_t)c->Rpad * c->kr_Kpad[a]);
        }
        const size_t esz = kind == 1 ? 4 : 2;
        if (kr_elems) {
            TRY(dalloc(c, (uint8_t**)&c->kr_hi, kr_elems * esz));
            TRY(dalloc(c, (uint8_t**)&c->kr_lo, kr_elems * esz));
            if (hf) {
                TRY(dalloc(c, &c->kr_scale, (size_t)c->Rpad));
                TRY(dalloc(c, &c->kr_colinv, (size_t)c->Rpad));
            }
            for (int a = 0; a + 1 < N; ++a) {
                if (!c->kr_Kpad[a]) continue;
                int64_t P = 1, Q = 1;
                for (int k = 0; k < a; ++k) P *= dims[k];
                for (int k = a + 2; k < N; ++k) Q *= dims[k];
                c->kr_plan[a] = cpk::ttm_tc_plan(c->T, P, (int)(dims[a] * dims[a + 1]), Q, R, kind, c->kr_hi,
                                                 c->kr_lo, c->Rpad, c->kr_Kpad[a], tscale, c->kr_colinv);
                cpk::ttm_tc_set_depth_bound(c->kr_plan[a], true);
                // a contraction so long that even 64 K-slices leave deep accumulators
                // (K = s_a s_b beyond about 65536 per hi*hi accumulator) is not fused:
                // the tree then forms the level-1 node and contracts it by a multi-TTV
                if (c->kr_plan[a] && cpk::ttm_tc_depth_slices(c->kr_plan[a]) > 64) {
                    cpk::ttm_tc_plan_free(c->kr_plan[a]);
                    c->kr_plan[a] = nullptr;
                }
            }
        }
        // split-K workspace for contractions with few row tiles
        size_t ws = 0;
        auto need = [&](const cpk::TcPlan* p) {
            const int nsk = p ? cpk::ttm_tc_splitk(p, c->num_sms) : 1;
            if (nsk > 1) ws = std::max(ws, (size_t)nsk * (size_t)cpk::ttm_tc_rows(p) * R);
        };
        for (int m = 0; m < N; ++m) need(c->tc_plan[m]);
        for (int a = 0; a + 1 < N; ++a) need(c->kr_plan[a]);
        if (ws) TRY(dalloc(c, &c->splitk_ws, ws));
        // first-child pieces of the multi-sweep roots T x_0 and T x_{N-1}
        if (N >= 3) {
            size_t cw = 0;
            const int roots[2][2] = {{0, N - 1}, {N - 1, N - 2}};
            for (const auto& rc : roots)
                if (c->tc_plan[rc[0]] && cpk::ttm_tc_child_ok(c->tc_plan[rc[0]], (int)dims[rc[1]]))
                    cw = std::max(cw, (size_t)cpk::ttm_tc_child_ws_floats(c->tc_plan[rc[0]], (int)dims[rc[1]]));
            if (cw) TRY(dalloc(c, &c->child_ws, cw));
            c->child_ws_cap = cw;
        }
    }
    TRY(tensor_norm(c));
#undef TRY
#undef TRYC
    *out = c;
    return CP_OK;
}

void cp_free(cp_ctx* c) {
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    free_all(c);
    delete c;
}

const char* cp_last_error(const cp_ctx* c) { return c ? c->err.c_str() : "null context"; }

cp_status cp_mttkrp(cp_ctx* c, int mode, float* M_dev) {
    CKST(entry_check(c));
    if (mode < 0 || mode >= c->N || !M_dev) return CP_EINVAL;
    float* M = nullptr;
    bool fuse2 = false;
    std::vector<int> path = dt_path(c->N, mode, &fuse2);
    fuse2 = fuse2 && c->fuse_dt;
    CKST(mttkrp_leaf(c, path, &M, fuse2));
    CKCUDA(c, cudaMemcpyAsync(M_dev, M, sizeof(float) * c->dims[mode] * c->R, cudaMemcpyDeviceToDevice, c->st));
    return CP_OK;
}

cp_status cp_ttm(cp_ctx* c, int mode, float* X_dev) {
    CKST(entry_check(c));
    if (mode < 0 || mode >= c->N || !X_dev) return CP_EINVAL;
    return launch_ttm(c, mode, X_dev);
}

cp_status cp_load_tensor(cp_ctx* c, const float* T, int on_host) {
    CKST(entry_check(c));
    if (T && !c->T_owned) return fail(c, CP_ESTATE, "cp_load_tensor: the context borrows its tensor");
    if (on_host != 0 && on_host != 1) return CP_EINVAL;
    CKST(ahead_join(c));
    if (T)
        CKCUDA(c, cudaMemcpyAsync(c->T_owned, T, sizeof(float) * c->numel,
                                  on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->st));
    // every intermediate was contracted from the old tensor
    for (int k = 0; k <= CP_MAXN; ++k) {
        c->slot[k].valid = false;
        c->alt[k].valid = false;
    }
    c->pp_valid = false;
    drop_judge(c);
    c->have_last = false;
    CKST(tensor_norm(c));
    if (c->cfg.prec == CP_F16X3) CKST(tensor_exponent(c));
    CKST(fill_presplit(c));
    return CP_OK;
}

static cp_status sweeps_exact(cp_ctx* c, int nsweeps, bool msdt) {
    CKST(entry_check(c));
    if (nsweeps < 0) return CP_EINVAL;
    if (nsweeps == 0) return CP_OK;
    CKST(grow_hist(c, nsweeps));
    CKST(ensure_events(c, (size_t)nsweeps + 1));
    c->pp_valid = false;
    drop_judge(c);
    std::vector<int> kinds(nsweeps, msdt ? 1 : 0);
    CKCUDA(c, cudaEventRecord(c->events[0], c->st));
    for (int k = 0; k < nsweeps; ++k) {
        CKST(exact_sweep(c, msdt, k, msdt && k + 1 < nsweeps));
        CKCUDA(c, cudaEventRecord(c->events[k + 1], c->st));
    }
    CKST(harvest(c, nsweeps, kinds.data(), nullptr, 0));
    // regular sweeps: dA(i) = this sweep's change (Alg. 2, after a regular sweep)
    return CP_OK;
}

cp_status cp_set_option(cp_ctx* c, int option, int value) {
    CKST(entry_check(c));
    switch (option) {
        case CP_OPT_FUSE_DT:
            if (value != 0 && value != 1) return CP_EINVAL;
            c->fuse_dt = value != 0;
            return CP_OK;
        case CP_OPT_LOOKAHEAD:
            if (value < 0 || value > 8) return CP_EINVAL;
            c->lookahead = value != 0;
            if (value) c->ahead_blocks_per_sm = value;
            return CP_OK;
        case CP_OPT_FUSE_CHILD:
            if (value != 0 && value != 1) return CP_EINVAL;
            c->fuse_child = value != 0;
            return CP_OK;
        case CP_OPT_WAIT_LIMIT:
            if (value < 0) return CP_EINVAL;
            c->wait_limit = value;
            return CP_OK;
        case CP_OPT_SOLVE_FP64:
            if (value != 0 && value != 1) return CP_EINVAL;
            c->solve_fp64 = value != 0;
            return CP_OK;
        case CP_OPT_TTM_PRESPLIT:
            if (value < 0 || value > 2) return CP_EINVAL;
            if (c->presplit == value) return CP_OK;
            CKST(ahead_join(c));
            CKCUDA(c, cudaStreamSynchronize(c->st));
            c->presplit = value;
            if (c->presplit) CKST(alloc_presplit(c));
            else free_presplit(c);
            if (c->cfg.prec != CP_FP32_SIMT) make_mode_plans(c);
            return CP_OK;
        case CP_OPT_MSDT_LEVELS:
            if (value < 1 || value > std::max(1, c->N - 2)) return CP_EINVAL;
            CKST(ahead_join(c));
            c->msdt_levels = value;
            return CP_OK;
        default: return CP_EINVAL;
    }
}

cp_status cp_sweep_dt(cp_ctx* c, int nsweeps) { return sweeps_exact(c, nsweeps, false); }
cp_status cp_sweep_msdt(cp_ctx* c, int nsweeps) { return sweeps_exact(c, nsweeps, true); }

cp_status cp_pp_init(cp_ctx* c) {
    CKST(entry_check(c));
    drop_judge(c);
    return pp_init_impl(c);
}

cp_status cp_pp_mttkrp(cp_ctx* c, int mode, float* M_dev) {
    CKST(entry_check(c));
    if (mode < 0 || mode >= c->N || !M_dev) return CP_EINVAL;
    if (!c->pp_valid) return CP_ESTATE;
    // first-order terms (Eq. U_ni) on top of M_p(n), then V = A(n) W (Eq. V_nij)
    CKST(pp_mttkrp_impl(c, mode, c->Mt));
    CKST(launch_chol(c, mode, true, c->red_part));
    CKCUDA(c, cudaStreamWaitEvent(c->st, c->ev_chol, 0));
    c->chol_pending = false;
    LAUNCH(c, cpk::add_aw(c->Mt, c->A64[mode], c->W, (int)c->dims[mode], c->R, M_dev, c->st));
    return CP_OK;
}

void ema(double& v, double x) { v = (v < 0.0) ? x : 0.7 * v + 0.3 * x; }

// Running averages of what each choice costs on this problem.
void note_cost(cp_ctx* c, int kind, int init, double ms) {
    if (kind == 3) {
        // the cheapest regular sweep seen: early sweeps (refinement from a
        // random start) are slower than the steady state
        c->cost_exact = (c->cost_exact < 0.0) ? ms : std::min(c->cost_exact, ms);
        c->n_exact_seen++;
    } else if (kind == 2 && !init) {
        ema(c->cost_pp, ms);
    } else if (kind == 2 && init && c->cost_pp > 0.0) {
        ema(c->cost_init, std::max(0.0, ms - c->cost_pp));
    }
}

// undo every sweep since the rollback point (a failed judgement, or an
// approximated sweep whose normal equations broke down)
cp_status rollback(cp_ctx* c, int judge) {
    const size_t from = c->snap[1].trace_len;
    for (size_t t = from; t < c->trace.size(); ++t) c->trace[t].rolled_back = 1;
    const int done = c->sweeps_done;
    CKST(snap_restore(c, c->snap[1], false, false));
    c->sweeps_done = done;  // the undone sweeps stay in the count and the trace
    // regular sweeps for the next judge_every sweeps, twice as many after each
    // further rollback in a row (at most 64 judge_every)
    c->rollbacks_in_row = std::min(c->rollbacks_in_row + 1, 7);
    c->fallback_left = judge << (c->rollbacks_in_row - 1);
    c->since_judge = 0;
    c->snap_current = true;
    c->stats.rollbacks++;
    return CP_OK;
}

// The judge: the direct residual at the end of a run of approximated sweeps.  If
// it rose by more than the residual's own rounding noise (1e-5 relative: the
// model values are FP32 dot products), the factors return to the rollback point,
// the operators are dropped, the undone sweeps stay in the trace marked
// rolled_back, and Alg. 2's rule decides the next judge_every sweeps.
cp_status judge_now(cp_ctx* c, int judge) {
    CKCUDA(c, cudaEventRecord(c->events[2], c->st));
    double r;
    CKST(direct_resid(c, &r));
    if (r > c->judge_r * (1.0 + 1e-5)) {
        CKST(rollback(c, judge));
    } else {
        // a run that no longer lowers the residual (the approximation has
        // settled above the regular iteration's fixed point) also hands over
        // to regular sweeps
        if (c->judge_r - r < 1e-7 * r) c->fallback_left = judge;
        c->judge_r = r;
        c->rollbacks_in_row = 0;
        CKST(snap_take(c, c->snap[1]));
    }
    c->since_judge = 0;
    c->snap_current = true;
    CKCUDA(c, cudaEventRecord(c->events[3], c->st));
    CKCUDA(c, cudaEventSynchronize(c->events[3]));
    float jms = 0.f;
    CKCUDA(c, cudaEventElapsedTime(&jms, c->events[2], c->events[3]));
    if (!c->trace.empty()) c->trace.back().ms += jms;
    ema(c->cost_judge, jms);
    return CP_OK;
}

// rollback point = the current state (taken before a run of approximated sweeps)
cp_status judge_mark(cp_ctx* c) {
    CKCUDA(c, cudaEventRecord(c->events[2], c->st));
    CKST(direct_resid(c, &c->judge_r));
    CKST(snap_take(c, c->snap[1]));
    c->since_judge = 0;
    c->snap_current = true;
    CKCUDA(c, cudaEventRecord(c->events[3], c->st));
    CKCUDA(c, cudaEventSynchronize(c->events[3]));
    float jms = 0.f;
    CKCUDA(c, cudaEventElapsedTime(&jms, c->events[2], c->events[3]));
    c->pending_ms += jms;
    ema(c->cost_judge, jms);
    return CP_OK;
}

cp_status cp_sweep_pp(cp_ctx* c, int nsweeps, double eps, cp_policy* policy) {
    CKST(entry_check(c));
    if (nsweeps < 0 || !(eps > 0.0 && eps < 1.0)) return CP_EINVAL;
    CKST(grow_hist(c, 1));
    CKST(ensure_events(c, 4));
    const int judge = policy ? std::max(0, c->cfg.judge_every) : 0;
    if (!policy) drop_judge(c);
    for (int k = 0; k < nsweeps; ++k) {
        c->pending_ms = 0.0;
        float sc[2] = {-1.f, -1.f};
        int by = 0, choice;
        auto eps_rule = [&]() {
            // Alg. 2: enter / stay while every ||dA(i)|| < eps ||A(i)||
            bool small = true;
            for (int i = 0; i < c->N; ++i)
                if (!(c->dA_rel[i] < eps)) small = false;
            return !small ? CH_EXACT : (c->pp_valid ? CH_CUR : CH_NEW);
        };
        if (!policy) {
            choice = eps_rule();
        } else if (c->fallback_left > 0) {
            // after a rollback or a stalled run: regular sweeps
            choice = CH_EXACT;
            by = 2;
            c->fallback_left--;
        } else {
            // an approximated sweep is considered only while it is measured (or
            // not yet known) to cost less than a regular one, counting its share
            // of the judge and of the network query
            // (the first sweep is regular, as in Alg. 2 from a random start, and
            // gives the reference cost)
            const double extra = std::max(0.0, c->cost_query) + (judge ? std::max(0.0, c->cost_judge) / judge : 0.0);
            bool pp_pays = c->n_exact_seen >= 2 || !c->cfg.policy_gate;
            if (!c->cfg.policy_gate) {
                // consult the network before every sweep
            } else if (pp_pays && c->cost_pp < 0.0) {
                // not measured yet: explore only if the MTTKRP traffic an approximated
                // sweep avoids (at about 6 TB/s) can cover a network query (about
                // 30 us) and the judge's share (its residual: 2 numel R flops at
                // about 20 TFLOP/s)
                const double saved_ms = (c->sweep_mttkrp_bytes - pp_sweep_bytes(c)) / 6e9;
                const double judge_ms = c->cost_judge >= 0.0 ? c->cost_judge : 2.0 * c->numel * c->R / 20e9;
                const double over_ms = (c->cost_query >= 0.0 ? c->cost_query : 0.03) + (judge ? judge_ms / judge : 0.0);
                pp_pays = saved_ms > over_ms;
            } else if (pp_pays) {
                // measured: the approximated sweeps' all-in time per sweep (their
                // operator builds, judge and queries included) against 0.9 of the
                // cheapest regular sweep (a safe approximated sweep keeps at least
                // 90% of a regular sweep's progress)
                pp_pays = c->pp_n >= 3 ? c->pp_ms_total / c->pp_n < 0.9 * c->cost_exact
                                       : c->cost_pp + extra < c->cost_exact;
            }
            by = 1;
            choice = CH_EXACT;
            if (pp_pays) {
                CKCUDA(c, cudaEventRecord(c->events[0], c->st));
                bool valid = true;
                CKST(policy_scores(c, policy, sc, &valid));
                CKCUDA(c, cudaEventRecord(c->events[1], c->st));
                CKCUDA(c, cudaEventSynchronize(c->events[1]));
                float fms = 0.f;
                CKCUDA(c, cudaEventElapsedTime(&fms, c->events[0], c->events[1]));
                c->pending_ms += fms;
                ema(c->cost_query, fms);
                if (!valid) {
                    // the network gave no usable score: Alg. 2's rule decides
                    choice = eps_rule();
                    by = 4;
                } else if (c->pp_valid && sc[0] >= 0.5f) {
                    // the network's two queries: approximate with the current
                    // operators, or with operators rebuilt now; neither -> regular
                    choice = CH_CUR;
                } else if (sc[1] >= 0.5f) {
                    choice = CH_NEW;
                }
            }
        }
        if (judge) {
            if (choice == CH_EXACT && c->since_judge > 0) {
                CKST(judge_now(c, judge));  // judge a run of approximated sweeps before leaving it
                if (c->fallback_left > 0) {
                    by = 2;
                    c->fallback_left--;
                }
            }
            if (choice != CH_EXACT && c->since_judge == 0 && !(c->snap_current && c->snap[1].have))
                CKST(judge_mark(c));
        }
        CKCUDA(c, cudaEventRecord(c->events[0], c->st));
        const cp_status rs = run_choice(c, choice);
        if (rs == CP_ENOTSPD && judge && choice != CH_EXACT && c->snap[1].have && !c->poisoned) {
            // the approximation broke the normal equations: undo the run
            c->err.clear();
            CKST(rollback(c, judge));
            continue;
        }
        CKST(rs);
        c->snap_current = false;
        cp_trace_rec& rec = c->trace.back();
        rec.p_cur = sc[0];
        rec.p_new = sc[1];
        rec.decided_by = by;
        note_cost(c, rec.kind, rec.pp_init, rec.ms);
        rec.ms += c->pending_ms;
        const size_t rec_i = c->trace.size() - 1;
        if (judge && rec.kind == 2 && ++c->since_judge >= judge) CKST(judge_now(c, judge));
        if (policy && c->trace[rec_i].kind == 2) {
            c->pp_ms_total += c->trace[rec_i].ms;  // judge time lands on this record
            c->pp_n++;
        }
    }
    return CP_OK;
}

// Branch probe: the three choices from one state, each judged by the direct
// residual; the context then continues along `follow`.
cp_status cp_pp_probe(cp_ctx* c, int follow, cp_probe_rec* out) {
    CKST(entry_check(c));
    if (!out || follow < -1 || follow > 2 || (follow == CH_CUR && !c->pp_valid)) return CP_EINVAL;
    CKST(pp_alloc2(c));
    CKST(grow_hist(c, 1));
    CKST(ensure_events(c, 2));
    drop_judge(c);
    memset(out, 0, sizeof(*out));
    features(c, false, out->feat_cur);
    features(c, true, out->feat_new);
    out->has_ops = c->pp_valid ? 1 : 0;
    CKST(direct_resid(c, &out->r0));
    CKST(snap_take(c, c->snap[0]));
    auto branch = [&](int ch, double* r, double* ms) -> cp_status {
        CKCUDA(c, cudaEventRecord(c->events[0], c->st));
        const cp_status rs = run_choice(c, ch);
        if (rs == CP_ENOTSPD && ch != CH_EXACT && !c->poisoned) {
            // an approximated branch whose normal equations broke down: unsafe
            c->err.clear();
            *r = INFINITY;
            *ms = 0.0;
            return CP_OK;
        }
        CKST(rs);
        *ms = c->trace.back().ms;
        CKST(direct_resid(c, r));
        return CP_OK;
    };
    out->r_cur = NAN;
    if (out->has_ops) {
        CKST(branch(CH_CUR, &out->r_cur, &out->ms_cur));
        CKST(snap_restore(c, c->snap[0], true, true));
    }
    CKST(branch(CH_EXACT, &out->r_exact, &out->ms_exact));
    CKST(snap_restore(c, c->snap[0], true, true));
    CKST(branch(CH_NEW, &out->r_new, &out->ms_new));
    // safe: the approximated sweep achieves at least 90% of the regular sweep's
    // decrease of the direct residual (plus a rounding allowance)
    const double gain = std::max(0.0, out->r0 - out->r_exact);
    const double slack = 0.1 * gain + 1e-9 * out->r0;
    out->label_cur = (out->has_ops && out->r_cur - out->r_exact <= slack) ? 1 : 0;
    out->label_new = (out->r_new - out->r_exact <= slack) ? 1 : 0;
    int ch = follow;
    if (ch < 0) ch = out->label_cur ? CH_CUR : (out->label_new ? CH_NEW : CH_EXACT);
    double rf = out->r_new;
    if (ch != CH_NEW) {
        CKST(snap_restore(c, c->snap[0], true, true));
        double ms;
        CKST(branch(ch, &rf, &ms));
    }
    if (!isfinite(rf)) {
        // the requested branch broke down: back to the starting state
        CKST(snap_restore(c, c->snap[0], true, true));
        return fail(c, CP_ENOTSPD, "the followed PP branch broke the normal equations");
    }
    out->followed = ch;
    c->trace.back().decided_by = 3;
    return CP_OK;
}

cp_status cp_run(cp_ctx* c, int route, cp_policy* policy, int* nsweeps) {
    CKST(entry_check(c));
    if (nsweeps) *nsweeps = 0;
    const double delta = c->cfg.delta;
    const int cap = c->cfg.max_sweeps;
    if (route < 0 || route > 2 || (!(delta > 0.0) && cap <= 0)) return CP_EINVAL;
    double r = c->have_last ? c->last_resid : 1.0;
    for (int k = 0; cap <= 0 || k < cap; ++k) {
        if (route == 0) CKST(cp_sweep_dt(c, 1));
        else if (route == 1) CKST(cp_sweep_msdt(c, 1));
        else CKST(cp_sweep_pp(c, 1, c->cfg.pp_eps, policy));
        if (nsweeps) *nsweeps = k + 1;
        const double r_old = r;
        r = c->trace.back().resid;
        if (delta > 0.0 && fabs(r - r_old) <= delta) break;
    }
    return CP_OK;
}

cp_status cp_policy_features(cp_ctx* c, float* f16) {
    CKST(entry_check(c));
    if (!f16) return CP_EINVAL;
    features(c, false, f16);
    features(c, true, f16 + 8);
    return CP_OK;
}

cp_status cp_fit(cp_ctx* c, int exact, double* fit, double* resid) {
    CKST(entry_check(c));
    double r;
    if (!exact && c->have_last) {
        r = c->last_resid;
    } else {
        CKST(direct_resid(c, &r));
    }
    if (!isfinite(r)) return fail(c, CP_ENUMERIC, "non-finite residual");
    if (resid) *resid = r;
    if (fit) *fit = 1.0 - r;
    return CP_OK;
}

cp_status cp_get_factor(cp_ctx* c, int mode, double* A_host) {
    CKST(entry_check(c));
    if (mode < 0 || mode >= c->N || !A_host) return CP_EINVAL;
    CKCUDA(c, cudaMemcpyAsync(A_host, c->A64[mode], sizeof(double) * c->dims[mode] * c->R, cudaMemcpyDeviceToHost, c->st));
    CKCUDA(c, cudaStreamSynchronize(c->st));
    return CP_OK;
}

cp_status cp_set_factor(cp_ctx* c, int mode, const double* A_host) {
    CKST(entry_check(c));
    if (mode < 0 || mode >= c->N || !A_host) return CP_EINVAL;
    const int s = (int)c->dims[mode];
    CKCUDA(c, cudaMemcpyAsync(c->A64[mode], A_host, sizeof(double) * s * c->R, cudaMemcpyHostToDevice, c->st));
    LAUNCH(c, cpk::factor_copies(c->A64[mode], c->A32[mode], uses_bf16(c) ? c->bhi[mode] : nullptr,
                                 uses_bf16(c) ? c->blo[mode] : nullptr, uses_tf32(c) ? c->bt32[mode] : nullptr, s,
                                 c->R, c->Rpad, c->Kpad[mode], c->st));
    // with PP operators present, dA = A - A_p and dS = A^T dA follow the new factor
    const bool pp = c->pp_valid;
    if (pp)
        LAUNCH(c, cpk::pp_delta(c->A64[mode], c->Ap64[mode], c->dA32[mode], c->dA64[mode], (int64_t)s * c->R, c->st));
    CKST(regram(c, mode, pp));
    CKCUDA(c, cudaStreamSynchronize(c->st));
    c->ver[mode] = ++c->vclock;
    c->have_last = false;
    drop_judge(c);
    return CP_OK;
}

cp_status cp_get_trace(cp_ctx* c, cp_trace_rec* buf, size_t* len) {
    if (!c || !len) return CP_EINVAL;
    const size_t n = c->trace.size();
    if (buf) memcpy(buf, c->trace.data(), std::min(*len, n) * sizeof(cp_trace_rec));
    *len = n;
    return CP_OK;
}

cp_status cp_get_stats(cp_ctx* c, cp_stats* st) {
    if (!c || !st) return CP_EINVAL;
    *st = c->stats;
    return CP_OK;
}

// ---------------------------------------------------------------------- policy
cp_status cp_policy_create(cp_policy** out, const float* theta_host, void* stream) {
    if (!out || !theta_host) return CP_EINVAL;
    *out = nullptr;
    cp_policy* p = new cp_policy();
    p->st = (cudaStream_t)stream;
    const int n = cpk::mlp_nparams();
    bool ok = cudaMalloc(&p->theta, n * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&p->m, n * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&p->v, n * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&p->grad, n * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&p->loss, sizeof(float)) == cudaSuccess &&
              cudaMalloc(&p->scratch, cpk::mlp_scratch_floats() * sizeof(float)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cp_policy_free(p);
        return CP_ENOMEM;
    }
    if (cudaMemcpyAsync(p->theta, theta_host, n * sizeof(float), cudaMemcpyHostToDevice, p->st) != cudaSuccess ||
        cudaMemsetAsync(p->m, 0, n * sizeof(float), p->st) != cudaSuccess ||
        cudaMemsetAsync(p->v, 0, n * sizeof(float), p->st) != cudaSuccess ||
        cudaStreamSynchronize(p->st) != cudaSuccess) {
        cudaGetLastError();
        cp_policy_free(p);
        return CP_ECUDA;
    }
    *out = p;
    return CP_OK;
}

cp_status cp_policy_get(cp_policy* p, float* theta_host) {
    if (!p || !theta_host) return CP_EINVAL;
    if (cudaMemcpyAsync(theta_host, p->theta, cpk::mlp_nparams() * sizeof(float), cudaMemcpyDeviceToHost, p->st) !=
            cudaSuccess ||
        cudaStreamSynchronize(p->st) != cudaSuccess)
        return CP_ECUDA;
    return CP_OK;
}

cp_status cp_policy_forward(cp_policy* p, const float* X_dev, int B, float* prob_dev) {
    if (!p || B < 0 || (B > 0 && (!X_dev || !prob_dev))) return CP_EINVAL;
    return cpk::mlp_forward(p->theta, X_dev, B, prob_dev, p->st) == cudaSuccess ? CP_OK : CP_ECUDA;
}

cp_status cp_policy_grad(cp_policy* p, const float* X_dev, const float* y_dev, int B, float* loss_dev,
                         float* grad_dev) {
    if (!p || B < 1 || !X_dev || !y_dev || !grad_dev) return CP_EINVAL;
    return cpk::mlp_grad(p->theta, X_dev, y_dev, B, loss_dev, grad_dev, p->scratch, p->st) == cudaSuccess
               ? CP_OK
               : CP_ECUDA;
}

cp_status cp_policy_train(cp_policy* p, const float* X_dev, const float* y_dev, int B, int steps, float lr) {
    if (!p || B < 1 || !X_dev || !y_dev || steps < 0) return CP_EINVAL;
    for (int i = 0; i < steps; ++i) {
        if (cpk::mlp_grad(p->theta, X_dev, y_dev, B, p->loss, p->grad, p->scratch, p->st) != cudaSuccess)
            return CP_ECUDA;
        p->t++;
        if (cpk::mlp_adam(p->theta, p->grad, p->m, p->v, cpk::mlp_nparams(), p->t, lr, p->st) != cudaSuccess)
            return CP_ECUDA;
    }
    return CP_OK;
}

void cp_policy_free(cp_policy* p) {
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st);
    for (float* q : {p->theta, p->m, p->v, p->grad, p->loss, p->scratch})
        if (q) cudaFree(q);
    delete p;
}

}  // extern "C"
