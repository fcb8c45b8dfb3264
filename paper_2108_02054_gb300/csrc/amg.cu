// amg.cu -- context, hierarchy orchestration and the C ABI of libamgpr.so.
//
// Method: partial-reuse AMG setup amortisation (arXiv 2108.02054).
//   amg_full_setup       Alg. 1 (all GPU kernels; host only sequences them and
//                        reads back the sizes it must allocate)
//   amg_partial_rebuild  Alg. 4 body: numeric Galerkin products over the cached
//                        patterns (Sec. 5), smoothers, coarsest LU
//   amg_step             Alg. 3 / Alg. 4 / no-reuse time-step dispatch
//   amg_solve            CG with one V-cycle (Alg. 2) per iteration; the
//                        iteration's control state lives on the device
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

using namespace amgpr;

namespace amgpr {
static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(int64_t d) { g_launches.fetch_add(d, std::memory_order_relaxed); }
int64_t launch_total() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace amgpr

// CUDA-event timing of selected kernels on the context's stream (off unless
// amg_profile(ctx, 1)); slot numbers are the AMG_PROF_* values of amgpr.h
struct ProfData {
    bool on = false;
    bool eager = false;  // time the host-driven launch loop instead of an unrolled graph
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> rec[AMG_PROF_NSLOTS];
};

// The host-buffer entry point copies a partial step's fine values in row
// chunks; chunk c (rows row[c] .. row[c + 1] - 1, boundaries multiples of 32)
// is on the device once ev[c] has completed, and its ingest and its rows of
// the finest A P (whose terms read only those rows' values) wait only for it.
constexpr int kHostChunks = 8;
// Stage 2 follows in coarse-row ranges: once chunks 0 .. c have landed, the
// coarse rows before crow[c + 1] (the leading rows whose R rows reach no fine
// row of a later chunk) have every A P row they read.
struct FineChunks {
    const int32_t *row;     // kHostChunks + 1 row boundaries
    const int32_t *ap;      // the finest A P's entry offsets at those rows
    const int32_t *ac;      // the next level's entry offsets at the coarse boundaries crow
    const cudaEvent_t *ev;  // kHostChunks events on the copy stream
};

struct amg_ctx {
    amg_params prm{};
    cudaStream_t s = nullptr;
    cudaMemPool_t pool = nullptr;
    std::vector<void *> hier;     // hierarchy allocations (replaced by every full setup)
    std::vector<void *> persist;  // context-lifetime allocations
    std::string err;
    // fine pattern (persistent)
    int32_t n = 0, nnz = 0;
    int32_t *fine_ptr = nullptr, *fine_col = nullptr;
    bool pattern_ok = false;  // the stored pattern passed the row-pointer check
    // its compressed columns, when its rows use at most kMaxColOffsets offsets
    uint8_t *fine_cidx = nullptr;
    int32_t *fine_coff = nullptr, *coff_table = nullptr;
    int *coff_count = nullptr;
    int fine_ncoff = 0;
    // hierarchy
    int nlev = 0;
    Level lev[kMaxLevels];
    int32_t nL = 0;
    double *lu = nullptr, *inv = nullptr, *luT = nullptr;
    int32_t *piv = nullptr;
    bool have_setup = false;
    // system matrix of the solve (aliases level 0 except under full reuse)
    double *A_sys = nullptr;
    double *A_sys_own = nullptr;
    // CG
    double *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_q = nullptr, *cg_t = nullptr;
    // per-block partial sums of the CG reductions, one set per reduction so
    // that a kernel may read one set while writing another
    double *partial = nullptr;
    double *part_pq = nullptr, *part_rr = nullptr, *part_rz = nullptr, *part_rzo = nullptr, *part_tt = nullptr;
    CgState *cg = nullptr;
    CgState *h_cg = nullptr;  // pinned
    // BiCGStab: r^, s, s^ (r, p, p^, v, t reuse cg_r, cg_p, cg_z, cg_q, cg_t)
    double *bi_rh = nullptr, *bi_s = nullptr, *bi_sh = nullptr;
    BiState *bi = nullptr;
    BiState *h_bi = nullptr;  // pinned
    int *d_st = nullptr;
    int *h_st = nullptr;      // pinned
    // host-buffer staging
    double *stage_val = nullptr, *stage_f = nullptr, *stage_u = nullptr;
    ProfData prof;
    // whole-solve CUDA graph (rebuilt after a full setup or a new tolerance)
    cudaStream_t s_cap = nullptr, s_cap_main = nullptr, s_cap_if = nullptr;
    // host-buffer entry point: the right-hand side's copy runs beside the rebuild
    cudaStream_t s_copy = nullptr;
    cudaEvent_t ev_vals = nullptr, ev_f = nullptr;
    // ... and, for a partial step, the values arrive in row chunks (one event
    // each); the chunk boundaries are read once per hierarchy
    cudaEvent_t ev_chunk[kHostChunks] = {};
    int32_t ck_row[kHostChunks + 1] = {}, ck_e[kHostChunks + 1] = {}, ck_ap[kHostChunks + 1] = {};
    int32_t ck_crow[kHostChunks + 1] = {}, ck_ac[kHostChunks + 1] = {};
    int64_t setup_gen = 0, ck_gen = -1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    bool use_graph = true;
    bool use_gather = true;  // partial rebuilds apply the Galerkin product as gather operators
    bool graph_valid = false;
    double graph_tol = -1.0;
    double *cg_f = nullptr, *cg_u = nullptr;
    int64_t graph_pro = 0, graph_body = 0, graph_epi = 0, graph_branch = 0;  // kernels per part of the graph
    // time-step bookkeeping
    int last_iters = 0;
    int last_status = AMG_OK;
    int last_rebuilt = 0;
    int steps_since_full = 0;   // partial rebuilds since the last full setup
    int iters_after_full = -1;  // iterations of the first solve after it (-1: not yet known)
};

namespace {

amg_status set_err(amg_ctx *c, amg_status st, const std::string &msg) {
    if (c) c->err = msg;
    return st;
}

cudaEvent_t prof_event(amg_ctx *c) {
    if (c->prof.pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    cudaEvent_t e = c->prof.pool.back();
    c->prof.pool.pop_back();
    return e;
}

// record a timing event; on a capturing stream as an event-record node of
// the graph (a plain record there would only mark a capture dependency)
void prof_record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}

struct ProfScope {
    amg_ctx *c;
    int slot;
    cudaEvent_t b = nullptr;
    ProfScope(amg_ctx *c_, int slot_, bool active = true) : c(c_), slot(slot_) {
        if (c->prof.on && active) {
            b = prof_event(c);
            prof_record(b, c->s);
        }
    }
    // end the timed span now (the destructor then does nothing)
    void close() {
        if (!b) return;
        cudaEvent_t e = prof_event(c);
        prof_record(e, c->s);
        c->prof.rec[slot].push_back({b, e});
        b = nullptr;
    }
    ~ProfScope() { close(); }
};

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return set_err(ctx, e_ == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA, \
                           std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)

#define TRY(expr)                              \
    do {                                       \
        amg_status t_ = (expr);                \
        if (t_ != AMG_OK) return t_;           \
    } while (0)

template <class T>
amg_status alloc(amg_ctx *ctx, T **p, size_t count, bool persistent = false) {
    void *q = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMallocFromPoolAsync(&q, bytes, ctx->pool, ctx->s);
    if (e != cudaSuccess)
        return set_err(ctx, e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA,
                       std::string("device allocation of ") + std::to_string(bytes) + " bytes: " +
                           cudaGetErrorString(e));
    (persistent ? ctx->persist : ctx->hier).push_back(q);
    *p = (T *)q;
    return AMG_OK;
}

void free_hierarchy(amg_ctx *ctx) {
    for (void *p : ctx->hier) cudaFreeAsync(p, ctx->s);
    ctx->hier.clear();
    for (int l = 0; l < kMaxLevels; ++l) ctx->lev[l] = Level{};
    ctx->nlev = 0;
    ctx->have_setup = false;
    ctx->lu = ctx->inv = ctx->luT = nullptr;
    ctx->piv = nullptr;
    ctx->graph_valid = false;
}

// read the device status word (synchronises the stream) and map it
amg_status check_device(amg_ctx *ctx, const char *where) {
    CK(cudaMemcpyAsync(ctx->h_st, ctx->d_st, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    CK(cudaGetLastError());
    int st = *ctx->h_st;
    if (st == 0) return AMG_OK;
    std::string w(where);
    if (st & DEV_ERR_PATTERN)
        return set_err(ctx, AMG_ERR_PATTERN, w + ": unsorted or out-of-range columns, or a missing diagonal");
    if (st & DEV_ERR_NONFINITE) return set_err(ctx, AMG_ERR_NONFINITE, w + ": non-finite matrix values");
    if (st & DEV_ERR_SINGULAR) return set_err(ctx, AMG_ERR_SINGULAR, w + ": zero pivot in the coarsest LU");
    if (st & DEV_ERR_CAPACITY)
        return set_err(ctx, AMG_ERR_CAPACITY, w + ": a row of a Galerkin product exceeds the kernel capacity");
    if (st & DEV_ERR_OVERFLOW) return set_err(ctx, AMG_ERR_CAPACITY, w + ": an index count exceeds int32");
    if (st & DEV_ERR_TIMEOUT)
        return set_err(ctx, AMG_ERR_CUDA, w + ": a message between the CTAs of the coarsest LU did not arrive");
    return set_err(ctx, AMG_ERR_STATE, w + ": inconsistent hierarchy state");
}

amg_status reset_status(amg_ctx *ctx) {
    CK(cudaMemsetAsync(ctx->d_st, 0, sizeof(int), ctx->s));
    return AMG_OK;
}

template <class T>
amg_status read_scalar(amg_ctx *ctx, const T *d, T *h) {
    CK(cudaMemcpyAsync(h, d, sizeof(T), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    return AMG_OK;
}

amg_status scan(amg_ctx *ctx, const int32_t *in, int32_t *out, int64_t n) {
    int64_t *tmp = nullptr;
    TRY(alloc(ctx, &tmp, (size_t)scan_tmp_elems(n)));
    scan_counts(in, out, n, ctx->d_st, tmp, ctx->s);
    return AMG_OK;
}

bool mixed(const amg_ctx *ctx) { return ctx->prm.precision == AMG_PREC_MIXED; }
// 4 x 4 block-valued matrices (amg_params.block_size = 4)
bool blockmode(const amg_ctx *ctx) { return ctx->prm.block_size == 4; }
// unknowns of a vector on the fine level, values of the fine matrix
int64_t nvec(const amg_ctx *ctx) { return (int64_t)ctx->n * ctx->prm.block_size; }
size_t nvals(const amg_ctx *ctx) { return (size_t)ctx->nnz * (size_t)(ctx->prm.block_size * ctx->prm.block_size); }

amg_status alloc_level_vectors(amg_ctx *ctx, Level &L) {
    if (blockmode(ctx)) {
        TRY(alloc(ctx, &L.vd.u, 4 * (size_t)L.n));
        TRY(alloc(ctx, &L.vd.f, 4 * (size_t)L.n));
        TRY(alloc(ctx, &L.vd.r, 4 * (size_t)L.n));
        TRY(alloc(ctx, &L.vd.t, 4 * (size_t)L.n));
        TRY(alloc(ctx, &L.Minv, 16 * (size_t)L.n));
        return AMG_OK;
    }
    if (mixed(ctx)) {
        TRY(alloc(ctx, &L.vf.u, L.n));
        TRY(alloc(ctx, &L.vf.f, L.n));
        TRY(alloc(ctx, &L.vf.r, L.n));
        TRY(alloc(ctx, &L.vf.t, L.n));
        TRY(alloc(ctx, &L.mf, L.n));
        TRY(alloc(ctx, &L.A_valf, L.nnz));
    } else {
        TRY(alloc(ctx, &L.vd.u, L.n));
        TRY(alloc(ctx, &L.vd.f, L.n));
        TRY(alloc(ctx, &L.vd.r, L.n));
        TRY(alloc(ctx, &L.vd.t, L.n));
        TRY(alloc(ctx, &L.m, L.n));
    }
    return AMG_OK;
}

// symbolic C = X*Y (pattern only), allocating C's arrays
amg_status symbolic_product(amg_ctx *ctx, int32_t nrows, int32_t ncols, const int32_t *X_ptr, const int32_t *X_col,
                            const int32_t *Y_ptr, const int32_t *Y_col, int add_diag, int32_t **C_ptr,
                            int32_t **C_col, int32_t *C_nnz) {
    int32_t *len = nullptr;
    TRY(alloc(ctx, &len, (size_t)nrows));
    TRY(alloc(ctx, C_ptr, (size_t)nrows + 1));
    // the hash tables are sized for the longest row of terms
    int *d_max = nullptr;
    TRY(alloc(ctx, &d_max, 1));
    CK(cudaMemsetAsync(d_max, 0, sizeof(int), ctx->s));
    launch_row_terms_max(nrows, X_ptr, X_col, Y_ptr, add_diag, d_max, ctx->s);
    int32_t max_terms = 0;
    TRY(read_scalar(ctx, d_max, &max_terms));
    const int cap = spgemm_symbolic_cap(max_terms);
    // lanes per row from X's average row length (its entries are spread over the lanes)
    int32_t xnnz = 0;
    TRY(read_scalar(ctx, X_ptr + nrows, &xnnz));
    const double avg = nrows > 0 ? (double)xnnz / (double)nrows : 0.0;
    const int lanes = avg <= 8.0 ? 8 : avg <= 16.0 ? 16 : 32;
    launch_spgemm_symbolic(nrows, ncols, X_ptr, X_col, Y_ptr, Y_col, add_diag, cap, lanes, len, nullptr, nullptr,
                           ctx->d_st, ctx->s);
    TRY(scan(ctx, len, *C_ptr, nrows));
    TRY(check_device(ctx, "symbolic product"));
    TRY(read_scalar(ctx, *C_ptr + nrows, C_nnz));
    TRY(alloc(ctx, C_col, (size_t)*C_nnz));
    launch_spgemm_symbolic(nrows, ncols, X_ptr, X_col, Y_ptr, Y_col, add_diag, cap, lanes, len, *C_ptr, *C_col,
                           ctx->d_st, ctx->s);
    return AMG_OK;
}

amg_status max_row(amg_ctx *ctx, int32_t n, const int32_t *ptr, int32_t *out) {
    int *d = nullptr;
    TRY(alloc(ctx, &d, 1));
    CK(cudaMemsetAsync(d, 0, sizeof(int), ctx->s));
    launch_row_maxlen(n, ptr, d, ctx->s);
    int h = 0;
    TRY(read_scalar(ctx, d, &h));
    *out = h;
    return AMG_OK;
}

// Lanes per row for a level's matrix-vector kernels (A rows, R rows): about
// sixteen entries per lane, then more lanes until the level offers enough
// threads to fill the GPU (short fine-level rows keep one lane and the plain
// sequential row sum).  Measured against eight and thirty-two entries per
// lane: sixteen is fastest on the large levels at 128^3 and 192^3, and the
// occupancy rule leaves the 64^3 levels as they were.
int choose_lpr(int64_t rows, int64_t nnz) {
    if (rows <= 0) return 1;
    const double avg = (double)nnz / (double)rows;
    int p = 1;
    while (p < 32 && 16.0 * p < avg) p *= 2;
    while (p < 32 && rows * p < 152LL * 1024) p *= 2;
    return p;
}

// the coarsest direct solver: dense LU (FP64) and its explicit inverse
amg_status coarse_factor(amg_ctx *ctx) {
    Level &C = ctx->lev[ctx->nlev - 1];
    if (blockmode(ctx)) {
        const int32_t n4 = ctx->nL;
        CK(cudaMemsetAsync(ctx->lu, 0, sizeof(double) * (size_t)n4 * (size_t)n4, ctx->s));
        launch_block_to_dense(C.n, C.A_ptr, C.A_col, C.Ab, ctx->lu, ctx->s);
        { ProfScope ps_(ctx, AMG_PROF_LU, true); launch_dense_lu(n4, ctx->lu, ctx->piv, ctx->d_st, ctx->s, ctx->luT); }
        { ProfScope ps_(ctx, AMG_PROF_INV, true); launch_lu_inverse(n4, ctx->lu, ctx->piv, ctx->inv, ctx->s, ctx->luT); }
        return AMG_OK;
    }
    const bool mx = mixed(ctx);
    launch_csr_to_dense(C.n, C.A_ptr, C.A_col, mx ? nullptr : C.A_val, mx ? C.A_valf : nullptr, ctx->lu, ctx->s);
    { ProfScope ps_(ctx, AMG_PROF_LU, true); launch_dense_lu(C.n, ctx->lu, ctx->piv, ctx->d_st, ctx->s, ctx->luT); }
    { ProfScope ps_(ctx, AMG_PROF_INV, true); launch_lu_inverse(C.n, ctx->lu, ctx->piv, ctx->inv, ctx->s, ctx->luT); }
    return AMG_OK;
}

// Build, for level l, the two fixed gather operators of the numeric Galerkin
// product (AP = N a, A_c = M AP) from the slot metadata of the setup.  Done
// once per hierarchy, at the first partial rebuild (full rebuilds never pay it).
amg_status build_gather(amg_ctx *ctx, int l) {
    Level &L = ctx->lev[l];
    Level &C = ctx->lev[l + 1];
    const bool mx = mixed(ctx);
    const int64_t nt1 = L.nt1, nt2 = L.nt2;
    const int64_t tmax = std::max(nt1, nt2);
    int32_t *perm = nullptr, *idx_tmp = nullptr;
    double *w_tmp = nullptr;
    TRY(alloc(ctx, &perm, (size_t)tmax));
    TRY(alloc(ctx, &idx_tmp, (size_t)tmax));
    TRY(alloc(ctx, &w_tmp, (size_t)tmax));
    // stage 1: one output per entry of AP
    TRY(alloc(ctx, &L.g1_ptr, (size_t)L.nnzAP + 1));
    TRY(alloc(ctx, &L.g1_idx, (size_t)nt1));
    if (mx) TRY(alloc(ctx, &L.g1_wf, (size_t)nt1));
    else TRY(alloc(ctx, &L.g1_w, (size_t)nt1));
    launch_group_terms(L.n, L.t1ptr, L.slot1, L.AP_ptr, L.g1_ptr, perm, ctx->d_st, ctx->s);
    CK(cudaMemcpyAsync(L.g1_ptr + L.nnzAP, L.t1ptr + L.n, sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->s));
    launch_stage1_terms(L.n, L.A_ptr, L.A_col, L.P_ptr, L.P_val, L.t1ptr, idx_tmp, w_tmp, ctx->s);
    launch_permute_terms(nt1, perm, idx_tmp, w_tmp, L.g1_idx, mx ? nullptr : L.g1_w, mx ? L.g1_wf : nullptr, ctx->s);
    // stage 2: one output per entry of A_c
    TRY(alloc(ctx, &L.g2_ptr, (size_t)C.nnz + 1));
    TRY(alloc(ctx, &L.g2_idx, (size_t)nt2));
    if (mx) TRY(alloc(ctx, &L.g2_wf, (size_t)nt2));
    else TRY(alloc(ctx, &L.g2_w, (size_t)nt2));
    launch_group_terms(L.nc, L.t2ptr, L.slot2, C.A_ptr, L.g2_ptr, perm, ctx->d_st, ctx->s);
    CK(cudaMemcpyAsync(L.g2_ptr + C.nnz, L.t2ptr + L.nc, sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->s));
    launch_stage2_terms(L.nc, L.R_ptr, L.R_col, L.R_val, L.AP_ptr, L.t2ptr, idx_tmp, w_tmp, ctx->s);
    launch_permute_terms(nt2, perm, idx_tmp, w_tmp, L.g2_idx, mx ? nullptr : L.g2_w, mx ? L.g2_wf : nullptr, ctx->s);
    L.gather_ready = true;
    return AMG_OK;
}

// Alg. 4 body for the 4 x 4 block hierarchy: new fine blocks, then per
// level the damped block-Jacobi inverses and (galerkin) the coarse blocks
// through the fixed gather operators, then the coarsest factorisation
amg_status block_numeric_rebuild(amg_ctx *ctx, const double *d_val, bool galerkin) {
    Level &F = ctx->lev[0];
    if (d_val != F.Ab) {
        launch_check_finite((int64_t)nvals(ctx), d_val, ctx->d_st, ctx->s);
        { ProfScope ps_(ctx, AMG_PROF_INGEST); CK(cudaMemcpyAsync(F.Ab, d_val, sizeof(double) * nvals(ctx), cudaMemcpyDeviceToDevice, ctx->s)); }
    }
    for (int l = 0; l + 1 < ctx->nlev; ++l) {
        Level &L = ctx->lev[l];
        Level &C = ctx->lev[l + 1];
        launch_block_jacobi(L.n, L.dia, L.Ab, ctx->prm.jacobi_omega, L.Minv, ctx->s);
        if (galerkin) {
            { ProfScope ps_(ctx, AMG_PROF_AP_L0, l == 0); launch_block_gather(L.nnzAP, L.g1_ptr, L.g1_idx, L.g1_w, L.Ab, L.APb, ctx->s); }
            { ProfScope ps_(ctx, AMG_PROF_RAP_L0, l == 0); launch_block_gather(C.nnz, L.g2_ptr, L.g2_idx, L.g2_w, L.APb, C.Ab, ctx->s); }
        }
    }
    return coarse_factor(ctx);
}

// numeric part shared by the full setup and the partial rebuild (Alg. 4 body)
amg_status numeric_rebuild(amg_ctx *ctx, const double *d_val, bool galerkin, const FineChunks *ck = nullptr) {
    if (blockmode(ctx)) return block_numeric_rebuild(ctx, d_val, galerkin);
    const amg_params &p = ctx->prm;
    Level &F = ctx->lev[0];
    const bool mx = mixed(ctx);
    auto ingest = [&](int32_t r0, int32_t r1) {
        launch_ingest_fine(r0, r1, F.A_ptr, d_val, F.dia, p.smoother, p.jacobi_omega,
                           d_val == F.A_val ? nullptr : F.A_val, mx ? F.A_valf : nullptr, mx ? nullptr : F.m,
                           mx ? F.mf : nullptr, ctx->d_st, ctx->s);
    };
    // with chunks (the caller checked that the gather operators exist), each
    // chunk's ingest and its rows of the finest stage 1 run once it has arrived
    const bool ck_ap = ck && galerkin && ctx->nlev > 1;
    if (ck) {
        for (int c = 0; c < kHostChunks; ++c) {
            CK(cudaStreamWaitEvent(ctx->s, ck->ev[c], 0));
            ingest(ck->row[c], ck->row[c + 1]);
            if (!ck_ap) continue;
            const int64_t e0 = ck->ap[c], ne = (int64_t)ck->ap[c + 1] - e0;
            if (mx) launch_gather_apply<float>(ne, F.g1_ptr + e0, F.g1_idx, F.g1_wf, F.A_valf, F.AP_valf + e0, ctx->s);
            else launch_gather_apply<double>(ne, F.g1_ptr + e0, F.g1_idx, F.g1_w, F.A_val, F.AP_val + e0, ctx->s);
            // the coarse rows whose A P rows are now all there
            Level &C1 = ctx->lev[1];
            const int64_t o0 = ck->ac[c], no = (int64_t)ck->ac[c + 1] - o0;
            if (mx) launch_gather_apply<float>(no, F.g2_ptr + o0, F.g2_idx, F.g2_wf, F.AP_valf, C1.A_valf + o0, ctx->s);
            else launch_gather_apply<double>(no, F.g2_ptr + o0, F.g2_idx, F.g2_w, F.AP_val, C1.A_val + o0, ctx->s);
        }
    } else {
        ProfScope ps_(ctx, AMG_PROF_INGEST);
        ingest(0, F.n);
    }
    for (int l = 0; l + 1 < ctx->nlev; ++l) {
        Level &L = ctx->lev[l];
        Level &C = ctx->lev[l + 1];
        ProfScope pg_(ctx, AMG_PROF_GALERKIN, galerkin);
        if (galerkin && L.gather_ready) {
            const bool s1 = !(ck_ap && l == 0);  // the finest level's stages not yet applied
            if (mx) {
                if (s1) { ProfScope ps_(ctx, AMG_PROF_AP_L0, l == 0); launch_gather_apply<float>(L.nnzAP, L.g1_ptr, L.g1_idx, L.g1_wf, L.A_valf, L.AP_valf, ctx->s); }
                if (s1) { ProfScope ps_(ctx, AMG_PROF_RAP_L0, l == 0); launch_gather_apply<float>(C.nnz, L.g2_ptr, L.g2_idx, L.g2_wf, L.AP_valf, C.A_valf, ctx->s); }
            } else {
                if (s1) { ProfScope ps_(ctx, AMG_PROF_AP_L0, l == 0); launch_gather_apply<double>(L.nnzAP, L.g1_ptr, L.g1_idx, L.g1_w, L.A_val, L.AP_val, ctx->s); }
                if (s1) { ProfScope ps_(ctx, AMG_PROF_RAP_L0, l == 0); launch_gather_apply<double>(C.nnz, L.g2_ptr, L.g2_idx, L.g2_w, L.AP_val, C.A_val, ctx->s); }
            }
        } else if (galerkin) {
            if (mx) {
                { ProfScope ps_(ctx, AMG_PROF_AP_L0, l == 0); launch_ap_numeric_f32(L, L.A_valf, ctx->s); }
                { ProfScope ps_(ctx, AMG_PROF_RAP_L0, l == 0); launch_rap_numeric_f32(L, C.A_ptr, C.A_valf, ctx->s); }
            } else {
                { ProfScope ps_(ctx, AMG_PROF_AP_L0, l == 0); launch_ap_numeric_f64(L, L.A_val, ctx->s); }
                { ProfScope ps_(ctx, AMG_PROF_RAP_L0, l == 0); launch_rap_numeric_f64(L, C.A_ptr, C.A_val, ctx->s); }
            }
        }
        pg_.close();
        if (l + 1 < ctx->nlev - 1) {
            ProfScope psm_(ctx, AMG_PROF_SMOOTHERS);
            if (mx) launch_smoother_f32(C.n, C.A_ptr, C.A_valf, C.dia, p.smoother, p.jacobi_omega, C.mf, ctx->s);
            else launch_smoother_f64(C.n, C.A_ptr, C.A_val, C.dia, p.smoother, p.jacobi_omega, C.m, ctx->s);
        }
    }
    return coarse_factor(ctx);
}

// Two-byte column offsets for every level without the one-byte form: A's
// columns as column - row, P's as column - (int)(row * n_c / n); each kept
// where all of a level's offsets fit in 16 bits (a coarse level of a grid
// hierarchy: up to about 24,000 at 192^3; the finest level's P: about
// 11,000), so the matrix kernels and the prolongation move 2 bytes less per
// entry.  Built once per full setup: the patterns stay fixed across partial
// rebuilds.
amg_status build_delta16(amg_ctx *ctx) {
    if (blockmode(ctx)) return AMG_OK;
    int *flags = nullptr;
    TRY(alloc(ctx, &flags, (size_t)(2 * kMaxLevels)));
    CK(cudaMemsetAsync(flags, 0, sizeof(int) * 2 * kMaxLevels, ctx->s));
    int16_t *buf[kMaxLevels] = {}, *pbuf[kMaxLevels] = {};
    float ratio[kMaxLevels] = {};
    for (int l = 0; l < ctx->nlev; ++l) {
        Level &L = ctx->lev[l];
        if (!L.A_cidx && L.n > 0 && L.nnz > 0) {
            TRY(alloc(ctx, &buf[l], (size_t)L.nnz));
            launch_col_delta16(L.n, L.A_ptr, L.A_col, 0.0f, buf[l], flags + l, ctx->s);
        }
        // P (fine rows, coarse columns): offsets from the row's linear image
        // in the coarse numbering
        if (l + 1 < ctx->nlev && L.P_col && L.nnzP > 0 && L.nc > 0) {
            ratio[l] = (float)L.nc / (float)L.n;
            TRY(alloc(ctx, &pbuf[l], (size_t)L.nnzP));
            launch_col_delta16(L.n, L.P_ptr, L.P_col, ratio[l], pbuf[l], flags + kMaxLevels + l, ctx->s);
        }
    }
    int h[2 * kMaxLevels] = {};
    CK(cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    for (int l = 0; l < ctx->nlev; ++l) {
        if (buf[l] && h[l] == 0) ctx->lev[l].A_c16 = buf[l];
        if (pbuf[l] && h[kMaxLevels + l] == 0) {
            ctx->lev[l].P_c16 = pbuf[l];
            ctx->lev[l].P_ratio = ratio[l];
        }
    }
    return AMG_OK;
}

amg_status full_setup_impl(amg_ctx *ctx, const double *d_val) {
    const amg_params &p = ctx->prm;
    free_hierarchy(ctx);
    TRY(reset_status(ctx));
    const int32_t n = ctx->n, nnz = ctx->nnz;
    Level &F = ctx->lev[0];
    F.n = n;
    F.nnz = nnz;
    F.A_ptr = ctx->fine_ptr;
    F.A_col = ctx->fine_col;
    if (ctx->fine_ncoff) {
        F.A_cidx = ctx->fine_cidx;
        F.A_coff = ctx->fine_coff;
        F.A_ncoff = ctx->fine_ncoff;
    }
    TRY(alloc(ctx, &F.A_val, (size_t)nnz));
    TRY(alloc(ctx, &F.dia, (size_t)n));
    launch_check_pattern(n, F.A_ptr, F.A_col, F.dia, ctx->d_st, ctx->s);
    launch_check_finite((int64_t)nvals(ctx), d_val, ctx->d_st, ctx->s);
    if (blockmode(ctx)) {
        // the node graph carries the block norms
        TRY(alloc(ctx, &F.Ab, nvals(ctx)));
        CK(cudaMemcpyAsync(F.Ab, d_val, sizeof(double) * nvals(ctx), cudaMemcpyDeviceToDevice, ctx->s));
        launch_block_norms(nnz, F.Ab, F.A_val, ctx->s);
    } else {
        CK(cudaMemcpyAsync(F.A_val, d_val, sizeof(double) * (size_t)nnz, cudaMemcpyDeviceToDevice, ctx->s));
    }
    TRY(check_device(ctx, "full setup input"));
    ctx->nlev = 1;
    double theta = p.theta;
    for (;;) {
        Level &L = ctx->lev[ctx->nlev - 1];
        TRY(alloc_level_vectors(ctx, L));
        TRY(alloc(ctx, &L.agg, (size_t)L.n));
        TRY(alloc(ctx, &L.strong, (size_t)L.nnz));
        CK(cudaMemsetAsync(L.agg, 0xff, sizeof(int32_t) * (size_t)L.n, ctx->s));
        CK(cudaMemsetAsync(L.strong, 0, (size_t)L.nnz, ctx->s));
        L.lpr = choose_lpr(L.n, L.nnz);
        if (L.n <= p.coarse_enough || ctx->nlev >= p.max_levels || ctx->nlev >= kMaxLevels) break;
        // strength and aggregation
        int32_t *deg = nullptr, *root_id = nullptr, *agg1 = nullptr, *root_of = nullptr;
        int8_t *state = nullptr;
        int64_t *m1 = nullptr, *scan_tmp = nullptr;
        uint8_t *r1 = nullptr;
        int *counter = nullptr;
        TRY(alloc(ctx, &deg, (size_t)L.n));
        TRY(alloc(ctx, &root_id, (size_t)L.n + 1));
        TRY(alloc(ctx, &agg1, (size_t)L.n));
        TRY(alloc(ctx, &root_of, (size_t)L.n));
        TRY(alloc(ctx, &state, (size_t)L.n));
        TRY(alloc(ctx, &m1, (size_t)L.n));
        TRY(alloc(ctx, &r1, (size_t)L.n));
        TRY(alloc(ctx, &counter, 1));
        TRY(alloc(ctx, &scan_tmp, (size_t)scan_tmp_elems(L.n)));
        launch_strength(L.n, L.A_ptr, L.A_col, L.A_val, L.dia, theta * theta, L.strong, deg, ctx->s);
        int32_t nagg = run_aggregation(L.n, L.A_ptr, L.A_col, L.A_val, L.strong, deg, L.agg, state, m1, r1, root_id,
                                       agg1, root_of, counter, ctx->d_st, scan_tmp, ctx->s);
        if (nagg < 0) {
            CK(cudaGetLastError());
            return set_err(ctx, AMG_ERR_CUDA, "aggregation did not complete");
        }
        TRY(check_device(ctx, "aggregation"));
        if (nagg == 0 || nagg >= L.n) {
            // coarsening stalls: this level becomes the coarsest
            CK(cudaMemsetAsync(L.agg, 0xff, sizeof(int32_t) * (size_t)L.n, ctx->s));
            CK(cudaMemsetAsync(L.strong, 0, (size_t)L.nnz, ctx->s));
            break;
        }
        L.nc = nagg;
        // smoothed prolongation
        int32_t *plen = nullptr;
        TRY(alloc(ctx, &plen, (size_t)L.n));
        TRY(alloc(ctx, &L.P_ptr, (size_t)L.n + 1));
        launch_p_count(L.n, L.A_ptr, L.A_col, L.strong, L.agg, p.smoothed, plen, ctx->s);
        TRY(scan(ctx, plen, L.P_ptr, L.n));
        TRY(read_scalar(ctx, L.P_ptr + L.n, &L.nnzP));
        TRY(alloc(ctx, &L.P_col, (size_t)L.nnzP));
        TRY(alloc(ctx, &L.P_val, (size_t)L.nnzP));
        launch_p_fill(L.n, L.A_ptr, L.A_col, L.A_val, L.strong, L.dia, L.agg, p.omega, p.smoothed, L.P_ptr, L.P_col,
                      L.P_val, ctx->s);
        // R = P^T
        int32_t *cnt = nullptr, *cursor = nullptr;
        TRY(alloc(ctx, &cnt, (size_t)nagg));
        TRY(alloc(ctx, &cursor, (size_t)nagg));
        CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)nagg, ctx->s));
        CK(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)nagg, ctx->s));
        launch_count_cols(L.nnzP, L.P_col, cnt, ctx->s);
        TRY(alloc(ctx, &L.R_ptr, (size_t)nagg + 1));
        TRY(scan(ctx, cnt, L.R_ptr, nagg));
        L.nnzR = L.nnzP;
        TRY(alloc(ctx, &L.R_col, (size_t)L.nnzR));
        TRY(alloc(ctx, &L.R_val, (size_t)L.nnzR));
        launch_transpose_scatter(L.n, L.P_ptr, L.P_col, L.P_val, L.R_ptr, cursor, L.R_col, L.R_val, ctx->s);
        launch_sort_rows(nagg, L.R_ptr, L.R_col, L.R_val, ctx->s);
        L.lpr_r = choose_lpr(nagg, L.nnzR);
        // symbolic Galerkin product: AP = A*P, A_c = R*AP (+ diagonal)
        TRY(symbolic_product(ctx, L.n, nagg, L.A_ptr, L.A_col, L.P_ptr, L.P_col, 0, &L.AP_ptr, &L.AP_col,
                             &L.nnzAP));
        TRY(alloc(ctx, &L.AP_val, (size_t)L.nnzAP));
        Level &C = ctx->lev[ctx->nlev];
        C.n = nagg;
        TRY(symbolic_product(ctx, nagg, nagg, L.R_ptr, L.R_col, L.AP_ptr, L.AP_col, 1, &C.A_ptr, &C.A_col, &C.nnz));
        TRY(alloc(ctx, &C.A_val, (size_t)C.nnz));
        TRY(alloc(ctx, &C.dia, (size_t)C.n));
        launch_check_pattern(C.n, C.A_ptr, C.A_col, C.dia, ctx->d_st, ctx->s);
        TRY(max_row(ctx, L.n, L.AP_ptr, &L.max_ap_row));
        TRY(max_row(ctx, C.n, C.A_ptr, &L.max_ac_row));
        if (L.max_ap_row > 65535 || L.max_ac_row > 65535)
            return set_err(ctx, AMG_ERR_CAPACITY, "Galerkin row longer than 65535 entries");
        // gather metadata: slot of every term of the two numeric stages
        int32_t *tc = nullptr;
        TRY(alloc(ctx, &tc, (size_t)std::max(L.n, nagg)));
        TRY(alloc(ctx, &L.t1ptr, (size_t)L.n + 1));
        launch_t1_count(L.n, L.A_ptr, L.A_col, L.P_ptr, tc, ctx->s);
        TRY(scan(ctx, tc, L.t1ptr, L.n));
        int32_t nt1 = 0, nt2 = 0;
        TRY(check_device(ctx, "term count"));
        TRY(read_scalar(ctx, L.t1ptr + L.n, &nt1));
        L.nt1 = nt1;
        TRY(alloc(ctx, &L.slot1, (size_t)nt1));
        launch_t1_fill(L.n, L.A_ptr, L.A_col, L.P_ptr, L.P_col, L.AP_ptr, L.AP_col, L.t1ptr, L.slot1, ctx->d_st,
                       ctx->s);
        TRY(alloc(ctx, &L.t2ptr, (size_t)nagg + 1));
        launch_t2_count(nagg, L.R_ptr, L.R_col, L.AP_ptr, tc, ctx->s);
        TRY(scan(ctx, tc, L.t2ptr, nagg));
        TRY(check_device(ctx, "term count"));
        TRY(read_scalar(ctx, L.t2ptr + nagg, &nt2));
        L.nt2 = nt2;
        TRY(alloc(ctx, &L.slot2, (size_t)nt2));
        launch_t2_fill(nagg, L.R_ptr, L.R_col, L.AP_ptr, L.AP_col, C.A_ptr, C.A_col, L.t2ptr, L.slot2, ctx->d_st,
                       ctx->s);
        // numeric values of the next level now: its strength test needs them
        if (blockmode(ctx)) {
            // coarse blocks through the gather operators, then their norms
            TRY(build_gather(ctx, ctx->nlev - 1));
            TRY(alloc(ctx, &L.APb, 16 * (size_t)L.nnzAP));
            TRY(alloc(ctx, &C.Ab, 16 * (size_t)C.nnz));
            launch_block_gather(L.nnzAP, L.g1_ptr, L.g1_idx, L.g1_w, L.Ab, L.APb, ctx->s);
            launch_block_gather(C.nnz, L.g2_ptr, L.g2_idx, L.g2_w, L.APb, C.Ab, ctx->s);
            launch_block_norms(C.nnz, C.Ab, C.A_val, ctx->s);
        } else {
            launch_ap_numeric_f64(L, L.A_val, ctx->s);
            launch_rap_numeric_f64(L, C.A_ptr, C.A_val, ctx->s);
        }
        TRY(check_device(ctx, "Galerkin product"));
        if (mixed(ctx)) {
            TRY(alloc(ctx, &L.P_valf, (size_t)L.nnzP));
            TRY(alloc(ctx, &L.R_valf, (size_t)L.nnzR));
            TRY(alloc(ctx, &L.AP_valf, (size_t)L.nnzAP));
            launch_cast_f32(L.nnzP, L.P_val, L.P_valf, ctx->s);
            launch_cast_f32(L.nnzR, L.R_val, L.R_valf, ctx->s);
        }
        ctx->nlev++;
        if (p.theta_halving) theta = theta * 0.5;
    }
    // coarsest solver storage
    Level &C = ctx->lev[ctx->nlev - 1];
    ctx->nL = C.n * p.block_size;
    const int64_t nL = ctx->nL;
    if (nL * nL > (int64_t)1 << 28)
        return set_err(ctx, AMG_ERR_CAPACITY, "coarsest level too large for a dense LU");
    TRY(alloc(ctx, &ctx->lu, (size_t)(nL * nL)));
    TRY(alloc(ctx, &ctx->inv, (size_t)(nL * nL)));
    TRY(alloc(ctx, &ctx->piv, (size_t)nL));
    ctx->luT = nullptr;
    if (lu_wants_transpose((int32_t)nL)) TRY(alloc(ctx, &ctx->luT, (size_t)(nL * nL)));
    if (mixed(ctx))
        for (int l = 1; l < ctx->nlev; ++l) launch_cast_f32(ctx->lev[l].nnz, ctx->lev[l].A_val, ctx->lev[l].A_valf, ctx->s);
    TRY(build_delta16(ctx));
    TRY(numeric_rebuild(ctx, blockmode(ctx) ? ctx->lev[0].Ab : ctx->lev[0].A_val, false));
    TRY(check_device(ctx, "full setup"));
    ctx->have_setup = true;
    ctx->setup_gen += 1;
    return AMG_OK;
}

amg_status ensure_persistent(amg_ctx *ctx, int32_t n, int32_t nnz) {
    if (ctx->fine_ptr && ctx->n == n && ctx->nnz == nnz) return AMG_OK;
    for (void *q : ctx->persist) cudaFreeAsync(q, ctx->s);
    ctx->persist.clear();
    ctx->fine_cidx = nullptr;
    ctx->fine_coff = ctx->coff_table = nullptr;
    ctx->coff_count = nullptr;
    ctx->fine_ncoff = 0;
    ctx->n = n;
    ctx->nnz = nnz;
    TRY(alloc(ctx, &ctx->fine_ptr, (size_t)n + 1, true));
    TRY(alloc(ctx, &ctx->fine_col, (size_t)nnz, true));
    const size_t nv = (size_t)nvec(ctx);
    TRY(alloc(ctx, &ctx->cg_r, nv, true));
    TRY(alloc(ctx, &ctx->cg_z, nv, true));
    TRY(alloc(ctx, &ctx->cg_p, nv, true));
    TRY(alloc(ctx, &ctx->cg_q, nv, true));
    TRY(alloc(ctx, &ctx->cg_t, nv, true));
    TRY(alloc(ctx, &ctx->cg_f, nv, true));
    TRY(alloc(ctx, &ctx->cg_u, nv, true));
    ctx->graph_valid = false;
    {
        const size_t nb = (size_t)cg_blocks((int64_t)nv);
        TRY(alloc(ctx, &ctx->partial, 5 * nb, true));
        ctx->part_pq = ctx->partial;
        ctx->part_rr = ctx->partial + nb;
        ctx->part_rz = ctx->partial + 2 * nb;
        ctx->part_rzo = ctx->partial + 3 * nb;
        ctx->part_tt = ctx->partial + 4 * nb;
    }
    TRY(alloc(ctx, &ctx->cg, 1, true));
    // the reduction counters inside must start at zero; kernels leave them zero
    CK(cudaMemsetAsync(ctx->cg, 0, sizeof(CgState), ctx->s));
    if (ctx->prm.solver == AMG_SOLVER_BICGSTAB) {
        TRY(alloc(ctx, &ctx->bi_rh, nv, true));
        TRY(alloc(ctx, &ctx->bi_s, nv, true));
        TRY(alloc(ctx, &ctx->bi_sh, nv, true));
        TRY(alloc(ctx, &ctx->bi, 1, true));
        CK(cudaMemsetAsync(ctx->bi, 0, sizeof(BiState), ctx->s));
    }
    TRY(alloc(ctx, &ctx->stage_val, nvals(ctx), true));
    TRY(alloc(ctx, &ctx->stage_f, nv, true));
    TRY(alloc(ctx, &ctx->stage_u, nv, true));
    ctx->A_sys_own = nullptr;
    if (ctx->prm.mode == AMG_MODE_FULL_REUSE) TRY(alloc(ctx, &ctx->A_sys_own, nvals(ctx), true));
    return AMG_OK;
}

// The fine pattern's compressed columns: one byte per entry naming its offset
// column - row in a table of at most kMaxColOffsets, when the rows use no
// more (a stencil's handful); otherwise fine_ncoff = 0 and the kernels read
// the int32 columns.  The values and every operation stay the same; the
// finest level's matrix kernels then move 3 bytes less per entry.
amg_status compress_pattern(amg_ctx *ctx) {
    ctx->fine_ncoff = 0;
    if (blockmode(ctx) || ctx->n >= (1 << 30)) return AMG_OK;
    if (!ctx->fine_cidx) {
        TRY(alloc(ctx, &ctx->fine_cidx, (size_t)ctx->nnz, true));
        TRY(alloc(ctx, &ctx->fine_coff, (size_t)kMaxColOffsets, true));
        TRY(alloc(ctx, &ctx->coff_table, (size_t)kColOffsetSlots, true));
        TRY(alloc(ctx, &ctx->coff_count, 1, true));
    }
    CK(cudaMemsetAsync(ctx->coff_table, 0x80, sizeof(int32_t) * kColOffsetSlots, ctx->s));
    CK(cudaMemsetAsync(ctx->coff_count, 0, sizeof(int), ctx->s));
    launch_col_offsets_collect(ctx->n, ctx->fine_ptr, ctx->fine_col, ctx->coff_table, ctx->coff_count, ctx->s);
    std::vector<int32_t> tab(kColOffsetSlots);
    int cnt = 0;
    CK(cudaMemcpyAsync(tab.data(), ctx->coff_table, sizeof(int32_t) * kColOffsetSlots, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaMemcpyAsync(&cnt, ctx->coff_count, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    if (cnt < 1 || cnt > kMaxColOffsets) return AMG_OK;
    std::vector<int32_t> off;
    for (int32_t v : tab)
        if (v != kColOffsetEmpty) off.push_back(v);
    if ((int)off.size() != cnt) return AMG_OK;
    std::sort(off.begin(), off.end());
    CK(cudaMemcpyAsync(ctx->fine_coff, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice, ctx->s));
    TRY(reset_status(ctx));
    launch_col_offsets_encode(ctx->n, ctx->fine_ptr, ctx->fine_col, ctx->fine_coff, cnt, ctx->fine_cidx, ctx->d_st,
                              ctx->s);
    TRY(check_device(ctx, "column compression"));
    ctx->fine_ncoff = cnt;
    return AMG_OK;
}

amg_status set_pattern(amg_ctx *ctx, int32_t n, int32_t nnz, const int32_t *d_ptr, const int32_t *d_col) {
    if (n <= 0 || nnz < n || !d_ptr || !d_col) return set_err(ctx, AMG_ERR_ARG, "bad matrix size or null pattern");
    TRY(ensure_persistent(ctx, n, nnz));
    if (d_ptr == ctx->fine_ptr && d_col == ctx->fine_col)
        return ctx->pattern_ok ? AMG_OK : set_err(ctx, AMG_ERR_PATTERN, "the stored pattern did not pass its checks");
    ctx->pattern_ok = false;
    CK(cudaMemcpyAsync(ctx->fine_ptr, d_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, ctx->s));
    CK(cudaMemcpyAsync(ctx->fine_col, d_col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, ctx->s));
    // the row pointers first: every later kernel reads the columns they delimit
    TRY(reset_status(ctx));
    launch_check_rowptr(n, nnz, ctx->fine_ptr, ctx->d_st, ctx->s);
    if (check_device(ctx, "row pointers") != AMG_OK)
        return set_err(ctx, AMG_ERR_PATTERN, "row pointers: not 0 at row 0, decreasing, or not ending at nnz");
    TRY(compress_pattern(ctx));
    ctx->pattern_ok = true;
    return AMG_OK;
}

// the finest level's column indices as the matrix kernels read them
ColIdx fine_cols(const amg_ctx *ctx) {
    return ColIdx{ctx->fine_col, ctx->fine_ncoff ? ctx->fine_cidx : nullptr, ctx->fine_coff, ctx->fine_ncoff,
                  ctx->nlev > 0 ? ctx->lev[0].A_c16 : nullptr};
}

void update_sys(amg_ctx *ctx) {
    ctx->A_sys = ctx->A_sys_own ? ctx->A_sys_own : blockmode(ctx) ? ctx->lev[0].Ab : ctx->lev[0].A_val;
}

// ---------------------------------------------------------------- V-cycle
template <class V>
struct Vops;
template <>
struct Vops<double> {
    static VecSet<double> &vec(Level &L) { return L.vd; }
    static const double *A(const Level &L) { return L.A_val; }
    static const double *m(const Level &L) { return L.m; }
    static const double *P(const Level &L) { return L.P_val; }
    static const double *R(const Level &L) { return L.R_val; }
};
template <>
struct Vops<float> {
    static VecSet<float> &vec(Level &L) { return L.vf; }
    static const float *A(const Level &L) { return L.A_valf; }
    static const float *m(const Level &L) { return L.mf; }
    static const float *P(const Level &L) { return L.P_valf; }
    static const float *R(const Level &L) { return L.R_valf; }
};

// pre-smoothing from a zero guess and the residual on level l (input f of type TF);
// returns the level's current iterate pointer.  u0_ready: the producer of f
// has already written the first smoothing step u = m o f into the level's u.
template <class V, class TF>
V *down_level(amg_ctx *ctx, int l, const TF *f, const int *skip, bool u0_ready) {
    Level &L = ctx->lev[l];
    VecSet<V> &v = Vops<V>::vec(L);
    const V *A = Vops<V>::A(L), *m = Vops<V>::m(L);
    const int npre = ctx->prm.npre;
    V *u = v.u, *t = v.t;
    if (npre <= 0) {
        cudaMemsetAsync(u, 0, sizeof(V) * (size_t)L.n, ctx->s);
        launch_copy_cast<TF, V>(L.n, f, v.r, skip, ctx->s);
        return u;
    }
    if (u0_ready) {
        for (int k = 1; k < npre; ++k) {
            launch_smooth_sweep<V, TF, V>(L, A, m, f, u, t, skip, ctx->s);
            std::swap(u, t);
        }
        { ProfScope ps_(ctx, AMG_PROF_SMOOTH0_L0, l == 0); launch_residual<V, TF>(L, A, f, u, v.r, skip, ctx->s); }
        return u;
    }
    { ProfScope ps_(ctx, AMG_PROF_SMOOTH0_L0, l == 0); launch_smooth0_residual<V, TF>(L, A, m, f, u, v.r, skip, ctx->s); }
    if (npre > 1) {
        for (int k = 1; k < npre; ++k) {
            launch_smooth_sweep<V, TF, V>(L, A, m, f, u, t, skip, ctx->s);
            std::swap(u, t);
        }
        launch_residual<V, TF>(L, A, f, u, v.r, skip, ctx->s);
    }
    return u;
}

// post-smoothing on the finest level; the last sweep writes z and, when
// rz_partial is given, the per-block partials of r.z (r = f here)
template <class V>
void up_finest(amg_ctx *ctx, const double *f, V *u, double *out, double *rz_partial, const int *skip) {
    Level &L = ctx->lev[0];
    VecSet<V> &v = Vops<V>::vec(L);
    const V *A = Vops<V>::A(L), *m = Vops<V>::m(L);
    V *t = (u == v.u) ? v.t : v.u;
    const int npost = ctx->prm.npost;
    for (int k = 0; k < npost; ++k) {
        if (k == npost - 1) {
            if (rz_partial) {
                ProfScope ps_(ctx, AMG_PROF_SWEEP_L0);
                launch_smooth_sweep_dot<V>(L, A, m, f, u, out, rz_partial, ctx->cg, skip, ctx->s);
            } else {
                ProfScope ps_(ctx, AMG_PROF_SWEEP_L0);
                launch_smooth_sweep<V, double, double>(L, A, m, f, u, out, skip, ctx->s);
            }
            return;
        }
        launch_smooth_sweep<V, double, V>(L, A, m, f, u, t, skip, ctx->s);
        std::swap(u, t);
    }
    launch_copy_cast<V, double>(L.n, u, out, skip, ctx->s);
    if (rz_partial) launch_dot(ctx->n, f, out, rz_partial, skip, ctx->cg, 1, ctx->s);
}

// post-smoothing on level l; the last sweep writes `out` (type TO) when given
template <class V, class TF, class TO>
void up_level(amg_ctx *ctx, int l, const TF *f, V *u, TO *out, const int *skip) {
    Level &L = ctx->lev[l];
    VecSet<V> &v = Vops<V>::vec(L);
    const V *A = Vops<V>::A(L), *m = Vops<V>::m(L);
    V *t = (u == v.u) ? v.t : v.u;
    const int npost = ctx->prm.npost;
    for (int k = 0; k < npost; ++k) {
        if (k == npost - 1 && out) {
            { ProfScope ps_(ctx, AMG_PROF_SWEEP_L0, l == 0); launch_smooth_sweep<V, TF, TO>(L, A, m, f, u, out, skip, ctx->s); }
            return;
        }
        launch_smooth_sweep<V, TF, V>(L, A, m, f, u, t, skip, ctx->s);
        std::swap(u, t);
    }
    if (out) launch_copy_cast<V, TO>(L.n, u, out, skip, ctx->s);
}

template <class V>
void enqueue_vcycle(amg_ctx *ctx, const double *r, double *z, const int *skip, double *rz_partial, bool u0_ready) {
    const int nl = ctx->nlev;
    if (nl == 1) {
        launch_coarse_solve<V, double, double>(ctx->lev[0].n, ctx->inv, r, z, skip, ctx->s);
        if (rz_partial) launch_dot(ctx->n, r, z, rz_partial, skip, ctx->cg, 1, ctx->s);
        return;
    }
    // the restriction into a smoothed level also writes that level's u0 = m o f
    const bool pre = ctx->prm.npre > 0;
    auto m_of = [&](int l) -> const V * { return (pre && l < nl - 1) ? Vops<V>::m(ctx->lev[l]) : nullptr; };
    auto u_of = [&](int l) -> V * { return (pre && l < nl - 1) ? Vops<V>::vec(ctx->lev[l]).u : nullptr; };
    V *cur[kMaxLevels];
    cur[0] = down_level<V, double>(ctx, 0, r, skip, u0_ready);
    {
        ProfScope ps_(ctx, AMG_PROF_RESTRICT_L0);
        launch_restrict<V>(ctx->lev[0], Vops<V>::R(ctx->lev[0]), Vops<V>::vec(ctx->lev[0]).r,
                           Vops<V>::vec(ctx->lev[1]).f, m_of(1), u_of(1), skip, ctx->s);
    }
    for (int l = 1; l < nl - 1; ++l) {
        Level &L = ctx->lev[l];
        cur[l] = down_level<V, V>(ctx, l, Vops<V>::vec(L).f, skip, pre);
        launch_restrict<V>(L, Vops<V>::R(L), Vops<V>::vec(L).r, Vops<V>::vec(ctx->lev[l + 1]).f, m_of(l + 1),
                           u_of(l + 1), skip, ctx->s);
    }
    Level &Cst = ctx->lev[nl - 1];
    { ProfScope ps_(ctx, AMG_PROF_COARSE, true); launch_coarse_solve<V, V, V>(Cst.n, ctx->inv, Vops<V>::vec(Cst).f, Vops<V>::vec(Cst).u, skip, ctx->s); }
    cur[nl - 1] = Vops<V>::vec(Cst).u;
    for (int l = nl - 2; l >= 1; --l) {
        Level &L = ctx->lev[l];
        launch_prolong<V>(L, Vops<V>::P(L), cur[l + 1], cur[l], skip, ctx->s);
        // the post-smoothed iterate stays in this level's buffers
        V *u = cur[l];
        VecSet<V> &v = Vops<V>::vec(L);
        V *t = (u == v.u) ? v.t : v.u;
        for (int k = 0; k < ctx->prm.npost; ++k) {
            launch_smooth_sweep<V, V, V>(L, Vops<V>::A(L), Vops<V>::m(L), v.f, u, t, skip, ctx->s);
            std::swap(u, t);
        }
        cur[l] = u;
    }
    Level &F = ctx->lev[0];
    { ProfScope ps_(ctx, AMG_PROF_PROLONG_L0, true); launch_prolong<V>(F, Vops<V>::P(F), cur[1], cur[0], skip, ctx->s); }
    up_finest<V>(ctx, r, cur[0], z, rz_partial, skip);
}

// Alg. 2 on the 4 x 4 block hierarchy (damped block Jacobi, zero initial
// guess on every level, dense inverse on the coarsest), z = B r
void enqueue_block_vcycle(amg_ctx *ctx, const double *r, double *z, const int *skip) {
    const int nl = ctx->nlev;
    const int npre = ctx->prm.npre, npost = ctx->prm.npost;
    if (nl == 1) {
        launch_coarse_solve<double, double, double>(ctx->nL, ctx->inv, r, z, skip, ctx->s);
        return;
    }
    double *cur[kMaxLevels];
    for (int l = 0; l < nl - 1; ++l) {
        Level &L = ctx->lev[l];
        const double *f = l == 0 ? r : L.vd.f;
        double *u = L.vd.u, *t = L.vd.t;
        if (npre <= 0) {
            (void)(cudaMemsetAsync(u, 0, sizeof(double) * 4 * (size_t)L.n, ctx->s));
        } else {
            { ProfScope ps_(ctx, AMG_PROF_SMOOTH0_L0, l == 0); launch_block_smooth0(L.n, L.Minv, f, u, skip, ctx->s); }
            for (int k = 1; k < npre; ++k) {
                launch_block_sweep(L.n, L.A_ptr, L.A_col, L.Ab, L.Minv, f, u, t, skip, ctx->s);
                std::swap(u, t);
            }
        }
        launch_block_residual(L.n, L.A_ptr, L.A_col, L.Ab, f, u, L.vd.r, skip, ctx->s);
        { ProfScope ps_(ctx, AMG_PROF_RESTRICT_L0, l == 0); launch_block_restrict(L.nc, L.R_ptr, L.R_col, L.R_val, L.vd.r, ctx->lev[l + 1].vd.f, skip, ctx->s); }
        cur[l] = u;
    }
    Level &Cst = ctx->lev[nl - 1];
    { ProfScope ps_(ctx, AMG_PROF_COARSE, true); launch_coarse_solve<double, double, double>(ctx->nL, ctx->inv, Cst.vd.f, Cst.vd.u, skip, ctx->s); }
    cur[nl - 1] = Cst.vd.u;
    for (int l = nl - 2; l >= 0; --l) {
        Level &L = ctx->lev[l];
        const double *f = l == 0 ? r : L.vd.f;
        { ProfScope ps_(ctx, AMG_PROF_PROLONG_L0, l == 0); launch_block_prolong(L.n, L.P_ptr, L.P_col, L.P_val, cur[l + 1], cur[l], skip, ctx->s); }
        double *u = cur[l];
        double *t = (u == L.vd.u) ? L.vd.t : L.vd.u;
        for (int k = 0; k < npost; ++k) {
            double *out = (l == 0 && k == npost - 1) ? z : t;
            { ProfScope ps_(ctx, AMG_PROF_SWEEP_L0, l == 0 && k == npost - 1); launch_block_sweep(L.n, L.A_ptr, L.A_col, L.Ab, L.Minv, f, u, out, skip, ctx->s); }
            if (out == z) { u = z; break; }
            std::swap(u, t);
        }
        if (l == 0 && u != z)
            (void)(cudaMemcpyAsync(z, u, sizeof(double) * 4 * (size_t)L.n, cudaMemcpyDeviceToDevice, ctx->s));
        cur[l] = u;
    }
}

// z = B r; with rz_partial, also the per-block partials of r.z
// u0_ready: the producer of r has written the finest level's u0 (cg_smooth0)
void vcycle(amg_ctx *ctx, const double *r, double *z, const int *skip, double *rz_partial = nullptr,
            bool u0_ready = false) {
    if (blockmode(ctx)) enqueue_block_vcycle(ctx, r, z, skip);
    else if (mixed(ctx)) enqueue_vcycle<float>(ctx, r, z, skip, rz_partial, u0_ready);
    else enqueue_vcycle<double>(ctx, r, z, skip, rz_partial, u0_ready);
}

// ---------------------------------------------------------------- CG
// CG prologue: u = 0, r = f, z = B r, p = z, rz = r.z (device state in ctx->cg)
// the CG kernels that produce r also write the V-cycle's first finest-level
// smoothing step from zero, u0 = m o r (when the V-cycle has a smoothed level)
Smooth0Out cg_smooth0(amg_ctx *ctx) {
    Smooth0Out z0;
    if (ctx->nlev < 2 || ctx->prm.npre < 1 || blockmode(ctx)) return z0;
    Level &F = ctx->lev[0];
    if (mixed(ctx)) { z0.mf = F.mf; z0.uf = F.vf.u; }
    else { z0.m = F.m; z0.u = F.vd.u; }
    return z0;
}
bool cg_u0(amg_ctx *ctx) { return ctx->nlev >= 2 && ctx->prm.npre >= 1 && !blockmode(ctx); }

void enqueue_cg_prologue(amg_ctx *ctx, const double *f, double *u, double tol) {
    const int32_t n = ctx->n;
    CgState *cg = ctx->cg;
    launch_cg_init(n, f, u, ctx->cg_r, ctx->part_rr, cg, tol, ctx->prm.maxiter, cg_smooth0(ctx), ctx->s);
    vcycle(ctx, ctx->cg_r, ctx->cg_z, &cg->done, ctx->part_rz, cg_u0(ctx));
    launch_cg_set_rz_p(n, ctx->cg_z, ctx->cg_p, cg, ctx->s);
}

// One CG iteration in three parts; every kernel returns at once when the
// state says done.  A: q = A p, alpha, u and r, the recurrence residual check.
void enqueue_cg_iter_a(amg_ctx *ctx, double *u, int use_h, cudaGraphConditionalHandle hb) {
    const int32_t n = ctx->n;
    CgState *cg = ctx->cg;
    {
        ProfScope ps_(ctx, AMG_PROF_CG_SPMV, true);
        launch_spmv_dot(n, ctx->fine_ptr, fine_cols(ctx), ctx->A_sys, ctx->cg_p, ctx->cg_q, ctx->part_pq, cg,
                        ctx->s);
    }
    {
        ProfScope ps_(ctx, AMG_PROF_CG_UPDATE, true);
        // flexible variant: r_new.z_old in the same pass (z still holds the last z)
        const bool flex = mixed(ctx);
        launch_cg_update_ur(n, cg, ctx->cg_p, ctx->cg_q, u, ctx->cg_r, ctx->part_rr, flex ? ctx->cg_z : nullptr,
                            ctx->part_rzo, use_h, hb, cg_smooth0(ctx), ctx->s);
    }
}

// B: only when the recurrence met the tolerance: the true residual, and r
// replaced by it if it misses
void enqueue_cg_iter_b(amg_ctx *ctx, const double *f, double *u) {
    const int32_t n = ctx->n;
    CgState *cg = ctx->cg;
    launch_true_residual(n, ctx->fine_ptr, fine_cols(ctx), ctx->A_sys, f, u, ctx->cg_t, ctx->part_tt,
                         cg, 0, ctx->s);
    launch_replace_r(n, cg, ctx->cg_t, ctx->cg_r, mixed(ctx) ? ctx->cg_z : nullptr, ctx->part_rzo, cg_smooth0(ctx),
                     ctx->s);
}

// C: z = B r with the partials of r.z, beta and p (and the loop condition)
void enqueue_cg_iter_c(amg_ctx *ctx, int use_h, cudaGraphConditionalHandle h) {
    const int32_t n = ctx->n;
    CgState *cg = ctx->cg;
    // (the flexible variant's r_new.z_old was formed by the u / r update)
    vcycle(ctx, ctx->cg_r, ctx->cg_z, &cg->done, ctx->part_rz, cg_u0(ctx));
    {
        ProfScope ps_(ctx, AMG_PROF_CG_P, true);
        launch_cg_update_p(n, cg, ctx->cg_z, ctx->cg_p, use_h, h, ctx->s);
    }
}

// the true relative residual of the returned iterate
void enqueue_cg_epilogue(amg_ctx *ctx, const double *f, double *u) {
    const int32_t n = ctx->n;
    launch_true_residual(n, ctx->fine_ptr, fine_cols(ctx), ctx->A_sys, f, u, ctx->cg_t, ctx->part_tt,
                         ctx->cg, 1,
                         ctx->s);
}

void drop_graph(amg_ctx *ctx) {
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->graph_exec = nullptr;
    ctx->graph = nullptr;
}

// add a conditional node after the current capture dependencies of stream s
// and make it the stream's only dependency; returns its body graph
cudaError_t add_conditional(cudaStream_t s, cudaGraphConditionalNodeType type, unsigned def,
                            cudaGraphConditionalHandle *h, cudaGraphNode_t *node, cudaGraph_t *body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return e;
    e = cudaGraphConditionalHandleCreate(h, g, def, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = *h;
    cp.conditional.type = type;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(node, g, deps, nullptr, ndeps, &cp);
    if (e != cudaSuccess) return e;
    *body = cp.conditional.phGraph_out[0];
    return cudaSuccess;
}

// The whole solve as one graph: prologue, a WHILE conditional node whose body
// is one CG iteration (its last kernel sets the loop condition), epilogue.
// Inside the body, the true-residual branch sits in an IF conditional node
// that the convergence check opens.  It works on the context's own f / u
// buffers, so it stays valid until the hierarchy or the tolerance changes.
// Capture runs on private streams (the caller's stream may be the legacy
// default stream, which cannot be captured); the graph is launched on the
// caller's stream.
amg_status build_solve_graph(amg_ctx *ctx, double tol) {
    drop_graph(ctx);
    CK(cudaStreamSynchronize(ctx->s));
    cudaStream_t user_s = ctx->s;
    const double *f = ctx->cg_f;
    double *u = ctx->cg_u;
    const int64_t c0 = launch_total();
    int64_t c1 = c0, c2 = c0;
    CK(cudaStreamBeginCapture(ctx->s_cap_main, cudaStreamCaptureModeThreadLocal));
    ctx->s = ctx->s_cap_main;
    enqueue_cg_prologue(ctx, f, u, tol);
    c1 = launch_total();
    cudaGraphConditionalHandle h_loop = 0, h_true = 0;
    cudaGraphNode_t loop_node = nullptr, if_node = nullptr;
    cudaGraph_t body = nullptr, tbody = nullptr;
    cudaError_t e = add_conditional(ctx->s_cap_main, cudaGraphCondTypeWhile, 1, &h_loop, &loop_node, &body);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(ctx->s_cap, body, nullptr, nullptr, 0,
                                                            cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        ctx->s = ctx->s_cap;
        const int64_t ca = launch_total();
        // the IF handle belongs to the body graph; the check kernel sets it
        cudaError_t eh = cudaGraphConditionalHandleCreate(&h_true, body, 0, cudaGraphCondAssignDefault);
        if (eh == cudaSuccess) {
            enqueue_cg_iter_a(ctx, u, 1, h_true);
            cudaStreamCaptureStatus cs;
            cudaGraph_t g = nullptr;
            const cudaGraphNode_t *deps = nullptr;
            size_t ndeps = 0;
            eh = cudaStreamGetCaptureInfo(ctx->s_cap, &cs, nullptr, &g, &deps, nullptr, &ndeps);
            cudaGraphNodeParams cp = {};
            if (eh == cudaSuccess) {
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = h_true;
                cp.conditional.type = cudaGraphCondTypeIf;
                cp.conditional.size = 1;
                eh = cudaGraphAddNode(&if_node, g, deps, nullptr, ndeps, &cp);
            }
            if (eh == cudaSuccess) {
                tbody = cp.conditional.phGraph_out[0];
                eh = cudaStreamBeginCaptureToGraph(ctx->s_cap_if, tbody, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeThreadLocal);
            }
            if (eh == cudaSuccess) {
                ctx->s = ctx->s_cap_if;
                const int64_t cb = launch_total();
                enqueue_cg_iter_b(ctx, f, u);
                // the branch runs only in some iterations: counted when it does
                ctx->graph_branch = launch_total() - cb;
                ctx->s = ctx->s_cap;
                cudaGraph_t tmp = nullptr;
                eh = cudaStreamEndCapture(ctx->s_cap_if, &tmp);
            }
            if (eh == cudaSuccess)
                eh = cudaStreamUpdateCaptureDependencies(ctx->s_cap, &if_node, nullptr, 1,
                                                         cudaStreamSetCaptureDependencies);
            if (eh == cudaSuccess) enqueue_cg_iter_c(ctx, 1, h_loop);
        }
        c2 = launch_total() - ctx->graph_branch;
        (void)ca;
        ctx->s = ctx->s_cap_main;
        cudaGraph_t tmp = nullptr;
        e = cudaStreamEndCapture(ctx->s_cap, &tmp);
        if (e == cudaSuccess) e = eh;
    }
    if (e == cudaSuccess)
        e = cudaStreamUpdateCaptureDependencies(ctx->s_cap_main, &loop_node, nullptr, 1,
                                                cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) enqueue_cg_epilogue(ctx, f, u);
    const int64_t c3 = launch_total();
    // captured launches do not run now: they are counted when the graph runs
    add_launches(c0 - c3);
    ctx->graph_pro = c1 - c0;
    ctx->graph_body = (c2 - c1);
    ctx->graph_epi = c3 - c2 - ctx->graph_branch;
    ctx->s = user_s;
    cudaGraph_t done_graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(ctx->s_cap_main, &done_graph);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        if (done_graph) cudaGraphDestroy(done_graph);
        cudaGetLastError();
        return set_err(ctx, AMG_ERR_CUDA, std::string("building the solve graph: ") + cudaGetErrorString(e));
    }
    ctx->graph = done_graph;
    CK(cudaGraphInstantiate(&ctx->graph_exec, ctx->graph, 0));
    ctx->graph_tol = tol;
    ctx->graph_valid = true;
    return AMG_OK;
}

amg_status finish_solve(amg_ctx *ctx, amg_info *info) {
    CK(cudaMemcpyAsync(ctx->h_cg, ctx->cg, sizeof(CgState), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    CK(cudaGetLastError());
    const CgState &h = *ctx->h_cg;
    amg_status st = (amg_status)h.status;
    if (!h.done && st == AMG_OK) st = AMG_NOT_CONVERGED;
    ctx->last_iters = h.iter;
    ctx->last_status = st;
    if (ctx->iters_after_full < 0 && st == AMG_OK) ctx->iters_after_full = h.iter;
    if (info) {
        info->iters = h.iter;
        info->rel_resid = h.tres;
        info->status = st;
        info->rebuilt = ctx->last_rebuilt;
        info->nlevels = ctx->nlev;
    }
    if (st == AMG_ERR_BREAKDOWN) set_err(ctx, st, "CG breakdown: p'Ap <= 0 or not finite");
    else if (st == AMG_NOT_CONVERGED) set_err(ctx, st, "CG reached maxiter");
    return st;
}

// ---------------------------------------------------------------- BiCGStab
// Right-preconditioned BiCGStab (Sec. 4, the level-set systems): per
// iteration p^ = B p and s^ = B s, one V-cycle each.  Vectors: r = cg_r,
// p = cg_p, p^ = cg_z, v = cg_q, t = cg_t, with r^, s, s^ of their own.  The
// second half of an iteration skips itself (state flag `skip`) when |s|
// already meets the tolerance, and the true-residual check skips itself
// unless the recurrence reports convergence.
void enqueue_bi_prologue(amg_ctx *ctx, const double *f, double *u, double tol) {
    launch_bi_init((int32_t)nvec(ctx), f, u, ctx->cg_r, ctx->bi_rh, ctx->cg_p, ctx->cg_q, ctx->partial, ctx->bi, tol,
                   ctx->prm.maxiter, ctx->s);
}

void enqueue_bi_iter(amg_ctx *ctx, const double *f, double *u, int use_h, cudaGraphConditionalHandle h) {
    const int32_t n = (int32_t)nvec(ctx);
    const int bs = ctx->prm.block_size;
    BiState *st = ctx->bi;
    double *part = ctx->partial;
    launch_bi_rho(n, ctx->bi_rh, ctx->cg_r, part, st, ctx->s);
    launch_bi_p(n, ctx->cg_r, ctx->cg_q, ctx->cg_p, st, ctx->s);
    vcycle(ctx, ctx->cg_p, ctx->cg_z, &st->done);
    launch_bi_spmv_rv(n, bs, ctx->fine_ptr, ctx->fine_col, ctx->A_sys, ctx->cg_z, ctx->cg_q, ctx->bi_rh, part, st, ctx->s);
    launch_bi_s(n, ctx->cg_r, ctx->cg_q, ctx->bi_s, part, st, ctx->s);
    launch_bi_half(n, ctx->cg_z, ctx->bi_s, u, ctx->cg_r, st, ctx->s);
    vcycle(ctx, ctx->bi_s, ctx->bi_sh, &st->skip);
    launch_bi_spmv_t(n, bs, ctx->fine_ptr, ctx->fine_col, ctx->A_sys, ctx->bi_sh, ctx->bi_s, ctx->cg_t, part, st, ctx->s);
    launch_bi_xr(n, ctx->cg_z, ctx->bi_sh, ctx->bi_s, ctx->cg_t, u, ctx->cg_r, part, st, ctx->s);
    launch_bi_true(n, bs, ctx->fine_ptr, ctx->fine_col, ctx->A_sys, f, u, ctx->cg_t, part, st, 0, ctx->s);
    launch_bi_replace(n, ctx->cg_t, ctx->cg_r, st, ctx->s);
    launch_bi_end(st, use_h, h, ctx->s);
}

void enqueue_bi_epilogue(amg_ctx *ctx, const double *f, double *u) {
    launch_bi_true((int32_t)nvec(ctx), ctx->prm.block_size, ctx->fine_ptr, ctx->fine_col, ctx->A_sys, f, u, ctx->cg_t, ctx->partial, ctx->bi, 1,
                   ctx->s);
}

// the whole BiCGStab solve as one graph: prologue, a WHILE node over one
// iteration (its last kernel sets the loop condition), epilogue
amg_status build_bi_graph(amg_ctx *ctx, double tol) {
    drop_graph(ctx);
    CK(cudaStreamSynchronize(ctx->s));
    cudaStream_t user_s = ctx->s;
    const double *f = ctx->cg_f;
    double *u = ctx->cg_u;
    const int64_t c0 = launch_total();
    int64_t c1 = c0, c2 = c0;
    CK(cudaStreamBeginCapture(ctx->s_cap_main, cudaStreamCaptureModeThreadLocal));
    ctx->s = ctx->s_cap_main;
    enqueue_bi_prologue(ctx, f, u, tol);
    c1 = launch_total();
    cudaGraphConditionalHandle h_loop = 0;
    cudaGraphNode_t loop_node = nullptr;
    cudaGraph_t body = nullptr;
    cudaError_t e = add_conditional(ctx->s_cap_main, cudaGraphCondTypeWhile, 1, &h_loop, &loop_node, &body);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(ctx->s_cap, body, nullptr, nullptr, 0,
                                                            cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        ctx->s = ctx->s_cap;
        enqueue_bi_iter(ctx, f, u, 1, h_loop);
        c2 = launch_total();
        ctx->s = ctx->s_cap_main;
        cudaGraph_t tmp = nullptr;
        e = cudaStreamEndCapture(ctx->s_cap, &tmp);
    }
    if (e == cudaSuccess)
        e = cudaStreamUpdateCaptureDependencies(ctx->s_cap_main, &loop_node, nullptr, 1,
                                                cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) enqueue_bi_epilogue(ctx, f, u);
    const int64_t c3 = launch_total();
    add_launches(c0 - c3);
    ctx->graph_pro = c1 - c0;
    ctx->graph_body = c2 - c1;
    ctx->graph_epi = c3 - c2;
    ctx->graph_branch = 0;
    ctx->s = user_s;
    cudaGraph_t done_graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(ctx->s_cap_main, &done_graph);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        if (done_graph) cudaGraphDestroy(done_graph);
        cudaGetLastError();
        return set_err(ctx, AMG_ERR_CUDA, std::string("building the BiCGStab graph: ") + cudaGetErrorString(e));
    }
    ctx->graph = done_graph;
    CK(cudaGraphInstantiate(&ctx->graph_exec, ctx->graph, 0));
    ctx->graph_tol = tol;
    ctx->graph_valid = true;
    return AMG_OK;
}

amg_status finish_bi(amg_ctx *ctx, amg_info *info) {
    CK(cudaMemcpyAsync(ctx->h_bi, ctx->bi, sizeof(BiState), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    CK(cudaGetLastError());
    const BiState &h = *ctx->h_bi;
    amg_status st = (amg_status)h.status;
    if (!h.done && st == AMG_OK) st = AMG_NOT_CONVERGED;
    ctx->last_iters = h.iter;
    ctx->last_status = st;
    if (ctx->iters_after_full < 0 && st == AMG_OK) ctx->iters_after_full = h.iter;
    if (info) {
        info->iters = h.iter;
        info->rel_resid = h.tres;
        info->status = st;
        info->rebuilt = ctx->last_rebuilt;
        info->nlevels = ctx->nlev;
    }
    if (st == AMG_ERR_BREAKDOWN) set_err(ctx, st, "BiCGStab breakdown: a zero or non-finite scalar");
    else if (st == AMG_NOT_CONVERGED) set_err(ctx, st, "BiCGStab reached maxiter");
    return st;
}

amg_status solve_bi(amg_ctx *ctx, const double *f, double *u, double tol, amg_info *info) {
    const int64_t n = nvec(ctx);
    if (ctx->use_graph && !ctx->prof.on) {
        if (!ctx->graph_valid || ctx->graph_tol != tol) TRY(build_bi_graph(ctx, tol));
        CK(cudaMemcpyAsync(ctx->cg_f, f, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->s));
        CK(cudaGraphLaunch(ctx->graph_exec, ctx->s));
        CK(cudaMemcpyAsync(u, ctx->cg_u, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->s));
        amg_status st = finish_bi(ctx, info);
        add_launches(ctx->graph_pro + ctx->graph_epi + ctx->graph_body * (int64_t)ctx->h_bi->pad);
        return st;
    }
    enqueue_bi_prologue(ctx, f, u, tol);
    for (int it = 1; it <= ctx->prm.maxiter; ++it) {
        enqueue_bi_iter(ctx, f, u, 0, 0);
        CK(cudaMemcpyAsync(ctx->h_bi, ctx->bi, sizeof(BiState), cudaMemcpyDeviceToHost, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        if (ctx->h_bi->done) break;
    }
    enqueue_bi_epilogue(ctx, f, u);
    return finish_bi(ctx, info);
}

amg_status solve_impl(amg_ctx *ctx, const double *f, double *u, double tol, amg_info *info);

// Per-kernel timing of a CG solve (amg_profile on).  The host-driven loop
// leaves the GPU waiting for the next launch between short kernels, which
// would inflate every timed launch; instead the solve first runs unprofiled
// (the whole-solve graph) to learn its iteration count K, then once more as
// one straight-line graph of K iterations whose event-record nodes bracket
// the timed kernels (the last iteration, whose preconditioner kernels return
// at once, is not timed); every timed iteration also brackets nothing, which
// measures the overhead of an event pair in the graph (slot AMG_PROF_EMPTY).
// Both runs compute the same iterates.
amg_status solve_cg_profiled(amg_ctx *ctx, const double *f, double *u, double tol, amg_info *info) {
    ctx->prof.on = false;
    amg_status st = solve_impl(ctx, f, u, tol, nullptr);
    ctx->prof.on = true;
    if (st != AMG_OK && st != AMG_NOT_CONVERGED) return st;
    const int K = ctx->h_cg->iter;
    CK(cudaStreamSynchronize(ctx->s));
    cudaStream_t user_s = ctx->s;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    CK(cudaStreamBeginCapture(ctx->s_cap_main, cudaStreamCaptureModeThreadLocal));
    ctx->s = ctx->s_cap_main;
    enqueue_cg_prologue(ctx, f, u, tol);
    for (int it = 1; it <= K; ++it) {
        if (it == K) ctx->prof.on = false;
        { ProfScope cal_(ctx, AMG_PROF_EMPTY, true); }  // two adjacent event nodes: the timing overhead
        enqueue_cg_iter_a(ctx, u, 0, 0);
        enqueue_cg_iter_b(ctx, f, u);
        enqueue_cg_iter_c(ctx, 0, 0);
    }
    ctx->prof.on = true;
    enqueue_cg_epilogue(ctx, f, u);
    ctx->s = user_s;
    cudaError_t e = cudaStreamEndCapture(ctx->s_cap_main, &g);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, ctx->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->s);
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, AMG_ERR_CUDA, std::string("profiled solve graph: ") + cudaGetErrorString(e));
    }
    return finish_solve(ctx, info);
}

amg_status solve_impl(amg_ctx *ctx, const double *f, double *u, double tol, amg_info *info) {
    const int32_t n = ctx->n;
    if (ctx->prm.solver == AMG_SOLVER_BICGSTAB) return solve_bi(ctx, f, u, tol, info);
    if (ctx->prof.on && !ctx->prof.eager && ctx->use_graph) return solve_cg_profiled(ctx, f, u, tol, info);
    if (ctx->use_graph && !ctx->prof.on) {
        if (!ctx->graph_valid || ctx->graph_tol != tol) TRY(build_solve_graph(ctx, tol));
        CK(cudaMemcpyAsync(ctx->cg_f, f, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->s));
        CK(cudaGraphLaunch(ctx->graph_exec, ctx->s));
        CK(cudaMemcpyAsync(u, ctx->cg_u, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->s));
        amg_status st = finish_solve(ctx, info);
        // bodies executed = completed p updates plus the final (returning) pass;
        // the true-residual branch ran in 1 + replacements bodies when it converged
        const CgState &hc = *ctx->h_cg;
        const int64_t bodies = (int64_t)hc.pad + 1;
        const int64_t branches = (hc.status == AMG_OK && hc.iter > 0) ? 1 + hc.replacements : hc.replacements;
        add_launches(ctx->graph_pro + ctx->graph_epi + ctx->graph_body * bodies + ctx->graph_branch * branches);
        return st;
    }
    // eager path: the host checks the device state after every iteration
    enqueue_cg_prologue(ctx, f, u, tol);
    for (int it = 1; it <= ctx->prm.maxiter; ++it) {
        enqueue_cg_iter_a(ctx, u, 0, 0);
        enqueue_cg_iter_b(ctx, f, u);
        enqueue_cg_iter_c(ctx, 0, 0);
        CK(cudaMemcpyAsync(ctx->h_cg, ctx->cg, sizeof(CgState), cudaMemcpyDeviceToHost, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        if (ctx->h_cg->done) break;
    }
    enqueue_cg_epilogue(ctx, f, u);
    return finish_solve(ctx, info);
}

}  // namespace

// ======================================================================= C ABI
extern "C" {

amg_status amg_default_params(amg_params *prm) {
    if (!prm) return AMG_ERR_ARG;
    prm->theta = 0.08;
    prm->omega = 2.0 / 3.0;
    prm->jacobi_omega = 0.72;
    prm->smoother = AMG_SMOOTHER_SPAI0;
    prm->npre = 1;
    prm->npost = 1;
    prm->coarse_enough = 256;
    prm->max_levels = 20;
    prm->theta_halving = 1;
    prm->smoothed = 1;
    prm->precision = AMG_PREC_FP64;
    prm->mode = AMG_MODE_PARTIAL;
    prm->reuse_iter_limit = 100;
    prm->maxiter = 100;
    prm->rebuild_every = 0;
    prm->rebuild_iter_growth = 0.0;
    prm->solver = AMG_SOLVER_CG;
    prm->block_size = 1;
    return AMG_OK;
}

amg_status amg_create(amg_ctx **out, const amg_params *prm, void *cuda_stream) {
    if (!out) return AMG_ERR_ARG;
    *out = nullptr;
    amg_params p;
    if (prm) p = *prm;
    else amg_default_params(&p);
    if (p.npre < 0 || p.npost < 0 || p.max_levels < 1 || p.coarse_enough < 1 || p.maxiter < 0 ||
        (p.smoother != AMG_SMOOTHER_SPAI0 && p.smoother != AMG_SMOOTHER_JACOBI) ||
        (p.precision != AMG_PREC_FP64 && p.precision != AMG_PREC_MIXED) || p.mode < 0 || p.mode > 2 ||
        p.rebuild_every < 0 || !(p.rebuild_iter_growth >= 0.0) ||
        (p.solver != AMG_SOLVER_CG && p.solver != AMG_SOLVER_BICGSTAB) ||
        (p.block_size != 1 && p.block_size != 4) ||
        (p.block_size == 4 && (p.smoothed != 0 || p.smoother != AMG_SMOOTHER_JACOBI ||
                               p.precision != AMG_PREC_FP64 || p.solver != AMG_SOLVER_BICGSTAB)) ||
        !(p.theta >= 0.0) || !std::isfinite(p.omega))
        return AMG_ERR_ARG;
    amg_ctx *ctx = new amg_ctx();
    ctx->prm = p;
    ctx->s = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    if (cudaGetDevice(&dev) != cudaSuccess) { delete ctx; return AMG_ERR_CUDA; }
    props.location.id = dev;
    if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess) { delete ctx; return AMG_ERR_CUDA; }
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (cudaStreamCreateWithFlags(&ctx->s_cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->s_cap_main, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->s_cap_if, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->s_copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_vals, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_f, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&ctx->h_cg, sizeof(CgState)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_bi, sizeof(BiState)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_st, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&ctx->d_st, sizeof(int)) != cudaSuccess) {
        amg_destroy(ctx);
        return AMG_ERR_CUDA;
    }
    for (cudaEvent_t &e : ctx->ev_chunk)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            amg_destroy(ctx);
            return AMG_ERR_CUDA;
        }
    *out = ctx;
    return AMG_OK;
}

void amg_destroy(amg_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->s);
    for (void *p : ctx->hier) cudaFreeAsync(p, ctx->s);
    for (void *p : ctx->persist) cudaFreeAsync(p, ctx->s);
    cudaStreamSynchronize(ctx->s);
    drop_graph(ctx);
    if (ctx->s_cap) cudaStreamDestroy(ctx->s_cap);
    if (ctx->s_cap_main) cudaStreamDestroy(ctx->s_cap_main);
    if (ctx->s_cap_if) cudaStreamDestroy(ctx->s_cap_if);
    if (ctx->s_copy) {
        cudaStreamSynchronize(ctx->s_copy);
        cudaStreamDestroy(ctx->s_copy);
    }
    if (ctx->ev_vals) cudaEventDestroy(ctx->ev_vals);
    if (ctx->ev_f) cudaEventDestroy(ctx->ev_f);
    for (cudaEvent_t e : ctx->ev_chunk)
        if (e) cudaEventDestroy(e);
    for (auto &v : ctx->prof.rec)
        for (auto &pr : v) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->h_cg) cudaFreeHost(ctx->h_cg);
    if (ctx->h_bi) cudaFreeHost(ctx->h_bi);
    if (ctx->h_st) cudaFreeHost(ctx->h_st);
    if (ctx->d_st) cudaFree(ctx->d_st);
    delete ctx;
}

const char *amg_last_error(const amg_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

amg_status amg_full_setup(amg_ctx *ctx, int32_t n, int32_t nnz, const int32_t *d_ptr, const int32_t *d_col,
                          const double *d_val) {
    if (!ctx) return AMG_ERR_ARG;
    if (!d_val) return set_err(ctx, AMG_ERR_ARG, "null values");
    amg_status st = set_pattern(ctx, n, nnz, d_ptr, d_col);
    if (st != AMG_OK) {
        // the stored pattern was replaced: no hierarchy refers to it any more
        free_hierarchy(ctx);
        return st;
    }
    st = full_setup_impl(ctx, d_val);
    if (st != AMG_OK) {
        free_hierarchy(ctx);
        return st;
    }
    if (ctx->A_sys_own)
        CK(cudaMemcpyAsync(ctx->A_sys_own, d_val, sizeof(double) * nvals(ctx), cudaMemcpyDeviceToDevice, ctx->s));
    update_sys(ctx);
    ctx->last_rebuilt = 1;
    ctx->steps_since_full = 0;
    ctx->iters_after_full = -1;
    return AMG_OK;
}

namespace {
// the partial-mode step takes a preventive full setup (every rebuild_every
// steps, or when the last solve took rebuild_iter_growth times the iterations
// of the first solve after the last full setup)
bool preventive_rebuild_due(const amg_ctx *ctx) {
    const amg_params &p = ctx->prm;
    const bool regular = p.rebuild_every > 0 && ctx->steps_since_full + 1 >= p.rebuild_every;
    const bool growth = p.rebuild_iter_growth > 0.0 && ctx->iters_after_full > 0 &&
                        ctx->last_iters > p.rebuild_iter_growth * ctx->iters_after_full;
    return regular || growth;
}

amg_status partial_rebuild_impl(amg_ctx *ctx, const double *d_val, const FineChunks *ck) {
    TRY(reset_status(ctx));
    if (ctx->use_gather)
        for (int l = 0; l + 1 < ctx->nlev; ++l)
            if (!ctx->lev[l].gather_ready) TRY(build_gather(ctx, l));
    TRY(numeric_rebuild(ctx, d_val, true, ck));
    if (ctx->A_sys_own)
        CK(cudaMemcpyAsync(ctx->A_sys_own, d_val, sizeof(double) * nvals(ctx), cudaMemcpyDeviceToDevice,
                           ctx->s));
    TRY(check_device(ctx, "partial rebuild"));
    update_sys(ctx);
    ctx->last_rebuilt = 0;
    ctx->steps_since_full += 1;
    return AMG_OK;
}

// whether the host-buffer step can take its values in chunks: a partial
// rebuild (no preventive full setup due) of a scalar hierarchy whose gather
// operators exist, with per-kernel timing off
bool host_chunks_ok(const amg_ctx *ctx) {
    if (!ctx->have_setup || blockmode(ctx) || ctx->prof.on || ctx->prm.mode != AMG_MODE_PARTIAL || !ctx->use_gather ||
        preventive_rebuild_due(ctx))
        return false;
    for (int l = 0; l + 1 < ctx->nlev; ++l)
        if (!ctx->lev[l].gather_ready) return false;
    return true;
}

// chunk boundaries: rows (multiples of 32), their first value and their first
// entry of the finest A P, read once per hierarchy
amg_status prepare_chunks(amg_ctx *ctx) {
    if (ctx->ck_gen == ctx->setup_gen) return AMG_OK;
    const int32_t n = ctx->n;
    for (int c = 0; c < kHostChunks; ++c) ctx->ck_row[c] = (int32_t)(((int64_t)n * c / kHostChunks) & ~(int64_t)31);
    ctx->ck_row[kHostChunks] = n;
    const bool ap = ctx->nlev > 1 && ctx->lev[0].AP_ptr;
    for (int c = 0; c <= kHostChunks; ++c) {
        CK(cudaMemcpyAsync(&ctx->ck_e[c], ctx->fine_ptr + ctx->ck_row[c], sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->s));
        if (ap)
            CK(cudaMemcpyAsync(&ctx->ck_ap[c], ctx->lev[0].AP_ptr + ctx->ck_row[c], sizeof(int32_t),
                               cudaMemcpyDeviceToHost, ctx->s));
        else ctx->ck_ap[c] = 0;
    }
    CK(cudaStreamSynchronize(ctx->s));
    // coarse boundaries: the leading coarse rows whose R rows (sorted by fine
    // row) end before the chunk's last row, from the prefix maximum of each R
    // row's last column
    for (int c = 0; c <= kHostChunks; ++c) ctx->ck_crow[c] = ctx->ck_ac[c] = 0;
    if (ap) {
        const Level &L = ctx->lev[0];
        const int32_t nc = L.nc;
        std::vector<int32_t> last((size_t)nc, -1);
        int32_t *d_last = nullptr;
        TRY(alloc(ctx, &d_last, (size_t)nc));
        launch_row_last(nc, L.R_ptr, L.R_col, d_last, ctx->s);
        CK(cudaMemcpyAsync(last.data(), d_last, sizeof(int32_t) * (size_t)nc, cudaMemcpyDeviceToHost, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        int32_t I = 0, pmax = -1;
        for (int c = 1; c <= kHostChunks; ++c) {
            const int32_t lim = ctx->ck_row[c];  // rows before this have landed with chunks 0 .. c - 1
            while (I < nc && std::max(pmax, last[I]) < lim) pmax = std::max(pmax, last[(size_t)I++]);
            ctx->ck_crow[c] = c == kHostChunks ? nc : I;
        }
        for (int c = 0; c <= kHostChunks; ++c)
            CK(cudaMemcpyAsync(&ctx->ck_ac[c], ctx->lev[1].A_ptr + ctx->ck_crow[c], sizeof(int32_t),
                               cudaMemcpyDeviceToHost, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
    }
    ctx->ck_gen = ctx->setup_gen;
    return AMG_OK;
}
}  // namespace

amg_status amg_partial_rebuild(amg_ctx *ctx, const double *d_val) {
    if (!ctx) return AMG_ERR_ARG;
    if (!ctx->have_setup) return set_err(ctx, AMG_ERR_STATE, "partial rebuild before a full setup");
    if (!d_val) return set_err(ctx, AMG_ERR_ARG, "null values");
    return partial_rebuild_impl(ctx, d_val, nullptr);
}

amg_status amg_step(amg_ctx *ctx, int32_t n, int32_t nnz, const int32_t *d_ptr, const int32_t *d_col,
                    const double *d_val, amg_info *info) {
    if (!ctx) return AMG_ERR_ARG;
    if (!d_val) return set_err(ctx, AMG_ERR_ARG, "null values");
    if (ctx->have_setup && (n != ctx->n || nnz != ctx->nnz))
        return set_err(ctx, AMG_ERR_ARG, "size differs from the pattern of the first step");
    amg_status st = AMG_OK;
    const int mode = ctx->prm.mode;
    if (!ctx->have_setup) {
        st = amg_full_setup(ctx, n, nnz, d_ptr, d_col, d_val);
    } else if (mode == AMG_MODE_PARTIAL) {
        if (preventive_rebuild_due(ctx)) {
            st = full_setup_impl(ctx, d_val);
            if (st == AMG_OK) {
                update_sys(ctx);
                ctx->last_rebuilt = 1;
                ctx->steps_since_full = 0;
                ctx->iters_after_full = -1;
            } else {
                free_hierarchy(ctx);
            }
        } else {
            st = amg_partial_rebuild(ctx, d_val);
        }
    } else if (mode == AMG_MODE_FULL_REBUILD) {
        st = full_setup_impl(ctx, d_val);
        if (st == AMG_OK) { update_sys(ctx); ctx->last_rebuilt = 1; }
        else free_hierarchy(ctx);
    } else {
        bool rebuild = ctx->last_status != AMG_OK || ctx->last_iters > ctx->prm.reuse_iter_limit;
        if (rebuild) {
            st = full_setup_impl(ctx, d_val);
            if (st != AMG_OK) free_hierarchy(ctx);
        }
        if (st == AMG_OK) {
            CK(cudaMemcpyAsync(ctx->A_sys_own, d_val, sizeof(double) * nvals(ctx), cudaMemcpyDeviceToDevice,
                               ctx->s));
            update_sys(ctx);
            ctx->last_rebuilt = rebuild ? 1 : 0;
        }
    }
    if (info) {
        info->rebuilt = ctx->last_rebuilt;
        info->nlevels = ctx->nlev;
    }
    return st;
}

amg_status amg_solve(amg_ctx *ctx, const double *d_f, double *d_u, double tol, amg_info *info) {
    if (!ctx) return AMG_ERR_ARG;
    if (!ctx->have_setup) return set_err(ctx, AMG_ERR_STATE, "solve before a setup");
    if (!d_f || !d_u || !(tol >= 0.0)) return set_err(ctx, AMG_ERR_ARG, "null vector or bad tolerance");
    return solve_impl(ctx, d_f, d_u, tol, info);
}

amg_status amg_apply_vcycle(amg_ctx *ctx, const double *d_r, double *d_z) {
    if (!ctx) return AMG_ERR_ARG;
    if (!ctx->have_setup) return set_err(ctx, AMG_ERR_STATE, "V-cycle before a setup");
    if (!d_r || !d_z) return set_err(ctx, AMG_ERR_ARG, "null vector");
    if (blockmode(ctx)) {
        // the block kernels load 16-byte pairs: run on the context's own vectors
        const size_t bytes = sizeof(double) * (size_t)nvec(ctx);
        CK(cudaMemcpyAsync(ctx->cg_r, d_r, bytes, cudaMemcpyDeviceToDevice, ctx->s));
        vcycle(ctx, ctx->cg_r, ctx->cg_z, nullptr);
        CK(cudaMemcpyAsync(d_z, ctx->cg_z, bytes, cudaMemcpyDeviceToDevice, ctx->s));
    } else {
        vcycle(ctx, d_r, d_z, nullptr);
    }
    CK(cudaStreamSynchronize(ctx->s));
    CK(cudaGetLastError());
    return AMG_OK;
}

amg_status amg_step_solve_host(amg_ctx *ctx, const double *h_val, const double *h_f, double *h_u, double tol,
                               amg_info *info) {
    if (!ctx) return AMG_ERR_ARG;
    if (!ctx->fine_ptr) return set_err(ctx, AMG_ERR_STATE, "no pattern: call amg_full_setup or amg_step first");
    if (!h_val || !h_f || !h_u) return set_err(ctx, AMG_ERR_ARG, "null host buffer");
    // the caller's buffers stay in use until their copies end: an early
    // return waits for both streams
    auto drain = [ctx](amg_status r) {
        cudaStreamSynchronize(ctx->s);
        cudaStreamSynchronize(ctx->s_copy);
        return r;
    };
    auto ok = [ctx](cudaError_t e, const char *what) {
        if (e == cudaSuccess) return AMG_OK;
        return set_err(ctx, AMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    amg_status st = AMG_OK;
    const size_t vbytes = sizeof(double) * nvals(ctx), fbytes = sizeof(double) * (size_t)nvec(ctx);
    if (host_chunks_ok(ctx)) {
        // a partial step: the values go over the link in row chunks on the
        // copy stream, each chunk's ingest and finest A P rows start as soon as
        // it has arrived, and the right-hand side follows the values
        TRY(prepare_chunks(ctx));
        if ((st = ok(cudaEventRecord(ctx->ev_vals, ctx->s), "event")) != AMG_OK) return drain(st);
        if ((st = ok(cudaStreamWaitEvent(ctx->s_copy, ctx->ev_vals, 0), "event wait")) != AMG_OK) return drain(st);
        for (int c = 0; c < kHostChunks; ++c) {
            const size_t e0 = (size_t)ctx->ck_e[c], e1 = (size_t)ctx->ck_e[c + 1];
            if (e1 > e0 && (st = ok(cudaMemcpyAsync(ctx->stage_val + e0, h_val + e0, sizeof(double) * (e1 - e0),
                                                    cudaMemcpyHostToDevice, ctx->s_copy), "values copy")) != AMG_OK)
                return drain(st);
            if ((st = ok(cudaEventRecord(ctx->ev_chunk[c], ctx->s_copy), "event")) != AMG_OK) return drain(st);
        }
        if ((st = ok(cudaMemcpyAsync(ctx->stage_f, h_f, fbytes, cudaMemcpyHostToDevice, ctx->s_copy), "rhs copy")) !=
                AMG_OK ||
            (st = ok(cudaEventRecord(ctx->ev_f, ctx->s_copy), "event")) != AMG_OK)
            return drain(st);
        const FineChunks ck{ctx->ck_row, ctx->ck_ap, ctx->ck_ac, ctx->ev_chunk};
        st = partial_rebuild_impl(ctx, ctx->stage_val, &ck);
        if (info) {
            info->rebuilt = ctx->last_rebuilt;
            info->nlevels = ctx->nlev;
        }
    } else {
        if ((st = ok(cudaMemcpyAsync(ctx->stage_val, h_val, vbytes, cudaMemcpyHostToDevice, ctx->s), "values copy")) !=
            AMG_OK)
            return drain(st);
        // the right-hand side is needed only by the solve: copied on a side
        // stream while the step's rebuild runs, after the values (so the two
        // copies do not share the link)
        if ((st = ok(cudaEventRecord(ctx->ev_vals, ctx->s), "event")) != AMG_OK ||
            (st = ok(cudaStreamWaitEvent(ctx->s_copy, ctx->ev_vals, 0), "event wait")) != AMG_OK ||
            (st = ok(cudaMemcpyAsync(ctx->stage_f, h_f, fbytes, cudaMemcpyHostToDevice, ctx->s_copy), "rhs copy")) !=
                AMG_OK ||
            (st = ok(cudaEventRecord(ctx->ev_f, ctx->s_copy), "event")) != AMG_OK)
            return drain(st);
        st = amg_step(ctx, ctx->n, ctx->nnz, ctx->fine_ptr, ctx->fine_col, ctx->stage_val, info);
    }
    if (st != AMG_OK) return drain(st);
    if (cudaStreamWaitEvent(ctx->s, ctx->ev_f, 0) != cudaSuccess) return drain(AMG_ERR_CUDA);
    st = amg_solve(ctx, ctx->stage_f, ctx->stage_u, tol, info);
    if (st != AMG_OK && st != AMG_NOT_CONVERGED) return drain(st);
    CK(cudaMemcpyAsync(h_u, ctx->stage_u, sizeof(double) * (size_t)nvec(ctx), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    return st;
}

amg_status amg_num_levels(const amg_ctx *ctx, int32_t *nlevels) {
    if (!ctx || !nlevels) return AMG_ERR_ARG;
    *nlevels = ctx->nlev;
    return AMG_OK;
}

amg_status amg_level_sizes(const amg_ctx *ctx, int32_t level, int64_t *sizes) {
    if (!ctx || !sizes || level < 0 || level >= ctx->nlev) return AMG_ERR_ARG;
    const Level &L = ctx->lev[level];
    sizes[0] = L.n;
    sizes[1] = L.nnz;
    sizes[2] = L.nnzP;
    sizes[3] = L.nnzR;
    sizes[4] = L.nnzAP;
    sizes[5] = L.nc;
    return AMG_OK;
}

amg_status amg_export_csr(amg_ctx *ctx, int32_t level, int32_t which, int32_t *d_ptr, int32_t *d_col,
                          double *d_val) {
    if (!ctx || level < 0 || level >= ctx->nlev || which < 0 || which > 2) return AMG_ERR_ARG;
    Level &L = ctx->lev[level];
    int32_t nrows = which == 0 ? L.n : which == 1 ? L.n : L.nc;
    int32_t nnz = which == 0 ? L.nnz : which == 1 ? L.nnzP : L.nnzR;
    const int32_t *ptr = which == 0 ? L.A_ptr : which == 1 ? L.P_ptr : L.R_ptr;
    const int32_t *col = which == 0 ? L.A_col : which == 1 ? L.P_col : L.R_col;
    const double *val = which == 0 ? L.A_val : which == 1 ? L.P_val : L.R_val;
    const float *valf = which == 0 ? L.A_valf : which == 1 ? L.P_valf : L.R_valf;
    if (!ptr) return set_err(ctx, AMG_ERR_STATE, "no such operator on this level");
    if (d_ptr) CK(cudaMemcpyAsync(d_ptr, ptr, sizeof(int32_t) * ((size_t)nrows + 1), cudaMemcpyDeviceToDevice, ctx->s));
    if (d_col) CK(cudaMemcpyAsync(d_col, col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, ctx->s));
    if (d_val) {
        if (blockmode(ctx) && which == 0)
            CK(cudaMemcpyAsync(d_val, L.Ab, sizeof(double) * 16 * (size_t)nnz, cudaMemcpyDeviceToDevice, ctx->s));
        else if (mixed(ctx) && valf) launch_copy_cast<float, double>(nnz, valf, d_val, nullptr, ctx->s);
        else CK(cudaMemcpyAsync(d_val, val, sizeof(double) * (size_t)nnz, cudaMemcpyDeviceToDevice, ctx->s));
    }
    CK(cudaStreamSynchronize(ctx->s));
    return AMG_OK;
}

amg_status amg_export_level_vec(amg_ctx *ctx, int32_t level, int32_t *d_agg, uint8_t *d_strong, double *d_m) {
    if (!ctx || level < 0 || level >= ctx->nlev) return AMG_ERR_ARG;
    Level &L = ctx->lev[level];
    if (d_agg) CK(cudaMemcpyAsync(d_agg, L.agg, sizeof(int32_t) * (size_t)L.n, cudaMemcpyDeviceToDevice, ctx->s));
    if (d_strong) CK(cudaMemcpyAsync(d_strong, L.strong, (size_t)L.nnz, cudaMemcpyDeviceToDevice, ctx->s));
    if (d_m) {
        if (blockmode(ctx)) {
            if (L.Minv)
                CK(cudaMemcpyAsync(d_m, L.Minv, sizeof(double) * 16 * (size_t)L.n, cudaMemcpyDeviceToDevice, ctx->s));
        } else if (mixed(ctx)) launch_copy_cast<float, double>(L.n, L.mf, d_m, nullptr, ctx->s);
        else CK(cudaMemcpyAsync(d_m, L.m, sizeof(double) * (size_t)L.n, cudaMemcpyDeviceToDevice, ctx->s));
    }
    CK(cudaStreamSynchronize(ctx->s));
    return AMG_OK;
}

amg_status amg_pattern_info(const amg_ctx *ctx, int32_t *col_bytes, int32_t *noffsets) {
    if (!ctx || !col_bytes || !noffsets) return AMG_ERR_ARG;
    if (!ctx->fine_ptr) return AMG_ERR_STATE;
    *col_bytes = ctx->fine_ncoff ? 1 : (ctx->nlev > 0 && ctx->lev[0].A_c16 ? 2 : 4);
    *noffsets = ctx->fine_ncoff;
    return AMG_OK;
}

amg_status amg_export_coarse_lu(amg_ctx *ctx, double *d_lu, int32_t *d_piv) {
    if (!ctx || !ctx->have_setup) return AMG_ERR_ARG;
    size_t nn = (size_t)ctx->nL * (size_t)ctx->nL;
    if (d_lu) CK(cudaMemcpyAsync(d_lu, ctx->lu, sizeof(double) * nn, cudaMemcpyDeviceToDevice, ctx->s));
    if (d_piv) CK(cudaMemcpyAsync(d_piv, ctx->piv, sizeof(int32_t) * (size_t)ctx->nL, cudaMemcpyDeviceToDevice, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    return AMG_OK;
}

amg_status amg_profile(amg_ctx *ctx, int32_t enable) {
    if (!ctx) return AMG_ERR_ARG;
    if (enable < 0 || enable > 2) return AMG_ERR_ARG;
    ctx->prof.on = enable != 0;
    ctx->prof.eager = enable == 2;
    return AMG_OK;
}

amg_status amg_profile_read(amg_ctx *ctx, int32_t slot, double *total_ms, int64_t *launches) {
    if (!ctx || slot < 0 || slot >= AMG_PROF_NSLOTS || !total_ms || !launches) return AMG_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->s));
    double ms = 0.0;
    cudaError_t first_err = cudaSuccess;
    // every pair goes back to the pool, whatever happens (each event is owned
    // by exactly one of the two lists)
    for (auto &pr : ctx->prof.rec[slot]) {
        float t = 0.f;
        const cudaError_t e = cudaEventElapsedTime(&t, pr.first, pr.second);
        if (e == cudaSuccess) ms += t;
        else if (first_err == cudaSuccess) first_err = e;
        ctx->prof.pool.push_back(pr.first);
        ctx->prof.pool.push_back(pr.second);
    }
    *total_ms = ms;
    *launches = (int64_t)ctx->prof.rec[slot].size();
    ctx->prof.rec[slot].clear();
    if (first_err != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, AMG_ERR_CUDA, std::string("reading a timing event: ") + cudaGetErrorString(first_err));
    }
    return AMG_OK;
}

int64_t amg_kernel_launches(void) { return launch_total(); }

int64_t amg_poisson_nnz(int32_t dim, int32_t N) {
    if ((dim != 2 && dim != 3) || N < 1) return -1;
    int64_t n1 = N, nf = N - 1;
    return dim == 2 ? n1 * n1 + 4 * nf * n1 : n1 * n1 * n1 + 6 * nf * n1 * n1;
}

amg_status amg_poisson_pattern(int32_t dim, int32_t N, int32_t *d_ptr, int32_t *d_col, void *cuda_stream) {
    if ((dim != 2 && dim != 3) || N < 1 || !d_ptr || !d_col) return AMG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int64_t n = dim == 2 ? (int64_t)N * N : (int64_t)N * N * N;
    if (amg_poisson_nnz(dim, N) > INT32_MAX) return AMG_ERR_ARG;
    int32_t *len = nullptr;
    int64_t *tmp = nullptr;
    int *st = nullptr;
    // on a failed allocation the ones already made are released before returning
    if (cudaMallocAsync(&len, sizeof(int32_t) * (size_t)n, s) != cudaSuccess) return AMG_ERR_OOM;
    if (cudaMallocAsync(&tmp, sizeof(int64_t) * (size_t)scan_tmp_elems(n), s) != cudaSuccess) {
        cudaFreeAsync(len, s);
        return AMG_ERR_OOM;
    }
    if (cudaMallocAsync(&st, sizeof(int), s) != cudaSuccess) {
        cudaFreeAsync(len, s);
        cudaFreeAsync(tmp, s);
        return AMG_ERR_OOM;
    }
    cudaMemsetAsync(st, 0, sizeof(int), s);
    launch_poisson_rowlen(dim, N, len, s);
    scan_counts(len, d_ptr, n, st, tmp, s);
    launch_poisson_cols(dim, N, d_ptr, d_col, s);
    cudaFreeAsync(len, s);
    cudaFreeAsync(tmp, s);
    cudaFreeAsync(st, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return AMG_ERR_CUDA;
    return AMG_OK;
}

amg_status amg_poisson_values(int32_t dim, int32_t N, int32_t dirichlet_top, const double *d_rho,
                              const int32_t *d_ptr, double *d_val, void *cuda_stream) {
    if ((dim != 2 && dim != 3) || N < 1 || !d_rho || !d_ptr || !d_val) return AMG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    launch_poisson_vals(dim, N, dirichlet_top, d_rho, 0, d_ptr, d_val, s);
    if (cudaGetLastError() != cudaSuccess) return AMG_ERR_CUDA;
    return AMG_OK;
}

amg_status amg_poisson_values_log(int32_t dim, int32_t N, int32_t dirichlet_top, const double *d_theta,
                                  const int32_t *d_ptr, double *d_val, void *cuda_stream) {
    if ((dim != 2 && dim != 3) || N < 1 || !d_theta || !d_ptr || !d_val) return AMG_ERR_ARG;
    launch_poisson_vals(dim, N, dirichlet_top, d_theta, 1, d_ptr, d_val, (cudaStream_t)cuda_stream);
    if (cudaGetLastError() != cudaSuccess) return AMG_ERR_CUDA;
    return AMG_OK;
}

amg_status amg_levelset_values(int32_t dim, int32_t N, const double *d_fx, const double *d_fy, const double *d_fz,
                               const int32_t *d_ptr, double *d_val, void *cuda_stream) {
    if ((dim != 2 && dim != 3) || N < 1 || !d_fx || !d_fy || (dim == 3 && !d_fz) || !d_ptr || !d_val)
        return AMG_ERR_ARG;
    if (amg_poisson_nnz(dim, N) > INT32_MAX) return AMG_ERR_ARG;
    launch_levelset_vals(dim, N, d_fx, d_fy, d_fz, d_ptr, d_val, (cudaStream_t)cuda_stream);
    if (cudaGetLastError() != cudaSuccess) return AMG_ERR_CUDA;
    return AMG_OK;
}

amg_status amg_stokes_values(int32_t N, const double *d_rho, const double *d_mu, const double *d_fx,
                             const double *d_fy, const double *d_fz, double mass, const int32_t *d_ptr, double *d_val,
                             void *cuda_stream) {
    if (N < 1 || !d_rho || !d_mu || !d_fx || !d_fy || !d_fz || !d_ptr || !d_val || !std::isfinite(mass))
        return AMG_ERR_ARG;
    if (amg_poisson_nnz(3, N) > INT32_MAX / 16) return AMG_ERR_ARG;
    launch_stokes_vals(N, d_rho, d_mu, d_fx, d_fy, d_fz, mass, d_ptr, d_val, (cudaStream_t)cuda_stream);
    if (cudaGetLastError() != cudaSuccess) return AMG_ERR_CUDA;
    return AMG_OK;
}

amg_status amg_poisson_grad_theta(int32_t dim, int32_t N, int32_t dirichlet_top, const double *d_rho,
                                  const double *d_u, const double *d_lam, double *d_grad, void *cuda_stream) {
    if ((dim != 2 && dim != 3) || N < 1 || !d_rho || !d_u || !d_lam || !d_grad) return AMG_ERR_ARG;
    launch_poisson_grad(dim, N, dirichlet_top, d_rho, 0, d_u, d_lam, d_grad, (cudaStream_t)cuda_stream);
    if (cudaGetLastError() != cudaSuccess) return AMG_ERR_CUDA;
    return AMG_OK;
}

amg_status amg_poisson_grad_log(int32_t dim, int32_t N, int32_t dirichlet_top, const double *d_theta,
                                const double *d_u, const double *d_lam, double *d_grad, void *cuda_stream) {
    if ((dim != 2 && dim != 3) || N < 1 || !d_theta || !d_u || !d_lam || !d_grad) return AMG_ERR_ARG;
    launch_poisson_grad(dim, N, dirichlet_top, d_theta, 1, d_u, d_lam, d_grad, (cudaStream_t)cuda_stream);
    if (cudaGetLastError() != cudaSuccess) return AMG_ERR_CUDA;
    return AMG_OK;
}

}  // extern "C"
