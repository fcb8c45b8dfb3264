// common.cuh -- internal declarations shared by the CUDA translation units of
// libamgpr.so (partial-reuse smoothed-aggregation AMG, arXiv 2108.02054).
#pragma once
#include <cuda_runtime.h>
#include <utility>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/amgpr.h"

namespace amgpr {

// Bits of the device status word that kernels set with atomicOr instead of
// trapping; the host turns them into an amg_status.
enum : int {
    DEV_ERR_PATTERN = 1,
    DEV_ERR_CAPACITY = 2,
    DEV_ERR_NONFINITE = 4,
    DEV_ERR_STATE = 8,
    DEV_ERR_SINGULAR = 16,
    DEV_ERR_OVERFLOW = 32,
    DEV_ERR_TIMEOUT = 64,  // a bounded wait between the CTAs of a cluster ran out
};

constexpr int kMaxLevels = 32;
// symbolic product: per-warp open-addressing hash of at most this many slots
// (a row of a Galerkin pattern may hold half as many distinct columns)
constexpr int kHashCap = 4096;

// Device-resident state of the CG iteration; every CG kernel reads and writes
// it so that the loop needs no host round trip between its kernels.
enum { CG_CTR_INIT = 0, CG_CTR_PQ, CG_CTR_RR, CG_CTR_RZ, CG_CTR_RZO, CG_CTR_TT, CG_NCTR = 8 };
struct CgState {
    double rz, rz_next, rzo, pq, alpha, beta, rr, nf, res, tres, tol;
    unsigned ctr[CG_NCTR];  // arrival counters of the last-block reductions (zero between kernels)
    int iter, maxiter, done, status, replacements, need_true, copy_r;
    int pad;  // loop bodies executed (graph path)
};

// Device-resident state of the BiCGStab iteration (same scheme as CgState).
enum { BI_CTR_INIT = 0, BI_CTR_RHO, BI_CTR_RV, BI_CTR_SS, BI_CTR_T, BI_CTR_RR, BI_CTR_TRUE, BI_NCTR = 8 };
struct BiState {
    double rho, rho_old, alpha, omega, beta, rv, ts, tt, nf, res, sres, tres, tol;
    unsigned ctr[BI_NCTR];
    int iter, maxiter, done, status, replacements, half, need_true, copy_r, skip, pad;
};

// Column indices of a matrix: plain int32 (col); or, for a pattern whose
// rows use at most kMaxColOffsets distinct column offsets (column - row, as
// in a stencil), one byte per entry (cidx) naming its offset in a table
// (off, noff entries): column = row + off[cidx[p]]; or, when every offset
// column - row fits in 16 bits, two bytes per entry (c16): column = row +
// c16[p].  The kernels read the first form that is set.
constexpr int kMaxColOffsets = 256;
struct ColIdx {
    const int32_t *col = nullptr;
    const uint8_t *cidx = nullptr;
    const int32_t *off = nullptr;
    int noff = 0;
    const int16_t *c16 = nullptr;
};

template <class V>
struct VecSet {
    V *u = nullptr, *f = nullptr, *r = nullptr, *t = nullptr;
};

struct Level {
    int32_t n = 0, nnz = 0;
    int32_t *A_ptr = nullptr, *A_col = nullptr, *dia = nullptr;
    // the finest level's one-byte columns (when its pattern allows them);
    // otherwise the two-byte offsets of any level whose offsets fit
    const uint8_t *A_cidx = nullptr;
    const int32_t *A_coff = nullptr;
    int A_ncoff = 0;
    int16_t *A_c16 = nullptr;
    ColIdx cols() const { return ColIdx{A_col, A_cidx, A_coff, A_ncoff, A_c16}; }
    double *A_val = nullptr;   // FP64 values (level 0: the hierarchy's copy of the fine matrix)
    float *A_valf = nullptr;   // FP32 values (mixed precision)
    // transfer operators (absent on the coarsest level)
    int32_t nc = 0, nnzP = 0, nnzR = 0, nnzAP = 0;
    int32_t *P_ptr = nullptr, *P_col = nullptr;
    // P's columns as two-byte offsets from (int)(row * P_ratio), when they fit
    int16_t *P_c16 = nullptr;
    float P_ratio = 0.0f;
    double *P_val = nullptr;
    float *P_valf = nullptr;
    int32_t *R_ptr = nullptr, *R_col = nullptr;
    double *R_val = nullptr;
    float *R_valf = nullptr;
    int32_t *AP_ptr = nullptr, *AP_col = nullptr;
    double *AP_val = nullptr;
    float *AP_valf = nullptr;
    // gather metadata of the numeric Galerkin product (resolved once at setup)
    int64_t nt1 = 0, nt2 = 0;
    int32_t *t1ptr = nullptr, *t2ptr = nullptr;
    uint16_t *slot1 = nullptr, *slot2 = nullptr;
    int32_t max_ap_row = 0, max_ac_row = 0;
    // lanes per row of the matrix-vector pieces on this level (A rows, R rows)
    int lpr = 1, lpr_r = 8;
    // the same products as fixed gather operators, built at the first partial rebuild
    bool gather_ready = false;
    int32_t *g1_ptr = nullptr, *g1_idx = nullptr, *g2_ptr = nullptr, *g2_idx = nullptr;
    double *g1_w = nullptr, *g2_w = nullptr;
    float *g1_wf = nullptr, *g2_wf = nullptr;
    // aggregation (kept for inspection)
    int32_t *agg = nullptr;
    uint8_t *strong = nullptr;
    // smoother
    double *m = nullptr;
    float *mf = nullptr;
    // V-cycle vectors
    VecSet<double> vd;
    VecSet<float> vf;
    // 4 x 4 block mode: block values of A and A P (16 per entry; A_val then
    // holds the block norms that strength and aggregation see), damped
    // block-Jacobi inverses (16 per node); vd vectors hold 4 per node
    double *Ab = nullptr, *APb = nullptr, *Minv = nullptr;
};

// ------------------------------------------------------------------ launchers
// (all enqueue on `s`; `st` is the device status word)
// every launcher counts its kernel launches (process-wide)
void count_launch();

// Programmatic dependent launch for the solve's kernel chain: the launch of
// a kernel may be processed while its predecessor in the stream (or graph)
// completes, and the kernel's first statement, pdl_wait(), blocks until the
// predecessor has finished and its memory is visible.  Without a
// programmatic predecessor pdl_wait() returns at once.
__device__ __forceinline__ void pdl_wait() { cudaGridDependencySynchronize(); }
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // a launch error stays the runtime's last error, read by the status check
    (void)cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
void add_launches(int64_t d);
int64_t launch_total();
void scan_counts(const int32_t *in, int32_t *out, int64_t n, int *st, int64_t *tmp, cudaStream_t s);
int64_t scan_tmp_elems(int64_t n);

void launch_poisson_rowlen(int dim, int N, int32_t *len, cudaStream_t s);
void launch_poisson_cols(int dim, int N, const int32_t *ptr, int32_t *col, cudaStream_t s);
// logd != 0: rho holds the log-density theta and every density is exp(theta)
void launch_poisson_vals(int dim, int N, int top, const double *rho, int logd, const int32_t *ptr, double *val,
                         cudaStream_t s);
void launch_poisson_grad(int dim, int N, int top, const double *rho, int logd, const double *u, const double *lam,
                         double *grad, cudaStream_t s);
void launch_levelset_vals(int dim, int N, const double *fx, const double *fy, const double *fz, const int32_t *ptr,
                          double *val, cudaStream_t s);

// a caller's row pointers (ptr[0] = 0, non-decreasing, ptr[n] = nnz): DEV_ERR_PATTERN otherwise
void launch_check_rowptr(int32_t n, int32_t nnz, const int32_t *ptr, int *st, cudaStream_t s);
void launch_check_pattern(int32_t n, const int32_t *ptr, const int32_t *col, int32_t *dia, int *st,
                          cudaStream_t s);
void launch_check_finite(int64_t nnz, const double *val, int *st, cudaStream_t s);
void launch_strength(int32_t n, const int32_t *ptr, const int32_t *col, const double *val, const int32_t *dia,
                     double eps2, uint8_t *strong, int32_t *deg, cudaStream_t s);
// aggregation; returns the number of aggregates (host sync inside), or -1 on error
int32_t run_aggregation(int32_t n, const int32_t *ptr, const int32_t *col, const double *val,
                        const uint8_t *strong, const int32_t *deg, int32_t *agg, int8_t *state, int64_t *m1,
                        uint8_t *r1, int32_t *root_id, int32_t *agg1, int32_t *root_of, int *counter, int *st,
                        int64_t *scan_tmp, cudaStream_t s);
void launch_p_count(int32_t n, const int32_t *ptr, const int32_t *col, const uint8_t *strong, const int32_t *agg,
                    int smoothed, int32_t *plen, cudaStream_t s);
void launch_p_fill(int32_t n, const int32_t *ptr, const int32_t *col, const double *val, const uint8_t *strong,
                   const int32_t *dia, const int32_t *agg, double omega, int smoothed, const int32_t *P_ptr,
                   int32_t *P_col, double *P_val, cudaStream_t s);
void launch_count_cols(int64_t nnz, const int32_t *col, int32_t *cnt, cudaStream_t s);
void launch_transpose_scatter(int32_t n, const int32_t *P_ptr, const int32_t *P_col, const double *P_val,
                              const int32_t *R_ptr, int32_t *cursor, int32_t *R_col, double *R_val, cudaStream_t s);
void launch_sort_rows(int32_t nrows, const int32_t *ptr, int32_t *col, double *val, cudaStream_t s);
// symbolic C = X*Y pattern: pass 1 (C_ptr == nullptr) writes row lengths into len,
// pass 2 writes sorted columns into C_col at C_ptr
// the most terms of any row of C = X * Y (a bound on its distinct columns),
// into *out (atomic maximum; zero it first), and the hash-table capacity for it
void launch_row_terms_max(int32_t nrows, const int32_t *X_ptr, const int32_t *X_col, const int32_t *Y_ptr,
                          int add_diag, int *out, cudaStream_t s);
int spgemm_symbolic_cap(int32_t max_terms);
// (lanes per row: 8, 16 or 32, from X's average row length)
void launch_spgemm_symbolic(int32_t nrows, int32_t ncols, const int32_t *X_ptr, const int32_t *X_col,
                            const int32_t *Y_ptr, const int32_t *Y_col, int add_diag, int cap, int lanes,
                            int32_t *len, const int32_t *C_ptr, int32_t *C_col, int *st, cudaStream_t s);
void launch_t1_count(int32_t n, const int32_t *A_ptr, const int32_t *A_col, const int32_t *P_ptr, int32_t *cnt,
                     cudaStream_t s);
void launch_t1_fill(int32_t n, const int32_t *A_ptr, const int32_t *A_col, const int32_t *P_ptr,
                    const int32_t *P_col, const int32_t *AP_ptr, const int32_t *AP_col, const int32_t *t1ptr,
                    uint16_t *slot1, int *st, cudaStream_t s);
void launch_t2_count(int32_t nc, const int32_t *R_ptr, const int32_t *R_col, const int32_t *AP_ptr, int32_t *cnt,
                     cudaStream_t s);
void launch_t2_fill(int32_t nc, const int32_t *R_ptr, const int32_t *R_col, const int32_t *AP_ptr,
                    const int32_t *AP_col, const int32_t *Ac_ptr, const int32_t *Ac_col, const int32_t *t2ptr,
                    uint16_t *slot2, int *st, cudaStream_t s);
void launch_row_maxlen(int32_t n, const int32_t *ptr, int *out, cudaStream_t s);
void launch_row_last(int32_t n, const int32_t *ptr, const int32_t *col, int32_t *last, cudaStream_t s);
// gather operators of the numeric Galerkin product (AP = N a, A_c = M AP)
void launch_group_terms(int32_t nrows, const int32_t *tptr, const uint16_t *slot, const int32_t *out_ptr,
                        int32_t *eptr, int32_t *perm, int *st, cudaStream_t s);
void launch_stage1_terms(int32_t n, const int32_t *A_ptr, const int32_t *A_col, const int32_t *P_ptr,
                         const double *P_val, const int32_t *t1ptr, int32_t *idx, double *wgt, cudaStream_t s);
void launch_stage2_terms(int32_t nc, const int32_t *R_ptr, const int32_t *R_col, const double *R_val,
                         const int32_t *AP_ptr, const int32_t *t2ptr, int32_t *idx, double *wgt, cudaStream_t s);
void launch_permute_terms(int64_t nt, const int32_t *perm, const int32_t *idx_in, const double *w_in,
                          int32_t *idx_out, double *w_out, float *wf_out, cudaStream_t s);
template <class V>
void launch_gather_apply(int64_t nout, const int32_t *eptr, const int32_t *idx, const V *w, const V *x, V *y,
                         cudaStream_t s);

// numeric Galerkin product, FP64 (bit-exact accumulation order)
void launch_ap_numeric_f64(const Level &L, const double *A_val, cudaStream_t s);
void launch_rap_numeric_f64(const Level &L, const int32_t *Ac_ptr, double *Ac_val, cudaStream_t s);
// numeric Galerkin product, FP32 values with compensated accumulation
void launch_ap_numeric_f32(const Level &L, const float *A_valf, cudaStream_t s);
void launch_rap_numeric_f32(const Level &L, const int32_t *Ac_ptr, float *Ac_valf, cudaStream_t s);

// smoother diagonal; optional fused copy / cast of the values read
void launch_smoother_f64(int32_t n, const int32_t *ptr, const double *val, const int32_t *dia, int type, double wj,
                         double *m, cudaStream_t s);
void launch_smoother_f32(int32_t n, const int32_t *ptr, const float *val, const int32_t *dia, int type, double wj,
                         float *m, cudaStream_t s);
// level-0 ingest of rows row0 .. row1 - 1 (row0 a multiple of 32): copy new
// values to the hierarchy (and the FP32 copy), check them, build the smoother
void launch_ingest_fine(int32_t row0, int32_t row1, const int32_t *ptr, const double *val_in, const int32_t *dia,
                        int type, double wj, double *val_out, float *valf_out, double *m, float *mf, int *st,
                        cudaStream_t s);
void launch_cast_f32(int64_t n, const double *in, float *out, cudaStream_t s);

// coarsest level: dense LU and explicit inverse
void launch_csr_to_dense(int32_t n, const int32_t *ptr, const int32_t *col, const double *val, const float *valf,
                         double *dense, cudaStream_t s);
// aT (optional, n x n): a column-major copy of the factors, written when
// lu_wants_transpose(n); the inverse then reads it
bool lu_wants_transpose(int32_t n);
void launch_dense_lu(int32_t n, double *a, int32_t *piv, int *st, cudaStream_t s, double *aT = nullptr);
void launch_lu_inverse(int32_t n, const double *lu, const int32_t *piv, double *inv, cudaStream_t s,
                       const double *luT = nullptr);

// V-cycle pieces; `skip` (may be null) makes the kernel return at once when *skip != 0
template <class V, class TF>
void launch_smooth0_residual(const Level &L, const V *val, const V *m, const TF *f, V *u, V *r, const int *skip,
                             cudaStream_t s);
template <class V, class TF, class TO>
void launch_smooth_sweep(const Level &L, const V *val, const V *m, const TF *f, const V *u_in, TO *u_out,
                         const int *skip, cudaStream_t s);
template <class V, class TF>
void launch_residual(const Level &L, const V *val, const TF *f, const V *u, V *r, const int *skip, cudaStream_t s);
// last finest-level post-smoothing sweep fused with the CG product r.z (cg_blocks(n) partials)
template <class V>
void launch_smooth_sweep_dot(const Level &L, const V *val, const V *m, const double *f, const V *u_in, double *z,
                             double *partial, CgState *cg, const int *skip, cudaStream_t s);
template <class V>
void launch_restrict(const Level &L, const V *Rval, const V *r, V *fc, const V *mc, V *uc, const int *skip,
                     cudaStream_t s);
template <class V>
void launch_prolong(const Level &L, const V *Pval, const V *uc, V *u, const int *skip, cudaStream_t s);
template <class V, class TF, class TO>
void launch_coarse_solve(int32_t n, const double *inv, const TF *f, TO *u, const int *skip, cudaStream_t s);
template <class TI, class TO>
void launch_copy_cast(int64_t n, const TI *in, TO *out, const int *skip, cudaStream_t s);

// CG (FP64); reductions finish in the last block of the producing kernel
int cg_blocks(int64_t n);
// The V-cycle's first pre-smoothing step from u = 0 on the finest level,
// u0 = m o r, written by the kernel that produces r (so that step needs no
// per-entry product); at most one of the two pointer pairs is set.
struct Smooth0Out {
    const double *m = nullptr;
    double *u = nullptr;
    const float *mf = nullptr;
    float *uf = nullptr;
};
void launch_cg_init(int32_t n, const double *f, double *u, double *r, double *partial, CgState *cg, double tol,
                    int maxiter, const Smooth0Out &z0, cudaStream_t s);
// x.y into per-block partials; with cg, the last block stores the total
// (target 1: the new r.z, target 2: r_new.z_old)
void launch_dot(int32_t n, const double *x, const double *y, double *partial, const int *skip, CgState *cg, int target,
                cudaStream_t s);
void launch_cg_set_rz_p(int32_t n, const double *z, double *p, CgState *cg, cudaStream_t s);
void launch_spmv_dot(int32_t n, const int32_t *ptr, const ColIdx &col, const double *val, const double *p,
                     double *q, double *partial, CgState *cg, cudaStream_t s);
// the compressed form of a pattern: collect the distinct offsets column - row
// into an open-addressed table of kColOffsetSlots ints (empty:
// kColOffsetEmpty, the int of four 0x80 bytes; *count the distinct keys,
// capped), then encode every entry's offset index against the sorted table
// off (noff entries)
constexpr int kColOffsetSlots = 1024;
constexpr int32_t kColOffsetEmpty = (int32_t)0x80808080u;
// c16[p] = col[p] - base(row) for every entry, base(i) = i (ratio == 0) or
// (int)((float)i * ratio); *flag = 1 if an offset does not fit in 16 bits
void launch_col_delta16(int32_t n, const int32_t *ptr, const int32_t *col, float ratio, int16_t *c16, int *flag,
                        cudaStream_t s);
void launch_col_offsets_collect(int32_t n, const int32_t *ptr, const int32_t *col, int32_t *table, int *count,
                                cudaStream_t s);
void launch_col_offsets_encode(int32_t n, const int32_t *ptr, const int32_t *col, const int32_t *off, int noff,
                               uint8_t *cidx, int *st, cudaStream_t s);
// zo (flexible variant, else null): the previous z; r_new.z_old goes to cg->rzo
// through the partials part_zo
void launch_cg_update_ur(int32_t n, CgState *cg, const double *p, const double *q, double *u, double *r,
                         double *partial, const double *zo, double *part_zo, int use_h, cudaGraphConditionalHandle hb,
                         const Smooth0Out &z0, cudaStream_t s);
void launch_true_residual(int32_t n, const int32_t *ptr, const ColIdx &col, const double *val, const double *f,
                          const double *u, double *t, double *partial, CgState *cg, int force, cudaStream_t s);
void launch_replace_r(int32_t n, CgState *cg, const double *t, double *r, const double *zo, double *part_zo,
                      const Smooth0Out &z0, cudaStream_t s);
void launch_cg_update_p(int32_t n, CgState *cg, const double *z, double *p, int use_h, cudaGraphConditionalHandle h,
                        cudaStream_t s);

// BiCGStab (FP64), right-preconditioned; partial: 3 * cg_blocks(n) doubles
void launch_bi_init(int32_t n, const double *f, double *x, double *r, double *rh, double *p, double *v,
                    double *partial, BiState *st, double tol, int maxiter, cudaStream_t s);
void launch_bi_rho(int32_t n, const double *rh, const double *r, double *partial, BiState *st, cudaStream_t s);
void launch_bi_p(int32_t n, const double *r, const double *v, double *p, BiState *st, cudaStream_t s);
void launch_bi_spmv_rv(int32_t n, int bs, const int32_t *ptr, const int32_t *col, const double *val,
                       const double *ph, double *v, const double *rh, double *partial, BiState *st, cudaStream_t s);
void launch_bi_s(int32_t n, const double *r, const double *v, double *sv, double *partial, BiState *st,
                 cudaStream_t s);
void launch_bi_half(int32_t n, const double *ph, const double *sv, double *x, double *r, BiState *st, cudaStream_t s);
void launch_bi_spmv_t(int32_t n, int bs, const int32_t *ptr, const int32_t *col, const double *val,
                      const double *sh, const double *sv, double *t, double *partial, BiState *st, cudaStream_t s);
void launch_bi_xr(int32_t n, const double *ph, const double *sh, const double *sv, const double *t, double *x,
                  double *r, double *partial, BiState *st, cudaStream_t s);
void launch_bi_true(int32_t n, int bs, const int32_t *ptr, const int32_t *col, const double *val, const double *f,
                    const double *x, double *t, double *partial, BiState *st, int force, cudaStream_t s);
void launch_bi_replace(int32_t n, const double *t, double *r, BiState *st, cudaStream_t s);
void launch_bi_end(BiState *st, int use_h, cudaGraphConditionalHandle h, cudaStream_t s);
// (BiCGStab vectors have n = bs * nodes entries; bs = 4 for the block matrix)

// 4 x 4 block-valued hierarchy (block.cu): block CSR, 16 doubles per entry
void launch_stokes_vals(int N, const double *rho, const double *mu, const double *fx, const double *fy,
                        const double *fz, double mass, const int32_t *ptr, double *val, cudaStream_t s);
void launch_block_norms(int64_t nnz, const double *bv, double *out, cudaStream_t s);
void launch_block_gather(int64_t nout, const int32_t *eptr, const int32_t *idx, const double *w, const double *x,
                         double *y, cudaStream_t s);
void launch_block_jacobi(int32_t n, const int32_t *dia, const double *bv, double wj, double *minv, cudaStream_t s);
void launch_block_to_dense(int32_t n, const int32_t *ptr, const int32_t *col, const double *bv, double *dense,
                           cudaStream_t s);
void launch_block_smooth0(int32_t n, const double *minv, const double *f, double *u, const int *skip,
                          cudaStream_t s);
void launch_block_sweep(int32_t n, const int32_t *ptr, const int32_t *col, const double *bv, const double *minv,
                        const double *f, const double *uin, double *uout, const int *skip, cudaStream_t s);
void launch_block_residual(int32_t n, const int32_t *ptr, const int32_t *col, const double *bv, const double *f,
                           const double *u, double *r, const int *skip, cudaStream_t s);
void launch_block_restrict(int32_t nc, const int32_t *Rptr, const int32_t *Rcol, const double *Rval, const double *r,
                           double *fc, const int *skip, cudaStream_t s);
void launch_block_prolong(int32_t n, const int32_t *Pptr, const int32_t *Pcol, const double *Pval, const double *uc,
                          double *u, const int *skip, cudaStream_t s);

}  // namespace amgpr
