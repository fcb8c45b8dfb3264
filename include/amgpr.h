/*
 * amgpr.h -- C ABI of the partial-reuse AMG library (libamgpr.so).
 *
 * Method: D. E. Demidov, "Partial reuse AMG setup cost amortization strategy
 * for the solution of non-steady state problems" (arXiv 2108.02054).
 * Alg. 1 (AMG setup), Alg. 2 (V-cycle), Alg. 3 (full reuse), Alg. 4 (partial
 * reuse), Sec. 2 (Krylov solver with one V-cycle as the preconditioner),
 * Sec. 5 (reuse of the Galerkin product's pattern).
 *
 * Conventions for every entry point:
 *  - Matrices are CSR with int32 row pointers / column indices, columns sorted
 *    ascending within each row, the diagonal stored in every row.
 *  - Pointers named d_* are DEVICE pointers (current CUDA device), h_* are
 *    HOST pointers.  The caller owns every pointer it passes; the library only
 *    reads or writes it during the call (work is ordered on the context's
 *    stream; calls that return data synchronise that stream before returning
 *    unless stated otherwise).
 *  - Every function returns an amg_status and never aborts the process.  On
 *    an error, amg_last_error() describes it.  A CUDA error maps to
 *    AMG_ERR_CUDA; device-side checks report through a status word, never by
 *    trapping.
 *  - The library allocates its own device memory (cudaMalloc) for the
 *    hierarchy and work vectors; amg_destroy frees it.
 */
#ifndef AMGPR_H
#define AMGPR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amg_ctx amg_ctx;

typedef enum {
    AMG_OK = 0,
    AMG_NOT_CONVERGED = 1,     /* solve hit maxiter; u and info are filled in */
    AMG_ERR_ARG = -1,          /* null pointer, bad size, bad parameter */
    AMG_ERR_STATE = -2,        /* e.g. partial rebuild before a full setup */
    AMG_ERR_PATTERN = -3,      /* unsorted / out-of-range columns, missing diagonal */
    AMG_ERR_BREAKDOWN = -4,    /* CG breakdown: p'Ap <= 0 or non-finite */
    AMG_ERR_NONFINITE = -5,    /* NaN / Inf in the matrix values */
    AMG_ERR_CUDA = -6,         /* a CUDA runtime error */
    AMG_ERR_OOM = -7,          /* device allocation failed */
    AMG_ERR_SINGULAR = -8,     /* zero pivot in the coarsest LU */
    AMG_ERR_CAPACITY = -9      /* a row exceeds a fixed kernel capacity */
} amg_status;

enum { AMG_SMOOTHER_SPAI0 = 0, AMG_SMOOTHER_JACOBI = 1 };
enum { AMG_PREC_FP64 = 0, AMG_PREC_MIXED = 1 };
enum { AMG_MODE_PARTIAL = 0, AMG_MODE_FULL_REBUILD = 1, AMG_MODE_FULL_REUSE = 2 };
enum { AMG_SOLVER_CG = 0, AMG_SOLVER_BICGSTAB = 1 };

typedef struct {
    double theta;          /* strength threshold on the finest level (0.08) */
    double omega;          /* prolongation smoothing weight (2/3) */
    double jacobi_omega;   /* damped Jacobi weight when smoother = JACOBI (0.72) */
    int32_t smoother;      /* AMG_SMOOTHER_* (SPAI0) */
    int32_t npre, npost;   /* smoothing sweeps before / after the coarse correction (1, 1) */
    int32_t coarse_enough; /* stop coarsening at or below this many rows (256) */
    int32_t max_levels;    /* at most this many levels (20) */
    int32_t theta_halving; /* 1: theta halves on every coarser level (1) */
    int32_t smoothed;      /* 1: smoothed aggregation, 0: plain aggregation (1) */
    int32_t precision;     /* AMG_PREC_* (FP64) */
    int32_t mode;          /* AMG_MODE_* used by amg_step (PARTIAL) */
    int32_t reuse_iter_limit; /* full reuse: rebuild after a solve that needed more (100) */
    int32_t maxiter;       /* CG iteration cap (100) */
    /* PARTIAL mode, preventive full rebuilds (Sec. 3: "from time to time",
     * regularly or on a convergence criterion); 0 disables each rule:
     * rebuild_every: a full setup every this many steps;
     * rebuild_iter_growth: a full setup when the previous solve needed more
     * than this factor times the iterations of the first solve after the last
     * full setup. */
    int32_t rebuild_every;
    double rebuild_iter_growth;
    /* Krylov solver of amg_solve (Sec. 4): AMG_SOLVER_CG for the symmetric
     * pressure systems, AMG_SOLVER_BICGSTAB (right-preconditioned) for the
     * nonsymmetric level-set systems.  (CG) */
    int32_t solver;
    /* 1: scalar matrices.  4: 4 x 4 block-valued matrices (Sec. 4, the
     * monolithic Navier-Stokes systems): n and nnz of every call count nodes
     * and blocks, values are 16 doubles per block (row-major: component r of
     * the row node, component c of the column node), vectors hold the 4
     * components of each node consecutively (4 n doubles).  The hierarchy
     * then takes the paper's configuration for these systems and requires
     * smoothed = 0, smoother = JACOBI (damped block Jacobi), precision = FP64
     * and solver = BICGSTAB (else amg_create returns AMG_ERR_ARG).  Strength
     * and aggregation run on the node graph of the block Frobenius norms;
     * coarse_enough counts nodes.  amg_export_csr(which = 0) returns 16
     * values per entry and amg_export_level_vec's d_m the block-Jacobi
     * inverses w_J A_ii^-1 (16 per node).  (1) */
    int32_t block_size;
} amg_params;

typedef struct {
    int32_t iters;         /* Krylov iterations of the last solve */
    int32_t rebuilt;       /* 1 if the last amg_step ran a full setup */
    int32_t nlevels;       /* levels of the current hierarchy */
    int32_t status;        /* status of the last solve */
    double rel_resid;      /* true relative residual |f - A u| / |f| of the last solve */
} amg_info;

/* Default parameters (values in the comments above). */
amg_status amg_default_params(amg_params *prm);

/* Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *ctx is owned by the
 * caller and released with amg_destroy. */
amg_status amg_create(amg_ctx **ctx, const amg_params *prm, void *cuda_stream);
void amg_destroy(amg_ctx *ctx);
const char *amg_last_error(const amg_ctx *ctx);

/* Alg. 1: full setup from A (n rows, nnz entries; device CSR).  Copies the
 * pattern and values; builds strength, aggregates, tentative and smoothed P,
 * R = P^T, the Galerkin patterns with their gather metadata, every A_{l+1},
 * the smoothers and the coarsest LU.  Replaces any previous hierarchy.
 * AMG_ERR_PATTERN: row pointers not starting at 0, decreasing or not ending
 * at nnz (checked before any column is read), or unsorted / out-of-range
 * columns or a missing diagonal; the context then holds no hierarchy. */
amg_status amg_full_setup(amg_ctx *ctx, int32_t n, int32_t nnz, const int32_t *d_ptr,
                          const int32_t *d_col, const double *d_val);

/* Alg. 4 body: new values d_val (nnz doubles) on the pattern given to the
 * last full setup; keeps P and R, recomputes every A_{l+1} = R A_l P over
 * the cached coarse patterns (Sec. 5), the smoothers and the coarsest LU.
 * AMG_ERR_STATE without a prior full setup. */
amg_status amg_partial_rebuild(amg_ctx *ctx, const double *d_val);

/* One time step's setup under the context's mode (Alg. 3 / Alg. 4 / no
 * reuse): PARTIAL -> partial rebuild (full setup on the first call),
 * FULL_REBUILD -> full setup, FULL_REUSE -> keep the whole hierarchy unless
 * the previous solve needed more than reuse_iter_limit iterations or did not
 * converge.  The new values always become the system matrix of the next
 * amg_solve.  For the first call, d_ptr/d_col give the pattern (they are
 * ignored afterwards and may then be NULL). */
amg_status amg_step(amg_ctx *ctx, int32_t n, int32_t nnz, const int32_t *d_ptr,
                    const int32_t *d_col, const double *d_val, amg_info *info);

/* Solve A u = f with a Krylov solver preconditioned by one V-cycle per
 * application (Sec. 2, Alg. 2), u_0 = 0, to |f - A u| / |f| <= tol or
 * params.maxiter iterations.  params.solver picks CG (one V-cycle per
 * iteration) or right-preconditioned BiCGStab (two per iteration; converged
 * at the half step when |s| / |f| <= tol).  Convergence reported by the
 * recurrence is confirmed on the true residual, which replaces the recurrence
 * residual (at most twice) when it is above tol.  A is the system matrix of
 * the last setup / step.  d_f, d_u: n doubles.  Returns AMG_OK,
 * AMG_NOT_CONVERGED, AMG_ERR_BREAKDOWN (CG: p'Ap <= 0; BiCGStab: a zero or
 * non-finite (r^, r), (r^, v), (t, t) or omega) or another error; info may
 * be NULL. */
amg_status amg_solve(amg_ctx *ctx, const double *d_f, double *d_u, double tol, amg_info *info);

/* Apply one V-cycle z = B r from a zero initial guess (Alg. 2). */
amg_status amg_apply_vcycle(amg_ctx *ctx, const double *d_r, double *d_z);

/* End to end with host buffers: copies h_val (nnz doubles) and h_f (n doubles)
 * to the device, runs amg_step and amg_solve, copies u back to h_u (n
 * doubles) and synchronises.  h_f's copy runs on the context's own copy
 * stream while the step's rebuild runs.  When the step is a partial rebuild
 * whose gather operators already exist (from the second partial step on),
 * h_val goes over in eight row chunks on that stream. As soon as a chunk
 * has arrived, its ingest and its rows of the finest A P start, followed by
 * the finest Galerkin rows of the coarse rows whose R rows end within the
 * chunks that have arrived; the results are the same bit for bit.  Every copy has ended when the call
 * returns, whatever its status.  Pinned host buffers give the full copy
 * rate.  The pattern must already be known (a previous amg_full_setup or
 * amg_step). */
amg_status amg_step_solve_host(amg_ctx *ctx, const double *h_val, const double *h_f, double *h_u,
                               double tol, amg_info *info);

/* Hierarchy inspection (for parity tests). */
amg_status amg_num_levels(const amg_ctx *ctx, int32_t *nlevels);
/* sizes[0..5] = n, nnz(A), nnz(P), nnz(R), nnz(A*P), number of aggregates */
amg_status amg_level_sizes(const amg_ctx *ctx, int32_t level, int64_t *sizes);
/* which: 0 = A_l, 1 = P_l, 2 = R_l; copies into caller device buffers sized
 * from amg_level_sizes (d_val gets FP64 values; any pointer may be NULL). */
amg_status amg_export_csr(amg_ctx *ctx, int32_t level, int32_t which, int32_t *d_ptr,
                          int32_t *d_col, double *d_val);
/* aggregate per row (-1 isolated), strong flag per entry of A_l, smoother
 * diagonal (FP64); any pointer may be NULL. */
amg_status amg_export_level_vec(amg_ctx *ctx, int32_t level, int32_t *d_agg, uint8_t *d_strong,
                                double *d_m);
/* How the finest level's matrix kernels read column indices (no counterpart
 * in the paper; an implementation detail reported for the roofline).  When
 * the pattern's rows use at most 256 distinct column offsets (column - row,
 * as a stencil's do), each entry's column is stored as one byte naming its
 * offset in a table: *col_bytes = 1 and *noffsets = the table's size.
 * Otherwise, after a full setup, when every offset fits in 16 bits, the
 * offsets themselves are read: *col_bytes = 2 (the coarser levels use the
 * same rule).  Otherwise the int32 columns: *col_bytes = 4; *noffsets = 0 in
 * both cases.  Values and arithmetic are the same either way.
 * AMG_ERR_STATE before a pattern is set. */
amg_status amg_pattern_info(const amg_ctx *ctx, int32_t *col_bytes, int32_t *noffsets);
/* Coarsest LU factors (n_L x n_L row-major, FP64) and pivots. */
amg_status amg_export_coarse_lu(amg_ctx *ctx, double *d_lu, int32_t *d_piv);

/* Instrumentation (no counterpart in the paper; used to report per-kernel
 * time against the memory roofline).  amg_profile(ctx, 1) records a CUDA
 * event pair on the context's stream around every launch of the kernels named
 * by the AMG_PROF_* slots.  A CG solve is then run twice: once unprofiled (to
 * learn its iteration count K), then as one straight-line CUDA graph of K
 * iterations with event-record nodes, the last iteration untimed, so that the
 * timings carry no host launch gaps.  amg_profile(ctx, 2) times the
 * host-driven launch loop instead (each launch submitted from the host, the
 * state read back after every iteration); 0 switches timing off.
 * amg_profile_read synchronises the stream, returns the summed milliseconds
 * and the number of timed launches of one slot and clears it.
 * amg_kernel_launches returns the number of kernels this library has launched
 * in the process so far (all contexts). */
enum {
    AMG_PROF_CG_SPMV = 0,      /* CG: q = A p fused with p.q (fine level, FP64) */
    AMG_PROF_SMOOTH0_L0 = 1,   /* V-cycle, finest level: zero-guess smoothing + residual */
    AMG_PROF_SWEEP_L0 = 2,     /* V-cycle, finest level: last post-smoothing sweep */
    AMG_PROF_RESTRICT_L0 = 3,  /* V-cycle: f_2 = R r on the finest level */
    AMG_PROF_PROLONG_L0 = 4,   /* V-cycle: u += P u_2 on the finest level */
    AMG_PROF_AP_L0 = 5,        /* Galerkin stage 1 on the finest level: A P */
    AMG_PROF_RAP_L0 = 6,       /* Galerkin stage 2 on the finest level: R (A P) */
    AMG_PROF_INGEST = 7,       /* fine values in: copy / cast / smoother */
    AMG_PROF_LU = 8,           /* coarsest dense LU */
    AMG_PROF_INV = 9,          /* coarsest explicit inverse */
    AMG_PROF_CG_UPDATE = 10,   /* CG: u += alpha p, r -= alpha q, r.r */
    AMG_PROF_CG_P = 11,        /* CG: p = z + beta p */
    AMG_PROF_DOT = 12,         /* CG: r.z */
    AMG_PROF_COARSE = 13,      /* coarsest solve (dense inverse times vector) */
    AMG_PROF_EMPTY = 14,       /* an empty event pair in the same stream or graph: the timing overhead */
    AMG_PROF_GALERKIN = 15,    /* numeric Galerkin product of every level (one pair per level) */
    AMG_PROF_SMOOTHERS = 16,   /* smoother diagonals of the coarse levels (one pair per level) */
    AMG_PROF_NSLOTS = 17
};
amg_status amg_profile(amg_ctx *ctx, int32_t enable);
amg_status amg_profile_read(amg_ctx *ctx, int32_t slot, double *total_ms, int64_t *launches);
int64_t amg_kernel_launches(void);

/* Synthetic pressure-Poisson workload: -div((1/rho) grad p) on an N^dim cell
 * grid (dim 2 or 3), harmonic face coefficients 2/(rho_i + rho_j), Dirichlet
 * p = 0 on the top face through a ghost cell (A_ii += 2/rho_i) when
 * dirichlet_top != 0, Neumann elsewhere.  It stands in for the dam-break
 * matrices of Sec. 4.  Pattern: n = N^dim rows, nnz from amg_poisson_nnz. */
int64_t amg_poisson_nnz(int32_t dim, int32_t N);
amg_status amg_poisson_pattern(int32_t dim, int32_t N, int32_t *d_ptr, int32_t *d_col, void *cuda_stream);
amg_status amg_poisson_values(int32_t dim, int32_t N, int32_t dirichlet_top, const double *d_rho,
                              const int32_t *d_ptr, double *d_val, void *cuda_stream);
/* Level-set transport stand-in (Sec. 4, eq. 5): an implicit upwind
 * convection-diffusion step on the same pattern as amg_poisson_pattern (a
 * nonsymmetric M-matrix).  Row c, with w_f the outward flux through face f
 * (+velocity on the high face, -velocity on the low face, walls excluded):
 * A_cj = min(w_f, 0) - 0.1, A_cc = 1 + sum over faces in column order of
 * (max(w_f, 0) + 0.1).  Face velocities (device, FP64, x fastest):
 * d_fx[(z N + y)(N + 1) + x_face], d_fy[(z (N + 1) + y_face) N + x],
 * d_fz[(z_face N + y) N + x] (dim 3; ignored and may be NULL in 2D, where
 * z = 0).  d_val: nnz doubles in the order of amg_poisson_pattern's columns.
 * Asynchronous on cuda_stream. */
amg_status amg_levelset_values(int32_t dim, int32_t N, const double *d_fx, const double *d_fy,
                               const double *d_fz, const int32_t *d_ptr, double *d_val,
                               void *cuda_stream);
/* Monolithic Navier-Stokes stand-in (Sec. 4), 4 x 4 blocks (u, v, w, p)
 * per cell of an N^3 grid, on the pattern of amg_poisson_pattern(3, N): an
 * Oseen-type system in balanced form (pressure unknowns scaled by
 * kappa = mass rho + 6 mu).  For the face f between cells c and j in
 * direction d, side s = -1 / +1, outward flux phi = s * face velocity,
 * mu_f = (2 mu_c mu_j) / (mu_c + mu_j), beta_f = 2 / (1/kappa_c + 1/kappa_j):
 *   block (c, j): velocity diagonal min(phi, 0) - mu_f; (u_d, p) = (p, u_d)
 *     = (s / 2) beta_f; (p, p) = -beta_f.
 *   block (c, c): velocity diagonal mass rho_c + sum of (mu_f + max(phi, 0))
 *     + 2 mu_c per wall face; (u_d, p) = -(p, u_d) = sum over the wall
 *     faces of direction d of (s / 2) kappa_c; (p, p) = sum of beta_f, plus
 *     2 kappa_c on the top face (z = N - 1).
 * The pressure part is the pressure Poisson matrix of density 1/kappa, the
 * velocity-pressure coupling is skew-symmetric and the symmetric part is
 * positive definite.  d_rho, d_mu: N^3 doubles; face velocities as in
 * amg_levelset_values (dim 3); d_val: 16 * amg_poisson_nnz(3, N) doubles.
 * Asynchronous on cuda_stream. */
amg_status amg_stokes_values(int32_t N, const double *d_rho, const double *d_mu, const double *d_fx,
                             const double *d_fy, const double *d_fz, double mass, const int32_t *d_ptr,
                             double *d_val, void *cuda_stream);
/* Adjoint chain rule for theta = log rho: given u (A u = f) and lam
 * (A lam = dL/du), grad = dL/dtheta per cell (n doubles). */
amg_status amg_poisson_grad_theta(int32_t dim, int32_t N, int32_t dirichlet_top, const double *d_rho,
                                  const double *d_u, const double *d_lam, double *d_grad,
                                  void *cuda_stream);
/* The same two calls with the per-cell log-density theta = log rho as input
 * (device, n doubles): each kernel forms rho = exp(theta) itself, so a
 * differentiable solve over theta does all of its arithmetic in the library.
 * amg_poisson_values_log: the values of amg_poisson_values for rho = exp(theta).
 * amg_poisson_grad_log: dL/dtheta per cell, as amg_poisson_grad_theta for
 * rho = exp(theta), with the face terms -(lam_c - lam_j)(u_c - u_j) chained
 * through dk_f/dtheta_c = -2 rho_c / (rho_c + rho_j)^2 and the Dirichlet term
 * (-lam_c u_c)(-2 / rho_c).  Both asynchronous on cuda_stream; AMG_ERR_ARG on
 * a bad size or a null pointer. */
amg_status amg_poisson_values_log(int32_t dim, int32_t N, int32_t dirichlet_top, const double *d_theta,
                                  const int32_t *d_ptr, double *d_val, void *cuda_stream);
amg_status amg_poisson_grad_log(int32_t dim, int32_t N, int32_t dirichlet_top, const double *d_theta,
                                const double *d_u, const double *d_lam, double *d_grad, void *cuda_stream);

/* Allocation-free variant of amg_poisson_pattern (no counterpart in the
 * paper).  It exists for callers that must not allocate device memory at
 * the time of the call: a host framework whose caching allocator already
 * holds nearly all of the GPU's memory, or a latency-critical loop that
 * forbids allocation once it runs.  Same outputs as amg_poisson_pattern
 * (d_ptr: n + 1 int32, d_col: amg_poisson_nnz(dim, N) int32, device), written
 * in order on cuda_stream (asynchronous: the call does not synchronise).
 * It calls no allocator: the row lengths are scanned in place in d_ptr and
 * the scan's block sums live in a fixed device array inside the library
 * (about 128 KiB, held by every device that loads the library until the
 * process exits).
 *  - n = N^dim must not exceed AMG_NOALLOC_MAX_CELLS: larger grids return
 *    AMG_ERR_CAPACITY without launching anything.
 *  - The first call on a device looks up that array's device address (once
 *    per device, with that device current); make this first call before any
 *    stream capture.  The address is kept for the life of the process: after
 *    a cudaDeviceReset of a device, do not call this entry point on it again.
 *  - A CUDA error already pending when it is called (from earlier work) is
 *    returned as AMG_ERR_CUDA without launching anything and is not cleared.
 *  - All calls share the one array and it keeps the last call's contents;
 *    each call writes every entry it reads, so nothing needs clearing, but
 *    calls whose work overlaps on the GPU (on different streams, or from
 *    different threads) race on it: order them on one stream or synchronise. */
#define AMG_NOALLOC_MAX_CELLS (1LL << 26)
amg_status amg_poisson_pattern_noalloc(int32_t dim, int32_t N, int32_t *d_ptr, int32_t *d_col,
                                       void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* AMGPR_H */
