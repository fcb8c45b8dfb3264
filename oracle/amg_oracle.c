/*
 * amg_oracle.c -- serial FP64 oracle for partial-reuse smoothed-aggregation AMG.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (Demidov, "Partial reuse AMG setup cost amortization
 * strategy for the solution of non-steady state problems", arXiv 2108.02054):
 *   - Alg. 1 (AMG setup): per level, strength of connection, aggregation,
 *     smoothed prolongation P, R = P^T, smoother, Galerkin A_{l+1} = R A_l P,
 *     and a direct solver (dense LU) for the coarsest level.
 *   - Alg. 4 (partial reuse): keep P and R, per level rebuild the smoother and
 *     A_{l+1} = R A_l P numerically over the cached coarse pattern (Sec. 5 notes
 *     the symbolic phase of the product can be reused), refactor the LU.
 *   - Alg. 2 (V-cycle) used once per iteration as the preconditioner of CG
 *     (Sec. 2: a single V-cycle per preconditioning step).
 *   - The adjoint gradient of L = 1/2 |u - u*|^2 w.r.t. log-density per cell
 *     for the variable-coefficient Poisson assembly below.
 *   - Sec. 4's nonsymmetric systems: a level-set transport stand-in solved
 *     with right-preconditioned BiCGStab, and a monolithic 4 x 4 block
 *     (u, v, w, p) system standing in for the Navier-Stokes matrices, with a
 *     block-valued hierarchy (non-smoothed aggregation on the node graph of
 *     block norms, damped block Jacobi, BiCGStab), as the paper runs them.
 *
 * The paper delegates the smoothed-aggregation construction to its library;
 * the readings used here (strength test, aggregation order, P smoothing, the
 * summation order of every reduction) are fixed below, one per function.
 * Floating point: plain C doubles, built with -ffp-contract=off; every
 * accumulation that the GPU path must reproduce bit for bit uses C99 fma()
 * explicitly, everything else is separate multiply / add.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOT_CONVERGED 1
#define ORC_ERR_ARG (-1)
#define ORC_ERR_STATE (-2)
#define ORC_ERR_PATTERN (-3)
#define ORC_ERR_BREAKDOWN (-4)
#define ORC_ERR_SINGULAR (-8)

typedef struct {
    int32_t nrows, ncols;
    int32_t *ptr, *col;
    double *val;
} ocsr;

typedef struct {
    ocsr A;           /* level operator (pattern fixed after the full setup) */
    ocsr P, R;        /* kept across partial rebuilds */
    ocsr AP;          /* cached pattern of A*P (values are scratch) */
    int32_t *agg;     /* aggregate of each row, -1 = isolated */
    uint8_t *strong;  /* per entry of A: 1 if the connection is strong */
    int32_t nroots;
    double *m;        /* smoother diagonal */
    double *u, *f, *r; /* V-cycle work vectors */
} olevel;

typedef struct {
    double theta, omega, jacobi_omega;
    int smoother;      /* 0 = SPAI0, 1 = damped Jacobi */
    int npre, npost, coarse_enough, max_levels;
    int theta_halving; /* 1: theta_{l+1} = theta_l / 2 */
    int smoothed;      /* 1: smoothed aggregation, 0: plain (tentative) P */
} oparams;

typedef struct {
    oparams prm;
    int nlev;
    olevel lev[32];
    int nL;            /* size of the coarsest system */
    double *LU;        /* nL x nL row-major factors */
    int32_t *piv;
    double *wq, *wz, *wp, *wr; /* PCG work vectors (fine size) */
} ohier;

static void *xcalloc(size_t n, size_t sz) {
    if (n == 0) n = 1;
    return calloc(n, sz);
}

static void csr_free(ocsr *a) {
    free(a->ptr); free(a->col); free(a->val);
    memset(a, 0, sizeof(*a));
}

/* ------------------------------------------------------------------------ */
/* Problem assembly: variable-coefficient pressure Poisson -div((1/rho) grad p)
 * on an N^dim cell grid, cell index x + N*y (+ N^2*z), harmonic face
 * coefficients k_f = 2/(rho_i + rho_j), Dirichlet p = 0 on the top face (last
 * coordinate = N-1) through a ghost cell (A_ii += 2/rho_i), Neumann elsewhere.
 * Row entries are written in ascending column order; the diagonal is the sum of
 * the face coefficients in that order, then the Dirichlet term.
 * (Sec. 4 uses a two-fluid dam break; this synthetic system stands in for it.) */
long long orc_poisson_nnz(int dim, int N) {
    long long n1 = N, nf = (long long)(N - 1);
    if (dim == 2) return n1 * n1 + 4 * nf * n1;
    return n1 * n1 * n1 + 6 * nf * n1 * n1;
}

int orc_poisson_assemble(int dim, int N, int dirichlet_top, const double *rho,
                         int32_t *ptr, int32_t *col, double *val) {
    if ((dim != 2 && dim != 3) || N < 1) return ORC_ERR_ARG;
    long long n = (dim == 2) ? (long long)N * N : (long long)N * N * N;
    long long pos = 0;
    long long s1 = 1, s2 = N, s3 = (long long)N * N;
    for (long long c = 0; c < n; ++c) {
        long long x = c % N, y = (c / N) % N, z = (dim == 3) ? c / s3 : 0;
        long long nb[7];
        int nnb = 0;
        /* neighbours in ascending index order, the diagonal slot marked -1 */
        if (dim == 3 && z > 0) nb[nnb++] = c - s3;
        if (y > 0) nb[nnb++] = c - s2;
        if (x > 0) nb[nnb++] = c - s1;
        nb[nnb++] = -1;
        if (x < N - 1) nb[nnb++] = c + s1;
        if (y < N - 1) nb[nnb++] = c + s2;
        if (dim == 3 && z < N - 1) nb[nnb++] = c + s3;
        int top = (dim == 2) ? (y == N - 1) : (z == N - 1);
        ptr[c] = (int32_t)pos;
        double diag = 0.0;
        long long dpos = -1;
        for (int t = 0; t < nnb; ++t) {
            if (nb[t] < 0) {
                dpos = pos;
                col[pos++] = (int32_t)c;
                continue;
            }
            double k = 2.0 / (rho[c] + rho[nb[t]]);
            diag = diag + k;
            col[pos] = (int32_t)nb[t];
            val[pos++] = -k;
        }
        if (dirichlet_top && top) diag = diag + 2.0 / rho[c];
        val[dpos] = diag;
    }
    ptr[n] = (int32_t)pos;
    return ORC_OK;
}

/* Level-set transport step (the stand-in for eq. 5 of Sec. 4): implicit
 * upwind convection with diffusion on the same pattern,
 *   A_cc = 1 + sum_f (max(w_f, 0) + 0.1),  A_cj = min(w_f, 0) - 0.1,
 * where w_f is the outward (Courant-scaled) face velocity of cell c, taken
 * from the face arrays fx ((N+1) x N (x N)), fy, fz (x fastest); the diagonal
 * starts at 1 and adds the face terms in ascending neighbour order. */
int orc_levelset_assemble(int dim, int N, const double *fx, const double *fy, const double *fz,
                          int32_t *ptr, int32_t *col, double *val) {
    if ((dim != 2 && dim != 3) || N < 1) return ORC_ERR_ARG;
    long long n = (dim == 2) ? (long long)N * N : (long long)N * N * N;
    long long pos = 0;
    const long long N1 = N + 1;
    for (long long c = 0; c < n; ++c) {
        long long x = c % N, y = (c / N) % N, z = (dim == 3) ? c / ((long long)N * N) : 0;
        long long nb[7];
        double w[7];
        int nnb = 0;
        /* face arrays: fx[(z*N + y)*(N+1) + x_face], fy[(z*(N+1) + y_face)*N + x],
         * fz[(z_face*N + y)*N + x] (2D: z = 0) */
        if (dim == 3 && z > 0) { nb[nnb] = c - (long long)N * N; w[nnb++] = -fz[(z * N + y) * N + x]; }
        if (y > 0) { nb[nnb] = c - N; w[nnb++] = -fy[(z * N1 + y) * N + x]; }
        if (x > 0) { nb[nnb] = c - 1; w[nnb++] = -fx[(z * N + y) * N1 + x]; }
        nb[nnb] = -1; w[nnb++] = 0.0;
        if (x < N - 1) { nb[nnb] = c + 1; w[nnb++] = fx[(z * N + y) * N1 + x + 1]; }
        if (y < N - 1) { nb[nnb] = c + N; w[nnb++] = fy[(z * N1 + y + 1) * N + x]; }
        if (dim == 3 && z < N - 1) { nb[nnb] = c + (long long)N * N; w[nnb++] = fz[((z + 1) * N + y) * N + x]; }
        ptr[c] = (int32_t)pos;
        double diag = 1.0;
        long long dpos = -1;
        for (int t = 0; t < nnb; ++t) {
            if (nb[t] < 0) { dpos = pos; col[pos++] = (int32_t)c; continue; }
            const double wf = w[t];
            diag = diag + ((wf > 0.0 ? wf : 0.0) + 0.1);
            col[pos] = (int32_t)nb[t];
            val[pos++] = (wf < 0.0 ? wf : 0.0) - 0.1;
        }
        val[dpos] = diag;
    }
    ptr[n] = (int32_t)pos;
    return ORC_OK;
}

/* Adjoint gradient (chain rule of the assembly above).  With A u = f and
 * A lam = u - u*, dL/dk_f = -(lam_i - lam_j)(u_i - u_j) for an interior face,
 * dL/dA_ii = -lam_i u_i for the Dirichlet term 2/rho_i.  rho = exp(theta):
 * dk_f/dtheta_i = -2 rho_i / (rho_i + rho_j)^2, d(2/rho_i)/dtheta_i = -2/rho_i. */
int orc_poisson_grad_theta(int dim, int N, int dirichlet_top, const double *rho,
                           const double *u, const double *lam, double *grad) {
    if ((dim != 2 && dim != 3) || N < 1) return ORC_ERR_ARG;
    long long n = (dim == 2) ? (long long)N * N : (long long)N * N * N;
    long long s3 = (long long)N * N;
    for (long long c = 0; c < n; ++c) grad[c] = 0.0;
    for (long long c = 0; c < n; ++c) {
        long long x = c % N, y = (c / N) % N, z = (dim == 3) ? c / s3 : 0;
        long long up[3];
        int nu = 0;
        if (x < N - 1) up[nu++] = c + 1;
        if (y < N - 1) up[nu++] = c + N;
        if (dim == 3 && z < N - 1) up[nu++] = c + s3;
        for (int t = 0; t < nu; ++t) {
            long long j = up[t];
            double dLdk = -(lam[c] - lam[j]) * (u[c] - u[j]);
            double s = rho[c] + rho[j];
            grad[c] += dLdk * (-2.0 * rho[c] / (s * s));
            grad[j] += dLdk * (-2.0 * rho[j] / (s * s));
        }
        int top = (dim == 2) ? (y == N - 1) : (z == N - 1);
        if (dirichlet_top && top) grad[c] += (-lam[c] * u[c]) * (-2.0 / rho[c]);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Pattern checks: sorted, in range, diagonal present. */
static int check_pattern(int32_t n, const int32_t *ptr, const int32_t *col) {
    if (ptr[0] != 0) return ORC_ERR_PATTERN;
    for (int32_t i = 0; i < n; ++i) {
        if (ptr[i + 1] < ptr[i]) return ORC_ERR_PATTERN;
        int has_diag = 0;
        for (int32_t p = ptr[i]; p < ptr[i + 1]; ++p) {
            if (col[p] < 0 || col[p] >= n) return ORC_ERR_PATTERN;
            if (p > ptr[i] && col[p] <= col[p - 1]) return ORC_ERR_PATTERN;
            if (col[p] == i) has_diag = 1;
        }
        if (!has_diag) return ORC_ERR_PATTERN;
    }
    return ORC_OK;
}

static int32_t find_col(const ocsr *a, int32_t row, int32_t c) {
    int32_t lo = a->ptr[row], hi = a->ptr[row + 1];
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (a->col[mid] < c) lo = mid + 1; else hi = mid;
    }
    return (lo < a->ptr[row + 1] && a->col[lo] == c) ? lo : -1;
}

/* ------------------------------------------------------------------------ */
/* Strength of connection (Vanek-Mandel-Brezina): entry (i,j), j != i, is
 * strong in row i's direction iff a_ij^2 > eps^2 |a_ii a_jj|, eps = theta_l.
 * The relation used for aggregation is symmetrised: (i,j) is strong iff the
 * test holds in either direction (identical to the one-sided test whenever A is
 * symmetric).  Products are separately rounded (no fused operations). */
static int dir_strong(double aij, double aii, double ajj, double eps2) {
    return aij * aij > eps2 * fabs(aii * ajj);
}

static void strength(const ocsr *A, double eps2, uint8_t *strong, const int32_t *dia) {
    int32_t n = A->nrows;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
            int32_t j = A->col[p];
            strong[p] = 0;
            if (j == i) continue;
            double aii = A->val[dia[i]], ajj = A->val[dia[j]];
            int s = dir_strong(A->val[p], aii, ajj, eps2);
            if (!s) {
                int32_t t = find_col(A, j, i);
                if (t >= 0) s = dir_strong(A->val[t], ajj, aii, eps2);
            }
            strong[p] = (uint8_t)s;
        }
    }
}

/* Fixed priority of node i: the murmur3 32-bit finaliser, a bijection on
 * 32-bit integers, so no two nodes share a priority. */
uint32_t orc_priority(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

typedef struct { uint32_t key; int32_t idx; } prio_item;
static int prio_desc(const void *a, const void *b) {
    uint32_t x = ((const prio_item *)a)->key, y = ((const prio_item *)b)->key;
    return (x < y) - (x > y);
}

/* Aggregation.  Roots form the greedy distance-2 independent set of the strong
 * graph (non-isolated nodes visited by decreasing priority: a node becomes a
 * root unless a root is already within two strong edges).  Phase 1: a root and
 * its strong neighbours form one aggregate.  Phase 2: every remaining
 * non-isolated node joins the phase-1 aggregate of its strong neighbour with the
 * largest |a_ij| (ties: the aggregate whose root has the larger priority).
 * Aggregates are numbered by ascending root index.  Returns the number of
 * aggregates, or a negative status. */
static int32_t aggregate(const ocsr *A, const uint8_t *strong, int32_t *agg) {
    int32_t n = A->nrows;
    int8_t *state = (int8_t *)xcalloc((size_t)n, 1); /* 0 undecided, 1 root, 2 excluded, 3 isolated */
    prio_item *order = (prio_item *)xcalloc((size_t)n, sizeof(prio_item));
    int32_t no = 0;
    for (int32_t i = 0; i < n; ++i) {
        int iso = 1;
        for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p)
            if (strong[p]) { iso = 0; break; }
        if (iso) { state[i] = 3; continue; }
        order[no].key = orc_priority((uint32_t)i);
        order[no].idx = i;
        ++no;
    }
    qsort(order, (size_t)no, sizeof(prio_item), prio_desc);
    for (int32_t t = 0; t < no; ++t) {
        int32_t v = order[t].idx;
        if (state[v] != 0) continue;
        state[v] = 1;
        for (int32_t p = A->ptr[v]; p < A->ptr[v + 1]; ++p) {
            if (!strong[p]) continue;
            int32_t j = A->col[p];
            if (state[j] == 0) state[j] = 2;
            for (int32_t q = A->ptr[j]; q < A->ptr[j + 1]; ++q) {
                if (!strong[q]) continue;
                int32_t l = A->col[q];
                if (state[l] == 0) state[l] = 2;
            }
        }
    }
    int32_t *root_id = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
    int32_t nagg = 0;
    for (int32_t i = 0; i < n; ++i) root_id[i] = (state[i] == 1) ? nagg++ : -1;
    int32_t *root_of = (int32_t *)xcalloc((size_t)nagg, sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) if (root_id[i] >= 0) root_of[root_id[i]] = i;
    /* phase 1 */
    int32_t *agg1 = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) {
        agg1[i] = -1;
        if (state[i] == 3) continue;
        if (state[i] == 1) { agg1[i] = root_id[i]; continue; }
        for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p)
            if (strong[p] && state[A->col[p]] == 1) { agg1[i] = root_id[A->col[p]]; break; }
    }
    /* phase 2 */
    int32_t status = nagg;
    for (int32_t i = 0; i < n; ++i) {
        agg[i] = agg1[i];
        if (state[i] == 3 || agg1[i] >= 0) continue;
        int32_t best = -1;
        double bestv = -1.0;
        uint32_t bestk = 0;
        for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
            if (!strong[p]) continue;
            int32_t j = A->col[p];
            if (agg1[j] < 0) continue;
            double v = fabs(A->val[p]);
            uint32_t k = orc_priority((uint32_t)root_of[agg1[j]]);
            if (best < 0 || v > bestv || (v == bestv && k > bestk)) {
                best = agg1[j]; bestv = v; bestk = k;
            }
        }
        if (best < 0) status = ORC_ERR_STATE; /* cannot happen for a maximal set */
        agg[i] = best;
    }
    free(state); free(order); free(root_id); free(root_of); free(agg1);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Prolongation.  Tentative P: P_tent[i, agg(i)] = 1 (isolated rows empty).
 * Filtered matrix A_F: diagonal d_i = a_ii + (weak off-diagonals of row i, added
 * in column order), strong off-diagonals kept.  Smoothed P = (I - w D_F^-1 A_F)
 * P_tent, entry by entry: P[i,c] = [c == agg(i)] - sum over j in {i} U strong(i)
 * with agg(j) = c, in column order, of (w * A_F[i,j]) / d_i.  The pattern is
 * structural (numeric zeros kept).  With smoothed = 0, P = P_tent. */
static int build_P(const ocsr *A, const uint8_t *strong, const int32_t *dia,
                   const int32_t *agg, int32_t nagg, double omega, int smoothed, ocsr *P) {
    int32_t n = A->nrows;
    P->nrows = n; P->ncols = nagg;
    P->ptr = (int32_t *)xcalloc((size_t)n + 1, sizeof(int32_t));
    /* pass 1: count */
    long long total = 0;
    int32_t maxrow = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t len = A->ptr[i + 1] - A->ptr[i];
        if (len > maxrow) maxrow = len;
    }
    int32_t *cols = (int32_t *)xcalloc((size_t)maxrow + 1, sizeof(int32_t));
    for (int pass = 0; pass < 2; ++pass) {
        total = 0;
        for (int32_t i = 0; i < n; ++i) {
            int32_t nc = 0;
            if (agg[i] >= 0) {
                if (smoothed) {
                    for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
                        int32_t j = A->col[p];
                        if (j != i && !strong[p]) continue;
                        int32_t c = agg[j];
                        if (c < 0) continue;
                        /* insert c into the sorted unique list */
                        int32_t t = nc;
                        int dup = 0;
                        for (int32_t s = 0; s < nc; ++s) if (cols[s] == c) { dup = 1; break; }
                        if (dup) continue;
                        while (t > 0 && cols[t - 1] > c) { cols[t] = cols[t - 1]; --t; }
                        cols[t] = c;
                        ++nc;
                    }
                } else {
                    cols[0] = agg[i];
                    nc = 1;
                }
            }
            if (pass == 0) {
                P->ptr[i + 1] = nc;
            } else {
                int32_t base = P->ptr[i];
                double d = A->val[dia[i]];
                if (smoothed) {
                    for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p)
                        if (A->col[p] != i && !strong[p]) d = d + A->val[p];
                }
                for (int32_t s = 0; s < nc; ++s) {
                    int32_t c = cols[s];
                    double v = (c == agg[i]) ? 1.0 : 0.0;
                    if (smoothed) {
                        for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
                            int32_t j = A->col[p];
                            if (j != i && !strong[p]) continue;
                            if (agg[j] != c) continue;
                            double w = (j == i) ? d : A->val[p];
                            v = v - (omega * w) / d;
                        }
                    }
                    P->col[base + s] = c;
                    P->val[base + s] = v;
                }
            }
            total += nc;
        }
        if (pass == 0) {
            for (int32_t i = 0; i < n; ++i) P->ptr[i + 1] += P->ptr[i];
            P->col = (int32_t *)xcalloc((size_t)total, sizeof(int32_t));
            P->val = (double *)xcalloc((size_t)total, sizeof(double));
        }
    }
    free(cols);
    return ORC_OK;
}

/* R = P^T as an explicit CSR; each row lists its fine indices in ascending order. */
static void transpose(const ocsr *P, ocsr *R) {
    int32_t n = P->nrows, nc = P->ncols;
    R->nrows = nc; R->ncols = n;
    R->ptr = (int32_t *)xcalloc((size_t)nc + 1, sizeof(int32_t));
    int32_t nnz = P->ptr[n];
    R->col = (int32_t *)xcalloc((size_t)nnz, sizeof(int32_t));
    R->val = (double *)xcalloc((size_t)nnz, sizeof(double));
    for (int32_t p = 0; p < nnz; ++p) R->ptr[P->col[p] + 1]++;
    for (int32_t c = 0; c < nc; ++c) R->ptr[c + 1] += R->ptr[c];
    int32_t *cur = (int32_t *)xcalloc((size_t)nc + 1, sizeof(int32_t));
    memcpy(cur, R->ptr, sizeof(int32_t) * (size_t)nc);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t p = P->ptr[i]; p < P->ptr[i + 1]; ++p) {
            int32_t c = P->col[p];
            R->col[cur[c]] = i;
            R->val[cur[c]] = P->val[p];
            cur[c]++;
        }
    free(cur);
}

/* ------------------------------------------------------------------------ */
/* Sparse product pattern: row i of C = sorted union over k in row i of X of the
 * columns of row k of Y (optionally with the diagonal added). */
static void spgemm_pattern(const ocsr *X, const ocsr *Y, int add_diag, ocsr *C) {
    int32_t n = X->nrows, nc = Y->ncols;
    int32_t *mark = (int32_t *)xcalloc((size_t)nc, sizeof(int32_t));
    for (int32_t c = 0; c < nc; ++c) mark[c] = -1;
    C->nrows = n; C->ncols = nc;
    C->ptr = (int32_t *)xcalloc((size_t)n + 1, sizeof(int32_t));
    long long total = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t cnt = 0;
        if (add_diag && i < nc) { mark[i] = i; ++cnt; }
        for (int32_t p = X->ptr[i]; p < X->ptr[i + 1]; ++p) {
            int32_t k = X->col[p];
            for (int32_t q = Y->ptr[k]; q < Y->ptr[k + 1]; ++q) {
                int32_t c = Y->col[q];
                if (mark[c] != i) { mark[c] = i; ++cnt; }
            }
        }
        total += cnt;
        C->ptr[i + 1] = (int32_t)total;
    }
    C->col = (int32_t *)xcalloc((size_t)total, sizeof(int32_t));
    C->val = (double *)xcalloc((size_t)total, sizeof(double));
    for (int32_t c = 0; c < nc; ++c) mark[c] = -1;
    for (int32_t i = 0; i < n; ++i) {
        int32_t pos = C->ptr[i];
        if (add_diag && i < nc) { mark[i] = i; C->col[pos++] = i; }
        for (int32_t p = X->ptr[i]; p < X->ptr[i + 1]; ++p) {
            int32_t k = X->col[p];
            for (int32_t q = Y->ptr[k]; q < Y->ptr[k + 1]; ++q) {
                int32_t c = Y->col[q];
                if (mark[c] != i) { mark[c] = i; C->col[pos++] = c; }
            }
        }
        /* insertion sort of the row */
        for (int32_t a = C->ptr[i] + 1; a < pos; ++a) {
            int32_t v = C->col[a], b = a;
            while (b > C->ptr[i] && C->col[b - 1] > v) { C->col[b] = C->col[b - 1]; --b; }
            C->col[b] = v;
        }
    }
    free(mark);
}

/* Numeric product over a known pattern: C[i,c] = sum over k in row i of X (in
 * column order) and, within it, over the entries of row k of Y (in column
 * order) of X[i,k] * Y[k,c], accumulated with one fma per term from 0.0. */
static int spgemm_numeric(const ocsr *X, const ocsr *Y, ocsr *C, int32_t *pos) {
    /* pos: scratch of size Y->ncols, all -1 on entry and on exit */
    int32_t n = X->nrows;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t e = C->ptr[i]; e < C->ptr[i + 1]; ++e) { pos[C->col[e]] = e; C->val[e] = 0.0; }
        for (int32_t p = X->ptr[i]; p < X->ptr[i + 1]; ++p) {
            int32_t k = X->col[p];
            double x = X->val[p];
            for (int32_t q = Y->ptr[k]; q < Y->ptr[k + 1]; ++q) {
                int32_t e = pos[Y->col[q]];
                if (e < 0) return ORC_ERR_PATTERN;
                C->val[e] = fma(x, Y->val[q], C->val[e]);
            }
        }
        for (int32_t e = C->ptr[i]; e < C->ptr[i + 1]; ++e) pos[C->col[e]] = -1;
    }
    return ORC_OK;
}

/* Galerkin product A_c = R (A P): first AP row by row, then R times AP. */
static int galerkin_numeric(olevel *L, ocsr *Ac) {
    int32_t nmax = L->A.ncols > L->P.ncols ? L->A.ncols : L->P.ncols;
    int32_t *pos = (int32_t *)xcalloc((size_t)nmax, sizeof(int32_t));
    for (int32_t c = 0; c < nmax; ++c) pos[c] = -1;
    int st = spgemm_numeric(&L->A, &L->P, &L->AP, pos);
    if (st == ORC_OK) st = spgemm_numeric(&L->R, &L->AP, Ac, pos);
    free(pos);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Smoother diagonal.  SPAI0: m_i = a_ii / sum_j a_ij^2 (the diagonal M that
 * minimises |I - M A|_F row by row), 0 for an empty denominator; the sum runs in
 * column order with fma.  Damped Jacobi: m_i = w_J / a_ii. */
static void smoother_build(const ocsr *A, const int32_t *dia, int type, double wj, double *m) {
    for (int32_t i = 0; i < A->nrows; ++i) {
        double aii = A->val[dia[i]];
        if (type == 0) {
            double s = 0.0;
            for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) s = fma(A->val[p], A->val[p], s);
            m[i] = (s != 0.0) ? aii / s : 0.0;
        } else {
            m[i] = (aii != 0.0) ? wj / aii : 0.0;
        }
    }
}

/* Dense LU with partial pivoting (pivot: first entry of largest magnitude in
 * the column), in place, row-major. */
static int dense_lu(int n, double *a, int32_t *piv) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(a[(size_t)k * n + k]);
        for (int r = k + 1; r < n; ++r) {
            double v = fabs(a[(size_t)r * n + k]);
            if (v > best) { best = v; p = r; }
        }
        piv[k] = p;
        if (best == 0.0) return ORC_ERR_SINGULAR;
        if (p != k)
            for (int c = 0; c < n; ++c) {
                double t = a[(size_t)k * n + c];
                a[(size_t)k * n + c] = a[(size_t)p * n + c];
                a[(size_t)p * n + c] = t;
            }
        double akk = a[(size_t)k * n + k];
        for (int r = k + 1; r < n; ++r) {
            double l = a[(size_t)r * n + k] / akk;
            a[(size_t)r * n + k] = l;
            for (int c = k + 1; c < n; ++c)
                a[(size_t)r * n + c] = fma(-l, a[(size_t)k * n + c], a[(size_t)r * n + c]);
        }
    }
    return ORC_OK;
}

static void dense_lu_solve(int n, const double *a, const int32_t *piv, const double *b, double *x) {
    for (int i = 0; i < n; ++i) x[i] = b[i];
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    for (int r = 0; r < n; ++r) {
        double s = x[r];
        for (int c = 0; c < r; ++c) s = fma(-a[(size_t)r * n + c], x[c], s);
        x[r] = s;
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = x[r];
        for (int c = r + 1; c < n; ++c) s = fma(-a[(size_t)r * n + c], x[c], s);
        x[r] = s / a[(size_t)r * n + r];
    }
}

/* ------------------------------------------------------------------------ */
static int32_t *diag_positions(const ocsr *A) {
    int32_t *dia = (int32_t *)xcalloc((size_t)A->nrows, sizeof(int32_t));
    for (int32_t i = 0; i < A->nrows; ++i) dia[i] = find_col(A, i, i);
    return dia;
}

static void level_free(olevel *L) {
    csr_free(&L->A); csr_free(&L->P); csr_free(&L->R); csr_free(&L->AP);
    free(L->agg); free(L->strong); free(L->m); free(L->u); free(L->f); free(L->r);
    memset(L, 0, sizeof(*L));
}

void orc_destroy(ohier *h) {
    if (!h) return;
    for (int l = 0; l < h->nlev; ++l) level_free(&h->lev[l]);
    free(h->LU); free(h->piv); free(h->wq); free(h->wz); free(h->wp); free(h->wr);
    free(h);
}

/* Refactor the coarsest direct solver from the current values of A_L. */
static int coarse_factor(ohier *h) {
    olevel *L = &h->lev[h->nlev - 1];
    int n = L->A.nrows;
    memset(h->LU, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int i = 0; i < n; ++i)
        for (int32_t p = L->A.ptr[i]; p < L->A.ptr[i + 1]; ++p)
            h->LU[(size_t)i * n + L->A.col[p]] = L->A.val[p];
    return dense_lu(n, h->LU, h->piv);
}

/* Alg. 4 body: smoothers and Galerkin operators of every level from new fine
 * values on the fixed pattern, then the coarsest factorisation.  The full
 * setup runs the same numeric routines, so a rebuild on unchanged values
 * reproduces it exactly. */
int orc_rebuild(ohier *h, const double *val) {
    if (!h) return ORC_ERR_STATE;
    olevel *L1 = &h->lev[0];
    memcpy(L1->A.val, val, sizeof(double) * (size_t)L1->A.ptr[L1->A.nrows]);
    for (int l = 0; l < h->nlev; ++l) {
        olevel *L = &h->lev[l];
        int32_t *dia = diag_positions(&L->A);
        if (l < h->nlev - 1)
            smoother_build(&L->A, dia, h->prm.smoother, h->prm.jacobi_omega, L->m);
        free(dia);
        if (l < h->nlev - 1) {
            int st = galerkin_numeric(L, &h->lev[l + 1].A);
            if (st) return st;
        }
    }
    return coarse_factor(h);
}

/* Alg. 1: full setup from a CSR matrix (sorted columns, diagonal present). */
ohier *orc_setup(int32_t n, const int32_t *ptr, const int32_t *col, const double *val,
                 const double *dprm, const int32_t *iprm, int *status) {
    *status = ORC_OK;
    if (n <= 0 || check_pattern(n, ptr, col) != ORC_OK) { *status = ORC_ERR_PATTERN; return NULL; }
    ohier *h = (ohier *)xcalloc(1, sizeof(ohier));
    h->prm.theta = dprm[0]; h->prm.omega = dprm[1]; h->prm.jacobi_omega = dprm[2];
    h->prm.smoother = iprm[0]; h->prm.npre = iprm[1]; h->prm.npost = iprm[2];
    h->prm.coarse_enough = iprm[3]; h->prm.max_levels = iprm[4];
    h->prm.theta_halving = iprm[5]; h->prm.smoothed = iprm[6];
    if (h->prm.max_levels > 32) h->prm.max_levels = 32;
    if (h->prm.max_levels < 1) h->prm.max_levels = 1;
    olevel *L = &h->lev[0];
    int32_t nnz = ptr[n];
    L->A.nrows = L->A.ncols = n;
    L->A.ptr = (int32_t *)xcalloc((size_t)n + 1, sizeof(int32_t));
    L->A.col = (int32_t *)xcalloc((size_t)nnz, sizeof(int32_t));
    L->A.val = (double *)xcalloc((size_t)nnz, sizeof(double));
    memcpy(L->A.ptr, ptr, sizeof(int32_t) * ((size_t)n + 1));
    memcpy(L->A.col, col, sizeof(int32_t) * (size_t)nnz);
    memcpy(L->A.val, val, sizeof(double) * (size_t)nnz);
    h->nlev = 1;
    double theta = h->prm.theta;
    for (;;) {
        L = &h->lev[h->nlev - 1];
        int32_t nl = L->A.nrows;
        L->u = (double *)xcalloc((size_t)nl, sizeof(double));
        L->f = (double *)xcalloc((size_t)nl, sizeof(double));
        L->r = (double *)xcalloc((size_t)nl, sizeof(double));
        L->m = (double *)xcalloc((size_t)nl, sizeof(double));
        L->agg = (int32_t *)xcalloc((size_t)nl, sizeof(int32_t));
        for (int32_t i = 0; i < nl; ++i) L->agg[i] = -1;
        L->strong = (uint8_t *)xcalloc((size_t)L->A.ptr[nl], 1);
        if (nl <= h->prm.coarse_enough || h->nlev >= h->prm.max_levels) break;
        int32_t *dia = diag_positions(&L->A);
        strength(&L->A, theta * theta, L->strong, dia);
        int32_t nagg = aggregate(&L->A, L->strong, L->agg);
        if (nagg < 0) { free(dia); *status = nagg; orc_destroy(h); return NULL; }
        if (nagg == 0 || nagg >= nl) {
            for (int32_t i = 0; i < nl; ++i) L->agg[i] = -1;
            memset(L->strong, 0, (size_t)L->A.ptr[nl]);
            free(dia);
            break;
        }
        L->nroots = nagg;
        build_P(&L->A, L->strong, dia, L->agg, nagg, h->prm.omega, h->prm.smoothed, &L->P);
        free(dia);
        transpose(&L->P, &L->R);
        spgemm_pattern(&L->A, &L->P, 0, &L->AP);
        olevel *C = &h->lev[h->nlev];
        spgemm_pattern(&L->R, &L->AP, 1, &C->A);
        C->A.ncols = nagg;
        /* the next level's strength test needs its values now */
        int gst = galerkin_numeric(L, &C->A);
        h->nlev++;
        if (gst) { *status = gst; orc_destroy(h); return NULL; }
        if (h->prm.theta_halving) theta = theta * 0.5;
    }
    h->nL = h->lev[h->nlev - 1].A.nrows;
    h->LU = (double *)xcalloc((size_t)h->nL * (size_t)h->nL, sizeof(double));
    h->piv = (int32_t *)xcalloc((size_t)h->nL, sizeof(int32_t));
    h->wq = (double *)xcalloc((size_t)n, sizeof(double));
    h->wz = (double *)xcalloc((size_t)n, sizeof(double));
    h->wp = (double *)xcalloc((size_t)n, sizeof(double));
    h->wr = (double *)xcalloc((size_t)n, sizeof(double));
    /* a singular coarsest matrix (e.g. a pure-Neumann operator) still yields a
     * usable hierarchy for inspection; the status reports it */
    int st = orc_rebuild(h, val);
    if (st == ORC_ERR_SINGULAR) { *status = st; return h; }
    if (st) { *status = st; orc_destroy(h); return NULL; }
    return h;
}

/* ------------------------------------------------------------------------ */
/* y = A x (row sums in column order, fma). */
static void spmv(const ocsr *A, const double *vals, const double *x, double *y) {
    for (int32_t i = 0; i < A->nrows; ++i) {
        double s = 0.0;
        for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) s = fma(vals[p], x[A->col[p]], s);
        y[i] = s;
    }
}

/* u <- u + m o (f - A u) */
static void smooth_sweep(const olevel *L, double *u, const double *f, double *tmp) {
    spmv(&L->A, L->A.val, u, tmp);
    for (int32_t i = 0; i < L->A.nrows; ++i) tmp[i] = f[i] - tmp[i];
    for (int32_t i = 0; i < L->A.nrows; ++i) u[i] = fma(L->m[i], tmp[i], u[i]);
}

/* Alg. 2 as a preconditioner: one V-cycle from a zero initial guess. */
static void vcycle_level(ohier *h, int l) {
    olevel *L = &h->lev[l];
    int32_t n = L->A.nrows;
    if (l == h->nlev - 1) {
        dense_lu_solve(n, h->LU, h->piv, L->f, L->u);
        return;
    }
    for (int32_t i = 0; i < n; ++i) L->u[i] = 0.0;
    for (int s = 0; s < h->prm.npre; ++s) smooth_sweep(L, L->u, L->f, L->r);
    spmv(&L->A, L->A.val, L->u, L->r);
    for (int32_t i = 0; i < n; ++i) L->r[i] = L->f[i] - L->r[i];
    olevel *C = &h->lev[l + 1];
    spmv(&L->R, L->R.val, L->r, C->f);
    vcycle_level(h, l + 1);
    for (int32_t i = 0; i < n; ++i) {
        double s = L->u[i];
        for (int32_t p = L->P.ptr[i]; p < L->P.ptr[i + 1]; ++p)
            s = fma(L->P.val[p], C->u[L->P.col[p]], s);
        L->u[i] = s;
    }
    for (int s = 0; s < h->prm.npost; ++s) smooth_sweep(L, L->u, L->f, L->r);
}

void orc_vcycle(ohier *h, const double *r, double *z) {
    olevel *L = &h->lev[0];
    memcpy(L->f, r, sizeof(double) * (size_t)L->A.nrows);
    vcycle_level(h, 0);
    memcpy(z, L->u, sizeof(double) * (size_t)L->A.nrows);
}

static double dot(int32_t n, const double *x, const double *y) {
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) s = fma(x[i], y[i], s);
    return s;
}

/* Preconditioned CG (Hestenes-Stiefel) from u = 0.  Convergence: recurrence
 * residual |r|/|f| <= tol, confirmed by the true residual f - A u; if the true
 * residual misses tol, r is replaced by it and the iteration continues (at
 * most twice).  sys_val: values of the system matrix on the level-1 pattern
 * (NULL = the hierarchy's own level-1 values). */
int orc_pcg(ohier *h, const double *sys_val, const double *f, double *u, double tol,
            int maxiter, int *iters, double *relres) {
    olevel *L = &h->lev[0];
    int32_t n = L->A.nrows;
    const double *av = sys_val ? sys_val : L->A.val;
    double *r = h->wr, *z = h->wz, *p = h->wp, *q = h->wq;
    for (int32_t i = 0; i < n; ++i) { u[i] = 0.0; r[i] = f[i]; }
    double nf = sqrt(dot(n, f, f));
    *iters = 0;
    *relres = 0.0;
    if (nf == 0.0) return ORC_OK;
    orc_vcycle(h, r, z);
    for (int32_t i = 0; i < n; ++i) p[i] = z[i];
    double rz = dot(n, r, z);
    int replacements = 0;
    int status = ORC_NOT_CONVERGED;
    for (int it = 1; it <= maxiter; ++it) {
        spmv(&L->A, av, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { *iters = it; status = ORC_ERR_BREAKDOWN; break; }
        double alpha = rz / pq;
        for (int32_t i = 0; i < n; ++i) { u[i] = fma(alpha, p[i], u[i]); r[i] = fma(-alpha, q[i], r[i]); }
        *iters = it;
        double res = sqrt(dot(n, r, r)) / nf;
        *relres = res;
        if (res <= tol) {
            spmv(&L->A, av, u, q);
            for (int32_t i = 0; i < n; ++i) q[i] = f[i] - q[i];
            double tres = sqrt(dot(n, q, q)) / nf;
            *relres = tres;
            if (tres <= tol) { status = ORC_OK; break; }
            if (replacements >= 2) { status = ORC_NOT_CONVERGED; break; }
            ++replacements;
            for (int32_t i = 0; i < n; ++i) r[i] = q[i];
        }
        orc_vcycle(h, r, z);
        double rz_new = dot(n, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int32_t i = 0; i < n; ++i) p[i] = fma(beta, p[i], z[i]);
    }
    if (status == ORC_NOT_CONVERGED) {
        spmv(&L->A, av, u, q);
        for (int32_t i = 0; i < n; ++i) q[i] = f[i] - q[i];
        *relres = sqrt(dot(n, q, q)) / nf;
    }
    return status;
}

/* Right-preconditioned BiCGStab (the Krylov solver of Sec. 4), one V-cycle
 * per preconditioner application, x_0 = 0, shadow residual r^ = r_0 = f:
 *   rho = (r^, r); beta = (rho / rho_old)(alpha / omega); p = r + beta (p - omega v);
 *   p^ = M p; v = A p^; alpha = rho / (r^, v); s = r - alpha v;
 *   if |s|/|f| <= tol: x += alpha p^ (half step) and confirm;
 *   s^ = M s; t = A s^; omega = (t, s) / (t, t);
 *   x += alpha p^ + omega s^; r = s - omega t.
 * Convergence (recurrence |r|/|f| <= tol, or |s| at the half step) is
 * confirmed by the true residual; if that misses tol, r is replaced by it
 * (at most twice) and the iteration goes on.  Breakdown: rho, (r^, v) or
 * (t, t) zero or not finite, or omega = 0. */
typedef void (*orc_apply_fn)(void *ctx, const double *x, double *y);

/* The iteration itself, for any operator y = A x and preconditioner y = M x
 * on n unknowns. */
static int bicgstab_core(int32_t n, orc_apply_fn apply_A, orc_apply_fn apply_M, void *ctx, const double *f,
                         double *u, double tol, int maxiter, int *iters, double *relres) {
    double *r = (double *)xcalloc((size_t)n, sizeof(double));
    double *rh = (double *)xcalloc((size_t)n, sizeof(double));
    double *p = (double *)xcalloc((size_t)n, sizeof(double));
    double *v = (double *)xcalloc((size_t)n, sizeof(double));
    double *ph = (double *)xcalloc((size_t)n, sizeof(double));
    double *sv = (double *)xcalloc((size_t)n, sizeof(double));
    double *sh = (double *)xcalloc((size_t)n, sizeof(double));
    double *t = (double *)xcalloc((size_t)n, sizeof(double));
    for (int32_t i = 0; i < n; ++i) { u[i] = 0.0; r[i] = f[i]; rh[i] = f[i]; }
    double nf = sqrt(dot(n, f, f));
    *iters = 0;
    *relres = 0.0;
    int status = ORC_NOT_CONVERGED;
    if (nf == 0.0) { status = ORC_OK; goto done; }
    {
        double rho_old = 1.0, alpha = 1.0, omega = 1.0;
        int replacements = 0;
        for (int it = 1; it <= maxiter; ++it) {
            *iters = it;
            double rho = dot(n, rh, r);
            if (!(rho != 0.0) || !isfinite(rho)) { status = ORC_ERR_BREAKDOWN; break; }
            double beta = (rho / rho_old) * (alpha / omega);
            for (int32_t i = 0; i < n; ++i) p[i] = fma(beta, fma(-omega, v[i], p[i]), r[i]);
            apply_M(ctx, p, ph);
            apply_A(ctx, ph, v);
            double rv = dot(n, rh, v);
            if (!(rv != 0.0) || !isfinite(rv)) { status = ORC_ERR_BREAKDOWN; break; }
            alpha = rho / rv;
            rho_old = rho;
            for (int32_t i = 0; i < n; ++i) sv[i] = fma(-alpha, v[i], r[i]);
            int conv = 0;
            double sres = sqrt(dot(n, sv, sv)) / nf;
            if (sres <= tol) {
                for (int32_t i = 0; i < n; ++i) u[i] = fma(alpha, ph[i], u[i]);
                for (int32_t i = 0; i < n; ++i) r[i] = sv[i];
                conv = 1;
            } else {
                apply_M(ctx, sv, sh);
                apply_A(ctx, sh, t);
                double ts = dot(n, t, sv), tt = dot(n, t, t);
                if (!(tt != 0.0) || !isfinite(tt)) { status = ORC_ERR_BREAKDOWN; break; }
                omega = ts / tt;
                if (!(omega != 0.0) || !isfinite(omega)) { status = ORC_ERR_BREAKDOWN; break; }
                for (int32_t i = 0; i < n; ++i) {
                    u[i] = fma(omega, sh[i], fma(alpha, ph[i], u[i]));
                    r[i] = fma(-omega, t[i], sv[i]);
                }
                double res = sqrt(dot(n, r, r)) / nf;
                *relres = res;
                conv = res <= tol;
            }
            if (conv) {
                apply_A(ctx, u, t);
                for (int32_t i = 0; i < n; ++i) t[i] = f[i] - t[i];
                double tres = sqrt(dot(n, t, t)) / nf;
                *relres = tres;
                if (tres <= tol) { status = ORC_OK; break; }
                if (replacements >= 2) { status = ORC_NOT_CONVERGED; break; }
                ++replacements;
                for (int32_t i = 0; i < n; ++i) r[i] = t[i];
            }
        }
    }
    {
        double *q = t;
        apply_A(ctx, u, q);
        for (int32_t i = 0; i < n; ++i) q[i] = f[i] - q[i];
        *relres = sqrt(dot(n, q, q)) / nf;
    }
done:
    free(r); free(rh); free(p); free(v); free(ph); free(sv); free(sh); free(t);
    return status;
}

typedef struct { ohier *h; const double *av; } scalar_ops;
static void scalar_apply_A(void *c, const double *x, double *y) {
    scalar_ops *o = (scalar_ops *)c;
    spmv(&o->h->lev[0].A, o->av, x, y);
}
static void scalar_apply_M(void *c, const double *x, double *y) { orc_vcycle(((scalar_ops *)c)->h, x, y); }

int orc_bicgstab(ohier *h, const double *sys_val, const double *f, double *u, double tol, int maxiter,
                 int *iters, double *relres) {
    scalar_ops o = {h, sys_val ? sys_val : h->lev[0].A.val};
    return bicgstab_core(h->lev[0].A.nrows, scalar_apply_A, scalar_apply_M, &o, f, u, tol, maxiter, iters, relres);
}

/* ------------------------------------------------------------------------ */
/* Accessors for the tests. */
int orc_nlevels(const ohier *h) { return h->nlev; }

/* sizes[0..5] = n, nnz(A), nnz(P), nnz(R), nnz(AP), nagg */
void orc_level_sizes(const ohier *h, int l, int64_t *sizes) {
    const olevel *L = &h->lev[l];
    sizes[0] = L->A.nrows;
    sizes[1] = L->A.ptr[L->A.nrows];
    sizes[2] = L->P.ptr ? L->P.ptr[L->P.nrows] : 0;
    sizes[3] = L->R.ptr ? L->R.ptr[L->R.nrows] : 0;
    sizes[4] = L->AP.ptr ? L->AP.ptr[L->AP.nrows] : 0;
    sizes[5] = L->nroots;
}

static void copy_csr(const ocsr *a, int32_t nrows, int32_t *ptr, int32_t *col, double *val) {
    if (!a->ptr) return;
    int32_t nnz = a->ptr[nrows];
    if (ptr) memcpy(ptr, a->ptr, sizeof(int32_t) * ((size_t)nrows + 1));
    if (col) memcpy(col, a->col, sizeof(int32_t) * (size_t)nnz);
    if (val) memcpy(val, a->val, sizeof(double) * (size_t)nnz);
}

/* which: 0 = A, 1 = P, 2 = R, 3 = AP (values of the last product) */
void orc_export_csr(const ohier *h, int l, int which, int32_t *ptr, int32_t *col, double *val) {
    const olevel *L = &h->lev[l];
    const ocsr *a = which == 0 ? &L->A : which == 1 ? &L->P : which == 2 ? &L->R : &L->AP;
    copy_csr(a, a->nrows, ptr, col, val);
}

void orc_export_level_vec(const ohier *h, int l, int32_t *agg, uint8_t *strong, double *m) {
    const olevel *L = &h->lev[l];
    if (agg) memcpy(agg, L->agg, sizeof(int32_t) * (size_t)L->A.nrows);
    if (strong) memcpy(strong, L->strong, (size_t)L->A.ptr[L->A.nrows]);
    if (m) memcpy(m, L->m, sizeof(double) * (size_t)L->A.nrows);
}

void orc_export_lu(const ohier *h, double *lu, int32_t *piv) {
    if (lu) memcpy(lu, h->LU, sizeof(double) * (size_t)h->nL * (size_t)h->nL);
    if (piv) memcpy(piv, h->piv, sizeof(int32_t) * (size_t)h->nL);
}

/* Standalone pieces, for the pins. */
int orc_dense_lu(int n, double *a, int32_t *piv) { return dense_lu(n, a, piv); }
void orc_dense_lu_solve(int n, const double *a, const int32_t *piv, const double *b, double *x) {
    dense_lu_solve(n, a, piv, b, x);
}

/* ======================================================================== */
/* Block-valued (4 x 4) hierarchy: the monolithic Navier-Stokes systems of
 * Sec. 4, which the paper solves with BiCGStab preconditioned by
 * non-smoothed aggregation AMG with damped Jacobi smoothing, on a backend
 * whose matrix values are statically sized 4 x 4 blocks.
 * Block CSR: the pattern is a scalar CSR over nodes; entry e holds 16
 * doubles, row-major (component r of the row node, component c of the column
 * node), at val[16 e].  Vectors hold the 4 components of a node
 * consecutively, so the block matrix is the scalar matrix of 4n unknowns
 * with entry (4i + r, 4j + c) = block (i, j)[r][c]. */
#define OB2 16

/* Synthetic monolithic Oseen-type system on an N^3 cell grid (a stand-in for
 * the stabilised P1 Navier-Stokes matrices of Sec. 4), unknowns (u, v, w, p)
 * per cell, on the 7-point pattern of orc_poisson_assemble.  For the face f
 * between cell c and its neighbour j in direction d with side s = -1 / +1
 * (outward flux phi = s * face velocity, face viscosity
 * mu_f = (2 mu_c mu_j) / (mu_c + mu_j), pressure coefficient
 * tau_f = 2 / (rho_c + rho_j)):
 *   off-diagonal block: velocity rows min(phi, 0) - mu_f on the diagonal of
 *   the 3 x 3 velocity part; (u_d, p) = (p, u_d) = s / 2; (p, p) = -tau_f.
 *   diagonal block: velocity a = mass rho_c + sum over faces in neighbour
 *   order of (mu_f + max(phi, 0)), plus 2 mu_c per wall face (no-slip
 *   ghost); (u_d, p) = g_d = sum of s / 2 over the wall faces of direction d
 *   (zero-gradient ghost pressure), (p, u_d) = -g_d; (p, p) = sum of tau_f in
 *   neighbour order, plus 2 / rho_c on the top face (z = N - 1).
 * The pressure part is exactly the pressure Poisson matrix; the
 * velocity-pressure coupling is skew-symmetric, so the symmetric part of the
 * matrix is block diagonal (velocity, pressure) and positive definite.
 * Faces are visited in ascending neighbour order z-, y-, x-, x+, y+, z+. */
int orc_stokes_assemble(int N, const double *rho, const double *mu, const double *fx, const double *fy,
                        const double *fz, double mass, int32_t *ptr, int32_t *col, double *bval) {
    if (N < 1) return ORC_ERR_ARG;
    const long long n = (long long)N * N * N, s3 = (long long)N * N, N1 = N + 1;
    long long pos = 0;
    for (long long c = 0; c < n; ++c) {
        const long long x = c % N, y = (c / N) % N, z = c / s3;
        const int has[6] = {z > 0, y > 0, x > 0, x < N - 1, y < N - 1, z < N - 1};
        const long long nbr[6] = {c - s3, c - N, c - 1, c + 1, c + N, c + s3};
        const int dir[6] = {2, 1, 0, 0, 1, 2};
        const double sg[6] = {-1.0, -1.0, -1.0, 1.0, 1.0, 1.0};
        const double wv[6] = {fz[(z * N + y) * N + x], fy[(z * N1 + y) * N + x], fx[(z * N + y) * N1 + x],
                              fx[(z * N + y) * N1 + x + 1], fy[(z * N1 + y + 1) * N + x],
                              fz[((z + 1) * N + y) * N + x]};
        ptr[c] = (int32_t)pos;
        const double kap_c = mass * rho[c] + 6.0 * mu[c];
        const double rinv_c = 1.0 / kap_c;
        double a = mass * rho[c], s = 0.0;
        double g[3] = {0.0, 0.0, 0.0};
        long long dpos = -1;
        for (int t = 0; t < 7; ++t) {
            if (t == 3) { dpos = pos; col[pos++] = (int32_t)c; continue; }
            const int q = t < 3 ? t : t - 1;
            const int d = dir[q];
            const double sig = sg[q];
            if (!has[q]) {
                a = a + 2.0 * mu[c];
                g[d] = g[d] + (0.5 * sig) * kap_c;
                continue;
            }
            const long long j = nbr[q];
            const double phi = sig * wv[q];
            const double muf = (2.0 * mu[c] * mu[j]) / (mu[c] + mu[j]);
            const double rinv_j = 1.0 / (mass * rho[j] + 6.0 * mu[j]);
            const double beta = 2.0 / (rinv_c + rinv_j);
            double *B = bval + OB2 * pos;
            for (int k = 0; k < OB2; ++k) B[k] = 0.0;
            const double off = (phi < 0.0 ? phi : 0.0) - muf;
            B[0] = off; B[5] = off; B[10] = off;
            B[d * 4 + 3] = (0.5 * sig) * beta;
            B[12 + d] = (0.5 * sig) * beta;
            B[15] = -beta;
            a = a + (muf + (phi > 0.0 ? phi : 0.0));
            s = s + beta;
            col[pos++] = (int32_t)j;
        }
        if (z == N - 1) s = s + 2.0 / rinv_c;
        double *D = bval + OB2 * dpos;
        for (int k = 0; k < OB2; ++k) D[k] = 0.0;
        D[0] = a; D[5] = a; D[10] = a;
        for (int d = 0; d < 3; ++d) { D[d * 4 + 3] = g[d]; D[12 + d] = -g[d]; }
        D[15] = s;
    }
    ptr[n] = (int32_t)pos;
    return ORC_OK;
}

/* Frobenius norm of a block: the square root of the sum, in storage order
 * with fma, of the squared entries.  The node graph that strength and
 * aggregation see carries these norms as its values. */
static double block_norm(const double *b) {
    double s = 0.0;
    for (int k = 0; k < OB2; ++k) s = fma(b[k], b[k], s);
    return sqrt(s);
}

/* 4 x 4 inverse by Gauss-Jordan elimination with partial pivoting (pivot:
 * first entry of largest magnitude in the column, rows swapped; pivot row
 * divided by the pivot, then eliminated from every other row with fma).
 * Returns 0 for a singular (or non-finite) block. */
static int inv4(const double *a_in, double *inv) {
    double a[OB2];
    memcpy(a, a_in, sizeof a);
    for (int k = 0; k < OB2; ++k) inv[k] = (k % 5 == 0) ? 1.0 : 0.0;
    for (int k = 0; k < 4; ++k) {
        int p = k;
        double best = fabs(a[k * 4 + k]);
        for (int r = k + 1; r < 4; ++r) {
            double v = fabs(a[r * 4 + k]);
            if (v > best) { best = v; p = r; }
        }
        if (!(best > 0.0) || !isfinite(best)) return 0;
        if (p != k)
            for (int c = 0; c < 4; ++c) {
                double t = a[k * 4 + c]; a[k * 4 + c] = a[p * 4 + c]; a[p * 4 + c] = t;
                t = inv[k * 4 + c]; inv[k * 4 + c] = inv[p * 4 + c]; inv[p * 4 + c] = t;
            }
        const double pv = a[k * 4 + k];
        for (int c = 0; c < 4; ++c) { a[k * 4 + c] = a[k * 4 + c] / pv; inv[k * 4 + c] = inv[k * 4 + c] / pv; }
        for (int r = 0; r < 4; ++r) {
            if (r == k) continue;
            const double f = a[r * 4 + k];
            for (int c = 0; c < 4; ++c) {
                a[r * 4 + c] = fma(-f, a[k * 4 + c], a[r * 4 + c]);
                inv[r * 4 + c] = fma(-f, inv[k * 4 + c], inv[r * 4 + c]);
            }
        }
    }
    return 1;
}

typedef struct {
    ocsr S;            /* node graph: pattern of A, values = block norms (setup only) */
    double *bv;        /* block values of A (16 per entry) */
    ocsr P, R;         /* scalar transfer operators: non-smoothed, P = P_tent, R = P^T */
    ocsr AP;           /* pattern of A P */
    double *apb;       /* block values of A P (scratch of the Galerkin product) */
    int32_t *agg;
    uint8_t *strong;
    int32_t nroots;
    double *Minv;      /* damped block Jacobi: w_J inv(A_ii), 16 per node (0 if singular) */
    double *u, *f, *r; /* 4 per node */
} oblevel;

typedef struct {
    oparams prm;
    int nlev;
    oblevel lev[32];
    int nL;            /* unknowns of the coarsest system (4 per node) */
    double *LU;
    int32_t *piv;
} obhier;

/* Block Galerkin product A_c = R (A P) with scalar P and R (each block is
 * scaled by the scalar entry, component by component): the loops and the
 * summation order of spgemm_numeric, one fma per term and component. */
static int block_galerkin(oblevel *L, oblevel *C) {
    const ocsr *A = &L->S, *P = &L->P, *R = &L->R;
    ocsr *AP = &L->AP, *Ac = &C->S;
    int32_t nmax = A->ncols > P->ncols ? A->ncols : P->ncols;
    int32_t *pos = (int32_t *)xcalloc((size_t)nmax, sizeof(int32_t));
    for (int32_t c = 0; c < nmax; ++c) pos[c] = -1;
    int st = ORC_OK;
    for (int32_t i = 0; i < A->nrows && st == ORC_OK; ++i) {
        for (int32_t e = AP->ptr[i]; e < AP->ptr[i + 1]; ++e) {
            pos[AP->col[e]] = e;
            for (int k = 0; k < OB2; ++k) L->apb[(size_t)OB2 * e + k] = 0.0;
        }
        for (int32_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
            const int32_t j = A->col[p];
            for (int32_t q = P->ptr[j]; q < P->ptr[j + 1]; ++q) {
                const int32_t e = pos[P->col[q]];
                if (e < 0) { st = ORC_ERR_PATTERN; break; }
                for (int k = 0; k < OB2; ++k)
                    L->apb[(size_t)OB2 * e + k] = fma(L->bv[(size_t)OB2 * p + k], P->val[q], L->apb[(size_t)OB2 * e + k]);
            }
        }
        for (int32_t e = AP->ptr[i]; e < AP->ptr[i + 1]; ++e) pos[AP->col[e]] = -1;
    }
    for (int32_t I = 0; I < R->nrows && st == ORC_OK; ++I) {
        for (int32_t e = Ac->ptr[I]; e < Ac->ptr[I + 1]; ++e) {
            pos[Ac->col[e]] = e;
            for (int k = 0; k < OB2; ++k) C->bv[(size_t)OB2 * e + k] = 0.0;
        }
        for (int32_t p = R->ptr[I]; p < R->ptr[I + 1]; ++p) {
            const int32_t i = R->col[p];
            for (int32_t q = AP->ptr[i]; q < AP->ptr[i + 1]; ++q) {
                const int32_t e = pos[AP->col[q]];
                if (e < 0) { st = ORC_ERR_PATTERN; break; }
                for (int k = 0; k < OB2; ++k)
                    C->bv[(size_t)OB2 * e + k] = fma(R->val[p], L->apb[(size_t)OB2 * q + k], C->bv[(size_t)OB2 * e + k]);
            }
        }
        for (int32_t e = Ac->ptr[I]; e < Ac->ptr[I + 1]; ++e) pos[Ac->col[e]] = -1;
    }
    free(pos);
    return st;
}

static void block_level_free(oblevel *L) {
    csr_free(&L->S); csr_free(&L->P); csr_free(&L->R); csr_free(&L->AP);
    free(L->bv); free(L->apb); free(L->agg); free(L->strong); free(L->Minv);
    free(L->u); free(L->f); free(L->r);
    memset(L, 0, sizeof(*L));
}

void orc_block_destroy(obhier *h) {
    if (!h) return;
    for (int l = 0; l < h->nlev; ++l) block_level_free(&h->lev[l]);
    free(h->LU); free(h->piv);
    free(h);
}

/* Coarsest level: the block matrix expanded to 4 n_L scalar unknowns, dense
 * LU with partial pivoting. */
static int block_coarse_factor(obhier *h) {
    const oblevel *L = &h->lev[h->nlev - 1];
    const int n4 = h->nL;
    memset(h->LU, 0, sizeof(double) * (size_t)n4 * (size_t)n4);
    for (int32_t i = 0; i < L->S.nrows; ++i)
        for (int32_t p = L->S.ptr[i]; p < L->S.ptr[i + 1]; ++p)
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c)
                    h->LU[(size_t)(4 * i + r) * n4 + 4 * L->S.col[p] + c] = L->bv[(size_t)OB2 * p + 4 * r + c];
    return dense_lu(n4, h->LU, h->piv);
}

/* Alg. 4 body for the block hierarchy: new fine block values, the damped
 * block-Jacobi inverses and the Galerkin blocks of every level over the kept
 * P, R and patterns, the coarsest LU. */
int orc_block_rebuild(obhier *h, const double *bval) {
    if (!h) return ORC_ERR_STATE;
    oblevel *L0 = &h->lev[0];
    memcpy(L0->bv, bval, sizeof(double) * OB2 * (size_t)L0->S.ptr[L0->S.nrows]);
    for (int l = 0; l + 1 < h->nlev; ++l) {
        oblevel *L = &h->lev[l];
        int32_t *dia = diag_positions(&L->S);
        for (int32_t i = 0; i < L->S.nrows; ++i) {
            double inv[OB2];
            int ok = inv4(L->bv + (size_t)OB2 * dia[i], inv);
            for (int k = 0; k < OB2; ++k) L->Minv[(size_t)OB2 * i + k] = ok ? h->prm.jacobi_omega * inv[k] : 0.0;
        }
        free(dia);
        int st = block_galerkin(L, &h->lev[l + 1]);
        if (st) return st;
    }
    return block_coarse_factor(h);
}

/* Alg. 1 for the block matrix (n nodes, block CSR).  Strength of connection
 * and aggregation run on the node graph whose values are the block norms
 * (the scalar routines above: the test ||A_ij||^2 > eps^2 ||A_ii|| ||A_jj||);
 * P is the tentative prolongation (non-smoothed aggregation, as the paper
 * uses for these systems), so every coarse block is a sum of fine blocks.
 * Parameters as orc_setup; smoother must be damped Jacobi (1) and smoothed 0;
 * coarse_enough counts nodes. */
obhier *orc_block_setup(int32_t n, const int32_t *ptr, const int32_t *col, const double *bval,
                        const double *dprm, const int32_t *iprm, int *status) {
    *status = ORC_OK;
    if (iprm[0] != 1 || iprm[6] != 0) { *status = ORC_ERR_ARG; return NULL; }
    if (n <= 0 || check_pattern(n, ptr, col) != ORC_OK) { *status = ORC_ERR_PATTERN; return NULL; }
    obhier *h = (obhier *)xcalloc(1, sizeof(obhier));
    h->prm.theta = dprm[0]; h->prm.omega = dprm[1]; h->prm.jacobi_omega = dprm[2];
    h->prm.smoother = iprm[0]; h->prm.npre = iprm[1]; h->prm.npost = iprm[2];
    h->prm.coarse_enough = iprm[3]; h->prm.max_levels = iprm[4];
    h->prm.theta_halving = iprm[5]; h->prm.smoothed = 0;
    if (h->prm.max_levels > 32) h->prm.max_levels = 32;
    if (h->prm.max_levels < 1) h->prm.max_levels = 1;
    oblevel *L = &h->lev[0];
    const int32_t nnz = ptr[n];
    L->S.nrows = L->S.ncols = n;
    L->S.ptr = (int32_t *)xcalloc((size_t)n + 1, sizeof(int32_t));
    L->S.col = (int32_t *)xcalloc((size_t)nnz, sizeof(int32_t));
    L->S.val = (double *)xcalloc((size_t)nnz, sizeof(double));
    L->bv = (double *)xcalloc((size_t)OB2 * nnz, sizeof(double));
    memcpy(L->S.ptr, ptr, sizeof(int32_t) * ((size_t)n + 1));
    memcpy(L->S.col, col, sizeof(int32_t) * (size_t)nnz);
    memcpy(L->bv, bval, sizeof(double) * OB2 * (size_t)nnz);
    for (int32_t e = 0; e < nnz; ++e) L->S.val[e] = block_norm(L->bv + (size_t)OB2 * e);
    h->nlev = 1;
    double theta = h->prm.theta;
    for (;;) {
        L = &h->lev[h->nlev - 1];
        const int32_t nl = L->S.nrows;
        L->u = (double *)xcalloc(4 * (size_t)nl, sizeof(double));
        L->f = (double *)xcalloc(4 * (size_t)nl, sizeof(double));
        L->r = (double *)xcalloc(4 * (size_t)nl, sizeof(double));
        L->Minv = (double *)xcalloc((size_t)OB2 * nl, sizeof(double));
        L->agg = (int32_t *)xcalloc((size_t)nl, sizeof(int32_t));
        for (int32_t i = 0; i < nl; ++i) L->agg[i] = -1;
        L->strong = (uint8_t *)xcalloc((size_t)L->S.ptr[nl], 1);
        if (nl <= h->prm.coarse_enough || h->nlev >= h->prm.max_levels) break;
        int32_t *dia = diag_positions(&L->S);
        strength(&L->S, theta * theta, L->strong, dia);
        int32_t nagg = aggregate(&L->S, L->strong, L->agg);
        if (nagg < 0) { free(dia); *status = nagg; orc_block_destroy(h); return NULL; }
        if (nagg == 0 || nagg >= nl) {
            for (int32_t i = 0; i < nl; ++i) L->agg[i] = -1;
            memset(L->strong, 0, (size_t)L->S.ptr[nl]);
            free(dia);
            break;
        }
        L->nroots = nagg;
        build_P(&L->S, L->strong, dia, L->agg, nagg, h->prm.omega, 0, &L->P);
        free(dia);
        transpose(&L->P, &L->R);
        spgemm_pattern(&L->S, &L->P, 0, &L->AP);
        oblevel *C = &h->lev[h->nlev];
        spgemm_pattern(&L->R, &L->AP, 1, &C->S);
        C->S.ncols = nagg;
        L->apb = (double *)xcalloc((size_t)OB2 * L->AP.ptr[L->AP.nrows], sizeof(double));
        C->bv = (double *)xcalloc((size_t)OB2 * C->S.ptr[nagg], sizeof(double));
        /* the next level's strength test needs its block values now */
        int gst = block_galerkin(L, C);
        for (int32_t e = 0; e < C->S.ptr[nagg]; ++e) C->S.val[e] = block_norm(C->bv + (size_t)OB2 * e);
        h->nlev++;
        if (gst) { *status = gst; orc_block_destroy(h); return NULL; }
        if (h->prm.theta_halving) theta = theta * 0.5;
    }
    h->nL = 4 * h->lev[h->nlev - 1].S.nrows;
    h->LU = (double *)xcalloc((size_t)h->nL * (size_t)h->nL, sizeof(double));
    h->piv = (int32_t *)xcalloc((size_t)h->nL, sizeof(int32_t));
    int st = orc_block_rebuild(h, bval);
    if (st == ORC_ERR_SINGULAR) { *status = st; return h; }
    if (st) { *status = st; orc_block_destroy(h); return NULL; }
    return h;
}

/* y = A x for the block matrix: component r of node i sums, in entry order
 * and within an entry in component order, A_e[r][c] x_j[c] with fma (the row
 * order of the expanded scalar matrix). */
static void block_spmv(const ocsr *S, const double *bv, const double *x, double *y) {
    for (int32_t i = 0; i < S->nrows; ++i)
        for (int r = 0; r < 4; ++r) {
            double s = 0.0;
            for (int32_t p = S->ptr[i]; p < S->ptr[i + 1]; ++p)
                for (int c = 0; c < 4; ++c) s = fma(bv[(size_t)OB2 * p + 4 * r + c], x[4 * (size_t)S->col[p] + c], s);
            y[4 * (size_t)i + r] = s;
        }
}

/* damped block Jacobi: u_i <- u_i + Minv_i (f - A u)_i */
static void block_sweep(const oblevel *L, double *u, const double *f, double *tmp) {
    const int32_t n = L->S.nrows;
    block_spmv(&L->S, L->bv, u, tmp);
    for (int32_t k = 0; k < 4 * n; ++k) tmp[k] = f[k] - tmp[k];
    for (int32_t i = 0; i < n; ++i) {
        double t[4];
        for (int c = 0; c < 4; ++c) t[c] = tmp[4 * (size_t)i + c];
        for (int r = 0; r < 4; ++r) {
            double s = u[4 * (size_t)i + r];
            for (int c = 0; c < 4; ++c) s = fma(L->Minv[(size_t)OB2 * i + 4 * r + c], t[c], s);
            u[4 * (size_t)i + r] = s;
        }
    }
}

static void block_vcycle_level(obhier *h, int l) {
    oblevel *L = &h->lev[l];
    const int32_t n = L->S.nrows;
    if (l == h->nlev - 1) {
        dense_lu_solve(h->nL, h->LU, h->piv, L->f, L->u);
        return;
    }
    for (int32_t k = 0; k < 4 * n; ++k) L->u[k] = 0.0;
    for (int s = 0; s < h->prm.npre; ++s) block_sweep(L, L->u, L->f, L->r);
    block_spmv(&L->S, L->bv, L->u, L->r);
    for (int32_t k = 0; k < 4 * n; ++k) L->r[k] = L->f[k] - L->r[k];
    oblevel *C = &h->lev[l + 1];
    for (int32_t I = 0; I < L->R.nrows; ++I)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int32_t p = L->R.ptr[I]; p < L->R.ptr[I + 1]; ++p)
                s = fma(L->R.val[p], L->r[4 * (size_t)L->R.col[p] + c], s);
            C->f[4 * (size_t)I + c] = s;
        }
    block_vcycle_level(h, l + 1);
    for (int32_t i = 0; i < n; ++i)
        for (int c = 0; c < 4; ++c) {
            double s = L->u[4 * (size_t)i + c];
            for (int32_t p = L->P.ptr[i]; p < L->P.ptr[i + 1]; ++p)
                s = fma(L->P.val[p], C->u[4 * (size_t)L->P.col[p] + c], s);
            L->u[4 * (size_t)i + c] = s;
        }
    for (int s = 0; s < h->prm.npost; ++s) block_sweep(L, L->u, L->f, L->r);
}

void orc_block_vcycle(obhier *h, const double *r, double *z) {
    oblevel *L = &h->lev[0];
    memcpy(L->f, r, sizeof(double) * 4 * (size_t)L->S.nrows);
    block_vcycle_level(h, 0);
    memcpy(z, L->u, sizeof(double) * 4 * (size_t)L->S.nrows);
}

typedef struct { obhier *h; const double *bv; } block_ops;
static void block_apply_A(void *c, const double *x, double *y) {
    block_ops *o = (block_ops *)c;
    block_spmv(&o->h->lev[0].S, o->bv, x, y);
}
static void block_apply_M(void *c, const double *x, double *y) { orc_block_vcycle(((block_ops *)c)->h, x, y); }

/* BiCGStab (as orc_bicgstab) on the 4n unknowns of the block system,
 * preconditioned by one block V-cycle. */
int orc_block_bicgstab(obhier *h, const double *sys_bval, const double *f, double *u, double tol, int maxiter,
                       int *iters, double *relres) {
    block_ops o = {h, sys_bval ? sys_bval : h->lev[0].bv};
    return bicgstab_core(4 * h->lev[0].S.nrows, block_apply_A, block_apply_M, &o, f, u, tol, maxiter, iters,
                         relres);
}

/* Accessors for the tests. */
int orc_block_nlevels(const obhier *h) { return h->nlev; }
void orc_block_level_sizes(const obhier *h, int l, int64_t *sizes) {
    const oblevel *L = &h->lev[l];
    sizes[0] = L->S.nrows;
    sizes[1] = L->S.ptr[L->S.nrows];
    sizes[2] = L->P.ptr ? L->P.ptr[L->P.nrows] : 0;
    sizes[3] = L->R.ptr ? L->R.ptr[L->R.nrows] : 0;
    sizes[4] = L->AP.ptr ? L->AP.ptr[L->AP.nrows] : 0;
    sizes[5] = L->nroots;
}
/* which: 0 = A (val: 16 per entry), 1 = P, 2 = R (scalar) */
void orc_block_export_csr(const obhier *h, int l, int which, int32_t *ptr, int32_t *col, double *val) {
    const oblevel *L = &h->lev[l];
    const ocsr *a = which == 0 ? &L->S : which == 1 ? &L->P : &L->R;
    if (!a->ptr) return;
    const int32_t nnz = a->ptr[a->nrows];
    if (ptr) memcpy(ptr, a->ptr, sizeof(int32_t) * ((size_t)a->nrows + 1));
    if (col) memcpy(col, a->col, sizeof(int32_t) * (size_t)nnz);
    if (val) {
        if (which == 0) memcpy(val, L->bv, sizeof(double) * OB2 * (size_t)nnz);
        else memcpy(val, a->val, sizeof(double) * (size_t)nnz);
    }
}
/* aggregates, strong flags, block-Jacobi inverses (16 per node), block norms
 * of the node graph (per entry); any pointer may be NULL */
void orc_block_export_vec(const obhier *h, int l, int32_t *agg, uint8_t *strong, double *minv, double *norms) {
    const oblevel *L = &h->lev[l];
    const int32_t n = L->S.nrows, nnz = L->S.ptr[n];
    if (agg) memcpy(agg, L->agg, sizeof(int32_t) * (size_t)n);
    if (strong) memcpy(strong, L->strong, (size_t)nnz);
    if (minv) memcpy(minv, L->Minv, sizeof(double) * OB2 * (size_t)n);
    if (norms) memcpy(norms, L->S.val, sizeof(double) * (size_t)nnz);
}
void orc_block_export_lu(const obhier *h, double *lu, int32_t *piv) {
    if (lu) memcpy(lu, h->LU, sizeof(double) * (size_t)h->nL * (size_t)h->nL);
    if (piv) memcpy(piv, h->piv, sizeof(int32_t) * (size_t)h->nL);
}
int orc_inv4(const double *a, double *inv) { return inv4(a, inv); }
double orc_block_norm(const double *b) { return block_norm(b); }
