// setup_kernels.cu -- full-setup kernels (Alg. 1 of arXiv 2108.02054) of the
// smoothed-aggregation hierarchy, all on the GPU: pattern checks, strength of
// connection, distance-2 maximal-independent-set aggregation, smoothed
// prolongation, R = P^T, the symbolic Galerkin product and the gather
// metadata that lets every later numeric product skip the symbolic phase
// (Sec. 5).  Also the synthetic pressure-Poisson assembly used as workload.
//
// Floating point that decides structure (strength test, aggregation ties, P
// values feeding coarser levels) is written as separately rounded IEEE
// operations in a fixed order; the library is built with --fmad=false so no
// multiply-add is contracted behind our back.
#include <climits>

#include "common.cuh"
#include "fdiv.cuh"

namespace amgpr {

namespace {

constexpr int kThreads = 256;

inline int nblocks(int64_t n, int t = kThreads) {
    int64_t b = (n + t - 1) / t;
    return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ uint32_t node_priority(uint32_t h) {
    // murmur3 32-bit finaliser: a bijection of the 32-bit integers
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ int32_t find_in_row(const int32_t *__restrict__ col, int32_t lo, int32_t hi, int32_t c) {
    while (lo < hi) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------ scan
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ int64_t block_exclusive_scan(int64_t v, int64_t *warp_tot, int64_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int64_t w = lane < nw ? warp_tot[lane] : 0;
        int64_t z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < nw) warp_tot[lane] = z - w;
        if (lane == 31) *total = z;
    }
    __syncthreads();
    int64_t r = warp_tot[warp] + x - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const int32_t *__restrict__ in, int64_t n, int64_t *__restrict__ bsum) {
    __shared__ int64_t wt[32];
    __shared__ int64_t tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        if (i < n) s += in[i];
    }
    block_exclusive_scan(s, wt, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_blocks(int64_t *__restrict__ bsum, int64_t nb) {
    __shared__ int64_t wt[32];
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        int64_t i = b0 + threadIdx.x;
        int64_t v = i < nb ? bsum[i] : 0;
        int64_t e = block_exclusive_scan(v, wt, &tot);
        if (i < nb) bsum[i] = carry + e;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_scan_final(const int32_t *__restrict__ in, int32_t *__restrict__ out, int64_t n,
                             const int64_t *__restrict__ bsum, int64_t nb, int *st) {
    __shared__ int64_t wt[32];
    __shared__ int64_t tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int64_t e = block_exclusive_scan(s, wt, &tot) + bsum[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) {
            if (e > INT32_MAX) atomicOr(st, DEV_ERR_OVERFLOW);
            out[base + k] = (int32_t)e;
        }
        e += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int64_t t = bsum[nb];
        if (t > INT32_MAX) atomicOr(st, DEV_ERR_OVERFLOW);
        out[n] = (int32_t)t;
    }
}

// ------------------------------------------------------------------ assembly
__device__ __forceinline__ void cell_coords(int dim, int N, int64_t c, int64_t &x, int64_t &y, int64_t &z) {
    x = c % N;
    y = (c / N) % N;
    z = dim == 3 ? c / ((int64_t)N * N) : 0;
}

__global__ void k_poisson_rowlen(int dim, int N, int64_t n, int32_t *__restrict__ len) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    int64_t x, y, z;
    cell_coords(dim, N, c, x, y, z);
    int l = 1 + (x > 0) + (x < N - 1) + (y > 0) + (y < N - 1);
    if (dim == 3) l += (z > 0) + (z < N - 1);
    len[c] = l;
}

__global__ void k_poisson_cols(int dim, int N, int64_t n, const int32_t *__restrict__ ptr, int32_t *__restrict__ col) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    int64_t x, y, z;
    cell_coords(dim, N, c, x, y, z);
    const int64_t s2 = N, s3 = (int64_t)N * N;
    int32_t p = ptr[c];
    if (dim == 3 && z > 0) col[p++] = (int32_t)(c - s3);
    if (y > 0) col[p++] = (int32_t)(c - s2);
    if (x > 0) col[p++] = (int32_t)(c - 1);
    col[p++] = (int32_t)c;
    if (x < N - 1) col[p++] = (int32_t)(c + 1);
    if (y < N - 1) col[p++] = (int32_t)(c + s2);
    if (dim == 3 && z < N - 1) col[p++] = (int32_t)(c + s3);
}

// per-cell density: the input itself, or exp of it when the input is the
// log-density theta = log rho
__device__ __forceinline__ double cell_rho(const double *__restrict__ in, int64_t c, int logd) {
    const double x = in[c];
    return logd ? exp(x) : x;
}

// Row c: neighbours in ascending index order, off-diagonal -2/(rho_c + rho_nb),
// diagonal = running sum of the face coefficients in that order, then the
// ghost-cell Dirichlet term 2/rho_c on the top face.
__global__ void k_poisson_vals(int dim, int N, int64_t n, int top, const double *__restrict__ rho, int logd,
                               const int32_t *__restrict__ ptr, double *__restrict__ val) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    int64_t x, y, z;
    cell_coords(dim, N, c, x, y, z);
    const int64_t s2 = N, s3 = (int64_t)N * N;
    int64_t nb[7];
    int nnb = 0;
    if (dim == 3 && z > 0) nb[nnb++] = c - s3;
    if (y > 0) nb[nnb++] = c - s2;
    if (x > 0) nb[nnb++] = c - 1;
    nb[nnb++] = -1;
    if (x < N - 1) nb[nnb++] = c + 1;
    if (y < N - 1) nb[nnb++] = c + s2;
    if (dim == 3 && z < N - 1) nb[nnb++] = c + s3;
    const double rc = cell_rho(rho, c, logd);
    double diag = 0.0;
    int32_t p = ptr[c], dpos = p;
    for (int t = 0; t < nnb; ++t, ++p) {
        if (nb[t] < 0) { dpos = p; continue; }
        double k = 2.0 / (rc + cell_rho(rho, nb[t], logd));
        diag = diag + k;
        val[p] = -k;
    }
    int is_top = dim == 2 ? (y == N - 1) : (z == N - 1);
    if (top && is_top) diag = diag + 2.0 / rc;
    val[dpos] = diag;
}

// Level-set transport stand-in (Sec. 4, eq. 5): implicit upwind
// convection-diffusion on the Poisson pattern.  With w_f the outward face
// flux of cell c (the face velocity, sign-flipped on the low faces):
// off-diagonal min(w_f, 0) - 0.1, diagonal 1 + sum over faces, in the
// neighbour order, of (max(w_f, 0) + 0.1).  Face arrays, x fastest:
// fx[(z N + y)(N + 1) + x_face], fy[(z (N + 1) + y_face) N + x],
// fz[(z_face N + y) N + x].
__global__ void k_levelset_vals(int dim, int N, int64_t n, const double *__restrict__ fx,
                                const double *__restrict__ fy, const double *__restrict__ fz,
                                const int32_t *__restrict__ ptr, double *__restrict__ val) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    int64_t x, y, z;
    cell_coords(dim, N, c, x, y, z);
    const int64_t N1 = N + 1;
    double w[7];
    int nnb = 0, dslot = 0;
    if (dim == 3 && z > 0) w[nnb++] = -fz[(z * N + y) * N + x];
    if (y > 0) w[nnb++] = -fy[(z * N1 + y) * N + x];
    if (x > 0) w[nnb++] = -fx[(z * N + y) * N1 + x];
    dslot = nnb;
    w[nnb++] = 0.0;
    if (x < N - 1) w[nnb++] = fx[(z * N + y) * N1 + x + 1];
    if (y < N - 1) w[nnb++] = fy[(z * N1 + y + 1) * N + x];
    if (dim == 3 && z < N - 1) w[nnb++] = fz[((z + 1) * N + y) * N + x];
    double diag = 1.0;
    const int32_t p0 = ptr[c];
    for (int t = 0; t < nnb; ++t) {
        if (t == dslot) continue;
        const double wf = w[t];
        diag = diag + ((wf > 0.0 ? wf : 0.0) + 0.1);
        val[p0 + t] = (wf < 0.0 ? wf : 0.0) - 0.1;
    }
    val[p0 + dslot] = diag;
}

// dL/dtheta for theta = log rho, gathered per cell (no atomics): every face
// of cell c contributes dL/dk_f * dk_f/dtheta_c with
// dL/dk_f = -(lam_c - lam_j)(u_c - u_j), dk_f/dtheta_c = -2 rho_c/(rho_c + rho_j)^2;
// the Dirichlet term contributes (-lam_c u_c) * (-2/rho_c).
__global__ void k_poisson_grad(int dim, int N, int64_t n, int top, const double *__restrict__ rho, int logd,
                               const double *__restrict__ u, const double *__restrict__ lam,
                               double *__restrict__ grad) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    int64_t x, y, z;
    cell_coords(dim, N, c, x, y, z);
    const int64_t s2 = N, s3 = (int64_t)N * N;
    int64_t nb[6];
    int nnb = 0;
    if (dim == 3 && z > 0) nb[nnb++] = c - s3;
    if (y > 0) nb[nnb++] = c - s2;
    if (x > 0) nb[nnb++] = c - 1;
    if (x < N - 1) nb[nnb++] = c + 1;
    if (y < N - 1) nb[nnb++] = c + s2;
    if (dim == 3 && z < N - 1) nb[nnb++] = c + s3;
    const double rc = cell_rho(rho, c, logd), lc = lam[c], uc = u[c];
    double g = 0.0;
    for (int t = 0; t < nnb; ++t) {
        int64_t j = nb[t];
        double dLdk = -(lc - lam[j]) * (uc - u[j]);
        double s = rc + cell_rho(rho, j, logd);
        g += dLdk * (-2.0 * rc / (s * s));
    }
    int is_top = dim == 2 ? (y == N - 1) : (z == N - 1);
    if (top && is_top) g += (-lc * uc) * (-2.0 / rc);
    grad[c] = g;
}

// ------------------------------------------------------------------ checks
// a caller's row pointers: ptr[0] = 0, non-decreasing, ptr[n] = nnz, checked
// before any kernel reads the columns they delimit
__global__ void k_check_rowptr(int32_t n, int32_t nnz, const int32_t *__restrict__ ptr, int *st) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = ptr[i];
        bool bad = v < 0 || v > nnz;
        if (i == 0) bad = bad || v != 0;
        if (i == n) bad = bad || v != nnz;
        else bad = bad || ptr[i + 1] < v;
        if (bad) atomicOr(st, DEV_ERR_PATTERN);
    }
}

__global__ void k_check_pattern(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                int32_t *__restrict__ dia, int *st) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && ptr[0] != 0) atomicOr(st, DEV_ERR_PATTERN);
    if (i >= n) return;
    int32_t b = ptr[i], e = ptr[i + 1];
    int32_t d = -1;
    bool bad = e < b;
    for (int32_t p = b; p < e && !bad; ++p) {
        int32_t c = col[p];
        if (c < 0 || c >= n || (p > b && c <= col[p - 1])) bad = true;
        if (c == i) d = p;
    }
    if (bad || d < 0) atomicOr(st, DEV_ERR_PATTERN);
    dia[i] = d < 0 ? b : d;
}

__global__ void k_check_finite(int64_t n, const double *__restrict__ v, int *st) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) { atomicOr(st, DEV_ERR_NONFINITE); return; }
}

// ------------------------------------------------------------------ strength
// (i,j), j != i, is strong iff a_ij^2 > eps^2 |a_ii a_jj| holds in row i's
// direction or in row j's; each product separately rounded.
__global__ void k_strength(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                           const double *__restrict__ val, const int32_t *__restrict__ dia, double eps2,
                           uint8_t *__restrict__ strong, int32_t *__restrict__ deg) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double aii = val[dia[i]];
    int32_t cnt = 0;
    for (int32_t p = ptr[i]; p < ptr[i + 1]; ++p) {
        int32_t j = col[p];
        uint8_t s = 0;
        if (j != i) {
            const double ajj = val[dia[j]];
            const double a = val[p];
            s = __dmul_rn(a, a) > __dmul_rn(eps2, fabs(__dmul_rn(aii, ajj)));
            if (!s) {
                int32_t b = ptr[j], e = ptr[j + 1];
                int32_t t = find_in_row(col, b, e, i);
                if (t < e && col[t] == i) {
                    const double at = val[t];
                    s = __dmul_rn(at, at) > __dmul_rn(eps2, fabs(__dmul_rn(ajj, aii)));
                }
            }
        }
        strong[p] = s;
        cnt += s;
    }
    deg[i] = cnt;
}

// ------------------------------------------------------------------ aggregation
// state: 0 undecided, 1 root, 2 excluded (within distance 2 of a root), 3 isolated
__global__ void k_mis_init(int32_t n, const int32_t *__restrict__ deg, int8_t *__restrict__ state) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) state[i] = deg[i] > 0 ? 0 : 3;
}

// m1[i] = largest priority among undecided nodes of {i} + strong(i), -1 if none
__global__ void k_mis_m1(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                         const uint8_t *__restrict__ strong, const int8_t *__restrict__ state,
                         int64_t *__restrict__ m1) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (state[i] == 3) { m1[i] = -1; return; }
    int64_t m = state[i] == 0 ? (int64_t)node_priority((uint32_t)i) : -1;
    for (int32_t p = ptr[i]; p < ptr[i + 1]; ++p) {
        if (!strong[p]) continue;
        int32_t j = col[p];
        if (state[j] == 0) {
            int64_t q = (int64_t)node_priority((uint32_t)j);
            m = q > m ? q : m;
        }
    }
    m1[i] = m;
}

// an undecided node whose priority is the largest among undecided nodes
// within strong distance 2 becomes a root
__global__ void k_mis_select(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                             const uint8_t *__restrict__ strong, int8_t *__restrict__ state,
                             const int64_t *__restrict__ m1) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || state[i] != 0) return;
    int64_t m = m1[i];
    for (int32_t p = ptr[i]; p < ptr[i + 1]; ++p)
        if (strong[p]) {
            int64_t q = m1[col[p]];
            m = q > m ? q : m;
        }
    if (m == (int64_t)node_priority((uint32_t)i)) state[i] = 1;
}

__global__ void k_mis_r1(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                         const uint8_t *__restrict__ strong, const int8_t *__restrict__ state,
                         uint8_t *__restrict__ r1) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint8_t r = state[i] == 1;
    for (int32_t p = ptr[i]; p < ptr[i + 1] && !r; ++p)
        if (strong[p] && state[col[p]] == 1) r = 1;
    r1[i] = r;
}

__global__ void k_mis_exclude(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                              const uint8_t *__restrict__ strong, int8_t *__restrict__ state,
                              const uint8_t *__restrict__ r1, int *__restrict__ undecided) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || state[i] != 0) return;
    bool ex = r1[i];
    for (int32_t p = ptr[i]; p < ptr[i + 1] && !ex; ++p)
        if (strong[p] && r1[col[p]]) ex = true;
    if (ex) state[i] = 2;
    else atomicAdd(undecided, 1);
}

__global__ void k_root_flags(int32_t n, const int8_t *__restrict__ state, int32_t *__restrict__ flag) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = state[i] == 1;
}

// phase 1: a root and its strong neighbours form aggregate root_id[root]
__global__ void k_agg_phase1(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                             const uint8_t *__restrict__ strong, const int8_t *__restrict__ state,
                             const int32_t *__restrict__ root_id, int32_t *__restrict__ agg1,
                             int32_t *__restrict__ root_of) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a = -1;
    if (state[i] == 1) {
        a = root_id[i];
        root_of[a] = i;
    } else if (state[i] != 3) {
        for (int32_t p = ptr[i]; p < ptr[i + 1]; ++p)
            if (strong[p] && state[col[p]] == 1) { a = root_id[col[p]]; break; }
    }
    agg1[i] = a;
}

// phase 2: a remaining non-isolated node joins the phase-1 aggregate of its
// strong neighbour with the largest |a_ij| (ties: larger root priority)
__global__ void k_agg_phase2(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                             const double *__restrict__ val, const uint8_t *__restrict__ strong,
                             const int8_t *__restrict__ state, const int32_t *__restrict__ agg1,
                             const int32_t *__restrict__ root_of, int32_t *__restrict__ agg, int *st) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a = agg1[i];
    if (state[i] != 3 && a < 0) {
        double bestv = -1.0;
        uint32_t bestk = 0;
        for (int32_t p = ptr[i]; p < ptr[i + 1]; ++p) {
            if (!strong[p]) continue;
            int32_t aj = agg1[col[p]];
            if (aj < 0) continue;
            double v = fabs(val[p]);
            uint32_t k = node_priority((uint32_t)root_of[aj]);
            if (a < 0 || v > bestv || (v == bestv && k > bestk)) { a = aj; bestv = v; bestk = k; }
        }
        if (a < 0) atomicOr(st, DEV_ERR_STATE);
    }
    agg[i] = a;
}

// ------------------------------------------------------------------ prolongation
// row i of smoothed P has one column per distinct aggregate among {i} + strong(i)
__global__ void k_p_count(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                          const uint8_t *__restrict__ strong, const int32_t *__restrict__ agg, int smoothed,
                          int32_t *__restrict__ plen) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (agg[i] < 0) { plen[i] = 0; return; }
    if (!smoothed) { plen[i] = 1; return; }
    int32_t cnt = 0;
    const int32_t b = ptr[i], e = ptr[i + 1];
    for (int32_t p = b; p < e; ++p) {
        int32_t j = col[p];
        if (j != i && !strong[p]) continue;
        int32_t c = agg[j];
        if (c < 0) continue;
        bool dup = false;
        for (int32_t q = b; q < p && !dup; ++q) {
            int32_t jq = col[q];
            if (jq != i && !strong[q]) continue;
            dup = agg[jq] == c;
        }
        cnt += !dup;
    }
    plen[i] = cnt;
}

// P = (I - w D_F^-1 A_F) P_tent: d_i = a_ii + weak off-diagonals (column order);
// P[i,c] = [c == agg(i)] - sum_{j in {i}+strong(i), agg(j) = c} (w * A_F[i,j]) / d_i
// in column order, A_F[i,i] = d_i.
__global__ void k_p_fill(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                         const double *__restrict__ val, const uint8_t *__restrict__ strong,
                         const int32_t *__restrict__ dia, const int32_t *__restrict__ agg, double omega,
                         int smoothed, const int32_t *__restrict__ P_ptr, int32_t *__restrict__ P_col,
                         double *__restrict__ P_val) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t ai = agg[i];
    if (ai < 0) return;
    const int32_t base = P_ptr[i];
    if (!smoothed) {
        P_col[base] = ai;
        P_val[base] = 1.0;
        return;
    }
    const int32_t b = ptr[i], e = ptr[i + 1];
    int32_t nc = 0;
    for (int32_t p = b; p < e; ++p) {
        int32_t j = col[p];
        if (j != i && !strong[p]) continue;
        int32_t c = agg[j];
        if (c < 0) continue;
        bool dup = false;
        for (int32_t s = 0; s < nc && !dup; ++s) dup = P_col[base + s] == c;
        if (dup) continue;
        int32_t t = nc;
        while (t > 0 && P_col[base + t - 1] > c) { P_col[base + t] = P_col[base + t - 1]; --t; }
        P_col[base + t] = c;
        ++nc;
    }
    double d = val[dia[i]];
    for (int32_t p = b; p < e; ++p)
        if (col[p] != i && !strong[p]) d = __dadd_rn(d, val[p]);
    // every term divides by d: its reciprocal once, then correctly rounded
    // quotients in integer arithmetic (the FP64 division bounds this kernel)
    const DivRecip rd = div_recip(d);
    for (int32_t s = 0; s < nc; ++s) {
        const int32_t c = P_col[base + s];
        double v = (c == ai) ? 1.0 : 0.0;
        for (int32_t p = b; p < e; ++p) {
            int32_t j = col[p];
            if (j != i && !strong[p]) continue;
            if (agg[j] != c) continue;
            double w = (j == i) ? d : val[p];
            v = __dsub_rn(v, div_rn(__dmul_rn(omega, w), rd));
        }
        P_val[base + s] = v;
    }
}

__global__ void k_count_cols(int64_t nnz, const int32_t *__restrict__ col, int32_t *__restrict__ cnt) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[p]], 1);
}

__global__ void k_transpose_scatter(int32_t n, const int32_t *__restrict__ P_ptr, const int32_t *__restrict__ P_col,
                                    const double *__restrict__ P_val, const int32_t *__restrict__ R_ptr,
                                    int32_t *__restrict__ cursor, int32_t *__restrict__ R_col,
                                    double *__restrict__ R_val) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t p = P_ptr[i]; p < P_ptr[i + 1]; ++p) {
        int32_t c = P_col[p];
        int32_t pos = R_ptr[c] + atomicAdd(&cursor[c], 1);
        R_col[pos] = i;
        R_val[pos] = P_val[p];
    }
}

// Sort each row of a CSR matrix by column (columns distinct within a row),
// one warp per row.  Rows of up to 128 entries are sorted in registers by a
// bitonic network over the warp (entry e = 32 j + lane in slot j; padding
// sorts last); longer rows by an insertion sort in place.
template <int E>
__device__ __forceinline__ void warp_bitonic(int32_t (&key)[E], double (&val)[E], int lane) {
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int s = k >> 1; s > 0; s >>= 1) {
            if (s >= 32) {
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const int jp = j ^ (s >> 5);
                    if (jp > j) {
                        const bool up = ((j * 32 + lane) & k) == 0;
                        if ((key[j] > key[jp]) == up) {
                            const int32_t tk = key[j];
                            key[j] = key[jp];
                            key[jp] = tk;
                            const double tv = val[j];
                            val[j] = val[jp];
                            val[jp] = tv;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const int e = j * 32 + lane;
                    const int32_t pk = __shfl_xor_sync(0xffffffffu, key[j], s);
                    const double pv = __shfl_xor_sync(0xffffffffu, val[j], s);
                    const bool up = (e & k) == 0, lower = (e & s) == 0;
                    if (lower == up ? pk < key[j] : pk > key[j]) {
                        key[j] = pk;
                        val[j] = pv;
                    }
                }
            }
        }
    }
}
template <int E>
__device__ __forceinline__ void warp_sort_row(int32_t b, int32_t len, int32_t *__restrict__ col,
                                              double *__restrict__ val, int lane) {
    int32_t key[E];
    double v[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int e = j * 32 + lane;
        key[j] = e < len ? col[b + e] : INT_MAX;
        v[j] = e < len ? val[b + e] : 0.0;
    }
    warp_bitonic<E>(key, v, lane);
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int e = j * 32 + lane;
        if (e < len) {
            col[b + e] = key[j];
            val[b + e] = v[j];
        }
    }
}
constexpr int kSortWarps = 4;
__global__ void __launch_bounds__(kSortWarps * 32)
k_sort_rows(int32_t nrows, const int32_t *__restrict__ ptr, int32_t *__restrict__ col, double *__restrict__ val) {
    const int lane = threadIdx.x & 31;
    const int32_t r = blockIdx.x * kSortWarps + (threadIdx.x >> 5);
    if (r >= nrows) return;  // warp-uniform
    const int32_t b = ptr[r], e = ptr[r + 1], len = e - b;
    if (len <= 1) return;
    if (len <= 64) warp_sort_row<2>(b, len, col, val, lane);
    else if (len <= 128) warp_sort_row<4>(b, len, col, val, lane);
    else if (lane == 0)
        for (int32_t a = b + 1; a < e; ++a) {
            int32_t c = col[a];
            double v = val[a];
            int32_t t = a;
            while (t > b && col[t - 1] > c) { col[t] = col[t - 1]; val[t] = val[t - 1]; --t; }
            col[t] = c;
            val[t] = v;
        }
}

// ------------------------------------------------------------------ symbolic product
// Each row's distinct columns go through a shared-memory hash table of `cap`
// slots (a power of two, at least twice the product's longest row of terms,
// so that a row's distinct columns always fit and probes stay short; at most
// kHashCap), then are ranked into sorted order.
constexpr int kSymSmemMax = 112 * 1024;

__device__ __forceinline__ bool hash_insert(int32_t *keys, int32_t *count, int32_t c, int cap, int shift) {
    uint32_t h = ((uint32_t)c * 2654435761u) >> shift;
    for (int probe = 0; probe < cap; ++probe) {
        int32_t old = atomicCAS(&keys[h], -1, c);
        if (old == -1) { atomicAdd(count, 1); return true; }
        if (old == c) return true;
        h = (h + 1) & (uint32_t)(cap - 1);
    }
    return false;
}

// the most terms (entries of the selected Y rows, plus the diagonal) of any
// row of C = X * Y: a bound on its distinct columns
__global__ void k_row_terms_max(int32_t nrows, const int32_t *__restrict__ X_ptr, const int32_t *__restrict__ X_col,
                                const int32_t *__restrict__ Y_ptr, int add_diag, int *out) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t c = 0;
    if (i < nrows) {
        c = add_diag ? 1 : 0;
        for (int32_t p = X_ptr[i]; p < X_ptr[i + 1]; ++p) {
            const int32_t k = X_col[p];
            c += Y_ptr[k + 1] - Y_ptr[k];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c = max(c, __shfl_xor_sync(0xffffffffu, c, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, c);
}

// G lanes per row of C = X * Y (32 / G rows per warp, each with its own hash
// table): the union of the Y-rows selected by X's row.  The warp's rows run
// the same code with warp-wide syncs; a row past the end takes part with no
// entries.
template <int G>
__global__ void k_spgemm_symbolic(int32_t nrows, int32_t ncols, const int32_t *__restrict__ X_ptr,
                                  const int32_t *__restrict__ X_col, const int32_t *__restrict__ Y_ptr,
                                  const int32_t *__restrict__ Y_col, int add_diag, int cap, int shift,
                                  int32_t *__restrict__ len, const int32_t *__restrict__ C_ptr,
                                  int32_t *__restrict__ C_col, int *st) {
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31, sub = lane % G;
    const int g = threadIdx.x / G;  // the row's group within the block
    const int lcap = cap / 2;       // distinct columns a row may hold
    int32_t *keys = smem + g * (cap + lcap + 2);
    int32_t *list = keys + cap;
    int32_t *cnt = list + lcap;
    const int32_t row = blockIdx.x * (blockDim.x / G) + g;
    const bool live = row < nrows;
    for (int h = sub; h < cap; h += G) keys[h] = -1;
    if (sub == 0) { cnt[0] = 0; cnt[1] = 0; }
    __syncwarp();
    bool ok = true;
    if (live && add_diag && row < ncols && sub == 0) ok = hash_insert(keys, &cnt[0], row, cap, shift);
    if (live)
        for (int32_t p = X_ptr[row] + sub; p < X_ptr[row + 1]; p += G) {
            int32_t k = X_col[p];
            for (int32_t q = Y_ptr[k]; q < Y_ptr[k + 1] && ok; ++q) ok = hash_insert(keys, &cnt[0], Y_col[q], cap, shift);
        }
    __syncwarp();
    const int32_t L = cnt[0];
    const bool bad = !__all_sync(0xffffffffu, ok) || __any_sync(0xffffffffu, live && L > lcap);
    if (bad) {
        if (lane == 0) atomicOr(st, DEV_ERR_CAPACITY);
        return;
    }
    if (C_ptr == nullptr) {
        if (live && sub == 0) len[row] = L;
        return;
    }
    for (int h = sub; h < cap; h += G) {
        int32_t c = keys[h];
        if (c >= 0) list[atomicAdd(&cnt[1], 1)] = c;
    }
    __syncwarp();
    if (!live) return;
    const int32_t base = C_ptr[row];
    if (C_ptr[row + 1] - base != L) {
        if (sub == 0) atomicOr(st, DEV_ERR_STATE);
        return;
    }
    for (int32_t e = sub; e < L; e += G) {
        int32_t v = list[e], rank = 0;
        for (int32_t x = 0; x < L; ++x) rank += list[x] < v;
        C_col[base + rank] = v;
    }
}

// ------------------------------------------------------------------ gather metadata
__global__ void k_t1_count(int32_t n, const int32_t *__restrict__ A_ptr, const int32_t *__restrict__ A_col,
                           const int32_t *__restrict__ P_ptr, int32_t *__restrict__ cnt) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = 0;
    for (int32_t p = A_ptr[i]; p < A_ptr[i + 1]; ++p) {
        int32_t k = A_col[p];
        c += P_ptr[k + 1] - P_ptr[k];
    }
    cnt[i] = c;
}

// slot1[t]: position within row i of A*P of the column of the t-th term
// (A entry (i,k) in column order, then P row k in column order)
__global__ void k_t1_fill(int32_t n, const int32_t *__restrict__ A_ptr, const int32_t *__restrict__ A_col,
                          const int32_t *__restrict__ P_ptr, const int32_t *__restrict__ P_col,
                          const int32_t *__restrict__ AP_ptr, const int32_t *__restrict__ AP_col,
                          const int32_t *__restrict__ t1ptr, uint16_t *__restrict__ slot1, int *st) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t t = t1ptr[i];
    const int32_t b = AP_ptr[i], e = AP_ptr[i + 1];
    for (int32_t p = A_ptr[i]; p < A_ptr[i + 1]; ++p) {
        int32_t k = A_col[p];
        for (int32_t q = P_ptr[k]; q < P_ptr[k + 1]; ++q) {
            int32_t c = P_col[q];
            int32_t pos = find_in_row(AP_col, b, e, c);
            if (pos >= e || AP_col[pos] != c) { atomicOr(st, DEV_ERR_STATE); pos = b; }
            slot1[t++] = (uint16_t)(pos - b);
        }
    }
}

__global__ void k_t2_count(int32_t nc, const int32_t *__restrict__ R_ptr, const int32_t *__restrict__ R_col,
                           const int32_t *__restrict__ AP_ptr, int32_t *__restrict__ cnt) {
    int32_t I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int32_t c = 0;
    for (int32_t r = R_ptr[I]; r < R_ptr[I + 1]; ++r) {
        int32_t i = R_col[r];
        c += AP_ptr[i + 1] - AP_ptr[i];
    }
    cnt[I] = c;
}

// slot2[t]: position within coarse row I of the column of the t-th term
// (R entry (I,i) in column order, then row i of A*P in column order).  One
// warp per coarse row: the row's columns of A_c staged in shared memory (rows
// of up to kT2Cols entries; longer ones are searched in place), the lanes over
// the R entries, the prefix of their A P row lengths giving each term's index
constexpr int kT2Warps = 4;
constexpr int kT2Cols = 1024;
__global__ void __launch_bounds__(kT2Warps * 32)
k_t2_fill(int32_t nc, const int32_t *__restrict__ R_ptr, const int32_t *__restrict__ R_col,
               const int32_t *__restrict__ AP_ptr, const int32_t *__restrict__ AP_col,
               const int32_t *__restrict__ Ac_ptr, const int32_t *__restrict__ Ac_col,
               const int32_t *__restrict__ t2ptr, uint16_t *__restrict__ slot2, int *st) {
    __shared__ int32_t s_cols[kT2Warps][kT2Cols];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t I = blockIdx.x * kT2Warps + w;
    if (I >= nc) return;  // warp-uniform
    const int32_t b = Ac_ptr[I], L = Ac_ptr[I + 1] - b;
    const int32_t *cols = Ac_col + b;
    if (L <= kT2Cols) {
        for (int32_t x = lane; x < L; x += 32) s_cols[w][x] = cols[x];
        __syncwarp();
        cols = s_cols[w];
    }
    const int64_t t0 = t2ptr[I];
    const int32_t r1 = R_ptr[I + 1];
    int64_t carry = 0;
    for (int32_t rc = R_ptr[I]; rc < r1; rc += 32) {
        const int32_t r = rc + lane;
        int32_t q0 = 0, len = 0;
        if (r < r1) {
            const int32_t i = R_col[r];
            q0 = AP_ptr[i];
            len = AP_ptr[i + 1] - q0;
        }
        int32_t inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int64_t t = t0 + carry + (inc - len);
        for (int32_t q = 0; q < len; ++q) {
            const int32_t c = AP_col[q0 + q];
            int32_t pos = find_in_row(cols, 0, L, c);
            if (pos >= L || cols[pos] != c) { atomicOr(st, DEV_ERR_STATE); pos = 0; }
            slot2[t + q] = (uint16_t)pos;
        }
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
}

// ------------------------------------------------------------------ gather operators
// With P and R fixed, the numeric Galerkin product is linear in the values:
// AP = N a and A_c = M AP, with fixed sparse N (coefficients P_kJ) and M
// (coefficients R_Ii).  These kernels build N and M from the slot metadata:
// each output entry's terms are grouped, keeping their sequential order.

constexpr int kGroupWarps = 4;
constexpr int kGroupSlots = 2048;

// One warp per output row: a stable counting sort of the row's terms by slot.
// eptr[out_ptr[row] + s] = first sorted position of slot s; perm[pos] = term.
__global__ void __launch_bounds__(kGroupWarps * 32)
k_group_terms(int32_t nrows, const int32_t *__restrict__ tptr, const uint16_t *__restrict__ slot,
              const int32_t *__restrict__ out_ptr, int32_t *__restrict__ eptr, int32_t *__restrict__ perm,
              int *st) {
    __shared__ int32_t cnt[kGroupWarps][kGroupSlots];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t row = blockIdx.x * kGroupWarps + w;
    if (row >= nrows) return;  // warp-uniform
    const int32_t t0 = tptr[row], t1 = tptr[row + 1];
    const int32_t ob = out_ptr[row], L = out_ptr[row + 1] - ob;
    if (L > kGroupSlots) {
        if (lane == 0) atomicOr(st, DEV_ERR_CAPACITY);
        return;
    }
    int32_t *c = cnt[w];
    for (int s = lane; s < L; s += 32) c[s] = 0;
    __syncwarp();
    for (int32_t t = t0 + lane; t < t1; t += 32) atomicAdd(&c[slot[t]], 1);
    __syncwarp();
    int32_t carry = 0;
    for (int32_t s0 = 0; s0 < L; s0 += 32) {
        const int32_t s = s0 + lane;
        const int32_t v = s < L ? c[s] : 0;
        int32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (s < L) {
            const int32_t start = carry + inc - v;
            c[s] = start;
            eptr[ob + s] = t0 + start;
        }
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    __syncwarp();
    for (int32_t base = t0; base < t1; base += 32) {
        const int32_t t = base + lane;
        const bool valid = t < t1;
        const unsigned active = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const int sl = slot[t];
            const unsigned peers = __match_any_sync(active, sl);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            perm[t0 + c[sl] + rank] = t;
            __syncwarp(active);
            if (rank == 0) c[sl] += __popc(peers);
        }
        __syncwarp();
    }
}

// term attributes in the sequential order, stage 1: A entry and P value
__global__ void k_stage1_terms(int32_t n, const int32_t *__restrict__ A_ptr, const int32_t *__restrict__ A_col,
                               const int32_t *__restrict__ P_ptr, const double *__restrict__ P_val,
                               const int32_t *__restrict__ t1ptr, int32_t *__restrict__ idx,
                               double *__restrict__ wgt) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t t = t1ptr[i];
    for (int32_t p = A_ptr[i]; p < A_ptr[i + 1]; ++p) {
        const int32_t k = A_col[p];
        for (int32_t q = P_ptr[k]; q < P_ptr[k + 1]; ++q) {
            idx[t] = p;
            wgt[t] = P_val[q];
            ++t;
        }
    }
}

// stage 2: AP entry and R value
__global__ void k_stage2_terms(int32_t nc, const int32_t *__restrict__ R_ptr, const int32_t *__restrict__ R_col,
                               const double *__restrict__ R_val, const int32_t *__restrict__ AP_ptr,
                               const int32_t *__restrict__ t2ptr, int32_t *__restrict__ idx,
                               double *__restrict__ wgt) {
    const int32_t I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int64_t t = t2ptr[I];
    for (int32_t r = R_ptr[I]; r < R_ptr[I + 1]; ++r) {
        const int32_t i = R_col[r];
        const double x = R_val[r];
        for (int32_t e = AP_ptr[i]; e < AP_ptr[i + 1]; ++e) {
            idx[t] = e;
            wgt[t] = x;
            ++t;
        }
    }
}

// sorted operator: idx_out[pos] = idx_in[perm[pos]], weights likewise (FP64 or FP32)
__global__ void k_permute_terms(int64_t nt, const int32_t *__restrict__ perm, const int32_t *__restrict__ idx_in,
                                const double *__restrict__ w_in, int32_t *__restrict__ idx_out,
                                double *__restrict__ w_out, float *__restrict__ wf_out) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nt; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = perm[p];
        idx_out[p] = idx_in[t];
        const double w = w_in[t];
        if (w_out) w_out[p] = w;
        if (wf_out) wf_out[p] = (float)w;
    }
}

// last[i]: the last column of row i (rows sorted), -1 for an empty row
__global__ void k_row_last(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                           int32_t *__restrict__ last) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t e = ptr[i + 1];
    last[i] = e > ptr[i] ? col[e - 1] : -1;
}

__global__ void k_row_maxlen(int32_t n, const int32_t *__restrict__ ptr, int *out) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    int l = i < n ? ptr[i + 1] - ptr[i] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l = max(l, __shfl_xor_sync(0xffffffffu, l, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, l);
}

}  // namespace

// ======================================================================= launchers
int64_t scan_tmp_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 2; }

void scan_counts(const int32_t *in, int32_t *out, int64_t n, int *st, int64_t *tmp, cudaStream_t s) {
    if (n <= 0) {
        cudaMemsetAsync(out, 0, sizeof(int32_t), s);
        return;
    }
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    count_launch();
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp);
    count_launch();
    k_scan_blocks<<<1, kScanThreads, 0, s>>>(tmp, nb);
    count_launch();
    k_scan_final<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, tmp, nb, st);
}

void launch_poisson_rowlen(int dim, int N, int32_t *len, cudaStream_t s) {
    int64_t n = dim == 2 ? (int64_t)N * N : (int64_t)N * N * N;
    count_launch();
    k_poisson_rowlen<<<nblocks(n), kThreads, 0, s>>>(dim, N, n, len);
}
void launch_poisson_cols(int dim, int N, const int32_t *ptr, int32_t *col, cudaStream_t s) {
    int64_t n = dim == 2 ? (int64_t)N * N : (int64_t)N * N * N;
    count_launch();
    k_poisson_cols<<<nblocks(n), kThreads, 0, s>>>(dim, N, n, ptr, col);
}
void launch_poisson_vals(int dim, int N, int top, const double *rho, int logd, const int32_t *ptr, double *val,
                         cudaStream_t s) {
    int64_t n = dim == 2 ? (int64_t)N * N : (int64_t)N * N * N;
    count_launch();
    k_poisson_vals<<<nblocks(n), kThreads, 0, s>>>(dim, N, n, top, rho, logd, ptr, val);
}
void launch_poisson_grad(int dim, int N, int top, const double *rho, int logd, const double *u, const double *lam,
                         double *grad, cudaStream_t s) {
    int64_t n = dim == 2 ? (int64_t)N * N : (int64_t)N * N * N;
    count_launch();
    k_poisson_grad<<<nblocks(n), kThreads, 0, s>>>(dim, N, n, top, rho, logd, u, lam, grad);
}

void launch_levelset_vals(int dim, int N, const double *fx, const double *fy, const double *fz, const int32_t *ptr,
                          double *val, cudaStream_t s) {
    int64_t n = dim == 2 ? (int64_t)N * N : (int64_t)N * N * N;
    count_launch();
    k_levelset_vals<<<nblocks(n), kThreads, 0, s>>>(dim, N, n, fx, fy, fz, ptr, val);
}

void launch_check_rowptr(int32_t n, int32_t nnz, const int32_t *ptr, int *st, cudaStream_t s) {
    const int64_t b = nblocks((int64_t)n + 1);
    count_launch();
    k_check_rowptr<<<(unsigned)(b > 4096 ? 4096 : b), kThreads, 0, s>>>(n, nnz, ptr, st);
}
void launch_check_pattern(int32_t n, const int32_t *ptr, const int32_t *col, int32_t *dia, int *st,
                          cudaStream_t s) {
    count_launch();
    k_check_pattern<<<nblocks(n), kThreads, 0, s>>>(n, ptr, col, dia, st);
}
void launch_check_finite(int64_t nnz, const double *val, int *st, cudaStream_t s) {
    int64_t b = nblocks(nnz);
    count_launch();
    k_check_finite<<<(unsigned)(b > 4096 ? 4096 : b), kThreads, 0, s>>>(nnz, val, st);
}
void launch_strength(int32_t n, const int32_t *ptr, const int32_t *col, const double *val, const int32_t *dia,
                     double eps2, uint8_t *strong, int32_t *deg, cudaStream_t s) {
    count_launch();
    k_strength<<<nblocks(n), kThreads, 0, s>>>(n, ptr, col, val, dia, eps2, strong, deg);
}

int32_t run_aggregation(int32_t n, const int32_t *ptr, const int32_t *col, const double *val,
                        const uint8_t *strong, const int32_t *deg, int32_t *agg, int8_t *state, int64_t *m1,
                        uint8_t *r1, int32_t *root_id, int32_t *agg1, int32_t *root_of, int *counter, int *st,
                        int64_t *scan_tmp, cudaStream_t s) {
    const int nb = nblocks(n);
    count_launch();
    k_mis_init<<<nb, kThreads, 0, s>>>(n, deg, state);
    // every round turns at least the undecided node of largest priority into
    // a root, so at most n rounds; in practice a few dozen
    for (int32_t round = 0; round <= n; ++round) {
        count_launch();
        k_mis_m1<<<nb, kThreads, 0, s>>>(n, ptr, col, strong, state, m1);
        count_launch();
        k_mis_select<<<nb, kThreads, 0, s>>>(n, ptr, col, strong, state, m1);
        count_launch();
        k_mis_r1<<<nb, kThreads, 0, s>>>(n, ptr, col, strong, state, r1);
        cudaMemsetAsync(counter, 0, sizeof(int), s);
        count_launch();
        k_mis_exclude<<<nb, kThreads, 0, s>>>(n, ptr, col, strong, state, r1, counter);
        int h = -1;
        if (cudaMemcpyAsync(&h, counter, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
        if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
        if (h == 0) break;
        if (round == n) return -1;
    }
    count_launch();
    k_root_flags<<<nb, kThreads, 0, s>>>(n, state, agg);
    scan_counts(agg, root_id, n, st, scan_tmp, s);
    int32_t nagg = 0;
    if (cudaMemcpyAsync(&nagg, root_id + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    count_launch();
    k_agg_phase1<<<nb, kThreads, 0, s>>>(n, ptr, col, strong, state, root_id, agg1, root_of);
    count_launch();
    k_agg_phase2<<<nb, kThreads, 0, s>>>(n, ptr, col, val, strong, state, agg1, root_of, agg, st);
    return nagg;
}

void launch_p_count(int32_t n, const int32_t *ptr, const int32_t *col, const uint8_t *strong, const int32_t *agg,
                    int smoothed, int32_t *plen, cudaStream_t s) {
    count_launch();
    k_p_count<<<nblocks(n), kThreads, 0, s>>>(n, ptr, col, strong, agg, smoothed, plen);
}
void launch_p_fill(int32_t n, const int32_t *ptr, const int32_t *col, const double *val, const uint8_t *strong,
                   const int32_t *dia, const int32_t *agg, double omega, int smoothed, const int32_t *P_ptr,
                   int32_t *P_col, double *P_val, cudaStream_t s) {
    count_launch();
    k_p_fill<<<nblocks(n), kThreads, 0, s>>>(n, ptr, col, val, strong, dia, agg, omega, smoothed, P_ptr, P_col,
                                             P_val);
}
void launch_count_cols(int64_t nnz, const int32_t *col, int32_t *cnt, cudaStream_t s) {
    int64_t b = nblocks(nnz);
    count_launch();
    k_count_cols<<<(unsigned)(b > 8192 ? 8192 : b), kThreads, 0, s>>>(nnz, col, cnt);
}
void launch_transpose_scatter(int32_t n, const int32_t *P_ptr, const int32_t *P_col, const double *P_val,
                              const int32_t *R_ptr, int32_t *cursor, int32_t *R_col, double *R_val,
                              cudaStream_t s) {
    count_launch();
    k_transpose_scatter<<<nblocks(n), kThreads, 0, s>>>(n, P_ptr, P_col, P_val, R_ptr, cursor, R_col, R_val);
}
void launch_sort_rows(int32_t nrows, const int32_t *ptr, int32_t *col, double *val, cudaStream_t s) {
    count_launch();
    if (nrows <= 0) return;
    k_sort_rows<<<(unsigned)((nrows + kSortWarps - 1) / kSortWarps), kSortWarps * 32, 0, s>>>(nrows, ptr, col, val);
}

void launch_row_terms_max(int32_t nrows, const int32_t *X_ptr, const int32_t *X_col, const int32_t *Y_ptr,
                          int add_diag, int *out, cudaStream_t s) {
    if (nrows <= 0) return;
    count_launch();
    k_row_terms_max<<<nblocks(nrows), kThreads, 0, s>>>(nrows, X_ptr, X_col, Y_ptr, add_diag, out);
}
int spgemm_symbolic_cap(int32_t max_terms) {
    int cap = 64;
    while (cap < kHashCap && cap < 2 * max_terms) cap *= 2;
    return cap;
}
namespace {
template <int G>
void launch_symbolic_g(int32_t nrows, int32_t ncols, const int32_t *X_ptr, const int32_t *X_col,
                       const int32_t *Y_ptr, const int32_t *Y_col, int add_diag, int cap, int shift, int32_t *len,
                       const int32_t *C_ptr, int32_t *C_col, int *st, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_spgemm_symbolic<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSymSmemMax);
        attr_set = true;
    }
    const size_t per_row = (size_t)(cap + cap / 2 + 2) * sizeof(int32_t);
    int warps = 8;
    while (warps > 1 && per_row * (size_t)(warps * 32 / G) > (size_t)kSymSmemMax) warps >>= 1;
    const int rows = warps * 32 / G;
    const unsigned grid = (unsigned)((nrows + rows - 1) / rows);
    count_launch();
    k_spgemm_symbolic<G><<<grid, warps * 32, per_row * (size_t)rows, s>>>(nrows, ncols, X_ptr, X_col, Y_ptr, Y_col,
                                                                         add_diag, cap, shift, len, C_ptr, C_col, st);
}
}  // namespace

void launch_spgemm_symbolic(int32_t nrows, int32_t ncols, const int32_t *X_ptr, const int32_t *X_col,
                            const int32_t *Y_ptr, const int32_t *Y_col, int add_diag, int cap, int lanes,
                            int32_t *len, const int32_t *C_ptr, int32_t *C_col, int *st, cudaStream_t s) {
    if (nrows <= 0) return;
    int shift = 32;
    for (int c = cap; c > 1; c >>= 1) --shift;  // cap = 2^(32 - shift)
    if (lanes <= 8)
        launch_symbolic_g<8>(nrows, ncols, X_ptr, X_col, Y_ptr, Y_col, add_diag, cap, shift, len, C_ptr, C_col, st, s);
    else if (lanes <= 16)
        launch_symbolic_g<16>(nrows, ncols, X_ptr, X_col, Y_ptr, Y_col, add_diag, cap, shift, len, C_ptr, C_col, st,
                              s);
    else
        launch_symbolic_g<32>(nrows, ncols, X_ptr, X_col, Y_ptr, Y_col, add_diag, cap, shift, len, C_ptr, C_col, st,
                              s);
}

void launch_t1_count(int32_t n, const int32_t *A_ptr, const int32_t *A_col, const int32_t *P_ptr, int32_t *cnt,
                     cudaStream_t s) {
    count_launch();
    k_t1_count<<<nblocks(n), kThreads, 0, s>>>(n, A_ptr, A_col, P_ptr, cnt);
}
void launch_t1_fill(int32_t n, const int32_t *A_ptr, const int32_t *A_col, const int32_t *P_ptr,
                    const int32_t *P_col, const int32_t *AP_ptr, const int32_t *AP_col, const int32_t *t1ptr,
                    uint16_t *slot1, int *st, cudaStream_t s) {
    count_launch();
    k_t1_fill<<<nblocks(n), kThreads, 0, s>>>(n, A_ptr, A_col, P_ptr, P_col, AP_ptr, AP_col, t1ptr, slot1, st);
}
void launch_t2_count(int32_t nc, const int32_t *R_ptr, const int32_t *R_col, const int32_t *AP_ptr, int32_t *cnt,
                     cudaStream_t s) {
    count_launch();
    k_t2_count<<<nblocks(nc), kThreads, 0, s>>>(nc, R_ptr, R_col, AP_ptr, cnt);
}
void launch_t2_fill(int32_t nc, const int32_t *R_ptr, const int32_t *R_col, const int32_t *AP_ptr,
                    const int32_t *AP_col, const int32_t *Ac_ptr, const int32_t *Ac_col, const int32_t *t2ptr,
                    uint16_t *slot2, int *st, cudaStream_t s) {
    count_launch();
    if (nc <= 0) return;
    k_t2_fill<<<(unsigned)((nc + kT2Warps - 1) / kT2Warps), kT2Warps * 32, 0, s>>>(nc, R_ptr, R_col, AP_ptr,
                                                                                     AP_col, Ac_ptr, Ac_col, t2ptr,
                                                                                     slot2, st);
}
void launch_group_terms(int32_t nrows, const int32_t *tptr, const uint16_t *slot, const int32_t *out_ptr,
                        int32_t *eptr, int32_t *perm, int *st, cudaStream_t s) {
    if (nrows <= 0) return;
    count_launch();
    k_group_terms<<<(unsigned)((nrows + kGroupWarps - 1) / kGroupWarps), kGroupWarps * 32, 0, s>>>(
        nrows, tptr, slot, out_ptr, eptr, perm, st);
}
void launch_stage1_terms(int32_t n, const int32_t *A_ptr, const int32_t *A_col, const int32_t *P_ptr,
                         const double *P_val, const int32_t *t1ptr, int32_t *idx, double *wgt, cudaStream_t s) {
    count_launch();
    k_stage1_terms<<<nblocks(n), kThreads, 0, s>>>(n, A_ptr, A_col, P_ptr, P_val, t1ptr, idx, wgt);
}
void launch_stage2_terms(int32_t nc, const int32_t *R_ptr, const int32_t *R_col, const double *R_val,
                         const int32_t *AP_ptr, const int32_t *t2ptr, int32_t *idx, double *wgt, cudaStream_t s) {
    count_launch();
    k_stage2_terms<<<nblocks(nc, 128), 128, 0, s>>>(nc, R_ptr, R_col, R_val, AP_ptr, t2ptr, idx, wgt);
}
void launch_permute_terms(int64_t nt, const int32_t *perm, const int32_t *idx_in, const double *w_in,
                          int32_t *idx_out, double *w_out, float *wf_out, cudaStream_t s) {
    if (nt <= 0) return;
    int64_t b = nblocks(nt);
    count_launch();
    k_permute_terms<<<(unsigned)(b > 8192 ? 8192 : b), kThreads, 0, s>>>(nt, perm, idx_in, w_in, idx_out, w_out,
                                                                         wf_out);
}
void launch_row_last(int32_t n, const int32_t *ptr, const int32_t *col, int32_t *last, cudaStream_t s) {
    if (n <= 0) return;
    count_launch();
    k_row_last<<<nblocks(n), kThreads, 0, s>>>(n, ptr, col, last);
}
void launch_row_maxlen(int32_t n, const int32_t *ptr, int *out, cudaStream_t s) {
    count_launch();
    k_row_maxlen<<<nblocks(n), kThreads, 0, s>>>(n, ptr, out);
}

}  // namespace amgpr
