// block.cu -- kernels of the 4 x 4 block-valued hierarchy.
//
// Sec. 4 solves its monolithic Navier-Stokes systems with BiCGStab
// preconditioned by non-smoothed aggregation AMG with damped Jacobi
// smoothing, on a backend whose matrix values are 4 x 4 blocks.  Block CSR:
// the pattern is a scalar CSR over nodes; entry e holds 16 doubles, row-major
// (component r of the row node, component c of the column node), at
// val[16 e]; vectors hold the 4 components of a node consecutively.
//
// Strength of connection and aggregation run on the node graph whose values
// are the block norms (the scalar kernels); with P = P_tent the Galerkin
// product is two fixed gather operators applied to 16 values per entry.
// Every kernel reproduces the summation order of the serial definition, so
// structure and values match it bit for bit.
#include "common.cuh"

namespace amgpr {
namespace {

constexpr int kBThreads = 128;
inline int bblocks(int64_t n, int t = kBThreads) { return (int)((n + t - 1) / t); }

// ------------------------------------------------------------------ assembly
// Synthetic monolithic Oseen-type system (the stand-in for the stabilised
// Navier-Stokes matrices of Sec. 4), one thread per cell.  kappa = mass rho +
// 6 mu; for the face to neighbour j in direction d, side s (outward flux phi
// = s * face velocity, mu_f = (2 mu_c mu_j) / (mu_c + mu_j),
// beta_f = 2 / (1/kappa_c + 1/kappa_j)):
//   off-diagonal block: velocity diagonal min(phi, 0) - mu_f,
//   (u_d, p) = (p, u_d) = (s / 2) beta_f, (p, p) = -beta_f;
//   diagonal block: velocity a = mass rho_c + sum of (mu_f + max(phi, 0)),
//   plus 2 mu_c per wall face; (u_d, p) = g_d = sum over the wall faces of
//   direction d of (s / 2) kappa_c, (p, u_d) = -g_d; (p, p) = sum of beta_f,
//   plus 2 kappa_c (as 2 / (1/kappa_c)) on the top face.
// Faces in ascending neighbour order z-, y-, x-, x+, y+, z+.
__global__ void k_stokes_vals(int N, int64_t n, const double *__restrict__ rho, const double *__restrict__ mu,
                              const double *__restrict__ fx, const double *__restrict__ fy,
                              const double *__restrict__ fz, double mass, const int32_t *__restrict__ ptr,
                              double *__restrict__ val) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int64_t s3 = (int64_t)N * N, N1 = N + 1;
    const int64_t x = c % N, y = (c / N) % N, z = c / s3;
    const bool has[6] = {z > 0, y > 0, x > 0, x < N - 1, y < N - 1, z < N - 1};
    const int64_t nbr[6] = {c - s3, c - N, c - 1, c + 1, c + N, c + s3};
    const int dir[6] = {2, 1, 0, 0, 1, 2};
    const double sg[6] = {-1.0, -1.0, -1.0, 1.0, 1.0, 1.0};
    const double wv[6] = {fz[(z * N + y) * N + x], fy[(z * N1 + y) * N + x], fx[(z * N + y) * N1 + x],
                          fx[(z * N + y) * N1 + x + 1], fy[(z * N1 + y + 1) * N + x],
                          fz[((z + 1) * N + y) * N + x]};
    const double kap_c = mass * rho[c] + 6.0 * mu[c];
    const double rinv_c = 1.0 / kap_c;
    double a = mass * rho[c], s = 0.0;
    double g[3] = {0.0, 0.0, 0.0};
    int32_t p = ptr[c], dpos = p;
    for (int t = 0; t < 7; ++t) {
        if (t == 3) { dpos = p++; continue; }
        const int q = t < 3 ? t : t - 1;
        const int d = dir[q];
        const double sig = sg[q];
        if (!has[q]) {
            a = a + 2.0 * mu[c];
            g[d] = g[d] + (0.5 * sig) * kap_c;
            continue;
        }
        const int64_t j = nbr[q];
        const double phi = sig * wv[q];
        const double muf = (2.0 * mu[c] * mu[j]) / (mu[c] + mu[j]);
        const double rinv_j = 1.0 / (mass * rho[j] + 6.0 * mu[j]);
        const double beta = 2.0 / (rinv_c + rinv_j);
        double *B = val + (int64_t)16 * p;
        const double off = (phi < 0.0 ? phi : 0.0) - muf;
        const double cpl = (0.5 * sig) * beta;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            double v = 0.0;
            if (k == 0 || k == 5 || k == 10) v = off;
            else if (k == d * 4 + 3 || k == 12 + d) v = cpl;
            else if (k == 15) v = -beta;
            B[k] = v;
        }
        a = a + (muf + (phi > 0.0 ? phi : 0.0));
        s = s + beta;
        ++p;
    }
    if (z == N - 1) s = s + 2.0 / rinv_c;
    double *D = val + (int64_t)16 * dpos;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        double v = 0.0;
        if (k == 0 || k == 5 || k == 10) v = a;
        else if (k == 15) v = s;
        else if (k % 4 == 3) v = g[k / 4];
        else if (k >= 12) v = -g[k - 12];
        D[k] = v;
    }
}

// ------------------------------------------------------------------ setup pieces
// Frobenius norm per block: fma sum of the squares in storage order, sqrt.
__global__ void k_block_norms(int64_t nnz, const double *__restrict__ bv, double *__restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const double2 *b = reinterpret_cast<const double2 *>(bv + 16 * e);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const double2 v = b[k];
        s = fma(v.x, v.x, s);
        s = fma(v.y, v.y, s);
    }
    out[e] = sqrt(s);
}

// y[16 e + k] = sum over the terms t of entry e, in order, of w_t x[16 idx_t + k]
// (fma from 0): the numeric Galerkin stages with scalar P / R entries; one
// thread per output value, 16 consecutive threads per block entry.
__global__ void k_block_gather(int64_t nout, const int32_t *__restrict__ eptr, const int32_t *__restrict__ idx,
                               const double *__restrict__ w, const double *__restrict__ x, double *__restrict__ y) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 16 * nout) return;
    const int64_t e = tid >> 4;
    const int k = (int)(tid & 15);
    double acc = 0.0;
    for (int32_t t = eptr[e]; t < eptr[e + 1]; ++t) acc = fma(w[t], x[(int64_t)16 * idx[t] + k], acc);
    y[tid] = acc;
}

// 4 x 4 Gauss-Jordan inverse with partial pivoting (first entry of largest
// magnitude; rows swapped; pivot row divided by the pivot; fma elimination
// from every other row); false for a singular or non-finite block.
__device__ bool inv4_dev(double *a, double *inv) {
#pragma unroll
    for (int k = 0; k < 16; ++k) inv[k] = (k % 5 == 0) ? 1.0 : 0.0;
    for (int k = 0; k < 4; ++k) {
        int p = k;
        double best = fabs(a[k * 4 + k]);
        for (int r = k + 1; r < 4; ++r) {
            const double v = fabs(a[r * 4 + k]);
            if (v > best) { best = v; p = r; }
        }
        if (!(best > 0.0) || !isfinite(best)) return false;
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
    return true;
}

// damped block Jacobi: Minv_i = w_J inv(A_ii), zero for a singular block
__global__ void k_block_jacobi(int32_t n, const int32_t *__restrict__ dia, const double *__restrict__ bv, double wj,
                               double *__restrict__ minv) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a[16], inv[16];
    const double *src = bv + (int64_t)16 * dia[i];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = src[k];
    const bool ok = inv4_dev(a, inv);
    double *dst = minv + (int64_t)16 * i;
#pragma unroll
    for (int k = 0; k < 16; ++k) dst[k] = ok ? wj * inv[k] : 0.0;
}

// coarsest level: the block matrix expanded to 4 n scalar rows (dense,
// row-major, zeroed beforehand)
__global__ void k_block_to_dense(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                 const double *__restrict__ bv, double *__restrict__ dense) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t n4 = 4 * (int64_t)n;
    for (int32_t e = ptr[i]; e < ptr[i + 1]; ++e)
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c)
                dense[(4 * (int64_t)i + r) * n4 + 4 * (int64_t)col[e] + c] = bv[(int64_t)16 * e + 4 * r + c];
}

// ------------------------------------------------------------------ V-cycle pieces (one thread per node)
__device__ __forceinline__ void load4(const double *p, double v[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void store4(double *p, const double v[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// (A x)_i, component r summing in entry order then component order (fma from 0)
__device__ __forceinline__ void block_row(int32_t i, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                          const double *__restrict__ bv, const double *__restrict__ x, double y[4]) {
    y[0] = y[1] = y[2] = y[3] = 0.0;
    for (int32_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        double xv[4];
        load4(x + (int64_t)4 * col[e], xv);
        const double2 *b = reinterpret_cast<const double2 *>(bv + (int64_t)16 * e);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const double2 lo = b[2 * r], hi = b[2 * r + 1];
            y[r] = fma(lo.x, xv[0], y[r]);
            y[r] = fma(lo.y, xv[1], y[r]);
            y[r] = fma(hi.x, xv[2], y[r]);
            y[r] = fma(hi.y, xv[3], y[r]);
        }
    }
}

// u_out = u_in + Minv_i t (fma from u_in, component order)
__device__ __forceinline__ void apply_minv(const double *__restrict__ m, const double t[4], const double uin[4],
                                           double uout[4]) {
    const double2 *M = reinterpret_cast<const double2 *>(m);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const double2 lo = M[2 * r], hi = M[2 * r + 1];
        double s = uin[r];
        s = fma(lo.x, t[0], s);
        s = fma(lo.y, t[1], s);
        s = fma(hi.x, t[2], s);
        s = fma(hi.y, t[3], s);
        uout[r] = s;
    }
}

// first pre-smoothing step from u = 0: u = Minv f
__global__ void k_block_smooth0(int32_t n, const double *__restrict__ minv, const double *__restrict__ f,
                                double *__restrict__ u, const int *skip) {
    pdl_wait();
    if (skip && *skip) return;
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double t[4], z[4] = {0.0, 0.0, 0.0, 0.0}, o[4];
    load4(f + (int64_t)4 * i, t);
    apply_minv(minv + (int64_t)16 * i, t, z, o);
    store4(u + (int64_t)4 * i, o);
}

// one damped block-Jacobi sweep: u_out = u_in + Minv (f - A u_in)
__global__ void k_block_sweep(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                              const double *__restrict__ bv, const double *__restrict__ minv,
                              const double *__restrict__ f, const double *__restrict__ uin, double *__restrict__ uout,
                              const int *skip) {
    pdl_wait();
    if (skip && *skip) return;
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double y[4], fv[4], t[4], u0[4], o[4];
    block_row(i, ptr, col, bv, uin, y);
    load4(f + (int64_t)4 * i, fv);
#pragma unroll
    for (int r = 0; r < 4; ++r) t[r] = fv[r] - y[r];
    load4(uin + (int64_t)4 * i, u0);
    apply_minv(minv + (int64_t)16 * i, t, u0, o);
    store4(uout + (int64_t)4 * i, o);
}

// r = f - A u
__global__ void k_block_residual(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                 const double *__restrict__ bv, const double *__restrict__ f,
                                 const double *__restrict__ u, double *__restrict__ r, const int *skip) {
    pdl_wait();
    if (skip && *skip) return;
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double y[4], fv[4];
    block_row(i, ptr, col, bv, u, y);
    load4(f + (int64_t)4 * i, fv);
#pragma unroll
    for (int k = 0; k < 4; ++k) fv[k] = fv[k] - y[k];
    store4(r + (int64_t)4 * i, fv);
}

// f_c = R r (scalar R, per component: fma from 0 in R's column order)
__global__ void k_block_restrict(int32_t nc, const int32_t *__restrict__ Rptr, const int32_t *__restrict__ Rcol,
                                 const double *__restrict__ Rval, const double *__restrict__ r,
                                 double *__restrict__ fc, const int *skip) {
    pdl_wait();
    if (skip && *skip) return;
    const int32_t I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int32_t p = Rptr[I]; p < Rptr[I + 1]; ++p) {
        double v[4];
        load4(r + (int64_t)4 * Rcol[p], v);
        const double w = Rval[p];
#pragma unroll
        for (int c = 0; c < 4; ++c) s[c] = fma(w, v[c], s[c]);
    }
    store4(fc + (int64_t)4 * I, s);
}

// u += P u_c
__global__ void k_block_prolong(int32_t n, const int32_t *__restrict__ Pptr, const int32_t *__restrict__ Pcol,
                                const double *__restrict__ Pval, const double *__restrict__ uc,
                                double *__restrict__ u, const int *skip) {
    pdl_wait();
    if (skip && *skip) return;
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s[4];
    load4(u + (int64_t)4 * i, s);
    for (int32_t p = Pptr[i]; p < Pptr[i + 1]; ++p) {
        double v[4];
        load4(uc + (int64_t)4 * Pcol[p], v);
        const double w = Pval[p];
#pragma unroll
        for (int c = 0; c < 4; ++c) s[c] = fma(w, v[c], s[c]);
    }
    store4(u + (int64_t)4 * i, s);
}

}  // namespace

// ======================================================================= launchers
void launch_stokes_vals(int N, const double *rho, const double *mu, const double *fx, const double *fy,
                        const double *fz, double mass, const int32_t *ptr, double *val, cudaStream_t s) {
    const int64_t n = (int64_t)N * N * N;
    count_launch();
    k_stokes_vals<<<bblocks(n), kBThreads, 0, s>>>(N, n, rho, mu, fx, fy, fz, mass, ptr, val);
}
void launch_block_norms(int64_t nnz, const double *bv, double *out, cudaStream_t s) {
    count_launch();
    k_block_norms<<<bblocks(nnz, 256), 256, 0, s>>>(nnz, bv, out);
}
void launch_block_gather(int64_t nout, const int32_t *eptr, const int32_t *idx, const double *w, const double *x,
                         double *y, cudaStream_t s) {
    if (nout <= 0) return;
    count_launch();
    k_block_gather<<<bblocks(16 * nout, 256), 256, 0, s>>>(nout, eptr, idx, w, x, y);
}
void launch_block_jacobi(int32_t n, const int32_t *dia, const double *bv, double wj, double *minv, cudaStream_t s) {
    count_launch();
    k_block_jacobi<<<bblocks(n), kBThreads, 0, s>>>(n, dia, bv, wj, minv);
}
void launch_block_to_dense(int32_t n, const int32_t *ptr, const int32_t *col, const double *bv, double *dense,
                           cudaStream_t s) {
    count_launch();
    k_block_to_dense<<<bblocks(n), kBThreads, 0, s>>>(n, ptr, col, bv, dense);
}
void launch_block_smooth0(int32_t n, const double *minv, const double *f, double *u, const int *skip,
                          cudaStream_t s) {
    count_launch();
    launch_pdl(k_block_smooth0, bblocks(n), kBThreads, 0, s, n, minv, f, u, skip);
}
void launch_block_sweep(int32_t n, const int32_t *ptr, const int32_t *col, const double *bv, const double *minv,
                        const double *f, const double *uin, double *uout, const int *skip, cudaStream_t s) {
    count_launch();
    launch_pdl(k_block_sweep, bblocks(n), kBThreads, 0, s, n, ptr, col, bv, minv, f, uin, uout, skip);
}
void launch_block_residual(int32_t n, const int32_t *ptr, const int32_t *col, const double *bv, const double *f,
                           const double *u, double *r, const int *skip, cudaStream_t s) {
    count_launch();
    launch_pdl(k_block_residual, bblocks(n), kBThreads, 0, s, n, ptr, col, bv, f, u, r, skip);
}
void launch_block_restrict(int32_t nc, const int32_t *Rptr, const int32_t *Rcol, const double *Rval, const double *r,
                           double *fc, const int *skip, cudaStream_t s) {
    count_launch();
    launch_pdl(k_block_restrict, bblocks(nc), kBThreads, 0, s, nc, Rptr, Rcol, Rval, r, fc, skip);
}
void launch_block_prolong(int32_t n, const int32_t *Pptr, const int32_t *Pcol, const double *Pval, const double *uc,
                          double *u, const int *skip, cudaStream_t s) {
    count_launch();
    launch_pdl(k_block_prolong, bblocks(n), kBThreads, 0, s, n, Pptr, Pcol, Pval, uc, u, skip);
}

}  // namespace amgpr
