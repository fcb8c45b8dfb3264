// solve_kernels.cu -- per-time-step kernels of partial-reuse AMG
// (arXiv 2108.02054, Alg. 4 body and Alg. 2 inside CG):
//   * numeric Galerkin product A_{l+1} = R (A_l P) over the cached coarse
//     pattern (Sec. 5): a gather through slot indices resolved at setup, an
//     atomic-free segmented reduction; FP64 with one fma per term in the
//     fixed order (A entries, then P entries; R entries, then A*P entries),
//     or FP32 values with double-float (compensated) accumulation;
//   * smoother diagonals (SPAI0 / damped Jacobi), the coarsest dense LU and
//     its explicit inverse;
//   * V-cycle pieces and the device-driven CG iteration.
#include <cfloat>

#include <cooperative_groups.h>

#include "common.cuh"
#include "fdiv.cuh"

namespace amgpr {

namespace {

constexpr int kThreads = 256;

inline int nblocks(int64_t n, int t = kThreads) {
    int64_t b = (n + t - 1) / t;
    return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ bool skipped(const int *skip) { return skip != nullptr && *skip != 0; }

// A compressed column pattern (ColIdx with cidx set) names entry p's column
// as row + off[cidx[p]].  Its offset table goes to shared memory once per
// block; every thread of the block must call this.
__device__ __forceinline__ void stage_col_offsets(const ColIdx &ci, int32_t *s_off) {
    if (!ci.cidx) return;
    for (int t = threadIdx.x; t < ci.noff; t += blockDim.x) s_off[t] = ci.off[t];
    __syncthreads();
}
// the column of entry p of row i, in whichever form the pattern is held
__device__ __forceinline__ int32_t col_at(const ColIdx &ci, const int32_t *s_off, int32_t i, int32_t p) {
    return ci.cidx ? i + s_off[ci.cidx[p]] : (ci.c16 ? i + (int32_t)ci.c16[p] : ci.col[p]);
}

// ------------------------------------------------------------------ Galerkin, FP64
constexpr int kApThreads = 128;
constexpr int kApSlots = 32;
constexpr int kRapWarps = 4;
constexpr int kRapSlots = 1024;

// stage 1: AP[i, :] = sum over k in row i of A (column order), over the
// entries of row k of P (column order), of fma(a_ik, P_kJ, acc)
__global__ void __launch_bounds__(kApThreads)
k_ap_numeric_f64(int32_t n, const int32_t *__restrict__ A_ptr, const int32_t *__restrict__ A_col,
                 const double *__restrict__ A_val, const int32_t *__restrict__ P_ptr,
                 const double *__restrict__ P_val, const int32_t *__restrict__ AP_ptr,
                 const int32_t *__restrict__ t1ptr, const uint16_t *__restrict__ slot1,
                 double *__restrict__ AP_val) {
    __shared__ double acc[kApSlots * kApThreads];
    const int32_t i = blockIdx.x * kApThreads + threadIdx.x;
    if (i >= n) return;
    const int32_t b = AP_ptr[i], L = AP_ptr[i + 1] - b;
    int64_t t = t1ptr[i];
    double *a;
    int stride;
    if (L <= kApSlots) { a = acc + threadIdx.x; stride = kApThreads; }
    else { a = AP_val + b; stride = 1; }
    for (int s = 0; s < L; ++s) a[s * stride] = 0.0;
    for (int32_t p = A_ptr[i]; p < A_ptr[i + 1]; ++p) {
        const int32_t k = A_col[p];
        const double x = A_val[p];
        for (int32_t q = P_ptr[k]; q < P_ptr[k + 1]; ++q) {
            const int s = slot1[t++];
            a[s * stride] = fma(x, P_val[q], a[s * stride]);
        }
    }
    if (L <= kApSlots)
        for (int s = 0; s < L; ++s) AP_val[b + s] = a[s * stride];
}

// ------------------------------------------------------------------ Galerkin, FP32 compensated
// double-float accumulation: (hi, lo) += x*y with the product error from fmaf
// and the addition error from a two-sum (error-free transformations)
__device__ __forceinline__ void df_acc(float &hi, float &lo, float x, float y) {
    const float p = x * y;
    const float pe = fmaf(x, y, -p);
    const float s = hi + p;
    const float bp = s - hi;
    const float se = (hi - (s - bp)) + (p - bp);
    hi = s;
    lo = lo + (se + pe);
}

__global__ void __launch_bounds__(kApThreads)
k_ap_numeric_f32(int32_t n, const int32_t *__restrict__ A_ptr, const int32_t *__restrict__ A_col,
                 const float *__restrict__ A_val, const int32_t *__restrict__ P_ptr,
                 const float *__restrict__ P_val, const int32_t *__restrict__ AP_ptr,
                 const int32_t *__restrict__ t1ptr, const uint16_t *__restrict__ slot1,
                 float *__restrict__ AP_val) {
    __shared__ float acc_hi[kApSlots * kApThreads];
    __shared__ float acc_lo[kApSlots * kApThreads];
    const int32_t i = blockIdx.x * kApThreads + threadIdx.x;
    if (i >= n) return;
    const int32_t b = AP_ptr[i], L = AP_ptr[i + 1] - b;
    int64_t t = t1ptr[i];
    if (L <= kApSlots) {
        float *hi = acc_hi + threadIdx.x, *lo = acc_lo + threadIdx.x;
        for (int s = 0; s < L; ++s) { hi[s * kApThreads] = 0.f; lo[s * kApThreads] = 0.f; }
        for (int32_t p = A_ptr[i]; p < A_ptr[i + 1]; ++p) {
            const int32_t k = A_col[p];
            const float x = A_val[p];
            for (int32_t q = P_ptr[k]; q < P_ptr[k + 1]; ++q) {
                const int s = slot1[t++] * kApThreads;
                df_acc(hi[s], lo[s], x, P_val[q]);
            }
        }
        for (int s = 0; s < L; ++s) AP_val[b + s] = hi[s * kApThreads] + lo[s * kApThreads];
    } else {
        // long rows (coarse levels only): plain FP32 accumulation in place
        for (int s = 0; s < L; ++s) AP_val[b + s] = 0.f;
        for (int32_t p = A_ptr[i]; p < A_ptr[i + 1]; ++p) {
            const int32_t k = A_col[p];
            const float x = A_val[p];
            for (int32_t q = P_ptr[k]; q < P_ptr[k + 1]; ++q) {
                const int s = slot1[t++];
                AP_val[b + s] = fmaf(x, P_val[q], AP_val[b + s]);
            }
        }
    }
}

// Galerkin stage 2, A_c = R (AP): one warp per coarse row I.  The row's terms
// (R entry r in column order, then the entries of row R_col[r] of AP in
// column order) are taken 32 at a time, one per lane; a lane finds its R entry
// by binary search in the staged prefix of AP row lengths.  Lanes whose terms
// hit the same slot apply them in lane order (rank among __match_any_sync
// peers), so every slot still accumulates in the sequential term order: the
// FP64 result is bit-identical to the plain row-by-row product, while the
// loads of 32 terms overlap.  FP32 accumulates in double-float pairs.
constexpr int kRapMaxR = 192;

template <class V>
__device__ __forceinline__ void rap_apply(V *hi, V *lo, bool comp, int s, V x, V y);
template <>
__device__ __forceinline__ void rap_apply<double>(double *hi, double *, bool, int s, double x, double y) {
    hi[s] = fma(x, y, hi[s]);
}
template <>
__device__ __forceinline__ void rap_apply<float>(float *hi, float *lo, bool comp, int s, float x, float y) {
    if (comp) df_acc(hi[s], lo[s], x, y);
    else hi[s] = fmaf(x, y, hi[s]);
}

template <class V>
__global__ void __launch_bounds__(kRapWarps * 32)
k_rap_terms(int32_t nc, const int32_t *__restrict__ R_ptr, const int32_t *__restrict__ R_col,
            const V *__restrict__ R_val, const int32_t *__restrict__ AP_ptr, const V *__restrict__ AP_val,
            const int32_t *__restrict__ Ac_ptr, const int32_t *__restrict__ t2ptr,
            const uint16_t *__restrict__ slot2, V *__restrict__ Ac_val) {
    __shared__ V acc_hi[kRapWarps][kRapSlots];
    __shared__ V acc_lo[kRapWarps][sizeof(V) == 4 ? kRapSlots : 1];
    __shared__ int32_t s_end[kRapWarps][kRapMaxR];
    __shared__ int32_t s_e0[kRapWarps][kRapMaxR];
    __shared__ V s_x[kRapWarps][kRapMaxR];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t I = blockIdx.x * kRapWarps + w;
    if (I >= nc) return;  // warp-uniform
    const int32_t rb = R_ptr[I], nr = R_ptr[I + 1] - rb;
    const int32_t b = Ac_ptr[I], L = Ac_ptr[I + 1] - b;
    const bool in_smem = L <= kRapSlots;
    const bool comp = sizeof(V) == 4 && in_smem;
    V *hi = in_smem ? acc_hi[w] : Ac_val + b;  // long coarse rows accumulate in place
    V *lo = acc_lo[w];
    for (int s = lane; s < L; s += 32) {
        hi[s] = V(0);
        if (comp) lo[s] = V(0);
    }
    __syncwarp();
    const int64_t t0 = t2ptr[I];
    if (nr > kRapMaxR) {
        // long R row: R entries in order, the lanes over one AP row's distinct slots
        int64_t t = t0;
        for (int32_t r = rb; r < rb + nr; ++r) {
            const int32_t i = R_col[r];
            const V x = R_val[r];
            const int32_t e0 = AP_ptr[i], le = AP_ptr[i + 1] - e0;
            for (int32_t e = lane; e < le; e += 32) rap_apply<V>(hi, lo, comp, slot2[t + e], x, AP_val[e0 + e]);
            t += le;
            __syncwarp();
        }
    } else {
        int32_t carry = 0;
        for (int32_t r0 = 0; r0 < nr; r0 += 32) {
            const int32_t r = r0 + lane;
            int32_t len = 0;
            if (r < nr) {
                const int32_t i = R_col[rb + r];
                const int32_t e0 = AP_ptr[i];
                len = AP_ptr[i + 1] - e0;
                s_e0[w][r] = e0;
                s_x[w][r] = R_val[rb + r];
            }
            int32_t inc = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (r < nr) s_end[w][r] = carry + inc;
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        __syncwarp();
        const int32_t nterms = carry;
        for (int32_t base = 0; base < nterms; base += 32) {
            const int32_t t = base + lane;
            const bool valid = t < nterms;
            int slot = 0;
            V x = V(0), y = V(0);
            if (valid) {
                int32_t lo_r = 0, hi_r = nr - 1;  // first r with s_end[r] > t
                while (lo_r < hi_r) {
                    const int32_t mid = (lo_r + hi_r) >> 1;
                    if (s_end[w][mid] > t) hi_r = mid; else lo_r = mid + 1;
                }
                const int32_t start = lo_r ? s_end[w][lo_r - 1] : 0;
                y = AP_val[s_e0[w][lo_r] + (t - start)];
                x = s_x[w][lo_r];
                slot = slot2[t0 + t];
            }
            const unsigned active = __ballot_sync(0xffffffffu, valid);
            int rank = 0;
            if (valid) {
                const unsigned peers = __match_any_sync(active, slot);
                rank = __popc(peers & ((1u << lane) - 1u));
            }
            const int maxrank = (int)__reduce_max_sync(0xffffffffu, (unsigned)rank);
            for (int k = 0; k <= maxrank; ++k) {
                if (valid && rank == k) rap_apply<V>(hi, lo, comp, slot, x, y);
                __syncwarp();
            }
        }
    }
    if (in_smem)
        for (int s = lane; s < L; s += 32) Ac_val[b + s] = comp ? V(hi[s] + lo[s]) : hi[s];
}

// ------------------------------------------------------------------ Galerkin as gather operators
// y[e] = sum over the terms t of entry e, in their sequential order, of
// w[t] * x[idx[t]]: the two stages of the numeric Galerkin product once P and
// R are fixed (w = P_kJ with x = a, then w = R_Ii with x = AP).  FP64: one fma
// per term from 0.0, the same operations as the row-by-row product; FP32:
// double-float accumulation.
template <class V>
__global__ void k_gather_apply(int64_t nout, const int32_t *__restrict__ eptr, const int32_t *__restrict__ idx,
                               const V *__restrict__ w, const V *__restrict__ x, V *__restrict__ y);
template <>
__global__ void k_gather_apply<double>(int64_t nout, const int32_t *__restrict__ eptr,
                                       const int32_t *__restrict__ idx, const double *__restrict__ w,
                                       const double *__restrict__ x, double *__restrict__ y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nout) return;
    double acc = 0.0;
    const int32_t t0 = eptr[e], t1 = eptr[e + 1];
    int32_t t = t0;
    // four terms' loads in flight at once; the fmas keep the term order
    for (; t + 4 <= t1; t += 4) {
        const int32_t i0 = idx[t], i1 = idx[t + 1], i2 = idx[t + 2], i3 = idx[t + 3];
        const double w0 = w[t], w1 = w[t + 1], w2 = w[t + 2], w3 = w[t + 3];
        const double x0 = x[i0], x1 = x[i1], x2 = x[i2], x3 = x[i3];
        acc = fma(w0, x0, acc);
        acc = fma(w1, x1, acc);
        acc = fma(w2, x2, acc);
        acc = fma(w3, x3, acc);
    }
    for (; t < t1; ++t) acc = fma(w[t], x[idx[t]], acc);
    y[e] = acc;
}
template <>
__global__ void k_gather_apply<float>(int64_t nout, const int32_t *__restrict__ eptr,
                                      const int32_t *__restrict__ idx, const float *__restrict__ w,
                                      const float *__restrict__ x, float *__restrict__ y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nout) return;
    float hi = 0.f, lo = 0.f;
    const int32_t t0 = eptr[e], t1 = eptr[e + 1];
    int32_t t = t0;
    for (; t + 4 <= t1; t += 4) {
        const int32_t i0 = idx[t], i1 = idx[t + 1], i2 = idx[t + 2], i3 = idx[t + 3];
        const float w0 = w[t], w1 = w[t + 1], w2 = w[t + 2], w3 = w[t + 3];
        const float x0 = x[i0], x1 = x[i1], x2 = x[i2], x3 = x[i3];
        df_acc(hi, lo, w0, x0);
        df_acc(hi, lo, w1, x1);
        df_acc(hi, lo, w2, x2);
        df_acc(hi, lo, w3, x3);
    }
    for (; t < t1; ++t) df_acc(hi, lo, w[t], x[idx[t]]);
    y[e] = hi + lo;
}

// ------------------------------------------------------------------ smoothers
// SPAI0: m_i = a_ii / sum_j a_ij^2 (fma, column order), 0 for a zero sum;
// damped Jacobi: m_i = w / a_ii.
template <class V>
__global__ void k_smoother(int32_t n, const int32_t *__restrict__ ptr, const V *__restrict__ val,
                           const int32_t *__restrict__ dia, int type, V wj, V *__restrict__ m) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const V aii = val[dia[i]];
    if (type == AMG_SMOOTHER_SPAI0) {
        V s = 0;
        for (int32_t p = ptr[i]; p < ptr[i + 1]; ++p) s = fma(val[p], val[p], s);
        m[i] = s != V(0) ? aii / s : V(0);
    } else {
        m[i] = aii != V(0) ? wj / aii : V(0);
    }
}

// fine level: copy the new values into the hierarchy (optionally an FP32
// copy as well), flag non-finite entries and build the smoother in one kernel
__global__ void k_ingest_fine(int32_t row0, int32_t n, const int32_t *__restrict__ ptr, const double *__restrict__ in,
                              const int32_t *__restrict__ dia, int type, double wj, double *__restrict__ out,
                              float *__restrict__ outf, double *__restrict__ m, float *__restrict__ mf, int *st) {
    // rows row0 .. n - 1 (row0 a multiple of 32); one warp per 32 consecutive
    // rows: their values are one contiguous range, copied, cast and checked
    // with coalesced accesses; then each lane forms its row's smoother from
    // the same values (now in L1/L2) in column order
    const int lane = threadIdx.x & 31;
    const int32_t r0 = row0 + (int32_t)((((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 5);
    if (r0 >= n) return;  // warp-uniform
    const int32_t r1 = min(r0 + 32, n);
    const int32_t p0 = ptr[r0], p1 = ptr[r1];
    // (the finiteness test, the FP32 cast and the division below are done in
    // integer arithmetic with the same results: on this part their FP64
    // instructions bound the kernel)
    bool finite = true;
    for (int32_t p = p0 + lane; p < p1; p += 32) {
        const double v = in[p];
        finite = finite && finite_bits(v);
        if (out) out[p] = v;
        if (outf) outf[p] = f64_to_f32_rn(v);
    }
    if (__any_sync(0xffffffffu, !finite) && lane == 0) atomicOr(st, DEV_ERR_NONFINITE);
    const int32_t i = r0 + lane;
    if (i >= n) return;
    double s = 0.0;
    for (int32_t p = ptr[i]; p < ptr[i + 1]; ++p) {
        const double v = in[p];
        s = fma(v, v, s);
    }
    const double aii = in[dia[i]];
    double mi;
    if (type == AMG_SMOOTHER_SPAI0) mi = s != 0.0 ? div_rn(aii, div_recip(s)) : 0.0;
    else mi = aii != 0.0 ? div_rn(wj, div_recip(aii)) : 0.0;
    if (m) m[i] = mi;
    if (mf) mf[i] = f64_to_f32_rn(mi);
}

__global__ void k_cast_f32(int64_t n, const double *__restrict__ in, float *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// ------------------------------------------------------------------ coarsest level
__global__ void k_csr_to_dense(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                               const double *__restrict__ val, const float *__restrict__ valf,
                               double *__restrict__ dense) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t p = ptr[i]; p < ptr[i + 1]; ++p)
        dense[(int64_t)i * n + col[p]] = val ? val[p] : (double)valf[p];
}

// Pivot candidates compare |a| through its IEEE bit pattern: with the sign
// bit cleared, the unsigned order of the bits is the order of the magnitudes,
// so the search needs no FP64 compares (slow on this part's FP64 pipe).  NaN
// patterns map to 0 and are never chosen.
struct KeyIdx {
    unsigned long long k;
    int i;
};
__device__ __forceinline__ unsigned long long mag_key(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    return b > 0x7ff0000000000000ull ? 0ull : b;
}
__device__ __forceinline__ KeyIdx better(KeyIdx a, KeyIdx b) {
    // larger magnitude wins; equal magnitudes: the lower row index
    if (b.k > a.k || (b.k == a.k && b.i < a.i)) return b;
    return a;
}

// LU with partial pivoting (first entry of largest magnitude), in place,
// row-major; l = a_rk / a_kk, a_rc = fma(-l, a_kc, a_rc); the result (factors
// and pivots) is that of the textbook row-swapping elimination.
// Small matrices (n <= kLuSmemN) are factorised in shared memory by one block
// with a lazy row permutation: rows are not moved during the elimination,
// perm[i] names the physical row at position i, and the factors are written
// out in position order at the end.  Larger ones use the cluster kernel (up to
// kLuClusterN rows) or the global-memory kernel.
constexpr int kLuSmemN = 160;
constexpr int kLuClusterN = 448;   // 8 CTAs x 56 rows x 448 columns fit in 227 KB each
constexpr int kLuThreads = 512;
__global__ void __launch_bounds__(kLuThreads) k_dense_lu_smem(int32_t n, double *__restrict__ g,
                                                              int32_t *__restrict__ piv, int *st) {
    extern __shared__ double a[];
    __shared__ int32_t perm[kLuSmemN];
    __shared__ int s_sing;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nw = kLuThreads / 32;
    const int64_t nn = (int64_t)n * n;
    for (int64_t e = tid; e < nn; e += kLuThreads) a[e] = g[e];
    for (int32_t i = tid; i < n; i += kLuThreads) perm[i] = i;
    __syncthreads();
    int32_t k = 0;
    for (; k < n; ++k) {
        if (warp == 0) {
            // pivot search by one warp: the largest magnitude key, then the
            // lowest position among equal keys (three warp reductions)
            unsigned long long key = 0ull;
            int32_t pos = n;
            for (int32_t i = k + lane; i < n; i += 32) {
                const unsigned long long q = mag_key(a[(int64_t)perm[i] * n + k]);
                if (q > key) { key = q; pos = i; }
            }
            const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
            const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
            const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
            const bool top = hi == mh && lo == ml && pos < n;
            const int32_t bi = (int32_t)__reduce_min_sync(0xffffffffu, top ? (unsigned)pos : (unsigned)n);
            if (lane == 0) {
                // no usable pivot (zero or NaN column): singular, identity pivots from here on
                const int sing = (mh | ml) == 0u || bi < k || bi >= n;
                const int32_t pp = sing ? k : bi;
                s_sing = sing;
                piv[k] = pp;
                const int32_t t = perm[k];
                perm[k] = perm[pp];
                perm[pp] = t;
            }
        }
        __syncthreads();
        if (s_sing) break;
        const int64_t rk = (int64_t)perm[k] * n;
        const double akk = a[rk + k];
        // all multipliers at once (one division latency per step), then the rank-1 update
        for (int32_t i = k + 1 + tid; i < n; i += kLuThreads) {
            const int64_t ri = (int64_t)perm[i] * n;
            a[ri + k] = a[ri + k] / akk;
        }
        __syncthreads();
        for (int32_t i = k + 1 + warp; i < n; i += nw) {
            const int64_t ri = (int64_t)perm[i] * n;
            const double l = a[ri + k];
            for (int32_t c = k + 1 + lane; c < n; c += 32) a[ri + c] = fma(-l, a[rk + c], a[ri + c]);
        }
        __syncthreads();
    }
    if (k < n) {
        if (tid == 0) atomicOr(st, DEV_ERR_SINGULAR);
        for (int32_t r = k + 1 + tid; r < n; r += kLuThreads) piv[r] = r;
    }
    for (int64_t e = tid; e < nn; e += kLuThreads) g[e] = a[(int64_t)perm[e / n] * n + e % n];
}

// Mid-size matrices (kLuSmemN < n <= kLuClusterN) are factorised by one
// thread-block cluster of eight CTAs (eight SMs' FP64 pipes): physical row r
// lives in the shared memory of CTA r % 8.  Each step, every CTA ranks its own
// rows (positions >= k; ties to the lower position), the CTAs read the eight
// candidates from one another's shared memory and all pick the same pivot,
// copy the pivot row from its owner, and update their own rows; two cluster
// barriers per step.  The permutation is kept lazily (perm / pos_of,
// replicated in every CTA), the divisions and fma updates are those of the
// one-block kernel, so factors and pivots are identical to it.  The factors
// are written in position order, and column-major as well for the inverse.
namespace cgr = cooperative_groups;
constexpr int kLuClusterCtas = 8;
constexpr int kLuClusterThreads = 512;
__global__ void __cluster_dims__(kLuClusterCtas, 1, 1) __launch_bounds__(kLuClusterThreads)
k_dense_lu_cluster(int32_t n, double *__restrict__ g, double *__restrict__ gT, int32_t *__restrict__ piv, int *st) {
    cgr::cluster_group cluster = cgr::this_cluster();
    const int rank = (int)cluster.block_rank();
    extern __shared__ double sm_lu[];
    const int32_t nloc = (n + kLuClusterCtas - 1) / kLuClusterCtas;
    double *a = sm_lu;                          // nloc rows of n
    double *prow = a + (int64_t)nloc * n;       // the step's pivot row
    double *lbuf = prow + n;                    // multipliers of this CTA's rows
    int32_t *perm = (int32_t *)(lbuf + nloc);   // position -> physical row
    int32_t *pos_of = perm + n;                 // physical row -> position
    __shared__ KeyIdx cand;
    __shared__ KeyIdx wbest[kLuClusterThreads / 32];
    __shared__ int s_sing;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nw = kLuClusterThreads / 32;
    const int32_t nmine = rank < n ? (n - rank + kLuClusterCtas - 1) / kLuClusterCtas : 0;
    for (int64_t e = tid; e < (int64_t)nmine * n; e += kLuClusterThreads) {
        const int32_t li = (int32_t)(e / n), c = (int32_t)(e % n);
        a[(int64_t)li * n + c] = g[(int64_t)(rank + kLuClusterCtas * li) * n + c];
    }
    for (int32_t i = tid; i < n; i += kLuClusterThreads) {
        perm[i] = i;
        pos_of[i] = i;
    }
    __syncthreads();
    int32_t k = 0;
    for (; k < n; ++k) {
        // this CTA's candidate
        KeyIdx best{0ull, n};
        for (int32_t li = tid; li < nmine; li += kLuClusterThreads) {
            const int32_t q = pos_of[rank + kLuClusterCtas * li];
            if (q >= k) best = better(best, KeyIdx{mag_key(a[(int64_t)li * n + k]), q});
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            KeyIdx other{__shfl_xor_sync(0xffffffffu, best.k, o), __shfl_xor_sync(0xffffffffu, best.i, o)};
            best = better(best, other);
        }
        if (lane == 0) wbest[warp] = best;
        __syncthreads();
        if (warp == 0) {
            KeyIdx bb = lane < nw ? wbest[lane] : KeyIdx{0ull, n};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                KeyIdx other{__shfl_xor_sync(0xffffffffu, bb.k, o), __shfl_xor_sync(0xffffffffu, bb.i, o)};
                bb = better(bb, other);
            }
            if (lane == 0) cand = bb;
        }
        cluster.sync();
        // the pivot: the best of the eight candidates, the same in every CTA
        if (warp == 0) {
            KeyIdx c{0ull, n};
            if (lane < kLuClusterCtas) c = *cluster.map_shared_rank(&cand, lane);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                KeyIdx other{__shfl_xor_sync(0xffffffffu, c.k, o), __shfl_xor_sync(0xffffffffu, c.i, o)};
                c = better(c, other);
            }
            if (lane == 0) {
                const int sing = c.k == 0ull || c.i < k || c.i >= n;
                const int32_t pos = sing ? k : c.i;
                s_sing = sing;
                if (rank == 0) piv[k] = pos;
                const int32_t pk = perm[k], pp = perm[pos];
                perm[k] = pp;
                perm[pos] = pk;
                pos_of[pp] = k;
                pos_of[pk] = pos;
            }
        }
        __syncthreads();
        if (s_sing) break;  // the same decision in every CTA
        const int32_t pr = perm[k];
        const double *src =
            cluster.map_shared_rank(a + (int64_t)(pr / kLuClusterCtas) * n, (unsigned)(pr % kLuClusterCtas));
        for (int32_t c = k + tid; c < n; c += kLuClusterThreads) prow[c] = src[c];
        __syncthreads();
        const double akk = prow[k];
        for (int32_t li = tid; li < nmine; li += kLuClusterThreads)
            if (pos_of[rank + kLuClusterCtas * li] > k) lbuf[li] = a[(int64_t)li * n + k] / akk;
        __syncthreads();
        for (int32_t li = warp; li < nmine; li += nw) {
            if (pos_of[rank + kLuClusterCtas * li] <= k) continue;
            const double l = lbuf[li];
            double *row = a + (int64_t)li * n;
            if (lane == 0) row[k] = l;
            for (int32_t c = k + 1 + lane; c < n; c += 32) row[c] = fma(-l, prow[c], row[c]);
        }
        cluster.sync();
    }
    if (k < n && rank == 0) {
        if (tid == 0) atomicOr(st, DEV_ERR_SINGULAR);
        for (int32_t r = k + 1 + tid; r < n; r += kLuClusterThreads) piv[r] = r;
    }
    for (int64_t e = tid; e < (int64_t)nmine * n; e += kLuClusterThreads) {
        const int32_t li = (int32_t)(e / n), c = (int32_t)(e % n);
        const int64_t q = pos_of[rank + kLuClusterCtas * li];
        const double v = a[(int64_t)li * n + c];
        g[q * n + c] = v;
        if (gT) gT[(int64_t)c * n + q] = v;
    }
    // no CTA leaves while another may still read its shared memory
    cluster.sync();
}

// ---- the coarsest LU for n <= kLuPipeN: a pipelined cluster factorisation
//
// On this part an FP64 instruction holds its SM sub-partition for about 64
// cycles whatever the number of active lanes, an FP64 division takes about
// 565 cycles and a cluster barrier about 400.  So the elimination keeps one
// pivot search, one division and one fma per step on its critical path, does
// the division in integer arithmetic (div_rn: the same IEEE quotient), and
// has no cluster-wide barrier between steps.
//
// Column j belongs to CTA (j / B) % C of a C-CTA cluster (blocks of B
// consecutive columns dealt round-robin), stored column-major in that CTA's
// shared memory, one row per lane of four compute warps; the columns of the
// block being factorised live in registers.  Step k is taken by the owner of
// column k alone (its column is already updated through step k-1): the
// pivot search (each warp's candidate carries the row's remaining block
// values and the reciprocal of its value, so one barrier serves the search),
// the multipliers l_r = a_rk / a_kk, and one message per step: a row of the
// multipliers and a header (pivot position, pivot row, singular flag) that a
// fifth warp copies into every other CTA's slot for step k with one bulk
// copy each; the copy's byte count completes that slot's mbarrier.  Every
// CTA applies the steps to its own columns in order, the next owner's block
// first, so a message's latency is paid once per block of B steps.
//
// Rows never move: every lane tracks the position of its row and the step at
// which the row became a pivot (the lazy form of the row swaps), and writes
// its row at its final position at the end.  Each entry sees the operations
// of the textbook row-swapping elimination in the same order (one division
// per multiplier, then a_rc = fma(-l_r, a_kc, a_rc) step by step), so the
// factors and pivots are identical to it.
//
// Every wait is bounded by a clock budget; on expiry the CTA sets
// DEV_ERR_TIMEOUT, waits no more and goes to the final cluster barrier, which
// every CTA then reaches.
constexpr int kLuPipeN = 128;
constexpr int kLuPipeMinN = 48;  // below: the one-CTA kernel is faster (fewer steps to pipeline)
constexpr int kLuPipeWarps = 4;                           // compute warps, one row per lane
constexpr int kLuPipeThreads = (kLuPipeWarps + 1) * 32;   // and the sender warp
constexpr int kLuPipeC = 8;                               // CTAs of the cluster
constexpr int kLuPipeB = 4;                               // columns per ownership block
constexpr long long kLuPipeWaitClocks = 2000000000ll;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_done(uint32_t bar) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar)
        : "memory");
    return ok != 0;
}
// bounded wait for phase 0 of an mbarrier; false when the budget ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar) {
    if (mbar_done(bar)) return true;
    const long long t0 = clock64();
    while (!mbar_done(bar))
        if (clock64() - t0 > kLuPipeWaitClocks) return false;
    return true;
}
__device__ __forceinline__ void bulk_to_peer(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst),
                 "r"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// barrier of the compute warps only (named barrier 1)
__device__ __forceinline__ void lu_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kLuPipeWarps * 32) : "memory"); }
__device__ __forceinline__ int lu_sync_or(int pred) {
    int r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.s32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"(pred), "n"(kLuPipeWarps * 32)
        : "memory");
    return r;
}

template <int B>
struct PivCand {
    unsigned long long key;
    int32_t pos, row;
    double vals[B];  // the row's values in the block's columns
    DivRecip rc;     // reciprocal of its value in the step's column
};
// header of step k: pivot position, pivot row, singular flag
__device__ __forceinline__ unsigned long long piv_header(int32_t p, int32_t row, bool sing) {
    return (unsigned long long)(uint32_t)p | ((unsigned long long)(uint32_t)row << 16) |
           ((unsigned long long)(sing ? 1u : 0u) << 32);
}

template <int C, int B>
struct LuPipeMap {
    int32_t n, nblk;
    __device__ int32_t owner(int32_t k) const { return (k / B) % C; }
    __device__ int32_t last_col(int32_t q) const {
        if (q >= nblk) return -1;
        const int32_t b = q + C * ((nblk - 1 - q) / C);
        return min(n, (b + 1) * B) - 1;
    }
    __device__ int32_t local(int32_t j) const { return ((j / B) / C) * B + j % B; }
    __device__ int32_t global(int32_t q, int32_t lc) const { return (q + C * (lc / B)) * B + lc % B; }
    __device__ int32_t ncols(int32_t q) const { return q < nblk ? local(last_col(q)) + 1 : 0; }
};

// shared memory: n_even mbarriers, n - 1 message rows of lu_pipe_row(n)
// doubles (multipliers, then the header at n_even), the own columns
__host__ __device__ inline int32_t lu_pipe_even(int32_t n) { return (n + 1) & ~1; }
__host__ __device__ inline int32_t lu_pipe_row(int32_t n) { return lu_pipe_even(n) + 2; }
size_t lu_pipe_smem(int32_t n, int C, int B) {
    const size_t nblk = (size_t)(n + B - 1) / B, per = (nblk + C - 1) / C * B;
    return ((size_t)lu_pipe_even(n) + (size_t)(n > 0 ? n - 1 : 0) * lu_pipe_row(n) + per * n) * 8;
}

template <int C, int B>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kLuPipeThreads)
k_dense_lu_pipe(int32_t n, double *__restrict__ g, double *__restrict__ gT, int32_t *__restrict__ piv, int *st) {
    extern __shared__ __align__(16) unsigned long long sm_pipe[];
    __shared__ PivCand<B> cand_buf[2][kLuPipeWarps];  // by step parity: a fast warp may write step k+1's
    __shared__ int s_quit;
    cgr::cluster_group cluster = cgr::this_cluster();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t rank = (int32_t)cluster.block_rank();
    const LuPipeMap<C, B> M{n, (n + B - 1) / B};
    const int32_t nmine = M.ncols(rank), ne = lu_pipe_even(n), row = lu_pipe_row(n);
    unsigned long long *bar = sm_pipe;                       // one mbarrier per step
    double *msg = (double *)(sm_pipe + ne);                  // message rows, [step][row]
    double *col = msg + (size_t)(n > 0 ? n - 1 : 0) * row;   // own columns, [local column][row]
    const uint32_t off_msg = 8u * (uint32_t)ne, row_bytes = 8u * (uint32_t)row;

    // setup: barriers (own steps: the compute warps arrive; others: one
    // arrival with the message's byte count), the own columns
    for (int32_t s = tid; s < n; s += kLuPipeThreads)
        mbar_init(smem_addr(bar + s), M.owner(s) == rank ? (uint32_t)kLuPipeWarps : 1u);
    if (tid == 0) s_quit = 0;
    __syncthreads();
    if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int32_t s = tid; s < n - 1; s += kLuPipeThreads)
        if (M.owner(s) != rank) mbar_arrive_expect(smem_addr(bar + s), row_bytes);
    for (int32_t e = tid; e < nmine * n; e += kLuPipeThreads) {
        const int32_t lc = e / n, r = e % n;
        col[e] = g[(int64_t)r * n + M.global(rank, lc)];
    }
    cluster.sync();

    if (warp == kLuPipeWarps) {
        // the sender: each own step's message row to every other CTA
        const uint32_t base = smem_addr(sm_pipe);
        bool stop = false;
        for (int32_t bk = rank; bk < M.nblk && !stop; bk += C)
            for (int32_t k = bk * B; k < min(n - 1, bk * B + B) && !stop; ++k) {
                const uint32_t b = smem_addr(bar + k);
                bool ready = mbar_done(b);
                const long long t0 = clock64();
                while (!ready) {
                    if (*(volatile int *)&s_quit) {
                        __threadfence_block();
                        ready = mbar_done(b);
                        if (!ready) stop = true;
                        break;
                    }
                    if (clock64() - t0 > kLuPipeWaitClocks) {
                        if (lane == 0) atomicOr(st, DEV_ERR_TIMEOUT);
                        stop = true;
                        break;
                    }
                    ready = mbar_done(b);
                }
                if (!ready) break;
                if (lane == 0) {
#pragma unroll 1
                    for (int q = 0; q < C; ++q)
                        if (q != rank) {
                            const uint32_t pb = peer_addr(base, (uint32_t)q);
                            bulk_to_peer(pb + off_msg + row_bytes * (uint32_t)k, smem_addr(msg + (size_t)k * row),
                                         row_bytes, pb + 8u * (uint32_t)k);
                        }
                }
                const unsigned long long h = (unsigned long long)__double_as_longlong(msg[(size_t)k * row + ne]);
                if ((h >> 32) & 1ull) stop = true;
            }
    } else {
        const int32_t r = tid;
        const bool valid = r < n;
        int32_t pos = r, pstep = n;  // position of this lane's row; step at which it became a pivot
        bool abort = false;
        int32_t kstop = n;  // step at which the elimination met a zero column

        // read the header of a received step: wait, then update the row bookkeeping
        auto consume = [&](int32_t s) -> bool {
            const int late = mbar_wait(smem_addr(bar + s)) ? 0 : 1;
            if (lu_sync_or(late)) {
                if (tid == 0) atomicOr(st, DEV_ERR_TIMEOUT);
                abort = true;
                return false;
            }
            const unsigned long long h = (unsigned long long)__double_as_longlong(msg[(size_t)s * row + ne]);
            if ((h >> 32) & 1ull) {
                kstop = s;
                return false;
            }
            const int32_t p = (int32_t)(h & 0xffffu), pr = (int32_t)((h >> 16) & 0xffffu);
            if (r == pr) { pos = s; pstep = s; }
            else if (pos == s) pos = p;
            return true;
        };
        // apply step s to the local columns [lo, hi) in shared memory
        auto apply = [&](int32_t s, int32_t lo, int32_t hi) {
            if (lo >= hi) return;
            const bool act = valid && pstep > s;
            if (!__any_sync(0xffffffffu, act)) return;
            const double *m = msg + (size_t)s * row;
            const int32_t pr = (int32_t)(((unsigned long long)__double_as_longlong(m[ne]) >> 16) & 0xffffu);
            const double l = act ? m[r] : 0.0;
            int32_t lc = lo;
            for (; lc + 4 <= hi; lc += 4) {
                double u[4], x[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    u[q] = col[(size_t)(lc + q) * n + pr];
                    x[q] = act ? col[(size_t)(lc + q) * n + r] : 0.0;
                }
                if (act)
#pragma unroll
                    for (int q = 0; q < 4; ++q) col[(size_t)(lc + q) * n + r] = fma(-l, u[q], x[q]);
            }
            for (; lc < hi; ++lc) {
                const double u = col[(size_t)lc * n + pr];
                if (act) col[(size_t)lc * n + r] = fma(-l, u, col[(size_t)lc * n + r]);
            }
        };

        int32_t s_all = 0;  // steps applied to every own column beyond the current block
        for (int32_t bk = rank; bk < M.nblk && kstop == n && !abort; bk += C) {
            const int32_t k0 = bk * B, k1 = min(n, k0 + B), nb = k1 - k0;
            const int32_t lb = M.local(k0), lb1 = lb + nb;  // the block's local columns
            // steps of the other CTAs since this CTA's previous block, the
            // block's columns first; the last one (which the block waits for)
            // on the block's columns only, in registers
            bool deferred = false;
            for (int32_t s = s_all; s + 1 < k0; ++s) {
                if (!consume(s)) break;
                apply(s, lb, nmine);  // the block's columns come first
            }
            if (kstop != n || abort) break;
            double vb[B];
            bool have_last = false;
            if (k0 > s_all && k0 >= 1) {
                if (!consume(k0 - 1)) break;
                have_last = true;
                deferred = true;
            }
#pragma unroll
            for (int t = 0; t < B; ++t) vb[t] = valid && t < nb ? col[(size_t)(lb + t) * n + r] : 0.0;
            if (have_last) {
                const double *m = msg + (size_t)(k0 - 1) * row;
                const int32_t pr = (int32_t)(((unsigned long long)__double_as_longlong(m[ne]) >> 16) & 0xffffu);
                const bool act = valid && pstep > k0 - 1;
                const double l = act ? m[r] : 0.0;
#pragma unroll
                for (int t = 0; t < B; ++t)
                    if (t < nb) {
                        const double u = col[(size_t)(lb + t) * n + pr];
                        if (act) vb[t] = fma(-l, u, vb[t]);
                    }
            }
            // the block's steps
            DivRecip rc = div_recip(vb[0]);  // reciprocal of this lane's value in the step's column
            int32_t pk[B];  // the block's pivots, stored at the end of the block
#pragma unroll
            for (int t = 0; t < B; ++t) {
                if (t >= nb) break;
                const int32_t k = k0 + t;
                const double v = vb[t];
                const bool cand_ok = valid && pstep >= k;
                const unsigned long long key = cand_ok ? mag_key(v) : 0ull;
                const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
                const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
                const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
                const bool top = cand_ok && hi == mh && lo == ml;
                const unsigned bp = __reduce_min_sync(0xffffffffu, top ? (unsigned)pos : 0xffffffffu);
                const unsigned wmask = __ballot_sync(0xffffffffu, top && (unsigned)pos == bp);
                PivCand<B> *cand = cand_buf[k & 1];
                if (wmask == 0u) {
                    if (lane == 0) {
                        cand[warp].key = 0ull;
                        cand[warp].pos = n;
                        cand[warp].row = -1;
                    }
                } else if (lane == __ffs(wmask) - 1) {
                    PivCand<B> &c = cand[warp];
                    c.key = key;
                    c.pos = pos;
                    c.row = r;
#pragma unroll
                    for (int q = 0; q < B; ++q) c.vals[q] = vb[q];
                    c.rc = rc;
                }
                lu_sync();
                int bw = 0;
                {
                    unsigned long long bk_ = cand[0].key;
                    int32_t bpos = cand[0].pos;
#pragma unroll
                    for (int w = 1; w < kLuPipeWarps; ++w) {
                        const unsigned long long kw = cand[w].key;
                        const int32_t pw = cand[w].pos;
                        if (kw > bk_ || (kw == bk_ && pw < bpos)) { bk_ = kw; bpos = pw; bw = w; }
                    }
                }
                const PivCand<B> &best = cand[bw];
                const int32_t brow = best.row, bpos = best.pos;
                const bool sing = best.key == 0ull || brow < 0;
                double *m = msg + (size_t)k * row;
                if (sing) {
                    // the receivers see the flag in the header; no multipliers
                    // follow (the last step has no message row)
                    kstop = k;
                    if (tid == 0) {
                        if (k < n - 1) m[ne] = __longlong_as_double((long long)piv_header(k, 0, true));
                        atomicOr(st, DEV_ERR_SINGULAR);
                        for (int32_t q = k; q < n; ++q) piv[q] = q;
                    }
                    if (k < n - 1) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(smem_addr(bar + k));
                    }
                    break;
                }
                if (r == brow) { pos = k; pstep = k; }
                else if (pos == k) pos = bpos;
                const bool act = valid && pstep > k;
                double l = 0.0;
                {
                    const DivRecip brc = best.rc;
                    if (act) l = div_rn(v, brc);
                }
                double u[B];
#pragma unroll
                for (int q = 0; q < B; ++q) u[q] = best.vals[q];
                // the block's next column first: the next step waits for it
                if (t + 1 < nb) {
                    if (act) vb[t + 1] = fma(-l, u[t + 1], vb[t + 1]);
                    rc = div_recip(vb[t + 1]);
                }
                if (act) {
                    vb[t] = l;
                    if (k < n - 1) m[r] = l;
                }
                pk[t] = bpos;
                if (tid == 0 && k < n - 1) m[ne] = __longlong_as_double((long long)piv_header(bpos, brow, false));
                if (k < n - 1) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_addr(bar + k));
                }
#pragma unroll
                for (int q = 0; q < B; ++q)
                    if (q > t + 1 && q < nb && act) vb[q] = fma(-l, u[q], vb[q]);
            }
            // the block's pivots, then the block back to shared memory, then
            // this CTA's later columns: the deferred step and the block's
            // steps (up to a zero column)
            if (tid == 0)
#pragma unroll
                for (int t = 0; t < B; ++t)
                    if (t < nb && k0 + t < kstop) piv[k0 + t] = pk[t];
            if (valid)
#pragma unroll
                for (int t = 0; t < B; ++t)
                    if (t < nb) col[(size_t)(lb + t) * n + r] = vb[t];
            const int32_t kend = kstop != n ? kstop : k1;
            lu_sync();
            for (int32_t s = deferred ? k0 - 1 : k0; s < kend; ++s) {
                apply(s, lb1, nmine);
                lu_sync();
            }
            s_all = k1;
        }
        // the headers after this CTA's last block (final positions)
        if (kstop == n && !abort)
            for (int32_t s = s_all; s < n - 1; ++s)
                if (!consume(s)) break;
        if (!abort && valid)
            for (int32_t lc = 0; lc < nmine; ++lc) {
                const int32_t j = M.global(rank, lc);
                const double v = col[(size_t)lc * n + r];
                g[(int64_t)pos * n + j] = v;
                if (gT) gT[(int64_t)j * n + pos] = v;
            }
        // every arrival is made: let the sender stop waiting
        lu_sync();
        if (tid == 0) {
            __threadfence_block();
            *(volatile int *)&s_quit = 1;
        }
    }
    // no CTA leaves while a message to or from it may be in flight
    cluster.sync();
}

__global__ void __launch_bounds__(1024) k_dense_lu(int32_t n, double *__restrict__ a, int32_t *__restrict__ piv,
                                                   int *st) {
    __shared__ KeyIdx wbest[32];
    __shared__ int s_p, s_sing;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int32_t k = 0; k < n; ++k) {
        KeyIdx best{0ull, n};
        for (int32_t r = k + tid; r < n; r += blockDim.x) best = better(best, KeyIdx{mag_key(a[(int64_t)r * n + k]), r});
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            KeyIdx other{__shfl_xor_sync(0xffffffffu, best.k, o), __shfl_xor_sync(0xffffffffu, best.i, o)};
            best = better(best, other);
        }
        if (lane == 0) wbest[warp] = best;
        __syncthreads();
        if (tid == 0) {
            KeyIdx bb = wbest[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) bb = better(bb, wbest[w]);
            s_sing = bb.k == 0ull || bb.i < k || bb.i >= n;
            s_p = s_sing ? k : bb.i;
            piv[k] = s_p;
        }
        __syncthreads();
        if (s_sing) {
            if (tid == 0) atomicOr(st, DEV_ERR_SINGULAR);
            for (int32_t r = k + 1 + tid; r < n; r += blockDim.x) piv[r] = r;
            break;
        }
        const int32_t p = s_p;
        if (p != k)
            for (int32_t c = tid; c < n; c += blockDim.x) {
                double t = a[(int64_t)k * n + c];
                a[(int64_t)k * n + c] = a[(int64_t)p * n + c];
                a[(int64_t)p * n + c] = t;
            }
        __syncthreads();
        const double akk = a[(int64_t)k * n + k];
        for (int32_t r = k + 1 + tid; r < n; r += blockDim.x) a[(int64_t)r * n + k] = a[(int64_t)r * n + k] / akk;
        __syncthreads();
        for (int32_t r = k + 1 + warp; r < n; r += (int32_t)(blockDim.x >> 5)) {
            const double l = a[(int64_t)r * n + k];
            for (int32_t c = k + 1 + lane; c < n; c += 32)
                a[(int64_t)r * n + c] = fma(-l, a[(int64_t)k * n + c], a[(int64_t)r * n + c]);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// explicit inverse from the LU factors: one warp per column j of A^-1, in
// column (axpy) form so that no step needs a reduction; the factors, the
// pivots, the reciprocals of U's diagonal and each warp's column are staged
// in shared memory when they fit (the reciprocals keep an FP64 division off
// every back-substitution step)
constexpr int kInvWarps = 4;
__global__ void __launch_bounds__(kInvWarps * 32)
k_lu_inverse(int32_t n, const double *__restrict__ lu_g, const int32_t *__restrict__ piv, double *__restrict__ inv) {
    extern __shared__ double sm_inv[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool staged = n <= kLuSmemN;
    const int64_t nn = (int64_t)n * n;
    const double *lu = lu_g;
    const int32_t *pv = piv;
    const double *rd = nullptr;
    if (staged) {
        for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) sm_inv[e] = lu_g[e];
        double *srd = sm_inv + nn + (int64_t)kInvWarps * n;
        for (int32_t e = threadIdx.x; e < n; e += blockDim.x) srd[e] = 1.0 / lu_g[(int64_t)e * n + e];
        int32_t *spv = (int32_t *)(srd + n);
        for (int32_t e = threadIdx.x; e < n; e += blockDim.x) spv[e] = piv[e];
        lu = sm_inv;
        pv = spv;
        rd = srd;
    }
    __syncthreads();
    const int32_t j = blockIdx.x * kInvWarps + w;
    if (j >= n) return;  // warp-uniform; no block barrier follows
    double *x;
    int64_t xs;
    if (staged) { x = sm_inv + nn + (int64_t)w * n; xs = 1; }
    else { x = inv + j; xs = n; }
    // P e_j is the unit vector at the position that the row swaps move j to
    int32_t pos = j;
    for (int32_t k = 0; k < n; ++k) {
        const int32_t p = pv[k];
        if (p < 0 || p >= n || p == k) continue;
        if (pos == k) pos = p;
        else if (pos == p) pos = k;
    }
    for (int32_t r = lane; r < n; r += 32) x[r * xs] = (r == pos) ? 1.0 : 0.0;
    __syncwarp();
    // L y = P e_j (unit lower triangular); entries before pos stay zero
    for (int32_t k = pos; k < n - 1; ++k) {
        const double xk = x[k * xs];
        for (int32_t r = k + 1 + lane; r < n; r += 32) x[r * xs] = fma(-lu[(int64_t)r * n + k], xk, x[r * xs]);
        __syncwarp();
    }
    // U x = y
    for (int32_t k = n - 1; k >= 0; --k) {
        if (lane == 0) x[k * xs] = rd ? x[k * xs] * rd[k] : x[k * xs] / lu[(int64_t)k * n + k];
        __syncwarp();
        const double xk = x[k * xs];
        for (int32_t r = lane; r < k; r += 32) x[r * xs] = fma(-lu[(int64_t)r * n + k], xk, x[r * xs]);
        __syncwarp();
    }
    if (staged)
        for (int32_t r = lane; r < n; r += 32) inv[(int64_t)r * n + j] = x[r];
}

// explicit inverse from the LU factors (n <= kLuSmemN): one block per column
// j of A^-1 with one row per thread (so each substitution step costs one fma
// and one block barrier, not a warp's serial chunks), the factors staged in
// shared memory.  The arithmetic per entry is that of k_lu_inverse: L y =
// P e_j, then U x = y with x_k = y_k * (1 / u_kk), each in step order.
__global__ void __launch_bounds__((kLuSmemN + 31) / 32 * 32)
k_lu_inverse_rows(int32_t n, const double *__restrict__ lu_g, const int32_t *__restrict__ piv,
                  double *__restrict__ inv) {
    extern __shared__ __align__(16) double sm_iv[];
    double *lu = sm_iv;                       // n x n, row-major
    double *xs = lu + (int64_t)n * n;          // x_k as each step finalises it
    int32_t *pv = (int32_t *)(xs + n);         // the pivots
    const int32_t j = blockIdx.x, r = threadIdx.x;
    const int64_t nn = (int64_t)n * n;
    // the factors by 16-byte asynchronous copies, all in flight at once; an
    // odd tail element (or an unaligned source) by plain copies
    if (((uintptr_t)lu_g & 15u) == 0u) {
        for (int64_t e = 2 * (int64_t)threadIdx.x; e + 1 < nn; e += 2 * (int64_t)blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(lu + e)), "l"(lu_g + e)
                         : "memory");
        if ((nn & 1) && threadIdx.x == 0) lu[nn - 1] = lu_g[nn - 1];
    } else {
        for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) lu[e] = lu_g[e];
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    const bool valid = r < n;
    if (valid) pv[r] = piv[r];
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    const double rd = valid ? 1.0 / lu_g[(int64_t)r * n + r] : 0.0;
    __syncthreads();
    // P e_j is the unit vector at the position that the row swaps move j to
    int32_t pos = j;
    for (int32_t k = 0; k < n; ++k) {
        const int32_t p = pv[k];
        if (p < 0 || p >= n || p == k) continue;
        if (pos == k) pos = p;
        else if (pos == p) pos = k;
    }
    double x = valid && r == pos ? 1.0 : 0.0;
    // L y = P e_j (unit lower triangular); entries before pos stay zero
    for (int32_t k = pos; k < n - 1; ++k) {
        if (r == k) xs[k] = x;
        __syncthreads();
        if (valid && r > k) x = fma(-lu[(int64_t)r * n + k], xs[k], x);
    }
    // U x = y
    for (int32_t k = n - 1; k >= 0; --k) {
        if (r == k) {
            x = x * rd;
            xs[k] = x;
        }
        __syncthreads();
        if (valid && r < k) x = fma(-lu[(int64_t)r * n + k], xs[k], x);
    }
    if (valid) inv[(int64_t)r * n + j] = x;
}

// explicit inverse from column-major factors (n > kLuSmemN): the factors stay
// in global memory (L2) and every step's loads are contiguous across lanes;
// the pivots, the reciprocals of U's diagonal and each warp's column live in
// shared memory
__global__ void __launch_bounds__(kInvWarps * 32)
k_lu_inverse_t(int32_t n, const double *__restrict__ luT, const int32_t *__restrict__ piv, double *__restrict__ inv) {
    extern __shared__ double sm_it[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double *xs = sm_it;                                   // kInvWarps columns
    double *rd = xs + (int64_t)kInvWarps * n;             // 1 / u_kk
    int32_t *pv = (int32_t *)(rd + n);
    for (int32_t e = threadIdx.x; e < n; e += blockDim.x) {
        rd[e] = 1.0 / luT[(int64_t)e * n + e];
        pv[e] = piv[e];
    }
    __syncthreads();
    const int32_t j = blockIdx.x * kInvWarps + w;
    if (j >= n) return;  // warp-uniform; no block barrier follows
    double *x = xs + (int64_t)w * n;
    int32_t pos = j;
    for (int32_t k = 0; k < n; ++k) {
        const int32_t p = pv[k];
        if (p < 0 || p >= n || p == k) continue;
        if (pos == k) pos = p;
        else if (pos == p) pos = k;
    }
    for (int32_t r = lane; r < n; r += 32) x[r] = (r == pos) ? 1.0 : 0.0;
    __syncwarp();
    for (int32_t k = pos; k < n - 1; ++k) {
        const double xk = x[k];
        const double *colk = luT + (int64_t)k * n;
        for (int32_t r = k + 1 + lane; r < n; r += 32) x[r] = fma(-colk[r], xk, x[r]);
        __syncwarp();
    }
    for (int32_t k = n - 1; k >= 0; --k) {
        if (lane == 0) x[k] = x[k] * rd[k];
        __syncwarp();
        const double xk = x[k];
        const double *colk = luT + (int64_t)k * n;
        for (int32_t r = lane; r < k; r += 32) x[r] = fma(-colk[r], xk, x[r]);
        __syncwarp();
    }
    for (int32_t r = lane; r < n; r += 32) inv[(int64_t)r * n + j] = x[r];
}

// ---- two-byte column offsets (built once per pattern)
__device__ __forceinline__ int32_t delta16_base(int32_t i, float ratio) {
    return ratio == 0.0f ? i : __float2int_rz((float)i * ratio);
}
__global__ void k_col_delta16(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                              float ratio, int16_t *__restrict__ c16, int *flag) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t b = delta16_base(i, ratio);
    bool wide = false;
    for (int32_t p = ptr[i]; p < ptr[i + 1]; ++p) {
        const int32_t d = col[p] - b;
        wide |= d < -32768 || d > 32767;
        c16[p] = (int16_t)d;
    }
    if (wide) atomicOr(flag, 1);
}

// ---- compressed columns of a pattern (built once per pattern)
// The distinct offsets column - row go into an open-addressed table; the
// lanes of a warp that share an offset insert it once (match), and a key is
// probed before any compare-and-swap, so almost every entry costs one read.
// Empty slots hold kColOffsetEmpty (the host fills the table with bytes 0x80;
// no offset of a pattern with fewer than 2^30 rows equals it).  *count counts
// the distinct keys; past kMaxColOffsets the pattern stays uncompressed and
// inserting stops.
__global__ void k_col_offsets_collect(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                      int32_t *table, int *count) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < n;
    const int32_t b = active ? ptr[i] : 0, len = active ? ptr[i + 1] - b : 0;
    const int32_t lmax = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)len);
    for (int32_t k = 0; k < lmax; ++k) {
        const bool has = k < len;
        const int32_t d = has ? col[b + k] - i : 0;
        const unsigned grp = __match_any_sync(0xffffffffu, has ? d : kColOffsetEmpty);
        const bool leader = has && (__ffs(grp) - 1) == (int)(threadIdx.x & 31);
        if (leader && *(volatile int *)count <= kMaxColOffsets) {
            unsigned h = ((unsigned)d * 2654435761u) & (kColOffsetSlots - 1);
            for (int probe = 0; probe < kColOffsetSlots; ++probe) {
                const int32_t cur = ((volatile int32_t *)table)[h];
                if (cur == d) break;
                if (cur == kColOffsetEmpty) {
                    const int32_t old = atomicCAS(table + h, kColOffsetEmpty, d);
                    if (old == kColOffsetEmpty) {
                        atomicAdd(count, 1);
                        break;
                    }
                    if (old == d) break;
                }
                h = (h + 1) & (kColOffsetSlots - 1);
            }
        }
    }
}

// cidx[p] = position of column - row in the sorted table off (binary search
// in shared memory); an offset missing from the table flags the status word
__global__ void k_col_offsets_encode(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                     const int32_t *__restrict__ off, int noff, uint8_t *__restrict__ cidx, int *st) {
    __shared__ int32_t s_off[kMaxColOffsets];
    for (int t = threadIdx.x; t < noff; t += blockDim.x) s_off[t] = off[t];
    __syncthreads();
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t p = ptr[i]; p < ptr[i + 1]; ++p) {
        const int32_t d = col[p] - i;
        int lo = 0, hi = noff - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_off[mid] < d) lo = mid + 1;
            else hi = mid;
        }
        if (noff == 0 || s_off[lo] != d) {
            atomicOr(st, DEV_ERR_STATE);
            lo = 0;
        }
        cidx[p] = (uint8_t)lo;
    }
}

// u = A_L^-1 f, one warp per row
template <class TF, class TO>
__global__ void k_coarse_solve(int32_t n, const double *__restrict__ inv, const TF *__restrict__ f,
                               TO *__restrict__ u, const int *skip) {
    pdl_wait();
    if (skipped(skip)) return;
    const int lane = threadIdx.x & 31;
    const int32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n) return;
    double s = 0.0;
    for (int32_t c = lane; c < n; c += 32) s = fma(inv[(int64_t)r * n + c], (double)f[c], s);
    s = warp_sum(s);
    if (lane == 0) u[r] = (TO)s;
}

// ------------------------------------------------------------------ V-cycle pieces
// Every matrix-vector piece takes LPR lanes per row (a power of two <= 32,
// chosen per level from the row length and count): the lanes stride over the
// row and combine with xor shuffles.  LPR = 1 is the plain sequential row sum.
template <int LPR, class V>
__device__ __forceinline__ V group_sum(V s) {
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// zero-guess pre-smoothing fused with the residual: u = m o f, r = f - A u
template <class V, class TF, int LPR>
__global__ void k_smooth0_residual(int32_t n, const int32_t *__restrict__ ptr, ColIdx ci,
                                   const V *__restrict__ val, const V *__restrict__ m, const TF *__restrict__ f,
                                   V *__restrict__ u, V *__restrict__ r, const int *skip) {
    __shared__ int32_t s_off[kMaxColOffsets];
    pdl_wait();
    if (skipped(skip)) return;
    stage_col_offsets(ci, s_off);
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(gt / LPR);
    const int sub = (int)(gt % LPR);
    V s = 0;
    if (i < n)
        for (int32_t p = ptr[i] + sub; p < ptr[i + 1]; p += LPR) {
            const int32_t j = col_at(ci, s_off, i, p);
            s = fma(val[p], m[j] * (V)f[j], s);
        }
    s = group_sum<LPR>(s);
    if (i < n && sub == 0) {
        const V fi = (V)f[i];
        u[i] = m[i] * fi;
        r[i] = fi - s;
    }
}

// u_out = u_in + m o (f - A u_in)
template <class V, class TF, class TO, int LPR>
__global__ void k_smooth_sweep(int32_t n, const int32_t *__restrict__ ptr, ColIdx ci,
                               const V *__restrict__ val, const V *__restrict__ m, const TF *__restrict__ f,
                               const V *__restrict__ u_in, TO *__restrict__ u_out, const int *skip) {
    __shared__ int32_t s_off[kMaxColOffsets];
    pdl_wait();
    if (skipped(skip)) return;
    stage_col_offsets(ci, s_off);
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(gt / LPR);
    const int sub = (int)(gt % LPR);
    V s = 0;
    if (i < n)
        for (int32_t p = ptr[i] + sub; p < ptr[i + 1]; p += LPR)
            s = fma(val[p], u_in[col_at(ci, s_off, i, p)], s);
    s = group_sum<LPR>(s);
    if (i < n && sub == 0) u_out[i] = (TO)fma(m[i], (V)f[i] - s, u_in[i]);
}

// the V-cycle's last finest-level sweep fused with the CG product r.z:
// z = u_in + m o (r - A u_in) and a per-block partial of r.z (block_sum order)
__device__ double block_sum(double v);
__device__ bool cg_reduce(double d, double *partial, unsigned *counter, double *total);
template <class V, int LPR>
__global__ void k_smooth_sweep_dot(int32_t n, const int32_t *__restrict__ ptr, ColIdx ci,
                                   const V *__restrict__ val, const V *__restrict__ m, const double *__restrict__ f,
                                   const V *__restrict__ u_in, double *__restrict__ z, double *__restrict__ partial,
                                   CgState *cg, const int *skip) {
    __shared__ int32_t s_off[kMaxColOffsets];
    pdl_wait();
    if (skipped(skip)) return;
    stage_col_offsets(ci, s_off);
    const int64_t total = (int64_t)n * LPR;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double d = 0.0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += stride) {
        const int64_t gt = base + threadIdx.x;
        const int32_t i = (int32_t)(gt / LPR);
        const int sub = (int)(gt % LPR);
        V s = 0;
        if (gt < total)
            for (int32_t p = ptr[i] + sub; p < ptr[i + 1]; p += LPR)
                s = fma(val[p], u_in[col_at(ci, s_off, i, p)], s);
        s = group_sum<LPR>(s);
        if (gt < total && sub == 0) {
            const double fi = f[i];
            const double zi = (double)fma(m[i], (V)fi - s, u_in[i]);
            z[i] = zi;
            d = fma(fi, zi, d);
        }
    }
    // the last block stores the new r.z in the CG state
    double rz = 0.0;
    if (cg_reduce(d, partial, &cg->ctr[CG_CTR_RZ], &rz) && threadIdx.x == 0) cg->rz_next = rz;
}

template <class V, class TF, int LPR>
__global__ void k_residual(int32_t n, const int32_t *__restrict__ ptr, ColIdx ci,
                           const V *__restrict__ val, const TF *__restrict__ f, const V *__restrict__ u,
                           V *__restrict__ r, const int *skip) {
    __shared__ int32_t s_off[kMaxColOffsets];
    pdl_wait();
    if (skipped(skip)) return;
    stage_col_offsets(ci, s_off);
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(gt / LPR);
    const int sub = (int)(gt % LPR);
    V s = 0;
    if (i < n)
        for (int32_t p = ptr[i] + sub; p < ptr[i + 1]; p += LPR)
            s = fma(val[p], u[col_at(ci, s_off, i, p)], s);
    s = group_sum<LPR>(s);
    if (i < n && sub == 0) r[i] = (V)f[i] - s;
}

// f_c = R r (R = P^T stored explicitly, rows sorted): a gather, no atomics
template <class V, int LPR>
__global__ void k_restrict(int32_t nc, const int32_t *__restrict__ R_ptr, const int32_t *__restrict__ R_col,
                           const V *__restrict__ R_val, const V *__restrict__ r, V *__restrict__ fc,
                           const V *__restrict__ mc, V *__restrict__ uc, const int *skip) {
    pdl_wait();
    if (skipped(skip)) return;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t I = (int32_t)(gt / LPR);
    const int sub = (int)(gt % LPR);
    V s = 0;
    if (I < nc)
        for (int32_t p = R_ptr[I] + sub; p < R_ptr[I + 1]; p += LPR) s = fma(R_val[p], r[R_col[p]], s);
    s = group_sum<LPR>(s);
    if (I < nc && sub == 0) {
        fc[I] = s;
        // the coarse level's first smoothing step from zero, u0 = m o f
        if (uc) uc[I] = mc[I] * s;
    }
}

// u += P u_c (P's columns as int32, or as two-byte offsets from
// (int)(row * ratio) when they fit)
template <class V>
__global__ void k_prolong(int32_t n, const int32_t *__restrict__ P_ptr, const int32_t *__restrict__ P_col,
                          const int16_t *__restrict__ P_c16, float ratio, const V *__restrict__ P_val,
                          const V *__restrict__ uc, V *__restrict__ u, const int *skip) {
    pdl_wait();
    if (skipped(skip)) return;
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V s = u[i];
    if (P_c16) {
        const int32_t b = delta16_base(i, ratio);
        for (int32_t p = P_ptr[i]; p < P_ptr[i + 1]; ++p) s = fma(P_val[p], uc[b + (int32_t)P_c16[p]], s);
    } else {
        for (int32_t p = P_ptr[i]; p < P_ptr[i + 1]; ++p) s = fma(P_val[p], uc[P_col[p]], s);
    }
    u[i] = s;
}

template <class TI, class TO>
__global__ void k_copy_cast(int64_t n, const TI *__restrict__ in, TO *__restrict__ out, const int *skip) {
    pdl_wait();
    if (skipped(skip)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (TO)in[i];
}

// ------------------------------------------------------------------ CG (FP64)
// Each reduction writes one partial per block; the block that finishes last
// (a fenced atomic counter, reset by that block) sums the partials in index
// order and takes the iteration's scalar step itself, so no separate
// single-block kernel is needed and the sums stay deterministic.
// 512 threads a block at every size (256 below kCgLargeN measured 1% slower
// per CG iteration at 64^3: 16 warps per SM hid less latency than 32)
constexpr int kCgThreads = 512;
constexpr int kCgMaxBlocks = 152 * 4;  // long vectors: four blocks of 512 per SM
constexpr int64_t kCgLargeN = (int64_t)152 * 8 * 256 * 4;
inline int cg_threads(int64_t) { return kCgThreads; }

// deterministic block sum (fixed lane / warp order)
__device__ double block_sum(double v) {
    __shared__ double ws[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

// true in every thread of the block that is the last of the grid to get here
__device__ bool cg_last_block(unsigned *counter) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return s_last != 0;
}

// the last block's sum of all partials, in index order (valid in thread 0)
__device__ double cg_sum_partials(const double *partial, int nblk) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += __ldcg(partial + b);
    return block_sum(s);
}

// publish this block's partial; the last block returns the total (thread 0)
__device__ bool cg_reduce(double d, double *partial, unsigned *counter, double *total) {
    d = block_sum(d);
    if (threadIdx.x == 0) partial[blockIdx.x] = d;
    if (!cg_last_block(counter)) return false;
    const double t = cg_sum_partials(partial, gridDim.x);
    if (threadIdx.x == 0) {
        *total = t;
        *counter = 0u;
    }
    return true;
}

// two sums at once, each with the arithmetic (and so the result) of cg_reduce
__device__ bool cg_reduce2(double d1, double d2, double *part1, double *part2, unsigned *counter, double *t1,
                           double *t2) {
    d1 = block_sum(d1);
    d2 = block_sum(d2);
    if (threadIdx.x == 0) {
        part1[blockIdx.x] = d1;
        part2[blockIdx.x] = d2;
    }
    if (!cg_last_block(counter)) return false;
    const double a = cg_sum_partials(part1, gridDim.x);
    const double b = cg_sum_partials(part2, gridDim.x);
    if (threadIdx.x == 0) {
        *t1 = a;
        *t2 = b;
        *counter = 0u;
    }
    return true;
}

__device__ __forceinline__ void put_smooth0(const Smooth0Out &z0, int32_t i, double ri) {
    if (z0.u) z0.u[i] = z0.m[i] * ri;
    if (z0.uf) z0.uf[i] = z0.mf[i] * (float)ri;
}

// u = 0, r = f; the last block initialises the iteration state from |f|
__global__ void k_cg_init(int32_t n, const double *__restrict__ f, double *__restrict__ u, double *__restrict__ r,
                          double *__restrict__ partial, CgState *cg, double tol, int maxiter, Smooth0Out z0) {
    pdl_wait();
    double s = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double fi = f[i];
        u[i] = 0.0;
        r[i] = fi;
        put_smooth0(z0, i, fi);
        s = fma(fi, fi, s);
    }
    double ff = 0.0;
    if (cg_reduce(s, partial, &cg->ctr[CG_CTR_INIT], &ff) && threadIdx.x == 0) {
        cg->nf = sqrt(ff);
        cg->tol = tol;
        cg->maxiter = maxiter;
        cg->done = (cg->nf == 0.0) || maxiter <= 0;
        cg->status = (maxiter <= 0 && cg->nf != 0.0) ? AMG_NOT_CONVERGED : AMG_OK;
        cg->iter = 0;
        cg->replacements = 0;
        cg->need_true = 0;
        cg->copy_r = 0;
        cg->pad = 0;
        cg->rz = cg->rz_next = cg->rzo = 0.0;
        cg->alpha = cg->beta = cg->pq = cg->rr = cg->res = cg->tres = 0.0;
    }
}

// x.y; with a state, the last block stores it (target 1: the new r.z,
// target 2: r_new.z_old of the flexible variant)
__global__ void k_dot(int32_t n, const double *__restrict__ x, const double *__restrict__ y,
                      double *__restrict__ partial, const int *skip, CgState *cg, int target) {
    pdl_wait();
    if (skipped(skip)) return;
    double s = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s = fma(x[i], y[i], s);
    if (!cg) {
        s = block_sum(s);
        if (threadIdx.x == 0) partial[blockIdx.x] = s;
        return;
    }
    double t = 0.0;
    if (cg_reduce(s, partial, &cg->ctr[target == 1 ? CG_CTR_RZ : CG_CTR_RZO], &t) && threadIdx.x == 0) {
        if (target == 1) cg->rz_next = t;
        else cg->rzo = t;
    }
}

// after the first preconditioner application: p = z, r.z becomes current
__global__ void k_cg_set_rz_p(int32_t n, const double *__restrict__ z, double *__restrict__ p, CgState *cg) {
    pdl_wait();
    if (cg->done) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) cg->rz = cg->rz_next;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = z[i];
}

// q = A p; the last block forms p.q and alpha = r.z / p.q (breakdown: p.q <= 0)
__global__ void k_spmv_dot(int32_t n, const int32_t *__restrict__ ptr, ColIdx ci,
                           const double *__restrict__ val, const double *__restrict__ p, double *__restrict__ q,
                           double *__restrict__ partial, CgState *cg) {
    __shared__ int32_t s_off[kMaxColOffsets];
    pdl_wait();
    if (cg->done) return;
    stage_col_offsets(ci, s_off);
    // r.z of the previous iteration becomes current (read only by the last block)
    if (blockIdx.x == 0 && threadIdx.x == 0) cg->rz = cg->rz_next;
    double d = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        if (ci.cidx)
            for (int32_t e = ptr[i]; e < ptr[i + 1]; ++e) s = fma(val[e], p[i + s_off[ci.cidx[e]]], s);
        else if (ci.c16)
            for (int32_t e = ptr[i]; e < ptr[i + 1]; ++e) s = fma(val[e], p[i + (int32_t)ci.c16[e]], s);
        else
            for (int32_t e = ptr[i]; e < ptr[i + 1]; ++e) s = fma(val[e], p[ci.col[e]], s);
        q[i] = s;
        d = fma(p[i], s, d);
    }
    double pq = 0.0;
    if (cg_reduce(d, partial, &cg->ctr[CG_CTR_PQ], &pq) && threadIdx.x == 0) {
        cg->pq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) {
            cg->iter += 1;
            cg->status = AMG_ERR_BREAKDOWN;
            cg->done = 1;
        } else {
            cg->alpha = __ldcg(&cg->rz) / pq;  // committed by block 0 of this kernel
        }
    }
}

// u += alpha p, r -= alpha q; the last block checks the recurrence residual
// (graph: opens the IF branch hb of the true-residual check when it meets tol).
// With zo (the flexible variant), also r_new.z_old into cg->rzo, summed as the
// separate dot kernel would sum it (same grid, same order).
__global__ void k_cg_update_ur(int32_t n, CgState *cg, const double *__restrict__ p, const double *__restrict__ q,
                               double *__restrict__ u, double *__restrict__ r, double *__restrict__ partial,
                               const double *__restrict__ zo, double *__restrict__ part_zo, int use_h,
                               cudaGraphConditionalHandle hb, Smooth0Out z0) {
    pdl_wait();
    if (cg->done) {
        if (use_h && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(hb, 0u);
        return;
    }
    const double alpha = cg->alpha;
    double s = 0.0, so = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        u[i] = fma(alpha, p[i], u[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        put_smooth0(z0, i, ri);
        s = fma(ri, ri, s);
        if (zo) so = fma(ri, zo[i], so);
    }
    double rr = 0.0, rzo = 0.0;
    const bool last = zo ? cg_reduce2(s, so, partial, part_zo, &cg->ctr[CG_CTR_RR], &rr, &rzo)
                         : cg_reduce(s, partial, &cg->ctr[CG_CTR_RR], &rr);
    if (last && threadIdx.x == 0) {
        if (zo) cg->rzo = rzo;
        cg->iter += 1;
        cg->rr = rr;
        cg->res = sqrt(rr) / cg->nf;
        cg->need_true = cg->res <= cg->tol;
        if (!cg->need_true && cg->iter >= cg->maxiter) {
            cg->done = 1;
            cg->status = AMG_NOT_CONVERGED;
        }
        if (use_h) cudaGraphSetConditional(hb, (cg->need_true && !cg->done) ? 1u : 0u);
    }
}

// t = f - A u, the true residual, when the recurrence reports convergence; the
// last block accepts convergence or schedules the replacement of r (twice at
// most).  With force: unconditionally, the final relative residual.
__global__ void k_true_residual(int32_t n, const int32_t *__restrict__ ptr, ColIdx ci,
                                const double *__restrict__ val, const double *__restrict__ f,
                                const double *__restrict__ u, double *__restrict__ t, double *__restrict__ partial,
                                CgState *cg, int force) {
    __shared__ int32_t s_off[kMaxColOffsets];
    pdl_wait();
    if (!force && (cg->done || !cg->need_true)) return;
    stage_col_offsets(ci, s_off);
    double d = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int32_t e = ptr[i]; e < ptr[i + 1]; ++e)
            s = fma(val[e], u[col_at(ci, s_off, i, e)], s);
        const double ti = f[i] - s;
        t[i] = ti;
        d = fma(ti, ti, d);
    }
    double tt = 0.0;
    if (cg_reduce(d, partial, &cg->ctr[CG_CTR_TT], &tt) && threadIdx.x == 0) {
        cg->tres = cg->nf > 0.0 ? sqrt(tt) / cg->nf : 0.0;
        if (!force) {
            if (cg->tres <= cg->tol) {
                cg->done = 1;
                cg->status = AMG_OK;
            } else if (cg->replacements >= 2 || cg->iter >= cg->maxiter) {
                cg->done = 1;
                cg->status = AMG_NOT_CONVERGED;
            } else {
                cg->replacements += 1;
                cg->copy_r = 1;
            }
        }
    }
}

// r = t when the true residual replaces the recurrence residual; with zo (the
// flexible variant), r_new.z_old is formed again from the new r
__global__ void k_replace_r(int32_t n, CgState *cg, const double *__restrict__ t, double *__restrict__ r,
                            const double *__restrict__ zo, double *__restrict__ part_zo, Smooth0Out z0) {
    pdl_wait();
    if (cg->done || !cg->copy_r) return;
    double so = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double ti = t[i];
        r[i] = ti;
        put_smooth0(z0, i, ti);
        if (zo) so = fma(ti, zo[i], so);
    }
    if (!zo) return;
    double rzo = 0.0;
    if (cg_reduce(so, part_zo, &cg->ctr[CG_CTR_RZO], &rzo) && threadIdx.x == 0) cg->rzo = rzo;
}

// beta = (r.z_new - r.z_old) / (r.z)_old, the flexible form (r.z_old = 0 for
// standard CG), p = z + beta p.  The new r.z becomes current in the next
// iteration's first kernel.  In the graph this is the body's last kernel: it
// keeps the while loop going while the iteration is not done, with a hard
// cap of maxiter + 4 bodies.
__global__ void k_cg_update_p(int32_t n, CgState *cg, const double *__restrict__ z, double *__restrict__ p,
                              int use_h, cudaGraphConditionalHandle h) {
    pdl_wait();
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    if (cg->done) {
        if (lead && use_h) cudaGraphSetConditional(h, 0u);
        return;
    }
    // one FP64 division per block, not per thread (FP64 runs at a small
    // fraction of the FP32 rate on this part)
    __shared__ double s_beta;
    if (threadIdx.x == 0) s_beta = (cg->rz_next - cg->rzo) / cg->rz;
    __syncthreads();
    const double beta = s_beta;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
    if (lead) {
        cg->beta = beta;
        cg->copy_r = 0;
        cg->need_true = 0;
        cg->pad += 1;  // loop bodies executed
        if (cg->pad > cg->maxiter + 4) {
            cg->done = 1;
            cg->status = AMG_NOT_CONVERGED;
        }
        if (use_h) cudaGraphSetConditional(h, cg->done ? 0u : 1u);
    }
}

// ------------------------------------------------------------------ BiCGStab (FP64)
// Right-preconditioned BiCGStab (the Krylov solver of Sec. 4) with the same
// device-resident control as CG: every kernel returns at once when the state
// says done; scalars are formed by the last block of the producing kernel.

// row i of y = A x for the scalar matrix (BS = 1) or the 4 x 4 block matrix
// seen as 4 n scalar rows (BS = 4: node i / 4, component i % 4; entry order,
// then component order)
template <int BS>
__device__ __forceinline__ double bi_row(int32_t i, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                         const double *__restrict__ val, const double *__restrict__ x) {
    double s = 0.0;
    if (BS == 1) {
        for (int32_t e = ptr[i]; e < ptr[i + 1]; ++e) s = fma(val[e], x[col[e]], s);
    } else {
        const int32_t node = i >> 2, r = i & 3;
        for (int32_t e = ptr[node]; e < ptr[node + 1]; ++e) {
            const double *b = val + (int64_t)16 * e + 4 * r;
            const double *xv = x + (int64_t)4 * col[e];
            s = fma(b[0], xv[0], s);
            s = fma(b[1], xv[1], s);
            s = fma(b[2], xv[2], s);
            s = fma(b[3], xv[3], s);
        }
    }
    return s;
}

// two sums published together; the last block returns both totals
__device__ bool bi_reduce2(double a, double b, double *pa, double *pb, unsigned *counter, double *ta, double *tb) {
    a = block_sum(a);
    b = block_sum(b);
    if (threadIdx.x == 0) {
        pa[blockIdx.x] = a;
        pb[blockIdx.x] = b;
    }
    if (!cg_last_block(counter)) return false;
    const double sa = cg_sum_partials(pa, gridDim.x);
    const double sb = cg_sum_partials(pb, gridDim.x);
    if (threadIdx.x == 0) {
        *ta = sa;
        *tb = sb;
        *counter = 0u;
    }
    return true;
}

// x = 0, r = r^ = f, p = v = 0; the last block initialises the state from |f|
__global__ void k_bi_init(int32_t n, const double *__restrict__ f, double *__restrict__ x, double *__restrict__ r,
                          double *__restrict__ rh, double *__restrict__ p, double *__restrict__ v,
                          double *__restrict__ partial, BiState *st, double tol, int maxiter) {
    pdl_wait();
    double s = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double fi = f[i];
        x[i] = 0.0;
        r[i] = fi;
        rh[i] = fi;
        p[i] = 0.0;
        v[i] = 0.0;
        s = fma(fi, fi, s);
    }
    double ff = 0.0;
    if (cg_reduce(s, partial, &st->ctr[BI_CTR_INIT], &ff) && threadIdx.x == 0) {
        st->nf = sqrt(ff);
        st->tol = tol;
        st->maxiter = maxiter;
        st->done = (st->nf == 0.0) || maxiter <= 0;
        st->status = (maxiter <= 0 && st->nf != 0.0) ? AMG_NOT_CONVERGED : AMG_OK;
        st->rho_old = st->alpha = st->omega = 1.0;
        st->rho = st->beta = st->rv = st->ts = st->tt = st->res = st->sres = st->tres = 0.0;
        st->iter = st->replacements = st->half = st->need_true = st->copy_r = st->pad = 0;
        st->skip = st->done;
    }
}

// rho = (r^, r); beta = (rho / rho_old)(alpha / omega)
__global__ void k_bi_rho(int32_t n, const double *__restrict__ rh, const double *__restrict__ r,
                         double *__restrict__ partial, BiState *st) {
    pdl_wait();
    if (st->done) return;
    double d = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) d = fma(rh[i], r[i], d);
    double rho = 0.0;
    if (cg_reduce(d, partial, &st->ctr[BI_CTR_RHO], &rho) && threadIdx.x == 0) {
        st->iter += 1;
        if (!(rho != 0.0) || !isfinite(rho)) {
            st->status = AMG_ERR_BREAKDOWN;
            st->done = st->skip = 1;
        } else {
            st->rho = rho;
            st->beta = (rho / st->rho_old) * (st->alpha / st->omega);
        }
    }
}

// p = r + beta (p - omega v)
__global__ void k_bi_p(int32_t n, const double *__restrict__ r, const double *__restrict__ v, double *__restrict__ p,
                       const BiState *st) {
    pdl_wait();
    if (st->done) return;
    const double beta = st->beta, omega = st->omega;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = fma(beta, fma(-omega, v[i], p[i]), r[i]);
}

// v = A p^, (r^, v); alpha = rho / (r^, v)
template <int BS>
__global__ void k_bi_spmv_rv(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                             const double *__restrict__ val, const double *__restrict__ ph, double *__restrict__ v,
                             const double *__restrict__ rh, double *__restrict__ partial, BiState *st) {
    pdl_wait();
    if (st->done) return;
    double d = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double s = bi_row<BS>(i, ptr, col, val, ph);
        v[i] = s;
        d = fma(rh[i], s, d);
    }
    double rv = 0.0;
    if (cg_reduce(d, partial, &st->ctr[BI_CTR_RV], &rv) && threadIdx.x == 0) {
        st->rv = rv;
        if (!(rv != 0.0) || !isfinite(rv)) {
            st->status = AMG_ERR_BREAKDOWN;
            st->done = st->skip = 1;
        } else {
            st->alpha = st->rho / rv;
            st->rho_old = st->rho;
        }
    }
}

// s = r - alpha v and |s|: converged at the half step when |s|/|f| <= tol
__global__ void k_bi_s(int32_t n, const double *__restrict__ r, const double *__restrict__ v, double *__restrict__ sv,
                       double *__restrict__ partial, BiState *st) {
    pdl_wait();
    if (st->done) return;
    const double alpha = st->alpha;
    double d = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double si = fma(-alpha, v[i], r[i]);
        sv[i] = si;
        d = fma(si, si, d);
    }
    double ss = 0.0;
    if (cg_reduce(d, partial, &st->ctr[BI_CTR_SS], &ss) && threadIdx.x == 0) {
        st->sres = sqrt(ss) / st->nf;
        st->half = st->sres <= st->tol;
        st->need_true = st->half;
        st->skip = st->half;
    }
}

// half step: x += alpha p^, r = s
__global__ void k_bi_half(int32_t n, const double *__restrict__ ph, const double *__restrict__ sv,
                          double *__restrict__ x, double *__restrict__ r, const BiState *st) {
    pdl_wait();
    if (st->done || !st->half) return;
    const double alpha = st->alpha;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = fma(alpha, ph[i], x[i]);
        r[i] = sv[i];
    }
}

// t = A s^, (t, s), (t, t); omega = (t, s) / (t, t)
template <int BS>
__global__ void k_bi_spmv_t(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                            const double *__restrict__ val, const double *__restrict__ sh,
                            const double *__restrict__ sv, double *__restrict__ t, double *__restrict__ partial,
                            BiState *st) {
    pdl_wait();
    if (st->skip) return;
    double a = 0.0, b = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double s = bi_row<BS>(i, ptr, col, val, sh);
        t[i] = s;
        a = fma(s, sv[i], a);
        b = fma(s, s, b);
    }
    const int nb = gridDim.x;
    double ts = 0.0, tt = 0.0;
    if (bi_reduce2(a, b, partial, partial + nb, &st->ctr[BI_CTR_T], &ts, &tt) && threadIdx.x == 0) {
        st->ts = ts;
        st->tt = tt;
        const double omega = ts / tt;
        if (!(tt != 0.0) || !isfinite(tt) || !(omega != 0.0) || !isfinite(omega)) {
            st->status = AMG_ERR_BREAKDOWN;
            st->done = st->skip = 1;
        } else {
            st->omega = omega;
        }
    }
}

// x += alpha p^ + omega s^, r = s - omega t, |r|
__global__ void k_bi_xr(int32_t n, const double *__restrict__ ph, const double *__restrict__ sh,
                        const double *__restrict__ sv, const double *__restrict__ t, double *__restrict__ x,
                        double *__restrict__ r, double *__restrict__ partial, BiState *st) {
    pdl_wait();
    if (st->skip) return;
    const double alpha = st->alpha, omega = st->omega;
    double d = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = fma(omega, sh[i], fma(alpha, ph[i], x[i]));
        const double ri = fma(-omega, t[i], sv[i]);
        r[i] = ri;
        d = fma(ri, ri, d);
    }
    double rr = 0.0;
    if (cg_reduce(d, partial, &st->ctr[BI_CTR_RR], &rr) && threadIdx.x == 0) {
        st->res = sqrt(rr) / st->nf;
        st->need_true = st->res <= st->tol;
    }
}

// the true residual when the recurrence (or the half step) reports
// convergence: accept, or replace r by it (twice at most); with force, the
// final relative residual
template <int BS>
__global__ void k_bi_true(int32_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                          const double *__restrict__ val, const double *__restrict__ f, const double *__restrict__ x,
                          double *__restrict__ t, double *__restrict__ partial, BiState *st, int force) {
    pdl_wait();
    if (!force && (st->done || !st->need_true)) return;
    double d = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double s = bi_row<BS>(i, ptr, col, val, x);
        const double ti = f[i] - s;
        t[i] = ti;
        d = fma(ti, ti, d);
    }
    double tt = 0.0;
    if (cg_reduce(d, partial, &st->ctr[BI_CTR_TRUE], &tt) && threadIdx.x == 0) {
        st->tres = st->nf > 0.0 ? sqrt(tt) / st->nf : 0.0;
        if (!force) {
            if (st->tres <= st->tol) {
                st->done = 1;
                st->status = AMG_OK;
            } else if (st->replacements >= 2) {
                st->done = 1;
                st->status = AMG_NOT_CONVERGED;
            } else {
                st->replacements += 1;
                st->copy_r = 1;
            }
        }
    }
}

__global__ void k_bi_replace(int32_t n, const double *__restrict__ t, double *__restrict__ r, const BiState *st) {
    pdl_wait();
    if (st->done || !st->copy_r) return;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) r[i] = t[i];
}

// end of an iteration: count it, clear the per-iteration flags, stop at
// maxiter (and, in the graph, keep the while loop going; hard cap maxiter + 4
// bodies)
__global__ void k_bi_end(BiState *st, int use_h, cudaGraphConditionalHandle h) {
    pdl_wait();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->pad += 1;  // bodies run (the graph's launch count)
    if (!st->done) {
        if (st->iter >= st->maxiter || st->pad > st->maxiter + 4) {
            st->done = 1;
            st->status = AMG_NOT_CONVERGED;
        }
    }
    st->half = st->need_true = st->copy_r = 0;
    st->skip = st->done;
    if (use_h) cudaGraphSetConditional(h, st->done ? 0u : 1u);
}

}  // namespace

// ======================================================================= launchers
void launch_ap_numeric_f64(const Level &L, const double *A_val, cudaStream_t s) {
    count_launch();
    k_ap_numeric_f64<<<nblocks(L.n, kApThreads), kApThreads, 0, s>>>(L.n, L.A_ptr, L.A_col, A_val, L.P_ptr, L.P_val,
                                                                     L.AP_ptr, L.t1ptr, L.slot1, L.AP_val);
}
void launch_rap_numeric_f64(const Level &L, const int32_t *Ac_ptr, double *Ac_val, cudaStream_t s) {
    unsigned g = (unsigned)((L.nc + kRapWarps - 1) / kRapWarps);
    count_launch();
    k_rap_terms<double><<<g, kRapWarps * 32, 0, s>>>(L.nc, L.R_ptr, L.R_col, L.R_val, L.AP_ptr, L.AP_val, Ac_ptr,
                                                     L.t2ptr, L.slot2, Ac_val);
}
void launch_ap_numeric_f32(const Level &L, const float *A_valf, cudaStream_t s) {
    count_launch();
    k_ap_numeric_f32<<<nblocks(L.n, kApThreads), kApThreads, 0, s>>>(L.n, L.A_ptr, L.A_col, A_valf, L.P_ptr,
                                                                     L.P_valf, L.AP_ptr, L.t1ptr, L.slot1, L.AP_valf);
}
void launch_rap_numeric_f32(const Level &L, const int32_t *Ac_ptr, float *Ac_valf, cudaStream_t s) {
    unsigned g = (unsigned)((L.nc + kRapWarps - 1) / kRapWarps);
    count_launch();
    k_rap_terms<float><<<g, kRapWarps * 32, 0, s>>>(L.nc, L.R_ptr, L.R_col, L.R_valf, L.AP_ptr, L.AP_valf, Ac_ptr,
                                                    L.t2ptr, L.slot2, Ac_valf);
}

template <class V>
void launch_gather_apply(int64_t nout, const int32_t *eptr, const int32_t *idx, const V *w, const V *x, V *y,
                         cudaStream_t s) {
    if (nout <= 0) return;
    count_launch();
    k_gather_apply<V><<<nblocks(nout), kThreads, 0, s>>>(nout, eptr, idx, w, x, y);
}
template void launch_gather_apply<double>(int64_t, const int32_t *, const int32_t *, const double *, const double *,
                                          double *, cudaStream_t);
template void launch_gather_apply<float>(int64_t, const int32_t *, const int32_t *, const float *, const float *,
                                         float *, cudaStream_t);

void launch_smoother_f64(int32_t n, const int32_t *ptr, const double *val, const int32_t *dia, int type, double wj,
                         double *m, cudaStream_t s) {
    count_launch();
    k_smoother<double><<<nblocks(n), kThreads, 0, s>>>(n, ptr, val, dia, type, wj, m);
}
void launch_smoother_f32(int32_t n, const int32_t *ptr, const float *val, const int32_t *dia, int type, double wj,
                         float *m, cudaStream_t s) {
    count_launch();
    k_smoother<float><<<nblocks(n), kThreads, 0, s>>>(n, ptr, val, dia, type, (float)wj, m);
}
void launch_ingest_fine(int32_t row0, int32_t row1, const int32_t *ptr, const double *val_in, const int32_t *dia,
                        int type, double wj, double *val_out, float *valf_out, double *m, float *mf, int *st,
                        cudaStream_t s) {
    if (row1 <= row0) return;
    count_launch();
    k_ingest_fine<<<nblocks(row1 - row0), kThreads, 0, s>>>(row0, row1, ptr, val_in, dia, type, wj, val_out, valf_out,
                                                            m, mf, st);
}
void launch_cast_f32(int64_t n, const double *in, float *out, cudaStream_t s) {
    int64_t b = nblocks(n);
    count_launch();
    k_cast_f32<<<(unsigned)(b > 8192 ? 8192 : b), kThreads, 0, s>>>(n, in, out);
}

void launch_csr_to_dense(int32_t n, const int32_t *ptr, const int32_t *col, const double *val, const float *valf,
                         double *dense, cudaStream_t s) {
    cudaMemsetAsync(dense, 0, sizeof(double) * (size_t)n * (size_t)n, s);
    count_launch();
    k_csr_to_dense<<<nblocks(n), kThreads, 0, s>>>(n, ptr, col, val, valf, dense);
}
size_t lu_cluster_smem(int32_t n) {
    const size_t nloc = (size_t)(n + kLuClusterCtas - 1) / kLuClusterCtas;
    return (nloc * n + n + nloc) * sizeof(double) + 2 * (size_t)n * sizeof(int32_t);
}
bool lu_wants_transpose(int32_t n) { return n > kLuSmemN && n <= kLuClusterN; }
void launch_dense_lu(int32_t n, double *a, int32_t *piv, int *st, cudaStream_t s, double *aT) {
    static bool attr = false;
    const int max_bytes = kLuSmemN * kLuSmemN * (int)sizeof(double);
    if (!attr) {
        cudaFuncSetAttribute(k_dense_lu_pipe<kLuPipeC, kLuPipeB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lu_pipe_smem(kLuPipeN, kLuPipeC, kLuPipeB));
        if (kLuPipeC > 8)
            cudaFuncSetAttribute(k_dense_lu_pipe<kLuPipeC, kLuPipeB>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(k_dense_lu_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(k_dense_lu_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lu_cluster_smem(kLuClusterN));
        cudaFuncSetAttribute(k_lu_inverse_t, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(((size_t)(kInvWarps + 1) * kLuClusterN) * sizeof(double) +
                                   (size_t)kLuClusterN * sizeof(int32_t)));
        attr = true;
    }
    count_launch();
    if (n > kLuPipeMinN && n <= kLuPipeN)
        k_dense_lu_pipe<kLuPipeC, kLuPipeB>
            <<<kLuPipeC, kLuPipeThreads, lu_pipe_smem(n, kLuPipeC, kLuPipeB), s>>>(n, a, aT, piv, st);
    else if (n <= kLuSmemN)
        k_dense_lu_smem<<<1, kLuThreads, (size_t)n * n * sizeof(double), s>>>(n, a, piv, st);
    else if (n <= kLuClusterN)
        k_dense_lu_cluster<<<kLuClusterCtas, kLuClusterThreads, lu_cluster_smem(n), s>>>(n, a, aT, piv, st);
    else
        k_dense_lu<<<1, 1024, 0, s>>>(n, a, piv, st);
}
void launch_lu_inverse(int32_t n, const double *lu, const int32_t *piv, double *inv, cudaStream_t s,
                       const double *luT) {
    if (luT && n > kLuSmemN && n <= kLuClusterN) {
        count_launch();
        const size_t bytes = ((size_t)(kInvWarps + 1) * n) * sizeof(double) + (size_t)n * sizeof(int32_t);
        k_lu_inverse_t<<<(unsigned)((n + kInvWarps - 1) / kInvWarps), kInvWarps * 32, bytes, s>>>(n, luT, piv, inv);
        return;
    }
    static bool attr = false;
    const int max_bytes = (kLuSmemN * kLuSmemN + (kInvWarps + 1) * kLuSmemN) * (int)sizeof(double) +
                          kLuSmemN * (int)sizeof(int32_t);
    if (!attr) {
        cudaFuncSetAttribute(k_lu_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(k_lu_inverse_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (kLuSmemN * kLuSmemN + kLuSmemN) * (int)sizeof(double) + kLuSmemN * (int)sizeof(int32_t));
        attr = true;
    }
    count_launch();
    if (n <= kLuSmemN) {
        const unsigned threads = (unsigned)((n + 31) / 32 * 32);
        k_lu_inverse_rows<<<(unsigned)n, threads,
                            ((size_t)n * n + (size_t)n) * sizeof(double) + (size_t)n * sizeof(int32_t), s>>>(n, lu, piv,
                                                                                                         inv);
        return;
    }
    k_lu_inverse<<<(unsigned)((n + kInvWarps - 1) / kInvWarps), kInvWarps * 32, 0, s>>>(n, lu, piv, inv);
}

#define LPR_DISPATCH(lpr, KCALL)                   \
    switch (lpr) {                                 \
        case 1: { constexpr int P_ = 1; KCALL; } break;   \
        case 2: { constexpr int P_ = 2; KCALL; } break;   \
        case 4: { constexpr int P_ = 4; KCALL; } break;   \
        case 8: { constexpr int P_ = 8; KCALL; } break;   \
        case 16: { constexpr int P_ = 16; KCALL; } break; \
        default: { constexpr int P_ = 32; KCALL; } break; \
    }

template <class V, class TF>
void launch_smooth0_residual(const Level &L, const V *val, const V *m, const TF *f, V *u, V *r, const int *skip,
                             cudaStream_t s) {
    count_launch();
    const unsigned g = (unsigned)nblocks((int64_t)L.n * L.lpr);
    LPR_DISPATCH(L.lpr, (launch_pdl(k_smooth0_residual<V, TF, P_>, g, kThreads, 0, s, L.n, L.A_ptr, L.cols(), val, m, f, u,
                                                                              r, skip)))
}
template <class V, class TF, class TO>
void launch_smooth_sweep(const Level &L, const V *val, const V *m, const TF *f, const V *u_in, TO *u_out,
                         const int *skip, cudaStream_t s) {
    count_launch();
    const unsigned g = (unsigned)nblocks((int64_t)L.n * L.lpr);
    LPR_DISPATCH(L.lpr, (launch_pdl(k_smooth_sweep<V, TF, TO, P_>, g, kThreads, 0, s, L.n, L.A_ptr, L.cols(), val, m, f,
                                                                              u_in, u_out, skip)))
}
template <class V>
void launch_smooth_sweep_dot(const Level &L, const V *val, const V *m, const double *f, const V *u_in, double *z,
                             double *partial, CgState *cg, const int *skip, cudaStream_t s) {
    count_launch();
    const unsigned g = (unsigned)cg_blocks(L.n);
    LPR_DISPATCH(L.lpr, (launch_pdl(k_smooth_sweep_dot<V, P_>, g, cg_threads(L.n), 0, s, L.n, L.A_ptr, L.cols(), val, m, f, u_in,
                                                                             z, partial, cg, skip)))
}
template void launch_smooth_sweep_dot<double>(const Level &, const double *, const double *, const double *,
                                              const double *, double *, double *, CgState *, const int *,
                                              cudaStream_t);
template void launch_smooth_sweep_dot<float>(const Level &, const float *, const float *, const double *,
                                             const float *, double *, double *, CgState *, const int *, cudaStream_t);
template <class V, class TF>
void launch_residual(const Level &L, const V *val, const TF *f, const V *u, V *r, const int *skip, cudaStream_t s) {
    count_launch();
    const unsigned g = (unsigned)nblocks((int64_t)L.n * L.lpr);
    LPR_DISPATCH(L.lpr, (launch_pdl(k_residual<V, TF, P_>, g, kThreads, 0, s, L.n, L.A_ptr, L.cols(), val, f, u, r, skip)))
}
template <class V>
void launch_restrict(const Level &L, const V *Rval, const V *r, V *fc, const V *mc, V *uc, const int *skip,
                     cudaStream_t s) {
    count_launch();
    const unsigned g = (unsigned)nblocks((int64_t)L.nc * L.lpr_r);
    LPR_DISPATCH(L.lpr_r, (launch_pdl(k_restrict<V, P_>, g, kThreads, 0, s, L.nc, L.R_ptr, L.R_col, Rval, r, fc, mc, uc,
                                                                    skip)))
}
template <class V>
void launch_prolong(const Level &L, const V *Pval, const V *uc, V *u, const int *skip, cudaStream_t s) {
    count_launch();
    launch_pdl(k_prolong<V>, nblocks(L.n), kThreads, 0, s, L.n, L.P_ptr, L.P_col, (const int16_t *)L.P_c16, L.P_ratio,
               Pval, uc, u, skip);
}
template <class V, class TF, class TO>
void launch_coarse_solve(int32_t n, const double *inv, const TF *f, TO *u, const int *skip, cudaStream_t s) {
    count_launch();
    launch_pdl(k_coarse_solve<TF, TO>, nblocks((int64_t)n * 32, 128), 128, 0, s, n, inv, f, u, skip);
}
template <class TI, class TO>
void launch_copy_cast(int64_t n, const TI *in, TO *out, const int *skip, cudaStream_t s) {
    int64_t b = nblocks(n);
    count_launch();
    launch_pdl(k_copy_cast<TI, TO>, (unsigned)(b > 8192 ? 8192 : b), kThreads, 0, s, n, in, out, skip);
}

#define INST_V(V, TF, TO)                                                                                           \
    template void launch_smooth_sweep<V, TF, TO>(const Level &, const V *, const V *, const TF *, const V *, TO *, \
                                                 const int *, cudaStream_t);
INST_V(double, double, double)
INST_V(float, float, float)
INST_V(float, double, double)
INST_V(float, double, float)
INST_V(float, float, double)
#undef INST_V
template void launch_smooth0_residual<double, double>(const Level &, const double *, const double *, const double *,
                                                      double *, double *, const int *, cudaStream_t);
template void launch_smooth0_residual<float, float>(const Level &, const float *, const float *, const float *,
                                                    float *, float *, const int *, cudaStream_t);
template void launch_smooth0_residual<float, double>(const Level &, const float *, const float *, const double *,
                                                     float *, float *, const int *, cudaStream_t);
template void launch_residual<double, double>(const Level &, const double *, const double *, const double *, double *,
                                              const int *, cudaStream_t);
template void launch_residual<float, float>(const Level &, const float *, const float *, const float *, float *,
                                            const int *, cudaStream_t);
template void launch_residual<float, double>(const Level &, const float *, const double *, const float *, float *,
                                             const int *, cudaStream_t);
template void launch_restrict<double>(const Level &, const double *, const double *, double *, const double *,
                                      double *, const int *, cudaStream_t);
template void launch_restrict<float>(const Level &, const float *, const float *, float *, const float *, float *,
                                     const int *, cudaStream_t);
template void launch_prolong<double>(const Level &, const double *, const double *, double *, const int *,
                                     cudaStream_t);
template void launch_prolong<float>(const Level &, const float *, const float *, float *, const int *, cudaStream_t);
template void launch_coarse_solve<double, double, double>(int32_t, const double *, const double *, double *,
                                                          const int *, cudaStream_t);
template void launch_coarse_solve<float, float, float>(int32_t, const double *, const float *, float *, const int *,
                                                       cudaStream_t);
template void launch_coarse_solve<float, double, double>(int32_t, const double *, const double *, double *,
                                                         const int *, cudaStream_t);
template void launch_copy_cast<float, float>(int64_t, const float *, float *, const int *, cudaStream_t);
template void launch_copy_cast<double, double>(int64_t, const double *, double *, const int *, cudaStream_t);
template void launch_copy_cast<double, float>(int64_t, const double *, float *, const int *, cudaStream_t);
template void launch_copy_cast<float, double>(int64_t, const float *, double *, const int *, cudaStream_t);

// Grid of the Krylov kernels (grid-stride loops, one partial per block).  The
// last-block reduction costs grow with the number of blocks (each block's
// partial, fence and counter update sit on the final block's critical path),
// so vectors up to about 1.2 M entries run on two blocks of 512 per SM; longer
// ones need full occupancy to keep enough loads in flight, reached with four
// blocks of 512 per SM (half the partials of eight blocks of 256, measured
// faster at 128^3 and 192^3).
int cg_blocks(int64_t n) {
    const int t = cg_threads(n);
    int64_t b = (n + t - 1) / t;
    const int64_t cap = n >= kCgLargeN ? kCgMaxBlocks : 152 * 2;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}
void launch_cg_init(int32_t n, const double *f, double *u, double *r, double *partial, CgState *cg, double tol,
                    int maxiter, const Smooth0Out &z0, cudaStream_t s) {
    count_launch();
    launch_pdl(k_cg_init, cg_blocks(n), cg_threads(n), 0, s, n, f, u, r, partial, cg, tol, maxiter, z0);
}
void launch_dot(int32_t n, const double *x, const double *y, double *partial, const int *skip, CgState *cg, int target,
                cudaStream_t s) {
    count_launch();
    launch_pdl(k_dot, cg_blocks(n), cg_threads(n), 0, s, n, x, y, partial, skip, cg, target);
}
void launch_cg_set_rz_p(int32_t n, const double *z, double *p, CgState *cg, cudaStream_t s) {
    count_launch();
    launch_pdl(k_cg_set_rz_p, cg_blocks(n), cg_threads(n), 0, s, n, z, p, cg);
}
void launch_spmv_dot(int32_t n, const int32_t *ptr, const ColIdx &col, const double *val, const double *p,
                     double *q, double *partial, CgState *cg, cudaStream_t s) {
    count_launch();
    launch_pdl(k_spmv_dot, cg_blocks(n), cg_threads(n), 0, s, n, ptr, col, val, p, q, partial, cg);
}
void launch_cg_update_ur(int32_t n, CgState *cg, const double *p, const double *q, double *u, double *r,
                         double *partial, const double *zo, double *part_zo, int use_h, cudaGraphConditionalHandle hb,
                         const Smooth0Out &z0, cudaStream_t s) {
    count_launch();
    launch_pdl(k_cg_update_ur, cg_blocks(n), cg_threads(n), 0, s, n, cg, p, q, u, r, partial, zo, part_zo, use_h, hb,
               z0);
}
void launch_col_delta16(int32_t n, const int32_t *ptr, const int32_t *col, float ratio, int16_t *c16, int *flag,
                        cudaStream_t s) {
    count_launch();
    k_col_delta16<<<nblocks(n), kThreads, 0, s>>>(n, ptr, col, ratio, c16, flag);
}
void launch_col_offsets_collect(int32_t n, const int32_t *ptr, const int32_t *col, int32_t *table, int *count,
                                cudaStream_t s) {
    count_launch();
    k_col_offsets_collect<<<nblocks(n), kThreads, 0, s>>>(n, ptr, col, table, count);
}
void launch_col_offsets_encode(int32_t n, const int32_t *ptr, const int32_t *col, const int32_t *off, int noff,
                               uint8_t *cidx, int *st, cudaStream_t s) {
    count_launch();
    k_col_offsets_encode<<<nblocks(n), kThreads, 0, s>>>(n, ptr, col, off, noff, cidx, st);
}
void launch_true_residual(int32_t n, const int32_t *ptr, const ColIdx &col, const double *val, const double *f,
                          const double *u, double *t, double *partial, CgState *cg, int force, cudaStream_t s) {
    count_launch();
    launch_pdl(k_true_residual, cg_blocks(n), cg_threads(n), 0, s, n, ptr, col, val, f, u, t, partial, cg, force);
}
void launch_replace_r(int32_t n, CgState *cg, const double *t, double *r, const double *zo, double *part_zo,
                      const Smooth0Out &z0, cudaStream_t s) {
    count_launch();
    launch_pdl(k_replace_r, cg_blocks(n), cg_threads(n), 0, s, n, cg, t, r, zo, part_zo, z0);
}
void launch_cg_update_p(int32_t n, CgState *cg, const double *z, double *p, int use_h, cudaGraphConditionalHandle h,
                        cudaStream_t s) {
    count_launch();
    launch_pdl(k_cg_update_p, cg_blocks(n), cg_threads(n), 0, s, n, cg, z, p, use_h, h);
}


void launch_bi_init(int32_t n, const double *f, double *x, double *r, double *rh, double *p, double *v,
                    double *partial, BiState *st, double tol, int maxiter, cudaStream_t s) {
    count_launch();
    launch_pdl(k_bi_init, cg_blocks(n), cg_threads(n), 0, s, n, f, x, r, rh, p, v, partial, st, tol, maxiter);
}
void launch_bi_rho(int32_t n, const double *rh, const double *r, double *partial, BiState *st, cudaStream_t s) {
    count_launch();
    launch_pdl(k_bi_rho, cg_blocks(n), cg_threads(n), 0, s, n, rh, r, partial, st);
}
void launch_bi_p(int32_t n, const double *r, const double *v, double *p, BiState *st, cudaStream_t s) {
    count_launch();
    launch_pdl(k_bi_p, cg_blocks(n), cg_threads(n), 0, s, n, r, v, p, st);
}
void launch_bi_spmv_rv(int32_t n, int bs, const int32_t *ptr, const int32_t *col, const double *val,
                       const double *ph, double *v, const double *rh, double *partial, BiState *st, cudaStream_t s) {
    count_launch();
    if (bs == 4) launch_pdl(k_bi_spmv_rv<4>, cg_blocks(n), cg_threads(n), 0, s, n, ptr, col, val, ph, v, rh, partial, st);
    else launch_pdl(k_bi_spmv_rv<1>, cg_blocks(n), cg_threads(n), 0, s, n, ptr, col, val, ph, v, rh, partial, st);
}
void launch_bi_s(int32_t n, const double *r, const double *v, double *sv, double *partial, BiState *st,
                 cudaStream_t s) {
    count_launch();
    launch_pdl(k_bi_s, cg_blocks(n), cg_threads(n), 0, s, n, r, v, sv, partial, st);
}
void launch_bi_half(int32_t n, const double *ph, const double *sv, double *x, double *r, BiState *st, cudaStream_t s) {
    count_launch();
    launch_pdl(k_bi_half, cg_blocks(n), cg_threads(n), 0, s, n, ph, sv, x, r, st);
}
void launch_bi_spmv_t(int32_t n, int bs, const int32_t *ptr, const int32_t *col, const double *val,
                      const double *sh, const double *sv, double *t, double *partial, BiState *st, cudaStream_t s) {
    count_launch();
    if (bs == 4) launch_pdl(k_bi_spmv_t<4>, cg_blocks(n), cg_threads(n), 0, s, n, ptr, col, val, sh, sv, t, partial, st);
    else launch_pdl(k_bi_spmv_t<1>, cg_blocks(n), cg_threads(n), 0, s, n, ptr, col, val, sh, sv, t, partial, st);
}
void launch_bi_xr(int32_t n, const double *ph, const double *sh, const double *sv, const double *t, double *x,
                  double *r, double *partial, BiState *st, cudaStream_t s) {
    count_launch();
    launch_pdl(k_bi_xr, cg_blocks(n), cg_threads(n), 0, s, n, ph, sh, sv, t, x, r, partial, st);
}
void launch_bi_true(int32_t n, int bs, const int32_t *ptr, const int32_t *col, const double *val, const double *f,
                    const double *x, double *t, double *partial, BiState *st, int force, cudaStream_t s) {
    count_launch();
    if (bs == 4) launch_pdl(k_bi_true<4>, cg_blocks(n), cg_threads(n), 0, s, n, ptr, col, val, f, x, t, partial, st, force);
    else launch_pdl(k_bi_true<1>, cg_blocks(n), cg_threads(n), 0, s, n, ptr, col, val, f, x, t, partial, st, force);
}
void launch_bi_replace(int32_t n, const double *t, double *r, BiState *st, cudaStream_t s) {
    count_launch();
    launch_pdl(k_bi_replace, cg_blocks(n), cg_threads(n), 0, s, n, t, r, st);
}
void launch_bi_end(BiState *st, int use_h, cudaGraphConditionalHandle h, cudaStream_t s) {
    count_launch();
    launch_pdl(k_bi_end, 1, 32, 0, s, st, use_h, h);
}

}  // namespace amgpr
