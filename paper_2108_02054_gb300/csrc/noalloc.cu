// noalloc.cu -- allocation-free variant of the pressure-Poisson pattern builder.
//
// amg_poisson_pattern scans the row lengths with scratch memory that it takes
// from the stream-ordered allocator.  Some callers cannot allocate device
// memory at that point: a host framework whose caching allocator has already
// reserved nearly all of the GPU's memory, or a latency-critical loop that
// forbids any allocation once it has started.  For them,
// amg_poisson_pattern_noalloc does the same work with its scan scratch in a
// fixed file-scope device array (kNoAllocMaxBlocks block sums, 128 KiB plus
// padding), which every device that loads this library keeps until the
// process exits.  The row lengths are written into the caller's d_ptr and
// scanned there in place.
#include <mutex>

#include "common.cuh"

namespace amgpr {
namespace {

constexpr int kNaThreads = 1024;
constexpr int kNaItems = 4;
constexpr int kNaTile = kNaThreads * kNaItems;
// at most AMG_NOALLOC_MAX_CELLS rows: one block sum per tile, plus the total
constexpr int64_t kNoAllocMaxBlocks = AMG_NOALLOC_MAX_CELLS / kNaTile;
constexpr int kMaxDevices = 64;

// shared by every call on a device; its last contents survive between calls
static __device__ __align__(256) int64_t g_scan_scratch[kNoAllocMaxBlocks + 2];

// device address of g_scan_scratch, resolved once per device
int64_t *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

__device__ int64_t na_block_exclusive_scan(int64_t v, int64_t *warp_tot, int64_t *total) {
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
        const int nw = blockDim.x >> 5;
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

// per-tile sums of the row lengths held in ptr[0..n)
__global__ void k_na_tile_sums(const int32_t *ptr, int64_t n, int64_t *bsum) {
    __shared__ int64_t wt[32];
    __shared__ int64_t tot;
    const int64_t base = (int64_t)blockIdx.x * kNaTile + (int64_t)threadIdx.x * kNaItems;
    int64_t s = 0;
    for (int k = 0; k < kNaItems; ++k)
        if (base + k < n) s += ptr[base + k];
    na_block_exclusive_scan(s, wt, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// exclusive scan of the tile sums, one block; bsum[nb] = total
__global__ void k_na_scan_tiles(int64_t *bsum, int64_t nb) {
    __shared__ int64_t wt[32];
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int64_t i = b0 + threadIdx.x;
        const int64_t v = i < nb ? bsum[i] : 0;
        const int64_t e = na_block_exclusive_scan(v, wt, &tot);
        if (i < nb) bsum[i] = carry + e;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

// in place: ptr[i] = sum of the lengths before row i, ptr[n] = total.  Every
// thread reads its own items before the block scan and writes them after it,
// and no other thread touches them, so reading and writing the same array is
// safe (no restrict qualifiers on purpose).
__global__ void k_na_scan_in_place(int32_t *ptr, int64_t n, const int64_t *bsum, int64_t nb) {
    __shared__ int64_t wt[32];
    __shared__ int64_t tot;
    const int64_t base = (int64_t)blockIdx.x * kNaTile + (int64_t)threadIdx.x * kNaItems;
    int64_t v[kNaItems];
    int64_t s = 0;
    for (int k = 0; k < kNaItems; ++k) {
        v[k] = (base + k < n) ? ptr[base + k] : 0;
        s += v[k];
    }
    int64_t e = na_block_exclusive_scan(s, wt, &tot) + bsum[blockIdx.x];
    for (int k = 0; k < kNaItems; ++k) {
        if (base + k < n) ptr[base + k] = (int32_t)e;
        e += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ptr[n] = (int32_t)bsum[nb];
}

// device address of the scratch array on the current device (first call per
// device resolves it; the host-side symbol itself is not a device address).
// The cached address belongs to the device's context: after a
// cudaDeviceReset it is stale, so a process that resets a device must not
// call this entry point on that device again.
amg_status scratch_for_current_device(int64_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AMG_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        int64_t *p = nullptr;
        if (cudaGetSymbolAddress((void **)&p, g_scan_scratch) != cudaSuccess || !p) return AMG_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return AMG_OK;
}

}  // namespace
}  // namespace amgpr

using namespace amgpr;

extern "C" amg_status amg_poisson_pattern_noalloc(int32_t dim, int32_t N, int32_t *d_ptr, int32_t *d_col,
                                                   void *cuda_stream) {
    if ((dim != 2 && dim != 3) || N < 1 || !d_ptr || !d_col) return AMG_ERR_ARG;
    const int64_t n = dim == 2 ? (int64_t)N * N : (int64_t)N * N * N;
    if (n > AMG_NOALLOC_MAX_CELLS) return AMG_ERR_CAPACITY;
    // an error left by earlier, unrelated work is reported without being
    // cleared, and nothing is launched on top of it
    if (cudaPeekAtLastError() != cudaSuccess) return AMG_ERR_CUDA;
    int64_t *scratch = nullptr;
    amg_status st = scratch_for_current_device(&scratch);
    if (st != AMG_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t nb = (n + kNaTile - 1) / kNaTile;
    launch_poisson_rowlen(dim, N, d_ptr, s);  // row lengths into the output, scanned below
    count_launch();
    k_na_tile_sums<<<(unsigned)nb, kNaThreads, 0, s>>>(d_ptr, n, scratch);
    count_launch();
    k_na_scan_tiles<<<1, kNaThreads, 0, s>>>(scratch, nb);
    count_launch();
    k_na_scan_in_place<<<(unsigned)nb, kNaThreads, 0, s>>>(d_ptr, n, scratch, nb);
    launch_poisson_cols(dim, N, d_ptr, d_col, s);
    if (cudaGetLastError() != cudaSuccess) return AMG_ERR_CUDA;
    return AMG_OK;
}
