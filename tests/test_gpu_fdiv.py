"""The integer FP64 division used for the coarsest LU's multipliers and the
finest smoother (csrc/fdiv.cuh) against IEEE division, and its FP64 -> FP32
conversion against the conversion instruction: a small CUDA program built
here runs
div_rn on classes of inputs chosen to hit its edges (random operands across
the normal range, raw 64-bit patterns with zeros, subnormals, infinities and
NaNs, significands near all-ones and near one, every pair of small integers,
quotients next to exact ones) and compares it bit for bit with the device's
division; a sample of the same quotients is compared with NumPy's IEEE
division on the host."""
import os
import subprocess

import numpy as np
import pytest

from paper_2108_02054_gb300 import build as PB

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_2108_02054_gb300", "csrc", "fdiv.cuh")

SRC = r'''
#include "%(header)s"
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
using namespace amgpr;

__device__ __forceinline__ unsigned long long mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double mk(unsigned long long s, unsigned long long e, unsigned long long m) {
    return __longlong_as_double((long long)((s << 63) | ((e & 0x7ff) << 52) | (m & 0xfffffffffffffull)));
}
__device__ void operands(int cls, long long i, double &x, double &d) {
    const unsigned long long a = mix(0x9E3779B97F4A7C15ull * (unsigned long long)(3 * i + 1) + cls);
    const unsigned long long b = mix(0x9E3779B97F4A7C15ull * (unsigned long long)(3 * i + 2) + cls);
    const unsigned long long c = mix(0x9E3779B97F4A7C15ull * (unsigned long long)(3 * i + 3) + cls);
    if (cls == 0) {
        x = mk(a >> 63, 1 + b %% 2046, a);
        d = mk(b >> 63, 1 + c %% 2046, c);
    } else if (cls == 1) {
        x = __longlong_as_double((long long)a);
        d = __longlong_as_double((long long)b);
        if ((c & 15) == 0) x = 0.0 * x;
    } else if (cls == 2) {
        const unsigned long long ma = (a & 1) ? (0xfffffffffffffull - (b & 0xfff)) : (b & 0xfff);
        const unsigned long long mb = (a & 2) ? (0xfffffffffffffull - (c & 0xfff)) : (c & 0xfff);
        x = mk((a >> 3) & 1, 1023 + (int)((a >> 8) %% 64) - 32, ma);
        d = mk((a >> 4) & 1, 1023 + (int)((a >> 20) %% 64) - 32, mb);
    } else if (cls == 3) {
        const long long q = i %% 601 - 300, r = (i / 601) %% 601 - 300;
        x = (double)q;
        d = (double)(r == 0 ? 7 : r);
    } else {
        d = mk(b >> 63, 1000 + c %% 40, c);
        const long long k = (long long)(a %% 64) - 32;
        x = d * (1.0 + (double)k * 0x1p-52);
        if (a & 0x100) x = __longlong_as_double(__double_as_longlong(x) + ((long long)(b %% 5) - 2));
    }
}
__global__ void k_check(int cls, long long n, unsigned long long *bad, long long ns, double *sx, double *sd,
                        double *sq) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double x, d;
        operands(cls, i, x, d);
        const double q = div_rn(x, div_recip(d)), h = x / d;
        const bool same = (q != q && h != h) || __double_as_longlong(q) == __double_as_longlong(h);
        if (!same) atomicAdd(bad, 1ull);
        if (i < ns) { sx[i] = x; sd[i] = d; sq[i] = q; }
    }
}
__global__ void k_cvt(int cls, long long n, unsigned long long *bad, long long ns, double *sx, float *sq) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long a = mix(0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1) + 77 + cls);
        unsigned long long b = a;
        if (cls == 1) b = (a & 0x800fffffffffffffull) | ((unsigned long long)(1023 - 160 + (a >> 56) %% 320) << 52);
        if (cls == 2) b = (a & 0x800000001fffffffull) | ((unsigned long long)(1023 - 150 + (a >> 58) %% 30) << 52) |
                          (((a >> 20) & 1ull) << 28);
        const double x = __longlong_as_double((long long)b);
        const float q = f64_to_f32_rn(x), h = (float)x;
        if (!((q != q && h != h) || __float_as_uint(q) == __float_as_uint(h))) atomicAdd(bad, 1ull);
        if (i < ns) { sx[i] = x; sq[i] = q; }
    }
}
int main(int argc, char **argv) {
    const long long n = atoll(argv[1]), ns = atoll(argv[2]);
    unsigned long long *bad; double *s;
    if (cudaMalloc(&bad, 8) != cudaSuccess || cudaMalloc(&s, 3 * 8 * ns) != cudaSuccess) return 2;
    FILE *f = fopen(argv[3], "wb");
    for (int cls = 0; cls < 5; ++cls) {
        cudaMemset(bad, 0, 8);
        const long long m = cls == 3 ? 601ll * 601ll : n;
        k_check<<<1216, 256>>>(cls, m, bad, ns, s, s + ns, s + 2 * ns);
        if (cudaDeviceSynchronize() != cudaSuccess) return 2;
        unsigned long long h;
        cudaMemcpy(&h, bad, 8, cudaMemcpyDeviceToHost);
        printf("%%d %%lld %%llu\n", cls, m, h);
        static double buf[3 * 2000000];
        const long long k = ns < m ? ns : m;
        cudaMemcpy(buf, s, 8 * k, cudaMemcpyDeviceToHost);
        cudaMemcpy(buf + k, s + ns, 8 * k, cudaMemcpyDeviceToHost);
        cudaMemcpy(buf + 2 * k, s + 2 * ns, 8 * k, cudaMemcpyDeviceToHost);
        fwrite(&k, 8, 1, f);
        fwrite(buf, 8, 3 * k, f);
    }
    // FP64 -> FP32: three classes (random bits, around the float range, near ties in the subnormal range)
    for (int cls = 0; cls < 3; ++cls) {
        cudaMemset(bad, 0, 8);
        k_cvt<<<1216, 256>>>(cls, n, bad, ns, s, (float *)(s + ns));
        if (cudaDeviceSynchronize() != cudaSuccess) return 2;
        unsigned long long h;
        cudaMemcpy(&h, bad, 8, cudaMemcpyDeviceToHost);
        printf("cvt%%d %%lld %%llu\n", cls, n, h);
        static double bx[2000000];
        static float bq[2000000];
        cudaMemcpy(bx, s, 8 * ns, cudaMemcpyDeviceToHost);
        cudaMemcpy(bq, s + ns, 4 * ns, cudaMemcpyDeviceToHost);
        fwrite(&ns, 8, 1, f);
        fwrite(bx, 8, ns, f);
        fwrite(bq, 4, ns, f);
    }
    fclose(f);
    return 0;
}
'''


@pytest.mark.gpu
def test_integer_fp64_arithmetic_is_ieee(tmp_path):
    src = tmp_path / "fdiv_check.cu"
    src.write_text(SRC % {"header": HEADER})
    exe = tmp_path / "fdiv_check"
    subprocess.check_call([PB._nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", str(exe), str(src)])
    samples = tmp_path / "samples.bin"
    out = subprocess.run([str(exe), "20000000", "400000", str(samples)], capture_output=True, text=True, check=True)
    rows = [line.split() for line in out.stdout.split("\n") if line.strip()]
    assert len(rows) == 8
    for cls, n, bad in rows:
        assert int(bad) == 0, (cls, n, bad)
    raw = np.fromfile(samples, dtype=np.uint8)
    off = 0
    for _ in range(5):
        k = int(raw[off:off + 8].view(np.int64)[0])
        off += 8
        vals = raw[off:off + 24 * k].view(np.float64).reshape(3, k)
        off += 24 * k
        x, d, q = vals
        with np.errstate(all="ignore"):
            ref = x / d
        same = (q.view(np.int64) == ref.view(np.int64)) | (np.isnan(q) & np.isnan(ref))
        assert same.all(), (x[~same][:3], d[~same][:3], q[~same][:3], ref[~same][:3])
    for _ in range(3):
        k = int(raw[off:off + 8].view(np.int64)[0])
        off += 8
        x = raw[off:off + 8 * k].view(np.float64)
        off += 8 * k
        q = raw[off:off + 4 * k].view(np.float32)
        off += 4 * k
        with np.errstate(all="ignore"):
            ref = x.astype(np.float32)
        same = (q.view(np.int32) == ref.view(np.int32)) | (np.isnan(q) & np.isnan(ref))
        assert same.all(), (x[~same][:3], q[~same][:3], ref[~same][:3])
