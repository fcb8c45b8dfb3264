"""Thin ctypes binding of libamgpr.so (C ABI in include/amgpr.h).

The functions keep the C names; every numeric step runs in the library's CUDA
kernels.  PyTorch is only used to own device memory and to name the stream.
There is no CPU fallback: without the compiled library, loading raises.

Method: partial-reuse AMG setup amortisation, arXiv 2108.02054 (Alg. 1 full
setup, Alg. 4 partial reuse, Alg. 3 full reuse, Alg. 2 V-cycle inside CG).
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from .build import LIB_PATH

AMG_OK, AMG_NOT_CONVERGED = 0, 1
AMG_ERR_ARG, AMG_ERR_STATE, AMG_ERR_PATTERN, AMG_ERR_BREAKDOWN = -1, -2, -3, -4
AMG_ERR_NONFINITE, AMG_ERR_CUDA, AMG_ERR_OOM, AMG_ERR_SINGULAR, AMG_ERR_CAPACITY = -5, -6, -7, -8, -9
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", -1: "ERR_ARG", -2: "ERR_STATE", -3: "ERR_PATTERN",
                -4: "ERR_BREAKDOWN", -5: "ERR_NONFINITE", -6: "ERR_CUDA", -7: "ERR_OOM", -8: "ERR_SINGULAR",
                -9: "ERR_CAPACITY"}
SMOOTHER_SPAI0, SMOOTHER_JACOBI = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
MODE_PARTIAL, MODE_FULL_REBUILD, MODE_FULL_REUSE = 0, 1, 2
SOLVER_CG, SOLVER_BICGSTAB = 0, 1

# every entry point declared in include/amgpr.h
EXPORTS = [
    "amg_default_params", "amg_create", "amg_destroy", "amg_last_error", "amg_full_setup", "amg_partial_rebuild",
    "amg_step", "amg_solve", "amg_apply_vcycle", "amg_step_solve_host", "amg_num_levels", "amg_level_sizes",
    "amg_export_csr", "amg_export_level_vec", "amg_export_coarse_lu", "amg_poisson_nnz", "amg_poisson_pattern",
    "amg_poisson_values", "amg_poisson_grad_theta", "amg_profile", "amg_profile_read", "amg_kernel_launches",
    "amg_poisson_pattern_noalloc", "amg_levelset_values", "amg_stokes_values", "amg_poisson_values_log",
    "amg_poisson_grad_log", "amg_pattern_info",
]
PROF_SLOTS = ["cg_spmv", "smooth0_l0", "sweep_l0", "restrict_l0", "prolong_l0", "ap_l0", "rap_l0", "ingest", "lu",
              "inv", "cg_update", "cg_p", "dot", "coarse", "empty", "galerkin", "smoothers"]


class amg_params(ctypes.Structure):
    _fields_ = [
        ("theta", ctypes.c_double), ("omega", ctypes.c_double), ("jacobi_omega", ctypes.c_double),
        ("smoother", ctypes.c_int32), ("npre", ctypes.c_int32), ("npost", ctypes.c_int32),
        ("coarse_enough", ctypes.c_int32), ("max_levels", ctypes.c_int32), ("theta_halving", ctypes.c_int32),
        ("smoothed", ctypes.c_int32), ("precision", ctypes.c_int32), ("mode", ctypes.c_int32),
        ("reuse_iter_limit", ctypes.c_int32), ("maxiter", ctypes.c_int32),
        ("rebuild_every", ctypes.c_int32), ("rebuild_iter_growth", ctypes.c_double),
        ("solver", ctypes.c_int32), ("block_size", ctypes.c_int32),
    ]


class amg_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("rebuilt", ctypes.c_int32), ("nlevels", ctypes.c_int32),
                ("status", ctypes.c_int32), ("rel_resid", ctypes.c_double)]


class AmgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32


def lib():
    """Load libamgpr.so (built by paper_2108_02054_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2108_02054_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            sig = {
                "amg_default_params": (_i32, [ctypes.POINTER(amg_params)]),
                "amg_create": (_i32, [ctypes.POINTER(_vp), ctypes.POINTER(amg_params), _vp]),
                "amg_destroy": (None, [_vp]),
                "amg_last_error": (ctypes.c_char_p, [_vp]),
                "amg_full_setup": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp]),
                "amg_partial_rebuild": (_i32, [_vp, _vp]),
                "amg_step": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp, ctypes.POINTER(amg_info)]),
                "amg_solve": (_i32, [_vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(amg_info)]),
                "amg_apply_vcycle": (_i32, [_vp, _vp, _vp]),
                "amg_step_solve_host": (_i32, [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(amg_info)]),
                "amg_num_levels": (_i32, [_vp, ctypes.POINTER(_i32)]),
                "amg_level_sizes": (_i32, [_vp, _i32, ctypes.POINTER(ctypes.c_int64)]),
                "amg_export_csr": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp]),
                "amg_export_level_vec": (_i32, [_vp, _i32, _vp, _vp, _vp]),
                "amg_export_coarse_lu": (_i32, [_vp, _vp, _vp]),
                "amg_poisson_nnz": (ctypes.c_int64, [_i32, _i32]),
                "amg_poisson_pattern": (_i32, [_i32, _i32, _vp, _vp, _vp]),
                "amg_poisson_values": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp, _vp]),
                "amg_poisson_grad_theta": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp]),
                "amg_profile": (_i32, [_vp, _i32]),
                "amg_profile_read": (_i32, [_vp, _i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
                "amg_kernel_launches": (ctypes.c_int64, []),
                "amg_poisson_pattern_noalloc": (_i32, [_i32, _i32, _vp, _vp, _vp]),
                "amg_levelset_values": (_i32, [_i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
                "amg_stokes_values": (_i32, [_i32, _vp, _vp, _vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp]),
                "amg_poisson_values_log": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp, _vp]),
                "amg_poisson_grad_log": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dptr(t, dtype=None, numel=None) -> int:
    """The device address of a contiguous CUDA tensor, checked against the
    element type and the least element count the call reads or writes (the
    kernels cannot check a buffer's extent)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected a {dtype} tensor, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"expected at least {numel} elements, got {t.numel()}")
    return t.data_ptr()


def _f64(t, numel=None) -> int:
    import torch
    return _dptr(t, torch.float64, numel)


def _i32p(t, numel=None) -> int:
    import torch
    return _dptr(t, torch.int32, numel)


def default_params(**overrides) -> amg_params:
    p = amg_params()
    lib().amg_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


@dataclass
class Info:
    iters: int
    rebuilt: int
    nlevels: int
    status: int
    rel_resid: float


def _info(i: amg_info) -> Info:
    return Info(i.iters, i.rebuilt, i.nlevels, i.status, i.rel_resid)


class AMG:
    """One hierarchy bound to a CUDA stream (owner of an amg_ctx)."""

    def __init__(self, params: amg_params | None = None, stream=None, **overrides):
        self.params = params if params is not None else default_params(**overrides)
        self._stream = _stream(stream)
        h = _vp()
        st = lib().amg_create(ctypes.byref(h), ctypes.byref(self.params), _vp(self._stream))
        if st != AMG_OK:
            raise AmgError(st, "amg_create failed")
        self._h = h
        self.n = 0
        self.nnz = 0

    def close(self):
        if getattr(self, "_h", None):
            lib().amg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, ok=(AMG_OK,)):
        if st not in ok:
            raise AmgError(st, (lib().amg_last_error(self._h) or b"").decode())
        return st

    # ------------------------------------------------------------ Alg. 1 / 3 / 4
    # values per matrix entry and per unknown of the vectors (4 x 4 blocks: 16, 4)
    def _vpe(self) -> int:
        return self.params.block_size * self.params.block_size

    def _vec(self) -> int:
        return self.n * self.params.block_size

    def full_setup(self, ptr, col, val):
        n, nnz = ptr.numel() - 1, col.numel()
        args = (_i32p(ptr), _i32p(col), _f64(val, nnz * self._vpe()))
        self.n, self.nnz = n, nnz
        self._check(lib().amg_full_setup(self._h, n, nnz, *args))

    def partial_rebuild(self, val):
        self._check(lib().amg_partial_rebuild(self._h, _f64(val, self.nnz * self._vpe())))

    def step(self, val, ptr=None, col=None) -> Info:
        info = amg_info()
        if (ptr is None) != (col is None):
            raise ValueError("give both ptr and col, or neither")
        n, nnz = (ptr.numel() - 1, col.numel()) if ptr is not None else (self.n, self.nnz)
        dp = _i32p(ptr) if ptr is not None else None
        dc = _i32p(col) if col is not None else None
        dv = _f64(val, nnz * self._vpe())
        self.n, self.nnz = n, nnz
        self._check(lib().amg_step(self._h, n, nnz, dp, dc, dv, ctypes.byref(info)))
        return _info(info)

    def solve(self, f, tol: float = 1e-8, u=None, allow_not_converged: bool = True):
        import torch
        if u is None:
            u = torch.empty_like(f)
        info = amg_info()
        ok = (AMG_OK, AMG_NOT_CONVERGED) if allow_not_converged else (AMG_OK,)
        self._check(lib().amg_solve(self._h, _f64(f, self._vec()), _f64(u, self._vec()), float(tol),
                                    ctypes.byref(info)), ok)
        return u, _info(info)

    def vcycle(self, r, z=None):
        import torch
        if z is None:
            z = torch.empty_like(r)
        self._check(lib().amg_apply_vcycle(self._h, _f64(r, self._vec()), _f64(z, self._vec())))
        return z

    def step_solve_host(self, h_val: np.ndarray, h_f: np.ndarray, h_u: np.ndarray, tol: float = 1e-8) -> Info:
        """Host buffers in and out (copies inside the call)."""
        info = amg_info()
        for a, need in ((h_val, self.nnz * self._vpe()), (h_f, self._vec()), (h_u, self._vec())):
            if a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError("host buffers must be contiguous float64")
            if a.size < need:
                raise ValueError(f"host buffer of {a.size} elements, the call copies {need}")
        self._check(lib().amg_step_solve_host(self._h, h_val.ctypes.data, h_f.ctypes.data, h_u.ctypes.data,
                                              float(tol), ctypes.byref(info)), (AMG_OK, AMG_NOT_CONVERGED))
        return _info(info)

    # ------------------------------------------------------------ inspection
    @property
    def nlevels(self) -> int:
        n = _i32()
        self._check(lib().amg_num_levels(self._h, ctypes.byref(n)))
        return n.value

    def level_sizes(self, level: int):
        s = (ctypes.c_int64 * 6)()
        self._check(lib().amg_level_sizes(self._h, level, s))
        return [int(x) for x in s]

    def pattern_info(self):
        """(column bytes per entry the finest level's kernels read, offset-table size)."""
        cb, no = _i32(), _i32()
        self._check(lib().amg_pattern_info(self._h, ctypes.byref(cb), ctypes.byref(no)))
        return cb.value, no.value

    def export_level(self, level: int) -> dict:
        """Copies of A, P, R (CSR), aggregates, strong flags and smoother on the host."""
        import torch
        n, nnzA, nnzP, nnzR, nnzAP, nagg = self.level_sizes(level)
        dev = torch.device("cuda", torch.cuda.current_device())
        out = {"n": n, "nagg": nagg, "nnzAP": nnzAP}
        bw = 16 if self.params.block_size == 4 else 1   # values per entry of A / per node of m
        for which, name, nrows, nnz in ((0, "A", n, nnzA), (1, "P", n, nnzP), (2, "R", nagg, nnzR)):
            if which > 0 and nnzP == 0:
                out[name] = None
                continue
            ptr = torch.empty(nrows + 1, dtype=torch.int32, device=dev)
            col = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
            w = bw if which == 0 else 1
            val = torch.empty(max(nnz, 1) * w, dtype=torch.float64, device=dev)
            self._check(lib().amg_export_csr(self._h, level, which, _dptr(ptr), _dptr(col), _dptr(val)))
            v = val[:nnz * w].cpu().numpy()
            out[name] = (ptr.cpu().numpy(), col[:nnz].cpu().numpy(), v.reshape(nnz, 16) if w == 16 else v)
        agg = torch.empty(n, dtype=torch.int32, device=dev)
        strong = torch.empty(max(nnzA, 1), dtype=torch.uint8, device=dev)
        m = torch.zeros(n * bw, dtype=torch.float64, device=dev)
        self._check(lib().amg_export_level_vec(self._h, level, _dptr(agg), _dptr(strong), _dptr(m)))
        out["agg"] = agg.cpu().numpy()
        out["strong"] = strong[:nnzA].cpu().numpy()
        out["m"] = m.cpu().numpy().reshape(n, 16) if bw == 16 else m.cpu().numpy()
        return out

    def profile(self, enable=True):
        """Per-kernel timing: True / 1 (unrolled graph), 2 (host-driven loop), False / 0 off."""
        self._check(lib().amg_profile(self._h, int(enable)))

    def profile_read(self) -> dict:
        """{slot name: (total ms, timed launches)} since the last read."""
        out = {}
        for k, name in enumerate(PROF_SLOTS):
            ms = ctypes.c_double()
            cnt = ctypes.c_int64()
            self._check(lib().amg_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(cnt)))
            out[name] = (ms.value, cnt.value)
        return out

    def coarse_lu(self):
        import torch
        nL = self.level_sizes(self.nlevels - 1)[0] * self.params.block_size
        lu = torch.empty(nL * nL, dtype=torch.float64, device="cuda")
        piv = torch.empty(nL, dtype=torch.int32, device="cuda")
        self._check(lib().amg_export_coarse_lu(self._h, _dptr(lu), _dptr(piv)))
        return lu.view(nL, nL).cpu().numpy(), piv.cpu().numpy()


# ---------------------------------------------------------------- workload assembly
def kernel_launches() -> int:
    """Kernels launched by libamgpr.so in this process so far."""
    return int(lib().amg_kernel_launches())


def poisson_nnz(dim: int, N: int) -> int:
    return int(lib().amg_poisson_nnz(dim, N))


def poisson_pattern(dim: int, N: int, stream=None):
    """Device CSR pattern (ptr, col) of the N^dim cell-grid pressure Poisson."""
    import torch
    n = N ** dim
    ptr = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(poisson_nnz(dim, N), dtype=torch.int32, device="cuda")
    st = lib().amg_poisson_pattern(dim, N, _dptr(ptr), _dptr(col), _vp(_stream(stream)))
    if st != AMG_OK:
        raise AmgError(st, "amg_poisson_pattern failed")
    return ptr, col


def poisson_values(dim: int, N: int, rho, ptr, dirichlet_top: bool = True, out=None, stream=None):
    """Device values of -div((1/rho) grad p) on the pattern from poisson_pattern."""
    import torch
    nnz, n = poisson_nnz(dim, N), N ** dim
    val = out if out is not None else torch.empty(nnz, dtype=torch.float64, device="cuda")
    st = lib().amg_poisson_values(dim, N, int(dirichlet_top), _f64(rho, n), _i32p(ptr, n + 1), _f64(val, nnz),
                                  _vp(_stream(stream)))
    if st != AMG_OK:
        raise AmgError(st, "amg_poisson_values failed")
    return val


def poisson_values_log(dim: int, N: int, theta, ptr, dirichlet_top: bool = True, out=None, stream=None):
    """poisson_values for rho = exp(theta), the exponential taken in the kernel."""
    import torch
    nnz, n = poisson_nnz(dim, N), N ** dim
    val = out if out is not None else torch.empty(nnz, dtype=torch.float64, device="cuda")
    st = lib().amg_poisson_values_log(dim, N, int(dirichlet_top), _f64(theta, n), _i32p(ptr, n + 1),
                                      _f64(val, nnz), _vp(_stream(stream)))
    if st != AMG_OK:
        raise AmgError(st, "amg_poisson_values_log failed")
    return val


def levelset_values(dim: int, N: int, fx, fy, fz, ptr, out=None, stream=None):
    """Device values of the upwind convection-diffusion (level-set) matrix on
    the pattern from poisson_pattern; fx, fy, fz are the face velocities (fz
    is ignored in 2D)."""
    import torch
    nnz, n = poisson_nnz(dim, N), N ** dim
    val = out if out is not None else torch.empty(nnz, dtype=torch.float64, device="cuda")
    faces = n // N * (N + 1)  # face values per direction: (N + 1) N^(dim - 1)
    fz_p = _f64(fz, faces) if dim == 3 else (_dptr(fz) if fz is not None and fz.numel() > 0 else 0)
    st = lib().amg_levelset_values(dim, N, _f64(fx, faces), _f64(fy, faces), fz_p, _i32p(ptr, n + 1),
                                   _f64(val, nnz), _vp(_stream(stream)))
    if st != AMG_OK:
        raise AmgError(st, "amg_levelset_values failed")
    return val


def stokes_values(N: int, rho, mu, fx, fy, fz, mass: float, ptr, out=None, stream=None):
    """Device block values (nnz x 16) of the 4 x 4 monolithic Navier-Stokes
    stand-in on the pattern from poisson_pattern(3, N)."""
    import torch
    nnz, n = poisson_nnz(3, N), N ** 3
    faces = N * N * (N + 1)
    val = out if out is not None else torch.empty((nnz, 16), dtype=torch.float64, device="cuda")
    st = lib().amg_stokes_values(N, _f64(rho, n), _f64(mu, n), _f64(fx, faces), _f64(fy, faces), _f64(fz, faces),
                                 float(mass), _i32p(ptr, n + 1), _f64(val, 16 * nnz), _vp(_stream(stream)))
    if st != AMG_OK:
        raise AmgError(st, "amg_stokes_values failed")
    return val


def block_params(**overrides) -> amg_params:
    """The paper's configuration for the 4 x 4 block systems (Sec. 4):
    non-smoothed aggregation, damped block Jacobi, BiCGStab, FP64."""
    kw = dict(block_size=4, smoothed=0, smoother=SMOOTHER_JACOBI, solver=SOLVER_BICGSTAB, precision=PREC_FP64)
    kw.update(overrides)
    return default_params(**kw)


def poisson_grad_theta(dim: int, N: int, rho, u, lam, dirichlet_top: bool = True, stream=None):
    import torch
    n = N ** dim
    g = torch.empty_like(u)
    st = lib().amg_poisson_grad_theta(dim, N, int(dirichlet_top), _f64(rho, n), _f64(u, n), _f64(lam, n),
                                      _f64(g, n), _vp(_stream(stream)))
    if st != AMG_OK:
        raise AmgError(st, "amg_poisson_grad_theta failed")
    return g


def poisson_grad_log(dim: int, N: int, theta, u, lam, dirichlet_top: bool = True, stream=None):
    """dL/dtheta per cell for rho = exp(theta) (the exponential taken in the kernel)."""
    import torch
    n = N ** dim
    g = torch.empty_like(u)
    st = lib().amg_poisson_grad_log(dim, N, int(dirichlet_top), _f64(theta, n), _f64(u, n), _f64(lam, n),
                                    _f64(g, n), _vp(_stream(stream)))
    if st != AMG_OK:
        raise AmgError(st, "amg_poisson_grad_log failed")
    return g
