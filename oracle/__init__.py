"""CPU FP64 oracle for partial-reuse smoothed-aggregation AMG (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg import this package; the product library never does.  The C
source (amg_oracle.c) is compiled on first use with gcc, FP contraction off.

Every function cites the part of the paper it follows (arXiv 2108.02054):
  Alg. 1  full setup                  -> Hierarchy(...)
  Alg. 4  partial reuse update        -> Hierarchy.rebuild(values)
  Alg. 2  V-cycle (one per PCG step)  -> Hierarchy.vcycle(r)
  Sec. 4  Krylov solve                -> Hierarchy.pcg / Hierarchy.bicgstab
  Sec. 4  4 x 4 block systems         -> BlockHierarchy (non-smoothed aggregation,
                                         damped block Jacobi, BiCGStab)
  Alg. 3  full reuse / no reuse modes -> run_time_steps(...)
Parity: every function is pinned by tests under tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, NOT_CONVERGED = 0, 1
ERR_ARG, ERR_STATE, ERR_PATTERN, ERR_BREAKDOWN, ERR_SINGULAR = -1, -2, -3, -4, -8


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_poisson_nnz.restype = ctypes.c_longlong
            L.orc_poisson_nnz.argtypes = [ctypes.c_int, ctypes.c_int]
            L.orc_poisson_assemble.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _f64p, _i32p, _i32p, _f64p]
            L.orc_poisson_grad_theta.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _f64p, _f64p, _f64p, _f64p]
            L.orc_priority.restype = ctypes.c_uint32
            L.orc_priority.argtypes = [ctypes.c_uint32]
            L.orc_setup.restype = ctypes.c_void_p
            L.orc_setup.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _i32p, ctypes.POINTER(ctypes.c_int)]
            L.orc_rebuild.argtypes = [ctypes.c_void_p, _f64p]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_vcycle.argtypes = [ctypes.c_void_p, _f64p, _f64p]
            L.orc_pcg.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _f64p, _f64p, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
            L.orc_nlevels.argtypes = [ctypes.c_void_p]
            L.orc_level_sizes.argtypes = [ctypes.c_void_p, ctypes.c_int, _i64p]
            L.orc_export_csr.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]
            L.orc_export_level_vec.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p]
            L.orc_export_lu.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_levelset_assemble.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, _i32p, _i32p, _f64p]
            L.orc_bicgstab.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _f64p, _f64p, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
            L.orc_stokes_assemble.argtypes = [ctypes.c_int, _f64p, _f64p, _f64p, _f64p, _f64p, ctypes.c_double,
                                              _i32p, _i32p, _f64p]
            L.orc_block_norm.restype = ctypes.c_double
            L.orc_block_norm.argtypes = [_f64p]
            L.orc_inv4.argtypes = [_f64p, _f64p]
            L.orc_block_setup.restype = ctypes.c_void_p
            L.orc_block_setup.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _i32p,
                                          ctypes.POINTER(ctypes.c_int)]
            L.orc_block_rebuild.argtypes = [ctypes.c_void_p, _f64p]
            L.orc_block_destroy.argtypes = [ctypes.c_void_p]
            L.orc_block_vcycle.argtypes = [ctypes.c_void_p, _f64p, _f64p]
            L.orc_block_bicgstab.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _f64p, _f64p, ctypes.c_double,
                                             ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_double)]
            L.orc_block_nlevels.argtypes = [ctypes.c_void_p]
            L.orc_block_level_sizes.argtypes = [ctypes.c_void_p, ctypes.c_int, _i64p]
            L.orc_block_export_csr.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]
            L.orc_block_export_vec.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]
            L.orc_block_export_lu.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_dense_lu.argtypes = [ctypes.c_int, _f64p, _i32p]
            L.orc_dense_lu_solve.argtypes = [ctypes.c_int, _f64p, _i32p, _f64p, _f64p]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


# --------------------------------------------------------------------------
# Problem assembly (the synthetic stand-in for the Sec. 4 dam-break matrices)

def poisson_assemble(dim: int, N: int, rho: np.ndarray, dirichlet_top: bool = True):
    """CSR (ptr, col, val) of -div((1/rho) grad p): harmonic face coefficients,
    Dirichlet top face through a ghost cell, Neumann elsewhere."""
    L = lib()
    n = N ** dim
    nnz = int(L.orc_poisson_nnz(dim, N))
    ptr = np.zeros(n + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz, np.float64)
    st = L.orc_poisson_assemble(dim, N, int(dirichlet_top), np.ascontiguousarray(rho, np.float64), ptr, col, val)
    if st != OK:
        raise ValueError(f"assembly failed: {st}")
    return ptr, col, val


def levelset_assemble(dim: int, N: int, fx, fy, fz):
    """CSR of the level-set transport step (implicit upwind convection with
    diffusion, the stand-in for eq. 5) on the pressure pattern."""
    L = lib()
    n = N ** dim
    nnz = int(L.orc_poisson_nnz(dim, N))
    ptr = np.zeros(n + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz, np.float64)
    fx, fy, fz = (np.ascontiguousarray(a, np.float64) for a in (fx, fy, fz))
    st = L.orc_levelset_assemble(dim, N, _ptr(fx), _ptr(fy), _ptr(fz) if fz.size else None, ptr, col, val)
    if st != OK:
        raise ValueError(f"assembly failed: {st}")
    return ptr, col, val


def poisson_grad_theta(dim, N, rho, u, lam, dirichlet_top=True):
    """dL/dtheta for theta = log rho, given the forward solution u and the
    adjoint solution lam of A lam = dL/du."""
    g = np.zeros(N ** dim, np.float64)
    lib().orc_poisson_grad_theta(dim, N, int(dirichlet_top), np.ascontiguousarray(rho, np.float64),
                                 np.ascontiguousarray(u, np.float64), np.ascontiguousarray(lam, np.float64), g)
    return g


def stokes_assemble(N: int, rho, mu, fx, fy, fz, mass: float):
    """Block CSR (ptr, col, val[nnz, 16]) of the synthetic monolithic Oseen-type
    system (the stand-in for the Sec. 4 Navier-Stokes matrices, 4 x 4 blocks
    (u, v, w, p) per cell) on the N^3 pressure pattern."""
    L = lib()
    n = N ** 3
    nnz = int(L.orc_poisson_nnz(3, N))
    ptr = np.zeros(n + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(16 * nnz, np.float64)
    a = [np.ascontiguousarray(x, np.float64) for x in (rho, mu, fx, fy, fz)]
    st = L.orc_stokes_assemble(N, *a, float(mass), ptr, col, val)
    if st != OK:
        raise ValueError(f"assembly failed: {st}")
    return ptr, col, val.reshape(nnz, 16)


def block_norm(b) -> float:
    """Frobenius norm of a 4 x 4 block, as the block hierarchy computes it."""
    return float(lib().orc_block_norm(np.ascontiguousarray(b, np.float64).reshape(16)))


def inv4(a):
    """(inverse, ok) of a 4 x 4 block by the hierarchy's Gauss-Jordan routine."""
    inv = np.zeros(16, np.float64)
    ok = lib().orc_inv4(np.ascontiguousarray(a, np.float64).reshape(16), inv)
    return inv.reshape(4, 4), bool(ok)


def priority(i: int) -> int:
    """Fixed aggregation priority of node i (murmur3 32-bit finaliser)."""
    return int(lib().orc_priority(ctypes.c_uint32(i)))


def dense_lu(a: np.ndarray):
    a = np.array(a, np.float64, order="C")
    piv = np.zeros(a.shape[0], np.int32)
    st = lib().orc_dense_lu(a.shape[0], a, piv)
    return a, piv, st


def dense_lu_solve(lu, piv, b):
    x = np.zeros_like(b, dtype=np.float64)
    lib().orc_dense_lu_solve(lu.shape[0], np.ascontiguousarray(lu), np.ascontiguousarray(piv),
                             np.ascontiguousarray(b, np.float64), x)
    return x


# --------------------------------------------------------------------------
@dataclass
class Params:
    """AMG parameters.  Defaults: theta = 0.08 halved per level, omega = 2/3,
    SPAI0, one pre- and one post-sweep, coarse_enough = 256, 20 levels."""

    theta: float = 0.08
    omega: float = 2.0 / 3.0
    jacobi_omega: float = 0.72
    smoother: int = 0          # 0 SPAI0, 1 damped Jacobi
    npre: int = 1
    npost: int = 1
    coarse_enough: int = 256
    max_levels: int = 20
    theta_halving: int = 1
    smoothed: int = 1          # 1 smoothed aggregation, 0 plain aggregation

    def arrays(self):
        d = np.array([self.theta, self.omega, self.jacobi_omega], np.float64)
        i = np.array([self.smoother, self.npre, self.npost, self.coarse_enough, self.max_levels,
                      self.theta_halving, self.smoothed], np.int32)
        return d, i


@dataclass
class CSR:
    ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    ncols: int = 0

    @property
    def nrows(self):
        return self.ptr.size - 1

    def dense(self):
        D = np.zeros((self.nrows, self.ncols))
        for i in range(self.nrows):
            for p in range(self.ptr[i], self.ptr[i + 1]):
                D[i, self.col[p]] += self.val[p]
        return D

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.ptr), shape=(self.nrows, self.ncols))


@dataclass
class Level:
    A: CSR
    P: CSR | None
    R: CSR | None
    AP: CSR | None
    agg: np.ndarray
    strong: np.ndarray
    m: np.ndarray
    nagg: int = 0


class Hierarchy:
    """Alg. 1 full setup on construction; rebuild() is the Alg. 4 update."""

    def __init__(self, ptr, col, val, params: Params | None = None, allow_singular: bool = False):
        self.params = params or Params()
        L = lib()
        self._ptr = np.ascontiguousarray(ptr, np.int32)
        self._col = np.ascontiguousarray(col, np.int32)
        d, i = self.params.arrays()
        st = ctypes.c_int(0)
        h = L.orc_setup(int(self._ptr.size - 1), self._ptr, self._col, np.ascontiguousarray(val, np.float64),
                        d, i, ctypes.byref(st))
        self.status = st.value
        if not h:
            raise ValueError(f"oracle setup failed: status {st.value}")
        if st.value == ERR_SINGULAR and not allow_singular:
            L.orc_destroy(h)
            raise ValueError("oracle setup: coarsest matrix singular")
        self._h = h
        self.n = int(self._ptr.size - 1)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def nlevels(self) -> int:
        return int(lib().orc_nlevels(self._h))

    def sizes(self, l: int):
        s = np.zeros(6, np.int64)
        lib().orc_level_sizes(self._h, l, s)
        return s

    def _csr(self, l, which, nrows, nnz, ncols):
        ptr = np.zeros(nrows + 1, np.int32)
        col = np.zeros(nnz, np.int32)
        val = np.zeros(nnz, np.float64)
        lib().orc_export_csr(self._h, l, which, _ptr(ptr), _ptr(col), _ptr(val))
        return CSR(ptr, col, val, ncols)

    def level(self, l: int) -> Level:
        n, nnzA, nnzP, nnzR, nnzAP, nagg = (int(x) for x in self.sizes(l))
        A = self._csr(l, 0, n, nnzA, n)
        P = R = AP = None
        if l < self.nlevels - 1:
            P = self._csr(l, 1, n, nnzP, nagg)
            R = self._csr(l, 2, nagg, nnzR, n)
            AP = self._csr(l, 3, n, nnzAP, nagg)
        agg = np.zeros(n, np.int32)
        strong = np.zeros(nnzA, np.uint8)
        m = np.zeros(n, np.float64)
        lib().orc_export_level_vec(self._h, l, _ptr(agg), _ptr(strong), _ptr(m))
        return Level(A, P, R, AP, agg, strong, m, nagg)

    def lu(self):
        nL = int(self.sizes(self.nlevels - 1)[0])
        lu = np.zeros((nL, nL), np.float64)
        piv = np.zeros(nL, np.int32)
        lib().orc_export_lu(self._h, _ptr(lu), _ptr(piv))
        return lu, piv

    def rebuild(self, val) -> int:
        """Alg. 4: smoothers and Galerkin operators from new fine values."""
        return int(lib().orc_rebuild(self._h, np.ascontiguousarray(val, np.float64)))

    def vcycle(self, r) -> np.ndarray:
        """Alg. 2, one cycle from a zero initial guess."""
        z = np.zeros(self.n, np.float64)
        lib().orc_vcycle(self._h, np.ascontiguousarray(r, np.float64), z)
        return z

    def bicgstab(self, f, tol=1e-8, maxiter=100, sys_val=None):
        """BiCGStab (Sec. 4) right-preconditioned by one V-cycle; (u, iters, relres, status)."""
        u = np.zeros(self.n, np.float64)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        sv = None if sys_val is None else np.ascontiguousarray(sys_val, np.float64)
        st = lib().orc_bicgstab(self._h, _ptr(sv), np.ascontiguousarray(f, np.float64), u, float(tol), int(maxiter),
                                ctypes.byref(it), ctypes.byref(rr))
        return u, it.value, rr.value, int(st)

    def pcg(self, f, tol=1e-8, maxiter=100, sys_val=None):
        """CG preconditioned with one V-cycle; returns (u, iters, relres, status)."""
        u = np.zeros(self.n, np.float64)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        sv = None if sys_val is None else np.ascontiguousarray(sys_val, np.float64)
        st = lib().orc_pcg(self._h, _ptr(sv), np.ascontiguousarray(f, np.float64), u, float(tol), int(maxiter),
                           ctypes.byref(it), ctypes.byref(rr))
        return u, it.value, rr.value, int(st)


# --------------------------------------------------------------------------
# Block-valued (4 x 4) hierarchy (Sec. 4, the monolithic Navier-Stokes systems)

def block_params(**kw) -> Params:
    """The paper's configuration for the block systems: non-smoothed
    aggregation, damped Jacobi (coarse_enough counts nodes)."""
    kw.setdefault("smoother", 1)
    kw.setdefault("smoothed", 0)
    return Params(**kw)


@dataclass
class BlockLevel:
    A: CSR              # val: (nnz, 16) block values
    P: CSR | None
    R: CSR | None
    agg: np.ndarray
    strong: np.ndarray
    minv: np.ndarray     # (n, 16) damped block-Jacobi inverses
    norms: np.ndarray    # block norms of the node graph (setup values)
    nagg: int = 0


class BlockHierarchy:
    """Alg. 1 on a 4 x 4 block matrix (node graph of block norms,
    non-smoothed aggregation, damped block Jacobi); rebuild() is Alg. 4."""

    def __init__(self, ptr, col, bval, params: Params | None = None):
        self.params = params or block_params()
        L = lib()
        self._ptr = np.ascontiguousarray(ptr, np.int32)
        self._col = np.ascontiguousarray(col, np.int32)
        d, i = self.params.arrays()
        st = ctypes.c_int(0)
        h = L.orc_block_setup(int(self._ptr.size - 1), self._ptr, self._col,
                              np.ascontiguousarray(bval, np.float64).reshape(-1), d, i, ctypes.byref(st))
        self.status = st.value
        if not h:
            raise ValueError(f"oracle block setup failed: status {st.value}")
        if st.value == ERR_SINGULAR:
            L.orc_block_destroy(h)
            raise ValueError("oracle block setup: coarsest matrix singular")
        self._h = h
        self.nodes = int(self._ptr.size - 1)
        self.n = 4 * self.nodes

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_block_destroy(h)
            self._h = None

    @property
    def nlevels(self) -> int:
        return int(lib().orc_block_nlevels(self._h))

    def sizes(self, l: int):
        s = np.zeros(6, np.int64)
        lib().orc_block_level_sizes(self._h, l, s)
        return s

    def level(self, l: int) -> BlockLevel:
        n, nnzA, nnzP, nnzR, _, nagg = (int(x) for x in self.sizes(l))

        def csr(which, nrows, nnz, ncols, width):
            ptr = np.zeros(nrows + 1, np.int32)
            col = np.zeros(nnz, np.int32)
            val = np.zeros(nnz * width, np.float64)
            lib().orc_block_export_csr(self._h, l, which, _ptr(ptr), _ptr(col), _ptr(val))
            return CSR(ptr, col, val.reshape(nnz, 16) if width == 16 else val, ncols)

        A = csr(0, n, nnzA, n, 16)
        P = R = None
        if l < self.nlevels - 1:
            P = csr(1, n, nnzP, nagg, 1)
            R = csr(2, nagg, nnzR, n, 1)
        agg = np.zeros(n, np.int32)
        strong = np.zeros(nnzA, np.uint8)
        minv = np.zeros(16 * n, np.float64)
        norms = np.zeros(nnzA, np.float64)
        lib().orc_block_export_vec(self._h, l, _ptr(agg), _ptr(strong), _ptr(minv), _ptr(norms))
        return BlockLevel(A, P, R, agg, strong, minv.reshape(n, 16), norms, nagg)

    def lu(self):
        nL = 4 * int(self.sizes(self.nlevels - 1)[0])
        lu = np.zeros((nL, nL), np.float64)
        piv = np.zeros(nL, np.int32)
        lib().orc_block_export_lu(self._h, _ptr(lu), _ptr(piv))
        return lu, piv

    def rebuild(self, bval) -> int:
        return int(lib().orc_block_rebuild(self._h, np.ascontiguousarray(bval, np.float64).reshape(-1)))

    def vcycle(self, r) -> np.ndarray:
        z = np.zeros(self.n, np.float64)
        lib().orc_block_vcycle(self._h, np.ascontiguousarray(r, np.float64), z)
        return z

    def bicgstab(self, f, tol=1e-8, maxiter=100, sys_val=None):
        """BiCGStab on the 4n unknowns, one block V-cycle per preconditioner
        application; (u, iters, relres, status)."""
        u = np.zeros(self.n, np.float64)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        sv = None if sys_val is None else np.ascontiguousarray(sys_val, np.float64).reshape(-1)
        st = lib().orc_block_bicgstab(self._h, _ptr(sv), np.ascontiguousarray(f, np.float64), u, float(tol),
                                      int(maxiter), ctypes.byref(it), ctypes.byref(rr))
        return u, it.value, rr.value, int(st)


def block_to_scipy(ptr, col, bval, ncols=None):
    """The expanded scalar matrix of a block CSR (4n x 4n), for the pins."""
    import scipy.sparse as sp
    n = ptr.size - 1
    ncols = n if ncols is None else ncols
    return sp.bsr_matrix((np.asarray(bval).reshape(-1, 4, 4), col, ptr), shape=(4 * n, 4 * ncols)).tocsr()


# --------------------------------------------------------------------------
MODE_PARTIAL, MODE_FULL_REBUILD, MODE_FULL_REUSE = 0, 1, 2


@dataclass
class StepRecord:
    step: int
    iters: int
    relres: float
    status: int
    rebuilt: bool
    u: np.ndarray | None = field(default=None, repr=False)


def run_time_steps(ptr, col, values_per_step, f, mode=MODE_PARTIAL, params=None, tol=1e-8, maxiter=100,
                   reuse_iter_limit=None, keep_u=False, rebuild_every=0, rebuild_iter_growth=0.0, solver="cg",
                   block=False):
    """Time loop of Alg. 3 (full reuse), Alg. 4 (partial reuse) or no reuse.

    Full reuse rebuilds when the previous step's solve did not converge within
    reuse_iter_limit iterations (default: maxiter), Sec. 3.  Partial reuse may
    add preventive full rebuilds (Sec. 3): every rebuild_every steps, or when
    the previous solve needed more than rebuild_iter_growth times the
    iterations of the first solve after the last full setup."""
    limit = maxiter if reuse_iter_limit is None else reuse_iter_limit
    recs = []
    H = None
    last_ok = True
    last_it = 0
    since_full = 0
    base_it = -1
    for k, val in enumerate(values_per_step):
        rebuilt = False
        preventive = mode == MODE_PARTIAL and k > 0 and (
            (rebuild_every > 0 and since_full + 1 >= rebuild_every)
            or (rebuild_iter_growth > 0 and base_it > 0 and last_it > rebuild_iter_growth * base_it))
        if k == 0 or mode == MODE_FULL_REBUILD or (mode == MODE_FULL_REUSE and not last_ok) or preventive:
            H = BlockHierarchy(ptr, col, val, params) if block else Hierarchy(ptr, col, val, params)
            rebuilt = True
            since_full = 0
            base_it = -1
        elif mode == MODE_PARTIAL:
            st = H.rebuild(val)
            if st != OK:
                raise RuntimeError(f"rebuild failed: {st}")
            since_full += 1
        solve = H.pcg if solver == "cg" else H.bicgstab
        u, it, rr, st = solve(f, tol, maxiter, sys_val=val)
        last_ok = (st == OK) and it <= limit
        last_it = it
        if base_it < 0 and st == OK:
            base_it = it
        recs.append(StepRecord(k, it, rr, st, rebuilt, u if keep_u else None))
    return recs
