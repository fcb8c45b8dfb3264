"""Seeded synthetic inputs for the collapsing-water-column pressure Poisson problems.

This module only draws random numbers and evaluates the problem geometry; it
contains none of the AMG arithmetic, so both the CUDA path and the CPU oracle
take their inputs from here.

The paper's measurements (Sec. 4) use matrices from a two-fluid dam-break
simulation that are not available; these fields stand in for them: a water
column (density 1000) in air (density 1) that collapses over T time steps, so
the matrix values change every step while the sparsity pattern stays fixed,
which is the situation the partial-reuse strategy targets (Sec. 3).

Geometry: unit square / cube, N cells per side, cell centre (i + 1/2)/N, cell
index x + N*y (+ N^2*z).  Water occupies {x < a(t), y < h(t)} in 2D and
{x < a(t), z < h(t)} in 3D with a(t) = 0.25 + 0.5 t/T, h(t) = 0.125/a(t),
t = k for k = 0..T-1 (strict inequalities: a centre on the line is air).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

RHO_WATER = 1000.0
RHO_AIR = 1.0


@dataclass(frozen=True)
class Workload:
    """One of the synthetic problem configurations."""

    name: str
    dim: int
    N: int
    T: int
    precision: str  # "fp64" or "mixed"

    @property
    def n(self) -> int:
        return self.N ** self.dim

    @property
    def nnz(self) -> int:
        N = self.N
        if self.dim == 2:
            return N * N + 4 * (N - 1) * N
        return N ** 3 + 6 * (N - 1) * N * N


WORKLOADS = {
    "2d32": Workload("2d32", 2, 32, 10, "fp64"),
    "3d64": Workload("3d64", 3, 64, 50, "fp64"),
    "3d128": Workload("3d128", 3, 128, 100, "mixed"),
    "3d192": Workload("3d192", 3, 192, 100, "mixed"),
    "3d64grad": Workload("3d64grad", 3, 64, 1, "fp64"),
}


def water_mask(dim: int, N: int, k: int, T: int) -> np.ndarray:
    """Boolean mask of water cells at time step k of T (flattened, x fastest)."""
    c = (np.arange(N, dtype=np.float64) + 0.5) / N
    a = 0.25 + 0.5 * k / T
    h = 0.125 / a
    inx = c < a
    iny = c < h
    if dim == 2:
        m = iny[:, None] & inx[None, :]  # [y, x]
    else:
        m = iny[:, None, None] & np.ones(N, dtype=bool)[None, :, None] & inx[None, None, :]  # [z, y, x]
    return m.reshape(-1)


def density(dim: int, N: int, k: int, T: int) -> np.ndarray:
    """Per-cell density rho at step k: 1000 in the water column, 1 elsewhere."""
    return np.where(water_mask(dim, N, k, T), RHO_WATER, RHO_AIR).astype(np.float64)


def rhs(n: int, seed: int = 0) -> np.ndarray:
    """Right-hand side f ~ U[-1, 1], the same vector at every step."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


def noisy_log_density(dim: int, N: int, seed: int = 1, sigma: float = 0.1) -> np.ndarray:
    """theta = log rho(t=0) + N(0, sigma^2): the differentiable-solve input."""
    theta0 = np.log(density(dim, N, 0, 1))
    return theta0 + np.random.default_rng(seed).normal(0.0, sigma, theta0.size)


def target_log_density(theta: np.ndarray, seed: int = 2, sigma: float = 0.1) -> np.ndarray:
    """Perturbed field whose solution serves as u_target."""
    return theta + np.random.default_rng(seed).normal(0.0, sigma, theta.size)


def fd_cells(n: int, count: int = 32, seed: int = 3) -> np.ndarray:
    """Distinct cell indices for the finite-difference gradient check."""
    return np.sort(np.random.default_rng(seed).choice(n, size=count, replace=False)).astype(np.int64)


def random_spd_like(n: int, density_: float, seed: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """A random symmetric, diagonally dominant sparse matrix in sorted CSR form
    (an irregular pattern for the edge-case tests)."""
    rng = np.random.default_rng(seed)
    upper = (rng.random((n, n)) < density_)
    upper = np.triu(upper, 1)
    w = -rng.uniform(0.01, 1.0, (n, n)) * upper
    M = w + w.T
    d = -M.sum(axis=1) + rng.uniform(0.0, 0.5, n) + 1e-3
    M[np.arange(n), np.arange(n)] = d
    ptr = [0]
    col = []
    val = []
    for i in range(n):
        nz = np.nonzero(M[i])[0]
        col.extend(nz.tolist())
        val.extend(M[i, nz].tolist())
        ptr.append(len(col))
    return np.asarray(ptr, np.int32), np.asarray(col, np.int32), np.asarray(val, np.float64)


def random_arrow_spd(n: int, density_: float, arm: int, seed: int):
    """random_spd_like plus one dense 'arrow' row and column (node 0 coupled to
    `arm` random nodes): rows far longer than a stencil's, for the edge cases
    of the row-length-dependent kernels.  Sorted CSR (ptr, col, val)."""
    ptr, col, val = random_spd_like(n, density_, seed)
    rng = np.random.default_rng(seed + 1000)
    M = np.zeros((n, n))
    for i in range(n):
        M[i, col[ptr[i]:ptr[i + 1]]] = val[ptr[i]:ptr[i + 1]]
    np.fill_diagonal(M, 0.0)
    nb = rng.choice(np.arange(1, n), size=arm, replace=False)
    w = -rng.uniform(0.01, 0.5, arm)
    M[0, nb] += w
    M[nb, 0] += w
    d = -M.sum(axis=1) + rng.uniform(0.0, 0.5, n) + 1e-3
    M[np.arange(n), np.arange(n)] = d
    p, c, v = [0], [], []
    for i in range(n):
        nz = np.nonzero(M[i])[0]
        c.extend(nz.tolist())
        v.extend(M[i, nz].tolist())
        p.append(len(c))
    return np.asarray(p, np.int32), np.asarray(c, np.int32), np.asarray(v, np.float64)


def random_banded_spd(n: int, band: int, density_: float, seed: int):
    """A random symmetric, diagonally dominant matrix whose entries lie within
    `band` of the diagonal (so its rows use at most 2 band + 1 distinct column
    offsets), in sorted CSR form."""
    rng = np.random.default_rng(seed)
    i, j = np.triu_indices(n, 1)
    keep = (j - i <= band) & (rng.random(i.size) < density_)
    M = np.zeros((n, n))
    w = -rng.uniform(0.01, 1.0, keep.sum())
    M[i[keep], j[keep]] = w
    M = M + M.T
    M[np.arange(n), np.arange(n)] = -M.sum(axis=1) + rng.uniform(0.0, 0.5, n) + 1e-3
    p, c, v = [0], [], []
    for r in range(n):
        nz = np.nonzero(M[r])[0]
        c.extend(nz.tolist())
        v.extend(M[r, nz].tolist())
        p.append(len(c))
    return np.asarray(p, np.int32), np.asarray(c, np.int32), np.asarray(v, np.float64)


def random_wide_spd(n: int, far: int, npairs: int, seed: int):
    """A random symmetric, diagonally dominant sparse matrix: a random
    tridiagonal band plus `npairs` symmetric couplings between rows at least
    `far` apart (so that column offsets exceed 16 bits when far > 32767), in
    sorted CSR form."""
    import scipy.sparse as sps
    rng = np.random.default_rng(seed)
    r = np.arange(n - 1)
    i = rng.integers(0, n - far, npairs)
    j = np.minimum(i + far + rng.integers(0, n, npairs) % np.maximum(n - far - i, 1), n - 1)
    rows = np.concatenate([r, i])
    cols = np.concatenate([r + 1, j])
    w = -rng.uniform(0.01, 1.0, rows.size)
    U = sps.coo_matrix((w, (rows, cols)), shape=(n, n))
    M = (U + U.T).tocsr()
    M.sum_duplicates()
    d = -np.asarray(M.sum(axis=1)).ravel() + rng.uniform(0.0, 0.5, n) + 1e-3
    M = (M + sps.diags(d)).tocsr()
    M.sort_indices()
    return M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64)


def revalue_symmetric(ptr, col, val, seed: int, spread: float = 0.5):
    """New values on the same symmetric pattern: every off-diagonal pair scaled
    by one seeded factor in [1 - spread, 1 + spread], the diagonal reset to the
    negated off-diagonal row sum plus a seeded margin (diagonally dominant)."""
    n = ptr.size - 1
    rng = np.random.default_rng(seed)
    lo = np.minimum(np.repeat(np.arange(n), np.diff(ptr)), col).astype(np.int64)
    hi = np.maximum(np.repeat(np.arange(n), np.diff(ptr)), col).astype(np.int64)
    key = lo * n + hi
    uk, inv = np.unique(key, return_inverse=True)
    fac = 1.0 + spread * rng.uniform(-1.0, 1.0, uk.size)
    rows = np.repeat(np.arange(n), np.diff(ptr))
    off = col != rows
    out = np.where(off, val * fac[inv], 0.0)
    rs = np.zeros(n)
    np.add.at(rs, rows, out)
    margin = rng.uniform(0.0, 0.5, n) + 1e-3
    out[~off] = -rs[rows[~off]] + margin[rows[~off]]
    return out


# ---------------------------------------------------------------- level-set transport stand-in
LEVELSET_COURANT = 2.0


def levelset_faces(dim: int, N: int, k: int, T: int, courant: float = LEVELSET_COURANT):
    """Face-normal velocities of the level-set stand-in (Sec. 4, eq. 5) at step k.

    A divergence-free rotating flow, in the x-y plane (2D) or the x-z plane
    (3D): u_x = -sin(pi x) cos(pi w), u_w = cos(pi x) sin(pi w), with w = y or z,
    scaled by s(t) = 1 + 0.5 sin(2 pi k / T) and by the Courant number, and
    sampled at the face centres.  It has no normal flow through the walls.
    Layouts (x fastest): fx[(z N + y)(N + 1) + x_face],
    fy[(z (N + 1) + y_face) N + x], fz[(z_face N + y) N + x]; in 2D z = 0 and
    fz is empty."""
    c = (np.arange(N, dtype=np.float64) + 0.5) / N
    e = np.arange(N + 1, dtype=np.float64) / N
    s = courant * (1.0 + 0.5 * np.sin(2.0 * np.pi * k / T))
    if dim == 2:
        fx = -np.sin(np.pi * e)[None, :] * np.cos(np.pi * c)[:, None]           # [y, x_face]
        fy = np.cos(np.pi * c)[None, :] * np.sin(np.pi * e)[:, None]            # [y_face, x]
        return (s * fx).reshape(-1), (s * fy).reshape(-1), np.zeros(0)
    ones = np.ones(N)
    fx = -np.sin(np.pi * e)[None, None, :] * np.cos(np.pi * c)[:, None, None] * ones[None, :, None]  # [z, y, xf]
    fy = np.zeros((N, N + 1, N))                                                                        # [z, yf, x]
    fz = np.cos(np.pi * c)[None, None, :] * np.sin(np.pi * e)[:, None, None] * ones[None, :, None]   # [zf, y, x]
    return (s * fx).reshape(-1), (s * fy).reshape(-1), (s * fz).reshape(-1)


# ---------------------------------------------------------------- monolithic Navier-Stokes stand-in
NS_MASS = 0.1          # mass coefficient: the velocity diagonal starts at NS_MASS * rho
NS_MU_WATER = 1.0      # dynamic viscosity in the water column
NS_MU_AIR = 0.018      # and in the air (about the water / air ratio)


# the 4 x 4 block workloads (unknowns 4 N^3): 48^3 has 110,592 nodes / 442,368
# unknowns, about the size of Sec. 4's Navier-Stokes system (417,604 unknowns)
NS_WORKLOADS = {
    "ns32": Workload("ns32", 3, 32, 20, "fp64"),
    "ns48": Workload("ns48", 3, 48, 50, "fp64"),
}


def ns_fields(N: int, k: int, T: int, courant: float = LEVELSET_COURANT):
    """Per-cell density and viscosity (the collapsing water column at step k)
    and the face velocities of the level-set flow: the inputs of the 4 x 4
    block system standing in for the monolithic Navier-Stokes matrices of
    Sec. 4 (3D, N^3 cells).  Returns (rho, mu, fx, fy, fz)."""
    rho = density(3, N, k, T)
    mu = np.where(rho == RHO_WATER, NS_MU_WATER, NS_MU_AIR)
    fx, fy, fz = levelset_faces(3, N, k, T, courant)
    return rho, mu, fx, fy, fz
