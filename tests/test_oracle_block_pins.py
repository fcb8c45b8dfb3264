"""Pins of the block-valued (4 x 4) oracle path against what the paper and the
mathematics fix, independently of the oracle's own formulas:

- the synthetic monolithic system: its pressure part is exactly the pressure
  Poisson matrix (an independently pinned routine) with density 1/kappa; the
  velocity-pressure coupling is skew-symmetric; its symmetric part is positive
  definite; a linear pressure field has the expected discrete gradient;
- a decoupled block system a_ij I_4 reduces to the scalar hierarchy (plain
  aggregation, damped Jacobi), structure and values;
- every block Galerkin operator equals the dense (P x I_4)^T A (P x I_4);
- the 4 x 4 inverse and block norm against numpy;
- BiCGStab: a direct solve, the exact-preconditioner (single level) case, and
  partial reuse keeping the iterations of the no-reuse strategy (Sec. 4,
  Table 2, Navier-Stokes rows).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_2108_02054_gb300 import inputs as I


def _system(N, k=2, T=10, mass=I.NS_MASS, uniform=False, still=False):
    rho, mu, fx, fy, fz = I.ns_fields(N, k, T)
    if uniform:
        rho = np.ones_like(rho)
        mu = np.ones_like(mu)
    if still:
        fx, fy, fz = np.zeros_like(fx), np.zeros_like(fy), np.zeros_like(fz)
    ptr, col, bv = O.stokes_assemble(N, rho, mu, fx, fy, fz, mass)
    return ptr, col, bv, rho, mu, mass


@pytest.mark.parametrize("N", [1, 2, 5, 9])
def test_stokes_pressure_part_is_the_poisson_matrix(N):
    ptr, col, bv, rho, mu, mass = _system(N)
    kap = mass * rho + 6.0 * mu
    pptr, pcol, pval = O.poisson_assemble(3, N, 1.0 / kap, dirichlet_top=True)
    assert np.array_equal(ptr, pptr) and np.array_equal(col, pcol)
    assert np.array_equal(bv[:, 15], pval)


@pytest.mark.parametrize("N", [2, 6])
def test_stokes_coupling_skew_and_positive_real(N):
    ptr, col, bv, *_ = _system(N)
    A = O.block_to_scipy(ptr, col, bv).toarray()
    n = 4 * N ** 3
    vel = np.array([i % 4 != 3 for i in range(n)])
    C = A[np.ix_(vel, ~vel)]
    D = A[np.ix_(~vel, vel)]
    assert np.array_equal(C, -D.T)
    # velocity part: the same scalar operator on u, v, w, no cross terms
    V = A[np.ix_(vel, vel)]
    for r in range(3):
        for c in range(3):
            blk = V[r::3, c::3]
            if r == c:
                assert np.array_equal(blk, V[0::3, 0::3])
            else:
                assert not blk.any()
    S = 0.5 * (A + A.T)
    assert np.linalg.eigvalsh(S).min() > 0.0


def test_stokes_still_uniform_closed_forms():
    """No flow, rho = mu = 1: the velocity operator is mass I + graph
    Laplacian + 2 per wall face (row sums = mass + 2 * walls); the pressure
    gradient of p = x in the u-rows of interior cells is kappa (central
    difference with weight kappa)."""
    N = 5
    ptr, col, bv, rho, mu, mass = _system(N, uniform=True, still=True)
    A = O.block_to_scipy(ptr, col, bv)
    n = N ** 3
    x = np.arange(n) % N
    y = (np.arange(n) // N) % N
    z = np.arange(n) // (N * N)
    walls = (x == 0).astype(int) + (x == N - 1) + (y == 0) + (y == N - 1) + (z == 0) + (z == N - 1)
    ones_u = np.zeros(4 * n)
    ones_u[0::4] = 1.0
    Au = A @ ones_u
    assert np.allclose(Au[0::4], mass + 2.0 * walls, rtol=0, atol=1e-13)
    assert not Au[1::4].any() and not Au[2::4].any()
    p = np.zeros(4 * n)
    p[3::4] = x
    g = (A @ p)[0::4]
    kap = mass + 6.0
    interior = (x > 0) & (x < N - 1)
    assert np.allclose(g[interior], kap, rtol=1e-14, atol=0)
    # on the x walls the ghost pressure equals the cell's: one-sided differences
    assert np.allclose(g[x == 0], 0.5 * kap * 1.0, rtol=1e-14)


def test_block_norm_and_inverse_against_numpy():
    rng = np.random.default_rng(5)
    for _ in range(50):
        a = rng.normal(size=(4, 4)) + 4 * np.eye(4) * rng.choice([-1, 1])
        assert abs(O.block_norm(a) - np.linalg.norm(a)) <= 1e-15 * np.linalg.norm(a)
        inv, ok = O.inv4(a)
        assert ok and np.allclose(inv @ a, np.eye(4), atol=1e-13)
    # zero leading pivot: row exchange needed
    a = np.array([[0, 1, 0, 0], [2, 0, 0, 0], [0, 0, 3, 1], [0, 0, 1, 3]], float)
    inv, ok = O.inv4(a)
    assert ok and np.allclose(inv, np.linalg.inv(a), rtol=1e-15, atol=1e-16)
    inv, ok = O.inv4(np.ones((4, 4)))
    assert not ok


@pytest.mark.parametrize("which", ["poisson", "levelset"])
def test_decoupled_block_system_reduces_to_scalar_hierarchy(which):
    """A_ij = a_ij I_4: aggregates, strength, P and the coarse operators are
    those of the scalar hierarchy (plain aggregation, damped Jacobi); the
    block-Jacobi inverse is w_J / a_ii I_4; BiCGStab needs the same work."""
    N = 10
    if which == "poisson":
        ptr, col, val = O.poisson_assemble(3, N, I.density(3, N, 3, 10))
    else:
        ptr, col, val = O.levelset_assemble(3, N, *I.levelset_faces(3, N, 3, 10))
    bv = np.zeros((val.size, 16))
    for r in range(4):
        bv[:, 5 * r] = val
    prm = O.block_params(coarse_enough=20)
    Hb = O.BlockHierarchy(ptr, col, bv, prm)
    Hs = O.Hierarchy(ptr, col, val, prm)
    assert Hb.nlevels == Hs.nlevels >= 3
    for l in range(Hs.nlevels):
        b, s = Hb.level(l), Hs.level(l)
        assert np.array_equal(b.A.ptr, s.A.ptr) and np.array_equal(b.A.col, s.A.col)
        assert np.array_equal(b.agg, s.agg) and np.array_equal(b.strong, s.strong)
        for r in range(4):
            assert np.array_equal(b.A.val[:, 5 * r], s.A.val)
        off = np.ones(16, bool)
        off[[0, 5, 10, 15]] = False
        assert not b.A.val[:, off].any()
        if l < Hs.nlevels - 1:
            assert np.array_equal(b.P.col, s.P.col) and np.array_equal(b.P.val, s.P.val)
            for r in range(4):
                assert np.allclose(b.minv[:, 5 * r], s.m, rtol=4.5e-16, atol=0)  # w (1/a) vs w / a: 2 ulp
    f = I.rhs(N ** 3)
    f4 = np.repeat(f, 4)
    u4, it4, rr4, st4 = Hb.bicgstab(f4, 1e-8)
    u, it, rr, st = Hs.bicgstab(f, 1e-8)
    assert st4 == st == O.OK and abs(it4 - it) <= 1
    assert np.allclose(u4.reshape(-1, 4), u[:, None], rtol=1e-6, atol=1e-10 * np.abs(u).max())


def test_block_galerkin_equals_dense_product():
    N = 6
    ptr, col, bv, *_ = _system(N)
    H = O.BlockHierarchy(ptr, col, bv, O.block_params(coarse_enough=8))
    assert H.nlevels >= 3
    for l in range(H.nlevels - 1):
        L, C = H.level(l), H.level(l + 1)
        A = O.block_to_scipy(L.A.ptr, L.A.col, L.A.val).toarray()
        P = np.kron(L.P.dense(), np.eye(4))
        ref = P.T @ A @ P
        bound = np.abs(P).T @ np.abs(A) @ np.abs(P)
        got = O.block_to_scipy(C.A.ptr, C.A.col, C.A.val).toarray()
        assert np.all(np.abs(got - ref) <= 1e-14 * bound)
        # tentative prolongation: one unit entry per aggregated row
        assert np.all(L.P.val == 1.0) and np.all(np.diff(L.P.ptr) == (L.agg >= 0))
        # the block-Jacobi inverse: Minv_i A_ii = w_J I
        dia = [L.A.ptr[i] + np.flatnonzero(L.A.col[L.A.ptr[i]:L.A.ptr[i + 1]] == i)[0] for i in range(L.A.nrows)]
        for i in range(0, L.A.nrows, 7):
            M = L.minv[i].reshape(4, 4)
            assert np.allclose(M @ L.A.val[dia[i]].reshape(4, 4), 0.72 * np.eye(4), atol=1e-13)


def test_block_partial_rebuild():
    """Alg. 4 on the block hierarchy: unchanged values reproduce the full
    setup bit for bit; new values give the Galerkin blocks of the kept P."""
    N = 8
    ptr, col, bv0, *_ = _system(N, k=0)
    _, _, bv5, *_ = _system(N, k=5)
    prm = O.block_params(coarse_enough=16)
    H = O.BlockHierarchy(ptr, col, bv0, prm)
    ref = [H.level(l) for l in range(H.nlevels)]
    assert H.rebuild(bv0) == 0
    for l in range(H.nlevels):
        assert np.array_equal(H.level(l).A.val, ref[l].A.val)
        assert np.array_equal(H.level(l).minv, ref[l].minv)
    assert H.rebuild(bv5) == 0
    for l in range(H.nlevels - 1):
        L, C = H.level(l), H.level(l + 1)
        assert np.array_equal(L.P.col, ref[l].P.col)
        A = O.block_to_scipy(L.A.ptr, L.A.col, L.A.val).toarray()
        P = np.kron(L.P.dense(), np.eye(4))
        got = O.block_to_scipy(C.A.ptr, C.A.col, C.A.val).toarray()
        assert np.all(np.abs(got - P.T @ A @ P) <= 1e-14 * (np.abs(P).T @ np.abs(A) @ np.abs(P)))


def test_block_bicgstab_direct_solve_and_exact_preconditioner():
    N = 8
    ptr, col, bv, *_ = _system(N)
    A = O.block_to_scipy(ptr, col, bv)
    f = I.rhs(4 * N ** 3)
    H = O.BlockHierarchy(ptr, col, bv, O.block_params(coarse_enough=16))
    u, it, rr, st = H.bicgstab(f, 1e-10)
    ud = sp.linalg.spsolve(A.tocsc(), f)
    assert st == O.OK and rr <= 1e-10
    assert np.linalg.norm(u - ud) <= 1e-7 * np.linalg.norm(ud)
    assert abs(np.linalg.norm(f - A @ u) / np.linalg.norm(f) - rr) <= 1e-3 * rr
    # one level: the coarse LU is exact, converged at the first half step
    H1 = O.BlockHierarchy(ptr, col, bv, O.block_params(coarse_enough=10 ** 6))
    assert H1.nlevels == 1
    u, it, rr, st = H1.bicgstab(f, 1e-10)
    assert st == O.OK and it == 1
    assert np.linalg.norm(u - ud) <= 1e-10 * np.linalg.norm(ud)
    u, it, rr, st = H.bicgstab(np.zeros_like(f))
    assert st == O.OK and it == 0 and not u.any()


def test_block_partial_reuse_keeps_iterations():
    """Sec. 4, Table 2 (Navier-Stokes): partial reuse keeps the iterations
    of the no-reuse strategy (16.9 vs 16.7 in the paper), full reuse does
    not."""
    N, T = 10, 6
    ptr, col, _, *_ = _system(N, k=0, T=T)
    vals = [_system(N, k=k, T=T)[2] for k in range(T)]
    f = I.rhs(4 * N ** 3)
    prm = O.block_params(coarse_enough=16)
    kw = dict(solver="bicgstab", block=True)
    full = O.run_time_steps(ptr, col, vals, f, O.MODE_FULL_REBUILD, prm, **kw)
    part = O.run_time_steps(ptr, col, vals, f, O.MODE_PARTIAL, prm, **kw)
    assert all(r.status == O.OK for r in full + part)
    assert sum(r.iters for r in part) <= 1.25 * sum(r.iters for r in full)
