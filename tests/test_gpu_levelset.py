"""GPU parity for the nonsymmetric path: the level-set transport stand-in
(Sec. 4, eq. 5) and right-preconditioned BiCGStab, through the C ABI,
against the CPU oracle on the same seeded inputs.

Bar: assembly bit-exact; hierarchy structure bit-exact and FP64 coarse values
bit-exact (the Galerkin summation order is the oracle's); solves to the same
relative residual with iteration counts within one; the time loop's rebuild
decisions identical.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_2108_02054_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2108_02054_gb300 import amg as B


def _faces(dim, N, k, T):
    return I.levelset_faces(dim, N, k, T)


def gpu_levelset(dim, N, k, T, ptr=None):
    fx, fy, fz = (torch.tensor(a, device="cuda") for a in _faces(dim, N, k, T))
    col = None
    if ptr is None:
        ptr, col = B.poisson_pattern(dim, N)
    return ptr, col, B.levelset_values(dim, N, fx, fy, fz, ptr)


def oracle_levelset(dim, N, k, T):
    return O.levelset_assemble(dim, N, *_faces(dim, N, k, T))


def _sp(ptr, col, val, n):
    return sp.csr_matrix((val, col, ptr), shape=(n, n))


@pytest.mark.parametrize("dim,N", [(2, 1), (2, 7), (2, 32), (3, 2), (3, 17), (3, 40)])
def test_levelset_assembly_bitwise(dim, N):
    ptr, col, val = gpu_levelset(dim, N, 3, 10)
    optr, ocol, oval = oracle_levelset(dim, N, 3, 10)
    assert np.array_equal(ptr.cpu().numpy(), optr)
    assert np.array_equal(col.cpu().numpy(), ocol)
    assert np.array_equal(val.cpu().numpy(), oval)


def test_levelset_values_argument_errors():
    ptr, col = B.poisson_pattern(3, 4)
    fx = torch.zeros(4 * 4 * 5, dtype=torch.float64, device="cuda")
    L = B.lib()
    v = torch.empty(B.poisson_nnz(3, 4), dtype=torch.float64, device="cuda")
    # 3D needs fz; bad dimension; null output
    assert L.amg_levelset_values(3, 4, fx.data_ptr(), fx.data_ptr(), 0, ptr.data_ptr(), v.data_ptr(), 0) == B.AMG_ERR_ARG
    assert L.amg_levelset_values(4, 4, fx.data_ptr(), fx.data_ptr(), fx.data_ptr(), ptr.data_ptr(), v.data_ptr(), 0) == B.AMG_ERR_ARG
    assert L.amg_levelset_values(3, 4, fx.data_ptr(), fx.data_ptr(), fx.data_ptr(), ptr.data_ptr(), 0, 0) == B.AMG_ERR_ARG


@pytest.mark.parametrize("dim,N,ce", [(2, 32, 64), (3, 24, 64), (3, 40, 256)])
def test_levelset_hierarchy_matches_oracle(dim, N, ce):
    """Nonsymmetric A: strength, aggregates, P, R = P^T and every A_{l+1}
    identical to the oracle's, before and after a partial rebuild."""
    T = 10
    ptr, col, v0 = gpu_levelset(dim, N, 0, T)
    G = B.AMG(coarse_enough=ce, solver=B.SOLVER_BICGSTAB)
    G.full_setup(ptr, col, v0)
    H = O.Hierarchy(*oracle_levelset(dim, N, 0, T), O.Params(coarse_enough=ce))
    assert G.nlevels == H.nlevels >= 2

    def check():
        for l in range(H.nlevels):
            g, o = G.export_level(l), H.level(l)
            gp, gc, gv = g["A"]
            assert np.array_equal(gp, o.A.ptr) and np.array_equal(gc, o.A.col), l
            assert np.array_equal(gv, o.A.val), l
            assert np.array_equal(g["agg"], o.agg) and np.array_equal(g["strong"], o.strong), l
            if l < H.nlevels - 1:
                assert np.array_equal(g["P"][1], o.P.col) and np.array_equal(g["P"][2], o.P.val), l
                assert np.allclose(g["m"], o.m, rtol=1e-13, atol=0), l
        lu, piv = G.coarse_lu()
        olu, opiv = H.lu()
        assert np.array_equal(piv, opiv)
        assert np.allclose(lu, olu, rtol=1e-12, atol=1e-14 * np.abs(olu).max())

    check()
    _, _, v5 = gpu_levelset(dim, N, 5, T, ptr)
    G.partial_rebuild(v5)
    assert H.rebuild(oracle_levelset(dim, N, 5, T)[2]) == 0
    check()


@pytest.mark.parametrize("dim,N", [(2, 32), (3, 40), (3, 64)])
def test_bicgstab_solve_matches_oracle(dim, N):
    T = 10
    ptr, col, v = gpu_levelset(dim, N, 4, T)
    G = B.AMG(solver=B.SOLVER_BICGSTAB)
    G.full_setup(ptr, col, v)
    optr, ocol, oval = oracle_levelset(dim, N, 4, T)
    H = O.Hierarchy(optr, ocol, oval)
    f = I.rhs(N ** dim)
    u, info = G.solve(torch.tensor(f, device="cuda"), 1e-8)
    uo, it, rr, st = H.bicgstab(f, 1e-8)
    assert info.status == B.AMG_OK and st == O.OK
    assert abs(info.iters - it) <= 1, (info.iters, it)
    assert info.rel_resid <= 1e-8
    un = u.cpu().numpy()
    A = _sp(optr, ocol, oval, N ** dim)
    res = np.linalg.norm(f - A @ un) / np.linalg.norm(f)
    assert res <= 1e-8 and abs(res - info.rel_resid) <= 1e-3 * res + 1e-15
    assert np.linalg.norm(un - uo) <= 1e-5 * np.linalg.norm(uo)


def test_bicgstab_on_symmetric_pressure_matrix():
    """BiCGStab is a general solver: on the SPD pressure matrix it matches the
    oracle's BiCGStab as well."""
    dim, N, T = 3, 32, 10
    rho = I.density(dim, N, 5, T)
    ptr, col = B.poisson_pattern(dim, N)
    v = B.poisson_values(dim, N, torch.tensor(rho, device="cuda"), ptr)
    G = B.AMG(solver=B.SOLVER_BICGSTAB)
    G.full_setup(ptr, col, v)
    H = O.Hierarchy(*O.poisson_assemble(dim, N, rho))
    f = I.rhs(N ** dim)
    _, info = G.solve(torch.tensor(f, device="cuda"), 1e-8)
    _, it, _, st = H.bicgstab(f, 1e-8)
    assert info.status == 0 and st == O.OK and abs(info.iters - it) <= 1


def test_bicgstab_half_step_and_edge_cases():
    """Single level (the coarsest LU is an exact preconditioner): converged
    at the half step of the first iteration.  Zero right-hand side: no
    iteration, u = 0.  maxiter = 1 on a multilevel hierarchy: NOT_CONVERGED
    after one iteration, with the true residual reported."""
    ptr, col, v = gpu_levelset(2, 8, 1, 4)
    G = B.AMG(solver=B.SOLVER_BICGSTAB)
    G.full_setup(ptr, col, v)
    assert G.nlevels == 1
    f = I.rhs(64)
    u, info = G.solve(torch.tensor(f, device="cuda"), 1e-10)
    assert info.status == 0 and info.iters == 1 and info.rel_resid <= 1e-10
    H = O.Hierarchy(*oracle_levelset(2, 8, 1, 4))
    uo, it, rr, st = H.bicgstab(f, 1e-10)
    assert it == 1 and st == O.OK
    assert np.allclose(u.cpu().numpy(), uo, rtol=1e-12, atol=1e-14)
    u, info = G.solve(torch.zeros(64, dtype=torch.float64, device="cuda"))
    assert info.status == 0 and info.iters == 0 and torch.all(u == 0)

    ptr, col, v = gpu_levelset(3, 24, 1, 4)
    G = B.AMG(solver=B.SOLVER_BICGSTAB, maxiter=1)
    G.full_setup(ptr, col, v)
    f = I.rhs(24 ** 3)
    u, info = G.solve(torch.tensor(f, device="cuda"), 1e-12)
    assert info.status == B.AMG_NOT_CONVERGED and info.iters == 1
    H = O.Hierarchy(*oracle_levelset(3, 24, 1, 4))
    _, it, rr, st = H.bicgstab(f, 1e-12, maxiter=1)
    assert st == O.NOT_CONVERGED and it == 1
    assert abs(info.rel_resid - rr) <= 1e-6 * rr


@pytest.mark.parametrize("precision", [0, 1])
def test_bicgstab_graph_equals_eager(precision):
    """The whole-solve graph runs the kernels of the host-driven loop:
    identical iterates and counts."""
    ptr, col, v = gpu_levelset(3, 40, 2, 10)
    G = B.AMG(precision=precision, solver=B.SOLVER_BICGSTAB)
    G.full_setup(ptr, col, v)
    f = torch.tensor(I.rhs(40 ** 3), device="cuda")
    u1, i1 = G.solve(f, 1e-8)
    u2, i2 = G.solve(f, 1e-8)
    G.profile(True)
    u3, i3 = G.solve(f, 1e-8)
    G.profile(False)
    G.profile_read()
    assert i1.iters == i2.iters == i3.iters and i1.status == i3.status == 0
    assert torch.equal(u1, u2) and torch.equal(u1, u3)
    assert i1.rel_resid <= 1e-8


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_levelset_time_series_matches_oracle(mode):
    """Sec. 4, level-set column of Table 2: the time loop under each mode,
    rebuild decisions and iteration counts against the oracle's loop."""
    dim, N, T = 3, 24, 8
    ptr, col, _ = gpu_levelset(dim, N, 0, T)
    f = I.rhs(N ** dim)
    ft = torch.tensor(f, device="cuda")
    optr, ocol, _ = oracle_levelset(dim, N, 0, T)
    vals = [oracle_levelset(dim, N, k, T)[2] for k in range(T)]
    recs = O.run_time_steps(optr, ocol, vals, f, mode, solver="bicgstab")
    G = B.AMG(mode=mode, solver=B.SOLVER_BICGSTAB)
    for k in range(T):
        _, _, vk = gpu_levelset(dim, N, k, T, ptr)
        si = G.step(vk, ptr, col)
        _, info = G.solve(ft, 1e-8)
        assert bool(si.rebuilt) == recs[k].rebuilt, k
        assert info.status == recs[k].status, k
        assert abs(info.iters - recs[k].iters) <= 1, (k, info.iters, recs[k].iters)
        if info.status == 0:
            assert info.rel_resid <= 1e-8


@pytest.mark.parametrize("dim,N", [(2, 32), (3, 64)])
def test_bicgstab_mixed_precision(dim, N):
    """FP32 hierarchy inside the FP64 BiCGStab: the same FP64 tolerance, a
    few more iterations at most."""
    T = 10
    ptr, col, v = gpu_levelset(dim, N, 6, T)
    G = B.AMG(precision=B.PREC_MIXED, solver=B.SOLVER_BICGSTAB)
    G.full_setup(ptr, col, v)
    optr, ocol, oval = oracle_levelset(dim, N, 6, T)
    H = O.Hierarchy(optr, ocol, oval)
    f = I.rhs(N ** dim)
    u, info = G.solve(torch.tensor(f, device="cuda"), 1e-8)
    _, it, _, st = H.bicgstab(f, 1e-8)
    assert info.status == 0 and info.iters <= it + 3
    A = _sp(optr, ocol, oval, N ** dim)
    assert np.linalg.norm(f - A @ u.cpu().numpy()) / np.linalg.norm(f) <= 1e-8
