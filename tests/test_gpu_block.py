"""GPU parity for the 4 x 4 block-valued hierarchy (Sec. 4, the monolithic
Navier-Stokes systems: non-smoothed aggregation on the node graph of block
norms, damped block Jacobi, BiCGStab), through the C ABI, against the CPU
oracle on the same seeded inputs.

Bar: assembly bit-exact; node graph, strength, aggregates, P and every coarse
block bit-exact; block-Jacobi inverses bit-exact; coarsest LU within 1e-12;
V-cycle within 1e-12 of the oracle's; solves to the same relative residual
with iteration counts within one; the time loop's rebuild decisions identical.
"""
import numpy as np
import pytest

import oracle as O
from paper_2108_02054_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2108_02054_gb300 import amg as B


def gpu_ns(N, k, T, ptr=None):
    col = None
    if ptr is None:
        ptr, col = B.poisson_pattern(3, N)
    rho, mu, fx, fy, fz = (torch.tensor(a, device="cuda") for a in I.ns_fields(N, k, T))
    return ptr, col, B.stokes_values(N, rho, mu, fx, fy, fz, I.NS_MASS, ptr)


def oracle_ns(N, k, T):
    return O.stokes_assemble(N, *I.ns_fields(N, k, T), I.NS_MASS)


@pytest.mark.parametrize("N", [1, 2, 5, 17])
def test_stokes_assembly_bitwise(N):
    ptr, col, v = gpu_ns(N, 3, 10)
    optr, ocol, ov = oracle_ns(N, 3, 10)
    assert np.array_equal(ptr.cpu().numpy(), optr) and np.array_equal(col.cpu().numpy(), ocol)
    assert np.array_equal(v.cpu().numpy(), ov)


def test_block_params_validation():
    for bad in (dict(block_size=3), dict(smoothed=1), dict(smoother=B.SMOOTHER_SPAI0),
                dict(precision=B.PREC_MIXED), dict(solver=B.SOLVER_CG)):
        with pytest.raises(B.AmgError) as e:
            B.AMG(B.block_params(**bad))
        assert e.value.status == B.AMG_ERR_ARG


def _compare(G, H):
    assert G.nlevels == H.nlevels
    for l in range(H.nlevels):
        g, o = G.export_level(l), H.level(l)
        gp, gc, gv = g["A"]
        assert np.array_equal(gp, o.A.ptr) and np.array_equal(gc, o.A.col), l
        assert np.array_equal(gv, o.A.val), l
        assert np.array_equal(g["agg"], o.agg) and np.array_equal(g["strong"], o.strong), l
        if l < H.nlevels - 1:
            assert np.array_equal(g["P"][0], o.P.ptr) and np.array_equal(g["P"][1], o.P.col), l
            assert np.array_equal(g["P"][2], o.P.val), l
            assert np.array_equal(g["m"], o.minv), l
    lu, piv = G.coarse_lu()
    olu, opiv = H.lu()
    assert np.array_equal(piv, opiv)
    assert np.allclose(lu, olu, rtol=1e-12, atol=1e-14 * np.abs(olu).max())


@pytest.mark.parametrize("N,ce", [(12, 16), (20, 64), (33, 64), (20, 100)])
def test_block_hierarchy_matches_oracle(N, ce):
    """(20, 100): an 86-node coarsest level, 344 unknowns, factorised by the
    cluster LU kernel."""
    T = 10
    ptr, col, v0 = gpu_ns(N, 0, T)
    G = B.AMG(B.block_params(coarse_enough=ce))
    G.full_setup(ptr, col, v0)
    H = O.BlockHierarchy(*oracle_ns(N, 0, T), O.block_params(coarse_enough=ce))
    assert H.nlevels >= 3
    _compare(G, H)
    # Alg. 4: the coarse blocks of new values over the kept P, R and patterns
    _, _, v6 = gpu_ns(N, 6, T, ptr)
    G.partial_rebuild(v6)
    assert H.rebuild(oracle_ns(N, 6, T)[2]) == 0
    _compare(G, H)


def test_block_vcycle_matches_oracle():
    N, T = 20, 10
    ptr, col, v = gpu_ns(N, 4, T)
    G = B.AMG(B.block_params(coarse_enough=64))
    G.full_setup(ptr, col, v)
    H = O.BlockHierarchy(*oracle_ns(N, 4, T), O.block_params(coarse_enough=64))
    r = I.rhs(4 * N ** 3, seed=11)
    z = G.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
    zo = H.vcycle(r)
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)


@pytest.mark.parametrize("N", [16, 24])
def test_block_bicgstab_matches_oracle(N):
    T = 10
    ptr, col, v = gpu_ns(N, 5, T)
    G = B.AMG(B.block_params())
    G.full_setup(ptr, col, v)
    optr, ocol, ov = oracle_ns(N, 5, T)
    H = O.BlockHierarchy(optr, ocol, ov)
    f = I.rhs(4 * N ** 3)
    u, info = G.solve(torch.tensor(f, device="cuda"), 1e-8)
    uo, it, rr, st = H.bicgstab(f, 1e-8)
    assert info.status == B.AMG_OK and st == O.OK
    assert abs(info.iters - it) <= 1, (info.iters, it)
    A = O.block_to_scipy(optr, ocol, ov)
    un = u.cpu().numpy()
    res = np.linalg.norm(f - A @ un) / np.linalg.norm(f)
    assert res <= 1e-8 and abs(res - info.rel_resid) <= 1e-3 * res + 1e-15
    assert np.linalg.norm(un - uo) <= 1e-5 * np.linalg.norm(uo)


def test_block_single_level_zero_rhs_and_host_entry():
    """One level: the dense inverse is exact, converged at the first half
    step.  Zero right-hand side: no iteration.  Host buffers in and out."""
    N, T = 6, 4
    ptr, col, v = gpu_ns(N, 1, T)
    G = B.AMG(B.block_params())
    G.full_setup(ptr, col, v)
    assert G.nlevels == 1
    f = I.rhs(4 * N ** 3)
    u, info = G.solve(torch.tensor(f, device="cuda"), 1e-10)
    assert info.status == 0 and info.iters == 1 and info.rel_resid <= 1e-10
    u, info = G.solve(torch.zeros(4 * N ** 3, dtype=torch.float64, device="cuda"))
    assert info.iters == 0 and not u.any()
    N = 14
    ptr, col, v = gpu_ns(N, 0, T)
    G = B.AMG(B.block_params())
    G.step(v, ptr, col)
    hv = np.ascontiguousarray(oracle_ns(N, 2, T)[2])
    f = I.rhs(4 * N ** 3)
    hu = np.zeros(4 * N ** 3)
    info = G.step_solve_host(hv, f, hu, 1e-8)
    H = O.BlockHierarchy(*oracle_ns(N, 0, T))
    assert H.rebuild(hv) == 0
    uo, it, rr, st = H.bicgstab(f, 1e-8)
    assert info.status == 0 and abs(info.iters - it) <= 1
    assert np.linalg.norm(hu - uo) <= 1e-5 * np.linalg.norm(uo)


def test_block_graph_equals_eager():
    N = 20
    ptr, col, v = gpu_ns(N, 2, 10)
    G = B.AMG(B.block_params())
    G.full_setup(ptr, col, v)
    f = torch.tensor(I.rhs(4 * N ** 3), device="cuda")
    u1, i1 = G.solve(f, 1e-8)
    u2, i2 = G.solve(f, 1e-8)
    G.profile(True)
    u3, i3 = G.solve(f, 1e-8)
    G.profile(False)
    G.profile_read()
    assert i1.iters == i2.iters == i3.iters and i1.status == i3.status == 0
    assert torch.equal(u1, u2) and torch.equal(u1, u3)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_block_time_series_matches_oracle(mode):
    """Sec. 4, Navier-Stokes rows of Table 2: the time loop under each mode,
    rebuild decisions and iterations against the oracle's loop."""
    N, T = 12, 6
    ptr, col, _ = gpu_ns(N, 0, T)
    optr, ocol, _ = oracle_ns(N, 0, T)
    vals = [oracle_ns(N, k, T)[2] for k in range(T)]
    f = I.rhs(4 * N ** 3)
    ft = torch.tensor(f, device="cuda")
    prm = O.block_params()
    recs = O.run_time_steps(optr, ocol, vals, f, mode, prm, solver="bicgstab", block=True)
    G = B.AMG(B.block_params(mode=mode))
    for k in range(T):
        _, _, vk = gpu_ns(N, k, T, ptr)
        si = G.step(vk, ptr, col)
        _, info = G.solve(ft, 1e-8)
        assert bool(si.rebuilt) == recs[k].rebuilt, k
        assert info.status == recs[k].status, k
        assert abs(info.iters - recs[k].iters) <= 1, (k, info.iters, recs[k].iters)
