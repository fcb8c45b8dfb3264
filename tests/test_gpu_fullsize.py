"""Parity at the full benchmark sizes, in the configuration bench.py times.

128^3 (mixed precision): the whole hierarchy structure against the FP64
oracle, bit for bit; coarse values after partial rebuilds within FP32
accuracy of the oracle's; the solution's FP64 residual recomputed on the host.

192^3 (mixed precision): the oracle's full setup is too slow for a test, so
this checks what holds at any size: the true FP64 residual of the solution,
recomputed on the host; sampled coarse rows recomputed as P^T A P from the
exported operators; symmetry of the coarse operators.
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


def _gpu_vals(w, k, ptr):
    return B.poisson_values(w.dim, w.N, torch.tensor(I.density(w.dim, w.N, k, w.T), device="cuda"), ptr)


def _sp(t, n, m):
    p, c, v = t
    return sp.csr_matrix((v, c, p), shape=(n, m))


def test_128cubed_mixed_against_oracle():
    w = I.WORKLOADS["3d128"]
    ptr, col = B.poisson_pattern(w.dim, w.N)
    G = B.AMG(precision=B.PREC_MIXED)
    G.step(_gpu_vals(w, 0, ptr), ptr, col)
    optr, ocol, ov0 = O.poisson_assemble(w.dim, w.N, I.density(w.dim, w.N, 0, w.T))
    H = O.Hierarchy(optr, ocol, ov0)
    assert G.nlevels == H.nlevels >= 4
    for l in range(H.nlevels):
        g, o = G.export_level(l), H.level(l)
        assert np.array_equal(g["A"][0], o.A.ptr) and np.array_equal(g["A"][1], o.A.col)
        assert np.array_equal(g["agg"], o.agg) and np.array_equal(g["strong"], o.strong)
        if l < H.nlevels - 1:
            assert np.array_equal(g["P"][0], o.P.ptr) and np.array_equal(g["P"][1], o.P.col)
    f = I.rhs(w.n)
    ft = torch.tensor(f, device="cuda")
    for k in (1, 50, 99):
        G.step(_gpu_vals(w, k, ptr))
        vk = O.poisson_assemble(w.dim, w.N, I.density(w.dim, w.N, k, w.T))[2]
        assert H.rebuild(vk) == 0
        # FP32 values and products: the error is measured against the nested
        # absolute-term bound B_0 = |A|, B_{l+1} = |P_l|^T B_l |P_l| (rounding of
        # FP32 inputs, ~6e-8 each, propagated through the coarse levels)
        Bd = abs(_sp((optr, ocol, vk), w.n, w.n))
        for l in range(1, H.nlevels):
            lo = H.level(l - 1)
            Pa = abs(_sp((lo.P.ptr, lo.P.col, lo.P.val), lo.A.nrows, lo.nagg))
            Bd = (Pa.T @ Bd @ Pa).tocsr()
            o = H.level(l)
            bd = np.asarray(Bd[np.repeat(np.arange(o.A.nrows), np.diff(o.A.ptr)), o.A.col]).ravel()
            gv = G.export_level(l)["A"][2]
            assert np.all(np.abs(gv - o.A.val) <= 1e-6 * bd + 1e-30), l
        u, info = G.solve(ft, 1e-8)
        assert info.status == 0
        A = _sp((optr, ocol, vk), w.n, w.n)
        res = np.linalg.norm(f - A @ u.cpu().numpy()) / np.linalg.norm(f)
        assert res <= 1e-8, res


def test_192cubed_mixed_properties():
    w = I.WORKLOADS["3d192"]
    ptr, col = B.poisson_pattern(w.dim, w.N)
    G = B.AMG(precision=B.PREC_MIXED)
    G.step(_gpu_vals(w, 0, ptr), ptr, col)
    v99 = _gpu_vals(w, 99, ptr)
    G.step(v99)
    f = I.rhs(w.n)
    u, info = G.solve(torch.tensor(f, device="cuda"), 1e-8)
    assert info.status == 0 and info.rel_resid <= 1e-8
    A = _sp((ptr.cpu().numpy(), col.cpu().numpy(), v99.cpu().numpy()), w.n, w.n)
    res = np.linalg.norm(f - A @ u.cpu().numpy()) / np.linalg.norm(f)
    assert res <= 1e-8, res
    rng = np.random.default_rng(7)
    for l in range(G.nlevels - 1):
        g, c = G.export_level(l), G.export_level(l + 1)
        n, nc = g["n"], g["nagg"]
        Al = _sp(g["A"], n, n)
        P = _sp(g["P"], n, nc)
        Ac = _sp(c["A"], nc, nc)
        # R is P^T, exactly
        R = _sp(g["R"], nc, n)
        assert (R != P.T.tocsr()).nnz == 0
        # sampled coarse rows: A_c[I, :] = P[:, I]^T A P, within FP32 accuracy
        rows = rng.choice(nc, size=min(nc, 200), replace=False)
        ref = (P[:, rows].T @ (Al @ P)).toarray()
        bound = (abs(P[:, rows]).T @ (abs(Al) @ abs(P))).toarray()
        got = Ac[rows].toarray()
        assert np.all(np.abs(got - ref) <= 2e-6 * bound + 1e-30)
        # the Galerkin operator of a symmetric A is symmetric (to FP32 rounding)
        d = abs(Ac - Ac.T).max()
        assert d <= 2e-6 * abs(Ac).max()
