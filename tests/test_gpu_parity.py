"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Bar: structure (strength flags, aggregates, P/R/A_c patterns, pivots) bit-exact;
FP64 values within 1e-12 of the oracle relative to the absolute-sum bound
(|P|^T |A| |P|) and, by construction of the summation order, bit-exact;
solutions to the same 1e-8 relative residual with iteration counts within one.
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


def gpu_problem(dim, N, k, T, dirichlet=True):
    rho = I.density(dim, N, k, T)
    ptr, col = B.poisson_pattern(dim, N)
    val = B.poisson_values(dim, N, torch.tensor(rho, device="cuda"), ptr, dirichlet_top=dirichlet)
    return ptr, col, val


def oracle_problem(dim, N, k, T, dirichlet=True):
    return O.poisson_assemble(dim, N, I.density(dim, N, k, T), dirichlet_top=dirichlet)


def _sp(ptr, col, val, ncols):
    return sp.csr_matrix((val, col, ptr), shape=(len(ptr) - 1, ncols))


def compare_hierarchy(G, H, values_bitwise=True, check_values=True):
    assert G.nlevels == H.nlevels
    for l in range(H.nlevels):
        g = G.export_level(l)
        o = H.level(l)
        assert g["n"] == o.A.nrows
        gp, gc, gv = g["A"]
        assert np.array_equal(gp, o.A.ptr) and np.array_equal(gc, o.A.col), f"A pattern level {l}"
        assert np.array_equal(g["agg"], o.agg), f"aggregates level {l}"
        assert np.array_equal(g["strong"], o.strong), f"strength level {l}"
        if check_values:
            if l > 0:
                lo = H.level(l - 1)
                Pa = abs(_sp(lo.P.ptr, lo.P.col, lo.P.val, lo.nagg))
                Aa = abs(_sp(lo.A.ptr, lo.A.col, lo.A.val, lo.A.nrows))
                bound = (Pa.T @ Aa @ Pa).tocsr()
                bound.sort_indices()
                bd = np.asarray(bound[np.repeat(np.arange(o.A.nrows), np.diff(o.A.ptr)), o.A.col]).ravel()
                assert np.all(np.abs(gv - o.A.val) <= 1e-12 * bd + 1e-300), f"A values level {l}"
            if values_bitwise:
                assert np.array_equal(gv, o.A.val), f"A values bitwise level {l}"
            if l < H.nlevels - 1:
                assert np.allclose(g["m"], o.m, rtol=1e-13, atol=0), f"smoother level {l}"
        if l < H.nlevels - 1:
            assert g["nagg"] == o.nagg
            for name, ref in (("P", o.P), ("R", o.R)):
                p_, c_, v_ = g[name]
                assert np.array_equal(p_, ref.ptr) and np.array_equal(c_, ref.col), f"{name} pattern level {l}"
                if check_values:
                    assert np.array_equal(v_, ref.val), f"{name} values level {l}"
            assert g["nnzAP"] == int(H.sizes(l)[4])


# ------------------------------------------------------------------ assembly
@pytest.mark.parametrize("dim,N,dirichlet", [(2, 32, True), (3, 17, True), (3, 64, True), (2, 9, False)])
def test_assembly_bitwise(dim, N, dirichlet):
    ptr, col, val = gpu_problem(dim, N, 3, 10, dirichlet)
    optr, ocol, oval = oracle_problem(dim, N, 3, 10, dirichlet)
    assert np.array_equal(ptr.cpu().numpy(), optr)
    assert np.array_equal(col.cpu().numpy(), ocol)
    assert np.array_equal(val.cpu().numpy(), oval)


# ------------------------------------------------------------------ full setup
@pytest.mark.parametrize("dim,N,ce", [(2, 32, 256), (3, 24, 64), (3, 33, 256), (3, 64, 256)])
def test_full_setup_matches_oracle(dim, N, ce):
    ptr, col, val = gpu_problem(dim, N, 2, 10)
    G = B.AMG(coarse_enough=ce)
    G.full_setup(ptr, col, val)
    H = O.Hierarchy(*oracle_problem(dim, N, 2, 10), O.Params(coarse_enough=ce))
    assert G.nlevels >= 2
    compare_hierarchy(G, H)
    lu, piv = G.coarse_lu()
    olu, opiv = H.lu()
    assert np.array_equal(piv, opiv)
    assert np.allclose(lu, olu, rtol=1e-12, atol=1e-14 * np.abs(olu).max())


@pytest.mark.parametrize("variant", ["jacobi", "plain", "const_theta", "npre2"])
def test_full_setup_variants(variant):
    kw, okw = {}, {}
    if variant == "jacobi":
        kw = okw = {"smoother": 1}
    elif variant == "plain":
        kw = okw = {"smoothed": 0}
    elif variant == "const_theta":
        kw = okw = {"theta_halving": 0}
    else:
        kw = okw = {"npre": 2, "npost": 2}
    ptr, col, val = gpu_problem(3, 20, 4, 10)
    G = B.AMG(coarse_enough=40, **kw)
    G.full_setup(ptr, col, val)
    H = O.Hierarchy(*oracle_problem(3, 20, 4, 10), O.Params(coarse_enough=40, **okw))
    compare_hierarchy(G, H)
    f = I.rhs(20 ** 3)
    u, info = G.solve(torch.tensor(f, device="cuda"), 1e-8)
    uo, it, rr, st = H.pcg(f, 1e-8)
    assert info.status == 0 and st == 0
    assert abs(info.iters - it) <= 1


def test_irregular_random_matrix():
    ptr, col, val = I.random_spd_like(700, 0.01, seed=9)
    G = B.AMG(coarse_enough=30)
    G.full_setup(*(torch.tensor(a, device="cuda") for a in (ptr, col, val)))
    H = O.Hierarchy(ptr, col, val, O.Params(coarse_enough=30))
    compare_hierarchy(G, H)


@pytest.mark.parametrize("case", ["random", "arrow"])
def test_partial_rebuild_irregular_patterns(case):
    """Alg. 4 on irregular patterns: a random symmetric pattern, and one with a
    dense arrow row (rows of about 300 entries on the finest level).  The whole
    hierarchy, values bit for bit, after two rebuilds with new values."""
    if case == "random":
        ptr, col, val = I.random_spd_like(900, 0.012, seed=11)
    else:
        ptr, col, val = I.random_arrow_spd(900, 0.006, 300, seed=12)
    assert np.diff(ptr).max() > 8 and (case == "random" or np.diff(ptr).max() > 256)
    G = B.AMG(coarse_enough=30)
    G.full_setup(*(torch.tensor(a, device="cuda") for a in (ptr, col, val)))
    H = O.Hierarchy(ptr, col, val, O.Params(coarse_enough=30))
    assert G.nlevels >= 3
    for seed in (21, 22):
        v = I.revalue_symmetric(ptr, col, val, seed)
        G.partial_rebuild(torch.tensor(v, device="cuda"))
        assert H.rebuild(v) == 0
        compare_hierarchy(G, H)


# ------------------------------------------------------------------ partial rebuild (Alg. 4)
FLAVOURS = {"sa_spai0": {}, "plain_jacobi": {"smoothed": 0, "smoother": 1}}


@pytest.mark.parametrize("flavour", sorted(FLAVOURS))
@pytest.mark.parametrize("dim,N,T", [(2, 32, 10), (3, 40, 20)])
def test_partial_rebuild_matches_oracle(dim, N, T, flavour):
    """Alg. 4 for smoothed aggregation + SPAI0 and for the paper's own flavour
    (plain aggregation + damped Jacobi, Sec. 4): hierarchy structure, P/R and
    every coarse value bit for bit, smoothers to rounding, LU pivots."""
    kw = FLAVOURS[flavour]
    ptr, col, v0 = gpu_problem(dim, N, 0, T)
    G = B.AMG(**kw)
    G.full_setup(ptr, col, v0)
    H = O.Hierarchy(*oracle_problem(dim, N, 0, T), O.Params(**kw))
    for k in (1, T // 2, T - 1):
        _, _, vk = gpu_problem(dim, N, k, T)
        G.partial_rebuild(vk)
        assert H.rebuild(oracle_problem(dim, N, k, T)[2]) == 0
        compare_hierarchy(G, H)
        lu, piv = G.coarse_lu()
        olu, opiv = H.lu()
        assert np.array_equal(piv, opiv)


def test_partial_rebuild_on_unchanged_values_equals_full_setup_bitwise():
    ptr, col, v0 = gpu_problem(3, 32, 3, 10)
    _, _, v1 = gpu_problem(3, 32, 8, 10)
    G = B.AMG()
    G.full_setup(ptr, col, v0)
    ref = [G.export_level(l) for l in range(G.nlevels)]
    G.partial_rebuild(v1)
    G.partial_rebuild(v0)
    for l in range(G.nlevels):
        g = G.export_level(l)
        assert np.array_equal(g["A"][2], ref[l]["A"][2])
        assert np.array_equal(g["m"], ref[l]["m"])


# ------------------------------------------------------------------ V-cycle and solve
def vcycle_envelope(H, r, npre=1, npost=1):
    """Alg. 2 with every operator and vector replaced by its absolute value
    (|A_l|, |m_l|, |R_l|, |P_l|, |A_L^-1|): an entrywise upper envelope of every
    term the V-cycle sums, so the rounding difference of two implementations
    of the same V-cycle is at most a small multiple of eps times this."""
    lv = [H.level(l) for l in range(H.nlevels)]
    nL = lv[-1].A.nrows
    invL = np.abs(np.linalg.inv(lv[-1].A.dense()))

    def cycle(l, f):
        if l == len(lv) - 1:
            return invL @ f
        L = lv[l]
        A = abs(_sp(L.A.ptr, L.A.col, L.A.val, L.A.nrows))
        m = np.abs(L.m)
        u = m * f
        for _ in range(npre - 1):
            u = u + m * (f + A @ u)
        fc = abs(_sp(L.R.ptr, L.R.col, L.R.val, L.A.nrows)) @ (f + A @ u)
        u = u + abs(_sp(L.P.ptr, L.P.col, L.P.val, L.nagg)) @ cycle(l + 1, fc)
        for _ in range(npost):
            u = u + m * (f + A @ u)
        return u

    assert nL == lv[-1].A.ncols
    return cycle(0, np.abs(r))


@pytest.mark.parametrize("dim,N", [(2, 32), (3, 40), (3, 48), (3, 64)])
def test_vcycle_matches_oracle(dim, N):
    """Entry by entry.  Every level's operators are bit-identical to the
    oracle's and every sweep keeps its order; the one difference is the
    coarsest solve (the GPU multiplies by the explicit inverse, the oracle
    substitutes through the LU factors).  Each entry must agree within 1e-9 of
    the V-cycle's absolute-term envelope, about 1e7 eps: room for the
    conditioning of the coarsest solve, far below what a wrong sweep on any
    row would leave."""
    ptr, col, v = gpu_problem(dim, N, 1, 5)
    G = B.AMG()
    G.full_setup(ptr, col, v)
    H = O.Hierarchy(*oracle_problem(dim, N, 1, 5))
    r = np.random.default_rng(5).normal(size=N ** dim)
    z = G.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
    zo = H.vcycle(r)
    env = vcycle_envelope(H, r)
    ratio = np.abs(z - zo) / env
    print(f"V-cycle {dim}D N={N}: max |z - z_o| / envelope = {ratio.max():.2e}, "
          f"envelope / |z_o| median {np.median(env / np.maximum(np.abs(zo), 1e-300)):.1f}")
    assert np.all(np.abs(z - zo) <= 1e-9 * env), ratio.max()


@pytest.mark.parametrize("dim,N,T", [(2, 32, 10), (3, 64, 50)])
def test_solve_matches_oracle(dim, N, T):
    ptr, col, v = gpu_problem(dim, N, T // 2, T)
    G = B.AMG()
    G.full_setup(ptr, col, v)
    H = O.Hierarchy(*oracle_problem(dim, N, T // 2, T))
    f = I.rhs(N ** dim)
    u, info = G.solve(torch.tensor(f, device="cuda"), 1e-8)
    uo, it, rr, st = H.pcg(f, 1e-8)
    assert info.status == B.AMG_OK and st == O.OK
    assert abs(info.iters - it) <= 1
    assert info.rel_resid <= 1e-8
    un = u.cpu().numpy()
    A = _sp(*oracle_problem(dim, N, T // 2, T), N ** dim)
    assert np.linalg.norm(f - A @ un) / np.linalg.norm(f) <= 1e-8
    assert np.linalg.norm(un - uo) <= 1e-5 * np.linalg.norm(uo)


def test_single_level_and_zero_rhs():
    ptr, col, v = gpu_problem(2, 8, 0, 2)
    G = B.AMG()
    G.full_setup(ptr, col, v)
    assert G.nlevels == 1
    f = torch.tensor(I.rhs(64), device="cuda")
    u, info = G.solve(f, 1e-10)
    assert info.status == 0 and info.iters == 1 and info.rel_resid <= 1e-10
    u, info = G.solve(torch.zeros(64, dtype=torch.float64, device="cuda"))
    assert info.iters == 0 and torch.all(u == 0)


# ------------------------------------------------------------------ time-step modes
@pytest.mark.parametrize("flavour", sorted(FLAVOURS))
@pytest.mark.parametrize("mode", [B.MODE_PARTIAL, B.MODE_FULL_REBUILD, B.MODE_FULL_REUSE] if torch.cuda.is_available() else [0])
def test_time_series_modes_match_oracle(mode, flavour):
    kw = FLAVOURS[flavour]
    dim, N, T = 2, 32, 10
    ptr, col, _ = gpu_problem(dim, N, 0, T)
    f = I.rhs(N * N)
    ft = torch.tensor(f, device="cuda")
    G = B.AMG(mode=mode, **kw)
    vals = [oracle_problem(dim, N, k, T)[2] for k in range(T)]
    recs = O.run_time_steps(*oracle_problem(dim, N, 0, T)[:2], vals, f, mode, params=O.Params(**kw))
    for k in range(T):
        _, _, vk = gpu_problem(dim, N, k, T)
        si = G.step(vk, ptr, col)
        u, info = G.solve(ft, 1e-8)
        assert bool(si.rebuilt) == recs[k].rebuilt, k
        assert info.status == recs[k].status, k
        assert abs(info.iters - recs[k].iters) <= 1, k
        if info.status == 0:
            assert info.rel_resid <= 1e-8


@pytest.mark.parametrize("pinned", [False, True])
def test_host_buffer_entry_point(pinned):
    """amg_step_solve_host against the oracle's rebuild + PCG, from pageable
    and from pinned host buffers (where the right-hand side's copy runs
    asynchronously beside the rebuild); two calls in a row with different
    values and right-hand sides, so a solve that started before its new
    right-hand side landed would fail the second comparison."""
    dim, N = 3, 24
    ptr, col, v0 = gpu_problem(dim, N, 0, 4)
    G = B.AMG()
    G.step(v0, ptr, col)
    H = O.Hierarchy(*oracle_problem(dim, N, 0, 4))

    def host(a):
        t = torch.tensor(np.ascontiguousarray(a))
        return (t.pin_memory() if pinned else t).numpy()

    for k, seed in ((2, 0), (3, 11)):
        f = host(I.rhs(N ** 3, seed=seed))
        hv = host(oracle_problem(dim, N, k, 4)[2])
        hu = host(np.zeros(N ** 3))
        info = G.step_solve_host(hv, f, hu, 1e-8)
        H.rebuild(np.array(hv))
        uo, it, rr, st = H.pcg(np.array(f), 1e-8)
        assert info.status == 0 and abs(info.iters - it) <= 1
        assert np.linalg.norm(hu - uo) <= 1e-5 * np.linalg.norm(uo)


@pytest.mark.parametrize("precision,dim,N,every", [("fp64", 3, 37, 0), ("mixed", 3, 40, 0), ("fp64", 2, 9, 0),
                                                   ("mixed", 3, 33, 3)])
def test_host_entry_point_chunked_equals_device_path(precision, dim, N, every):
    """From the second partial step on, amg_step_solve_host sends the values in
    row chunks and starts each chunk's ingest and its rows of the finest A P as
    soon as the chunk has landed.  Over consecutive steps its solutions,
    iteration counts and coarse operators are those of the device-buffer path
    bit for bit: on a grid whose row count the chunk boundaries do not divide
    (37^3), in mixed precision (40^3), and on a one-level hierarchy whose
    chunks are mostly empty (9^2 = 81 rows).  With a preventive full setup
    every third step (steps 2 and 5 chunked, step 3 a full setup), the chunk
    boundaries must follow the new hierarchy."""
    T = 6
    prec = B.PREC_MIXED if precision == "mixed" else B.PREC_FP64
    n = N ** dim
    ptr, col, v0 = gpu_problem(dim, N, 0, T)
    Gh, Gd = B.AMG(precision=prec, rebuild_every=every), B.AMG(precision=prec, rebuild_every=every)
    Gh.step(v0, ptr, col)
    Gd.step(v0, ptr, col)
    hu = torch.empty(n, dtype=torch.float64).pin_memory()
    for k in range(1, T):
        vk = gpu_problem(dim, N, k, T)[2]
        f = I.rhs(n, seed=k)
        hv, hf = vk.cpu().pin_memory(), torch.tensor(f).pin_memory()
        ih = Gh.step_solve_host(hv.numpy(), hf.numpy(), hu.numpy(), 1e-8)
        info = Gd.step(vk)
        ud, idd = Gd.solve(torch.tensor(f, device="cuda"), 1e-8)
        assert ih.status == idd.status == 0 and ih.rebuilt == info.rebuilt == (1 if every and k % every == 0 else 0)
        assert ih.iters == idd.iters, (k, ih.iters, idd.iters)
        assert np.array_equal(hu.numpy(), ud.cpu().numpy()), f"solution, step {k}"
        assert Gh.nlevels == Gd.nlevels
        for l in range(Gd.nlevels):
            gh, gd = Gh.export_level(l), Gd.export_level(l)
            assert np.array_equal(gh["A"][2], gd["A"][2]), f"A values level {l}, step {k}"
            if l < Gd.nlevels - 1:
                assert np.array_equal(gh["m"], gd["m"]), f"smoother level {l}, step {k}"
    Gh.close()
    Gd.close()


def test_host_entry_point_chunked_reports_nonfinite_values():
    """A non-finite value in any chunk of a chunked host-buffer step (first,
    middle, last entry) is reported as AMG_ERR_NONFINITE, every copy has ended
    when the call returns, and the next step with finite values gives the
    device path's solution bit for bit."""
    dim, N, T = 3, 24, 6
    n = N ** dim
    ptr, col, v0 = gpu_problem(dim, N, 0, T)
    Gh, Gd = B.AMG(), B.AMG()
    Gh.step(v0, ptr, col)
    Gd.step(v0, ptr, col)
    hu = torch.empty(n, dtype=torch.float64).pin_memory()
    hf = torch.tensor(I.rhs(n)).pin_memory()
    v1 = gpu_problem(dim, N, 1, T)[2]
    Gh.step_solve_host(v1.cpu().pin_memory().numpy(), hf.numpy(), hu.numpy(), 1e-8)  # builds the gather operators
    Gd.step(v1)
    Gd.solve(torch.tensor(hf.numpy(), device="cuda"), 1e-8)
    for k, (pos, bad) in enumerate(((0, float("nan")), (v0.numel() // 2 + 5, float("inf")),
                                    (v0.numel() - 1, float("nan"))), start=2):
        w = gpu_problem(dim, N, k, T)[2].cpu()
        w[pos] = bad
        with pytest.raises(B.AmgError) as e:
            Gh.step_solve_host(w.pin_memory().numpy(), hf.numpy(), hu.numpy(), 1e-8)
        assert e.value.status == B.AMG_ERR_NONFINITE
    vk = gpu_problem(dim, N, 5, T)[2]
    ih = Gh.step_solve_host(vk.cpu().pin_memory().numpy(), hf.numpy(), hu.numpy(), 1e-8)
    Gd.step(vk)
    ud, idd = Gd.solve(torch.tensor(hf.numpy(), device="cuda"), 1e-8)
    assert ih.status == idd.status == 0 and ih.iters == idd.iters
    assert np.array_equal(hu.numpy(), ud.cpu().numpy())
    Gh.close()
    Gd.close()


# ------------------------------------------------------------------ mixed precision
@pytest.mark.parametrize("dim,N,T", [(2, 32, 10), (3, 64, 50)])
def test_mixed_precision_reaches_fp64_tolerance(dim, N, T):
    ptr, col, v0 = gpu_problem(dim, N, 0, T)
    G = B.AMG(precision=B.PREC_MIXED)
    G.full_setup(ptr, col, v0)
    H = O.Hierarchy(*oracle_problem(dim, N, 0, T))
    f = I.rhs(N ** dim)
    ft = torch.tensor(f, device="cuda")
    for k in (0, T - 1):
        if k:
            _, _, vk = gpu_problem(dim, N, k, T)
            G.partial_rebuild(vk)
            H.rebuild(oracle_problem(dim, N, k, T)[2])
        # structure identical to the FP64 oracle; every coarse value within FP32
        # accuracy of the oracle's, entry by entry, against the nested
        # absolute-term bound B_0 = |A|, B_{l+1} = |P_l|^T B_l |P_l|
        compare_hierarchy(G, H, values_bitwise=False, check_values=False)
        optr, ocol, ovk = oracle_problem(dim, N, k, T)
        Bd = abs(_sp(optr, ocol, ovk, N ** dim))
        worst = 0.0
        for l in range(1, G.nlevels):
            lo, o = H.level(l - 1), H.level(l)
            Pa = abs(_sp(lo.P.ptr, lo.P.col, lo.P.val, lo.nagg))
            Bd = (Pa.T @ Bd @ Pa).tocsr()
            bd = np.asarray(Bd[np.repeat(np.arange(o.A.nrows), np.diff(o.A.ptr)), o.A.col]).ravel()
            gv = G.export_level(l)["A"][2]
            assert np.all(np.abs(gv - o.A.val) <= 1e-6 * bd), l
            worst = max(worst, float(np.max(np.abs(gv - o.A.val) / bd)))
        print(f"mixed {dim}D N={N} step {k}: max coarse |a - a_o| / bound = {worst:.2e}")
        u, info = G.solve(ft, 1e-8)
        uo, it, rr, st = H.pcg(f, 1e-8)
        assert info.status == 0 and info.rel_resid <= 1e-8
        assert info.iters <= it + 3
        assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-5 * np.linalg.norm(uo)


# ------------------------------------------------------------------ errors (all detected without faults)
def test_binding_rejects_wrong_types_and_extents():
    """The Python binding checks every tensor's element type and extent against
    what the call reads or writes (the kernels cannot), and raises before
    anything is launched."""
    N = 8
    n = N ** 3
    ptr, col = B.poisson_pattern(3, N)
    rho = torch.ones(n, dtype=torch.float64, device="cuda")
    for bad_rho, bad_ptr in ((rho.float(), ptr), (rho[:-1], ptr), (rho, ptr.long()), (rho, ptr[:-1])):
        with pytest.raises(ValueError):
            B.poisson_values(3, N, bad_rho, bad_ptr)
    with pytest.raises(ValueError):
        B.poisson_values(3, N, rho, ptr, out=torch.empty(col.numel() - 1, dtype=torch.float64, device="cuda"))
    v = B.poisson_values(3, N, rho, ptr)
    G = B.AMG(coarse_enough=64)
    for bad in (v.float(), v[:-3]):
        with pytest.raises(ValueError):
            G.full_setup(ptr, col, bad)
    with pytest.raises(ValueError):
        G.full_setup(ptr.long(), col, v)
    G.full_setup(ptr, col, v)
    with pytest.raises(ValueError):
        G.partial_rebuild(v[:-1])
    f = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        G.solve(f[:-1])
    with pytest.raises(ValueError):
        G.solve(f, u=torch.empty(n, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        G.step_solve_host(v.cpu().numpy(), np.zeros(n - 1), np.zeros(n), 1e-8)
    u, info = G.solve(f, 1e-8)
    assert info.status == 0
    G.close()


def test_error_statuses():
    ptr, col, v = gpu_problem(2, 16, 0, 2)
    G = B.AMG()
    with pytest.raises(B.AmgError) as e:
        G.partial_rebuild(v)
    assert e.value.status == B.AMG_ERR_STATE
    bad = col.clone()
    bad[1], bad[2] = col[2], col[1]
    with pytest.raises(B.AmgError) as e:
        G.full_setup(ptr, bad, v)
    assert e.value.status == B.AMG_ERR_PATTERN
    nan = v.clone()
    nan[5] = float("nan")
    with pytest.raises(B.AmgError) as e:
        G.full_setup(ptr, col, nan)
    assert e.value.status == B.AMG_ERR_NONFINITE
    G.full_setup(ptr, col, v)
    with pytest.raises(B.AmgError) as e:
        G.partial_rebuild(nan)
    assert e.value.status == B.AMG_ERR_NONFINITE
    # the check covers every group of 32 rows: a NaN in the last entry (the
    # last group) and an infinity mid-matrix
    for pos, bad_v in ((v.numel() - 1, float("nan")), (v.numel() // 2 + 3, float("inf"))):
        G.full_setup(ptr, col, v)
        w = v.clone()
        w[pos] = bad_v
        with pytest.raises(B.AmgError) as e:
            G.partial_rebuild(w)
        assert e.value.status == B.AMG_ERR_NONFINITE
    # row pointers inconsistent with nnz (a truncated column array), decreasing
    # or not starting at 0: reported before any kernel reads the columns they
    # delimit, and the context then takes a good pattern
    G3 = B.AMG()
    cases = [(ptr, col[:-5].clone(), v[:-5].clone())]
    for pos, val in ((4, None), (0, 1)):
        bp = ptr.clone()
        bp[pos] = bp[pos + 1] + 1 if val is None else val
        cases.append((bp, col, v))
    for bp, bc, bv in cases:
        with pytest.raises(B.AmgError) as e:
            G3.full_setup(bp, bc, bv)
        assert e.value.status == B.AMG_ERR_PATTERN
        with pytest.raises(B.AmgError) as e:
            G3.step_solve_host(bv.cpu().numpy(), np.zeros(256), np.zeros(256), 1e-8)
        assert e.value.status in (B.AMG_ERR_PATTERN, B.AMG_ERR_STATE)
    G3.full_setup(ptr, col, v)
    u3, i3 = G3.solve(torch.tensor(I.rhs(256), device="cuda"), 1e-8)
    assert i3.status == 0
    G.full_setup(ptr, col, v)
    f = torch.tensor(I.rhs(256), device="cuda")
    G1 = B.AMG(maxiter=1, coarse_enough=16)
    G1.full_setup(ptr, col, v)
    u, info = G1.solve(f, 1e-14)
    assert info.status == B.AMG_NOT_CONVERGED and info.iters == 1
    # an indefinite system breaks CG down: reported, not trapped
    G2 = B.AMG(coarse_enough=16)
    G2.full_setup(ptr, col, v)
    neg = -v
    G2.partial_rebuild(neg)
    with pytest.raises(B.AmgError) as e:
        G2.solve(f, 1e-8)
    assert e.value.status in (B.AMG_ERR_BREAKDOWN,)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_solve_equals_eager_solve(precision):
    """The whole-solve CUDA graph (while-conditional loop) runs exactly the
    kernels of the host-driven loop: identical iterates and counts."""
    ptr, col, v = gpu_problem(3, 40, 5, 10)
    G = B.AMG(precision=precision)
    G.full_setup(ptr, col, v)
    f = torch.tensor(I.rhs(40 ** 3), device="cuda")
    u1, i1 = G.solve(f, 1e-8)
    u2, i2 = G.solve(f, 1e-8)           # graph reused
    G.profile(2)                        # timing of the host-driven launch loop
    u3, i3 = G.solve(f, 1e-8)
    G.profile(1)                        # timing through an unrolled graph
    u5, i5 = G.solve(f, 1e-8)
    G.profile(False)
    prof = G.profile_read()
    assert prof["cg_spmv"][1] > 0 and prof["cg_spmv"][0] > 0
    assert i1.iters == i2.iters == i3.iters == i5.iters and i1.status == i3.status == i5.status == 0
    assert torch.equal(u1, u2) and torch.equal(u1, u3) and torch.equal(u1, u5)
    u4, i4 = G.solve(f, 1e-11)          # a new tolerance rebuilds the graph
    assert i4.iters > i1.iters and i4.rel_resid <= 1e-11


def test_preventive_rebuilds():
    dim, N, T = 2, 32, 10
    ptr, col, _ = gpu_problem(dim, N, 0, T)
    f = I.rhs(N * N)
    ft = torch.tensor(f, device="cuda")
    vals = [oracle_problem(dim, N, k, T)[2] for k in range(T)]
    # every 3rd step: the schedule and the iterations follow the oracle
    G = B.AMG(rebuild_every=3)
    recs = O.run_time_steps(*oracle_problem(dim, N, 0, T)[:2], vals, f, O.MODE_PARTIAL, rebuild_every=3)
    for k in range(T):
        si = G.step(gpu_problem(dim, N, k, T)[2], ptr, col)
        _, info = G.solve(ft, 1e-8)
        assert bool(si.rebuilt) == recs[k].rebuilt == (k % 3 == 0)
        assert info.status == 0 and abs(info.iters - recs[k].iters) <= 1
    # iteration growth: every decision follows the GPU's own iteration counts
    G = B.AMG(rebuild_iter_growth=1.1)
    base, last, rebuilt_any = None, None, False
    for k in range(T):
        si = G.step(gpu_problem(dim, N, k, T)[2], ptr, col)
        _, info = G.solve(ft, 1e-8)
        if k > 0:
            assert bool(si.rebuilt) == (last > 1.1 * base)
            rebuilt_any |= bool(si.rebuilt)
        if si.rebuilt:
            base = info.iters
        last = info.iters
    assert rebuilt_any


def test_time_series_64cubed_partial_and_full_reuse():
    """64^3, the benchmark's grid (one lane per finest-level row): the time
    loop under partial and full reuse follows the oracle's."""
    dim, N, T = 3, 64, 50
    ptr, col, _ = gpu_problem(dim, N, 0, T)
    f = I.rhs(N ** 3)
    ft = torch.tensor(f, device="cuda")
    steps = [0, 1, 2, 3]
    vals = [oracle_problem(dim, N, k, T)[2] for k in steps]
    for mode in (B.MODE_PARTIAL, B.MODE_FULL_REUSE):
        recs = O.run_time_steps(*oracle_problem(dim, N, 0, T)[:2], vals, f, mode)
        G = B.AMG(mode=mode)
        for j, k in enumerate(steps):
            si = G.step(gpu_problem(dim, N, k, T)[2], ptr, col)
            u, info = G.solve(ft, 1e-8)
            # (full reuse: the kept hierarchy misses the tolerance on some steps, as in the oracle)
            assert bool(si.rebuilt) == recs[j].rebuilt and info.status == recs[j].status
            assert abs(info.iters - recs[j].iters) <= 1, (mode, k, info.iters, recs[j].iters)
            A = _sp(*oracle_problem(dim, N, k, T), N ** 3)
            res = np.linalg.norm(f - A @ u.cpu().numpy()) / np.linalg.norm(f)
            assert abs(res - info.rel_resid) <= 1e-6 * res + 1e-15
            if info.status == 0:
                assert res <= 1e-8


def _dense_csr(M):
    n = M.shape[0]
    ptr = np.arange(0, n * n + 1, n, dtype=np.int32)
    col = np.tile(np.arange(n, dtype=np.int32), n)
    return ptr, col, np.ascontiguousarray(M, np.float64).ravel()


@pytest.mark.parametrize("n", [1, 2, 5, 31, 32, 33, 48, 49, 87, 100, 127, 128, 129, 160, 161, 250, 448, 449, 500])
@pytest.mark.parametrize("dup", [False, True])
def test_coarsest_lu_with_tied_pivots_and_singular_input(n, dup):
    """The coarsest dense LU of every kernel size class (one block up to 48
    rows, the pipelined eight-CTA cluster up to 128 with whole and partial
    last column blocks, one block again up to 160, the eight-CTA cluster up to
    448, the global-memory kernel above) on
    a one-level hierarchy whose matrix is dense with small-integer entries, so
    that many candidates tie in magnitude: the pivots (first position of the
    largest magnitude) and the factors equal the oracle's bit for bit.  With a
    duplicated row the matrix is singular: the setup reports ERR_SINGULAR
    exactly when the oracle's elimination meets an all-zero column."""
    rng = np.random.default_rng(1000 + n)
    M = rng.integers(-3, 4, (n, n)).astype(np.float64)
    if dup and n >= 2:
        M[n // 2] = M[0]
    olu, opiv, ost = O.dense_lu(M)
    ptr, col, val = (torch.tensor(a, device="cuda") for a in _dense_csr(M))
    G = B.AMG(coarse_enough=n)
    if ost == O.ERR_SINGULAR:
        with pytest.raises(B.AmgError) as e:
            G.full_setup(ptr, col, val)
        assert e.value.status == B.AMG_ERR_SINGULAR
        return
    assert ost == O.OK
    G.full_setup(ptr, col, val)
    assert G.nlevels == 1
    lu, piv = G.coarse_lu()
    assert np.array_equal(piv, opiv)
    assert np.array_equal(lu, olu)


@pytest.mark.parametrize("j", [0, 3, 4, 31, 32, 50, 85, 86])
def test_pipelined_lu_zero_column_at_every_position(j):
    """A zero column j makes the elimination meet an all-zero candidate column
    exactly at step j (earlier steps subtract multiples of zeros from it). In
    the pipelined cluster kernel (n = 87, four-column blocks dealt to eight
    CTAs) j = 0, 3, 4, 31, 32, 50, 85, 86 put that step first or last in an
    owner's block, at an owner change, and at the final step (which sends no
    message): the setup reports ERR_SINGULAR as the oracle does, and a
    regular matrix factorised next by the same context matches the oracle
    bit for bit (the kernel left nothing behind)."""
    n = 87
    rng = np.random.default_rng(300 + j)
    M = rng.integers(-3, 4, (n, n)).astype(np.float64) + np.eye(n) * 20.0
    Z = M.copy()
    Z[:, j] = 0.0
    _, _, ost = O.dense_lu(Z)
    assert ost == O.ERR_SINGULAR
    G = B.AMG(coarse_enough=n)
    ptr, col, val = (torch.tensor(a, device="cuda") for a in _dense_csr(Z))
    with pytest.raises(B.AmgError) as e:
        G.full_setup(ptr, col, val)
    assert e.value.status == B.AMG_ERR_SINGULAR
    olu, opiv, ost = O.dense_lu(M)
    assert ost == O.OK
    G.full_setup(*(torch.tensor(a, device="cuda") for a in _dense_csr(M)))
    lu, piv = G.coarse_lu()
    assert np.array_equal(piv, opiv) and np.array_equal(lu, olu)


@pytest.mark.parametrize("N,ce,nL", [(32, 250, 191), (40, 400, 369)])
def test_cluster_lu_for_mid_size_coarsest_level(N, ce, nL):
    """A coarsest level between 160 and 448 rows is factorised by the
    eight-CTA cluster kernel: pivots identical to the oracle's, factors within
    1e-12, and the V-cycle (which uses the inverse from the column-major
    factors) and the solve as the oracle's."""
    dim, T = 3, 10
    ptr, col, v = gpu_problem(dim, N, 3, T)
    G = B.AMG(coarse_enough=ce)
    G.full_setup(ptr, col, v)
    H = O.Hierarchy(*oracle_problem(dim, N, 3, T), O.Params(coarse_enough=ce))
    assert G.nlevels == H.nlevels and H.sizes(H.nlevels - 1)[0] == nL
    lu, piv = G.coarse_lu()
    olu, opiv = H.lu()
    assert np.array_equal(piv, opiv)
    assert np.allclose(lu, olu, rtol=1e-12, atol=1e-14 * np.abs(olu).max())
    r = I.rhs(N ** dim, seed=5)
    z = G.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
    zo = H.vcycle(r)
    assert np.linalg.norm(z - zo) <= 1e-11 * np.linalg.norm(zo)
    f = I.rhs(N ** dim)
    u, info = G.solve(torch.tensor(f, device="cuda"), 1e-8)
    _, it, _, st = H.pcg(f, 1e-8)
    assert info.status == 0 and st == O.OK and abs(info.iters - it) <= 1


@pytest.mark.parametrize("n", [1, 5, 33, 87, 150, 160, 161, 300])
def test_coarse_inverse_every_size_class(n):
    """On a one-level hierarchy the V-cycle is the coarsest solve, the explicit
    inverse (from the LU factors) times r: against a dense solve of the same
    diagonally dominant matrix, for the one-row-per-thread kernel (n <= 160)
    and the column-major kernel above."""
    rng = np.random.default_rng(2000 + n)
    M = rng.uniform(-1.0, 1.0, (n, n))
    M[np.arange(n), np.arange(n)] = np.abs(M).sum(axis=1) + 1.0
    ptr, col, val = (torch.tensor(a, device="cuda") for a in _dense_csr(M))
    G = B.AMG(coarse_enough=n)
    G.full_setup(ptr, col, val)
    assert G.nlevels == 1
    r = rng.normal(size=n)
    z = G.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
    ref = np.linalg.solve(M, r)
    assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref) * np.linalg.cond(M)


@pytest.mark.parametrize("form", ["one_byte", "two_byte", "int32"])
def test_patterns_through_every_column_form(form):
    """The finest level's matrix kernels read one byte per entry when the rows
    use at most 256 distinct column offsets (band 120: up to 241 offsets),
    two-byte offsets when they all fit in 16 bits (band 140: up to 281
    distinct ones), and the int32 columns otherwise (couplings 40,000 rows
    apart): the form reported, then hierarchy, V-cycle and solve against the
    oracle in each."""
    if form == "int32":
        n = 48000
        ptr, col, val = I.random_wide_spd(n, 40000, 300, seed=5)
    else:
        n = 1500
        band = 120 if form == "one_byte" else 140
        ptr, col, val = I.random_banded_spd(n, band, 0.04, seed=band)
    offs = np.unique(col - np.repeat(np.arange(n), np.diff(ptr)))
    assert (offs.size <= 256) == (form == "one_byte")
    assert (np.abs(offs).max() > 32767) == (form == "int32")
    G = B.AMG(coarse_enough=40)
    G.full_setup(*(torch.tensor(a, device="cuda") for a in (ptr, col, val)))
    assert G.pattern_info()[0] == {"one_byte": 1, "two_byte": 2, "int32": 4}[form]
    H = O.Hierarchy(ptr, col, val, O.Params(coarse_enough=40))
    compare_hierarchy(G, H)
    r = np.random.default_rng(9).normal(size=n)
    z = G.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
    zo = H.vcycle(r)
    assert np.all(np.abs(z - zo) <= 1e-9 * vcycle_envelope(H, r))
    f = I.rhs(n)
    u, info = G.solve(torch.tensor(f, device="cuda"), 1e-8)
    uo, it, rr, st = H.pcg(f, 1e-8)
    assert info.status == 0 and st == 0 and abs(info.iters - it) <= 1
    A = _sp(ptr, col, val, n)
    assert np.linalg.norm(f - A @ u.cpu().numpy()) <= 1e-8 * np.linalg.norm(f)
