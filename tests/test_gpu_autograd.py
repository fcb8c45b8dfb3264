"""Differentiable solve: adjoint gradients of L = 1/2 |u - u*|^2 with respect to
the per-cell log-density theta, where u = A(exp theta)^-1 f.

The backward pass solves A lam = u - u* with the hierarchy of the forward pass
(A is symmetric) and forms dL/dtheta in one kernel.  Checks:
  * small grid: against central differences of exact (dense) solves;
  * 64^3 (the differentiable-solve workload): against the FP64 oracle's
    adjoint gradient, in FP64 and in mixed precision, and against central
    differences (h = 2e-3, error estimated from h = 1e-3 and 4e-3) of GPU
    solves converged to a relative residual of 1e-15 on 32 seeded cells.
"""
import numpy as np
import pytest

import oracle as O
from paper_2108_02054_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2108_02054_gb300 import amg as B
    from paper_2108_02054_gb300.autograd import PoissonSolver, solve


def _dense(dim, N, theta):
    p, c, v = O.poisson_assemble(dim, N, np.exp(theta))
    return O.CSR(p, c, v, N ** dim).dense()


def test_adjoint_small_grid_against_dense_finite_differences():
    dim, N = 3, 10
    n = N ** dim
    theta0 = np.log(I.density(dim, N, 0, 1)) + np.random.default_rng(1).normal(0, 0.1, n)
    f = I.rhs(n)
    ut = np.linalg.solve(_dense(dim, N, theta0 + np.random.default_rng(2).normal(0, 0.1, n)), f)
    S = PoissonSolver(dim, N, tol=1e-13, coarse_enough=40)
    th = torch.tensor(theta0, device="cuda", requires_grad=True)
    ft = torch.tensor(f, device="cuda", requires_grad=True)
    u = solve(th, ft, S)
    L = 0.5 * ((u - torch.tensor(ut, device="cuda")) ** 2).sum()
    L.backward()
    g = th.grad.cpu().numpy()
    assert S.last_info.status == 0 and S.adjoint_info.status == 0

    def loss(t):
        return 0.5 * np.sum((np.linalg.solve(_dense(dim, N, t), f) - ut) ** 2)

    # the adjoint formula on exact (dense) solutions: the reference gradient
    A0 = _dense(dim, N, theta0)
    u_ex = np.linalg.solve(A0, f)
    lam = np.linalg.solve(A0, u_ex - ut)
    g_ex = O.poisson_grad_theta(dim, N, np.exp(theta0), u_ex, lam)
    gmax = np.abs(g_ex).max()
    assert np.abs(g - g_ex).max() <= 1e-6 * gmax, np.abs(g - g_ex).max() / gmax
    L0 = loss(theta0)
    h = 1e-6
    fd_round = 20 * np.finfo(float).eps * abs(L0) / h
    worst = 0.0
    for cell in I.fd_cells(n, 32, seed=3):
        e = np.zeros(n)
        e[cell] = h
        fd = (loss(theta0 + e) - loss(theta0 - e)) / (2 * h)
        # components are sums of face terms that cancel: the error is measured
        # against the gradient's size, plus the differences' rounding
        assert abs(g[cell] - fd) <= 1e-6 * gmax + fd_round, (cell, g[cell], fd)
        worst = max(worst, abs(g[cell] - fd) / gmax)
    print(f"small grid: |g - g_exact|/|g| = {np.abs(g - g_ex).max() / gmax:.2e}, FD worst {worst:.2e}")
    # dL/df = lam = A^-1 (u - u*)
    assert np.allclose(ft.grad.cpu().numpy(), lam, rtol=1e-8, atol=1e-10 * np.abs(lam).max())


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_64cubed_against_oracle_gradient_and_fd(precision):
    dim, N = 3, 64
    n = N ** dim
    theta0 = I.noisy_log_density(dim, N, seed=1)
    f = I.rhs(n)
    theta_t = I.target_log_density(theta0, seed=2)
    # the target and the gradient reference come from the FP64 oracle
    pt, ct, vt = O.poisson_assemble(dim, N, np.exp(theta_t))
    Ht = O.Hierarchy(pt, ct, vt)
    ut, _, _, st = Ht.pcg(f, 1e-13, 300)
    assert st == 0
    p0, c0, v0 = O.poisson_assemble(dim, N, np.exp(theta0))
    H0 = O.Hierarchy(p0, c0, v0)
    uo, _, _, st = H0.pcg(f, 1e-13, 300)
    lamo, _, _, st2 = H0.pcg(uo - ut, 1e-13, 300)
    assert st == 0 and st2 == 0
    go = O.poisson_grad_theta(dim, N, np.exp(theta0), uo, lamo)

    tol = 1e-13 if precision == 0 else 1e-12
    S = PoissonSolver(dim, N, tol=tol, precision=precision, maxiter=300)
    utt = torch.tensor(ut, device="cuda")
    th = torch.tensor(theta0, device="cuda", requires_grad=True)
    ft = torch.tensor(f, device="cuda")
    u = solve(th, ft, S)
    L = 0.5 * ((u - utt) ** 2).sum()
    L.backward()
    g = th.grad.cpu().numpy()
    assert S.last_info.status == 0 and S.adjoint_info.status == 0
    gmax = np.abs(go).max()
    err = np.abs(g - go).max() / gmax
    print(f"64^3 precision={precision}: |g - g_oracle|/|g| = {err:.2e}, iters fwd {S.last_info.iters} "
          f"adj {S.adjoint_info.iters}")
    assert err <= 1e-6, err
    # per cell against the FP64 oracle gradient: 1e-6 relative, plus a floor
    # of 1e-9 max|g| for cells whose gradient is far below the largest (the
    # solves stop at a relative residual of 1e-13 / 1e-12)
    gate = 1e-6 * np.abs(go) + 1e-9 * gmax
    assert np.all(np.abs(g - go) <= gate), np.max(np.abs(g - go) / gate)
    big = np.abs(go) >= 1e-3 * gmax
    rel = np.abs(g - go)[big] / np.abs(go)[big]
    print(f"64^3 precision={precision}: per cell |g - g_oracle|/|g_oracle| over the {big.sum()} cells with "
          f"|g| >= 1e-3 max|g|: median {np.median(rel):.2e}, max {rel.max():.2e}")

    # central differences of GPU solves (partial rebuilds of the same hierarchy).
    # L(t + he) - L(t - he) is formed from the two solutions as
    # 0.5 sum (u+ - u-)(u+ + u- - 2 u*): subtracting the two loss values
    # (|L| ~ 8e5, each a sum of n squares) would leave their rounding, about
    # log2(n) eps |L|, in every quotient (~1e-3 at h = 1e-6); this form rounds
    # relative to the difference itself.
    #
    # The probes' solves go to a relative residual of 1e-15 (the FP64 outer
    # CG's floor; a stagnating last digit is accepted): at the gradient's
    # 1e-13 / 1e-12 their error dominated the quotients
    def usol(t):
        with torch.no_grad():
            S.refresh(S.assemble(torch.tensor(t, device="cuda"))[1])
            uu, _ = S.amg.solve(ft.detach().contiguous(), 1e-15, allow_not_converged=True)
            return uu.clone()

    def quotient(cell, hh):
        e = np.zeros(n)
        e[cell] = hh
        up, um = usol(theta0 + e), usol(theta0 - e)
        prod = (up - um) * (up + um - 2.0 * utt)
        d = 0.5 * float(prod.sum())
        # rounding of the sum (pairwise, at most log2(n) levels) and of its terms
        rnd = (np.log2(n) + 4) * np.finfo(float).eps * 0.5 * float(prod.abs().sum())
        return d / (2 * hh), rnd / (2 * hh)

    # each quotient's own error: the solves' and the truncation. The solves
    # reach a relative residual of about 2e-15, and the attainable accuracy
    # of u still leaves about 6e-9 / h (relative) in a quotient (measured over
    # h = 1e-5 ... 1e-2: 6e-4 at 1e-5, 4e-5 at 1e-4, 9e-6 at 1e-3), while
    # truncation grows as h^2 past h ~ 3e-3.  So the quotient is taken at
    # h = 2e-3, and its error is estimated per cell as twice the spread of the
    # quotients at h = 1e-3, 2e-3 and 4e-3, plus rounding.
    fds, noise = {}, {}
    for cell in I.fd_cells(n, 32, seed=3):
        qs = [quotient(int(cell), hh) for hh in (1e-3, 2e-3, 4e-3)]
        vals = [q for q, _ in qs]
        fds[int(cell)] = vals[1]
        noise[int(cell)] = 2 * (max(vals) - min(vals)) + sum(r for _, r in qs)
    gm = np.abs(go).max()
    limited, rels = 0, []
    for cell, fd in fds.items():
        err = abs(g[cell] - fd)
        # per cell: 1e-6 relative to the difference quotient, plus its own error
        assert err <= 1e-6 * abs(fd) + noise[cell], (cell, g[cell], fd, noise[cell])
        rels.append(err / abs(fd))
        if noise[cell] > 1e-6 * abs(fd):
            limited += 1
    rels = np.array(rels)
    print(f"64^3 precision={precision}: FD (h=2e-3, 32 cells) per-cell |g - fd|/|fd|: median {np.median(rels):.2e}, "
          f"max {rels.max():.2e}; cells whose FD error estimate exceeds 1e-6 |fd|: {limited} of {len(fds)} "
          f"(largest estimate {max(noise.values()):.2e} = {max(noise.values()) / gm:.2e} max|g|)")


def test_log_density_assembly_and_gradient_kernels():
    """The log-density calls equal the density calls on rho = exp(theta)."""
    dim, N = 3, 12
    n = N ** dim
    theta = I.noisy_log_density(dim, N, seed=4)
    ptr, col = B.poisson_pattern(dim, N)
    th = torch.tensor(theta, device="cuda")
    v_log = B.poisson_values_log(dim, N, th, ptr).cpu().numpy()
    _, _, v_ref = O.poisson_assemble(dim, N, np.exp(theta))
    assert np.allclose(v_log, v_ref, rtol=4e-16 * 8, atol=0)
    rng = np.random.default_rng(6)
    u, lam = rng.normal(size=n), rng.normal(size=n)
    g_log = B.poisson_grad_log(dim, N, th, torch.tensor(u, device="cuda"),
                               torch.tensor(lam, device="cuda")).cpu().numpy()
    g_ref = O.poisson_grad_theta(dim, N, np.exp(theta), u, lam)
    assert np.allclose(g_log, g_ref, rtol=1e-13, atol=1e-13 * np.abs(g_ref).max())


def test_backward_after_a_second_forward_uses_its_own_theta():
    """forward(theta1), forward(theta2), then the backward of the first: the
    adjoint must solve with A(theta1), not with the hierarchy theta2 left."""
    dim, N = 3, 10
    n = N ** dim
    theta1 = np.log(I.density(dim, N, 0, 1)) + np.random.default_rng(1).normal(0, 0.1, n)
    theta2 = theta1 + np.random.default_rng(8).normal(0, 0.5, n)
    f = I.rhs(n)
    ut = np.linalg.solve(_dense(dim, N, theta1 + np.random.default_rng(2).normal(0, 0.1, n)), f)
    S = PoissonSolver(dim, N, tol=1e-13, coarse_enough=40)
    utt = torch.tensor(ut, device="cuda")
    ft = torch.tensor(f, device="cuda")
    th1 = torch.tensor(theta1, device="cuda", requires_grad=True)
    th2 = torch.tensor(theta2, device="cuda", requires_grad=True)
    L1 = 0.5 * ((solve(th1, ft, S) - utt) ** 2).sum()
    L2 = 0.5 * ((solve(th2, ft, S) - utt) ** 2).sum()
    L1.backward()
    A1 = _dense(dim, N, theta1)
    u1 = np.linalg.solve(A1, f)
    g1 = O.poisson_grad_theta(dim, N, np.exp(theta1), u1, np.linalg.solve(A1, u1 - ut))
    g = th1.grad.cpu().numpy()
    assert np.abs(g - g1).max() <= 1e-6 * np.abs(g1).max()
    L2.backward()
    A2 = _dense(dim, N, theta2)
    u2 = np.linalg.solve(A2, f)
    g2 = O.poisson_grad_theta(dim, N, np.exp(theta2), u2, np.linalg.solve(A2, u2 - ut))
    assert np.abs(th2.grad.cpu().numpy() - g2).max() <= 1e-6 * np.abs(g2).max()
