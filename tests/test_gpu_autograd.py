"""Differentiable solve: adjoint gradients of L = 1/2 |u - u*|^2 with respect to
the per-cell log-density theta, where u = A(exp theta)^-1 f.

The backward pass solves A lam = u - u* with the hierarchy of the forward pass
(A is symmetric) and forms dL/dtheta in one kernel.  Checks:
  * small grid: against central differences of exact (dense) solves;
  * 64^3 (the differentiable-solve workload): against the FP64 oracle's
    adjoint gradient, in FP64 and in mixed precision, and against central
    differences (h = 1e-6) of tightly converged GPU solves on 32 seeded cells.
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

    # central differences of GPU solves (partial rebuilds of the same hierarchy)
    tol_fd = tol

    def loss(t, tol_=tol_fd):
        S.tol = tol_
        with torch.no_grad():
            uu = solve(torch.tensor(t, device="cuda"), ft, S)
        S.tol = tol
        return 0.5 * float(((uu - utt) ** 2).sum())

    # each difference quotient's own error: solver noise (each loss value
    # carries its solve's error, which the +h and -h solves need not share)
    # plus rounding; estimated per cell as twice the change of the quotient
    # between h and 2 h (truncation, O(h^2), is far below it), plus 4 eps |L| / h
    h = 1e-6
    L0 = loss(theta0)
    fds, noise = {}, {}
    for cell in I.fd_cells(n, 32, seed=3):
        e = np.zeros(n)
        e[cell] = 1.0
        fd = (loss(theta0 + h * e) - loss(theta0 - h * e)) / (2 * h)
        fd2 = (loss(theta0 + 2 * h * e) - loss(theta0 - 2 * h * e)) / (4 * h)
        fds[int(cell)] = fd
        noise[int(cell)] = 2 * abs(fd - fd2) + 4 * np.finfo(float).eps * abs(L0) / h
    gm = np.abs(go).max()
    worst_rel, limited, rels = 0.0, 0, []
    for cell, fd in fds.items():
        err = abs(g[cell] - fd)
        # per cell: 1e-6 relative to the difference quotient, plus its own error
        assert err <= 1e-6 * abs(fd) + noise[cell], (cell, g[cell], fd, noise[cell])
        rels.append(err / abs(fd))
        if noise[cell] > 1e-6 * abs(fd):
            limited += 1
    rels = np.array(rels)
    print(f"64^3 precision={precision}: FD (h=1e-6, 32 cells) per-cell |g - fd|/|fd|: median {np.median(rels):.2e}, "
          f"max {rels.max():.2e}; cells whose FD error estimate exceeds 1e-6 |fd|: {limited} of {len(fds)} "
          f"(largest estimate {max(noise.values()):.2e} = {max(noise.values()) / gm:.2e} max|g|, |L| = {L0:.3e})")


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
