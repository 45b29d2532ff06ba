"""Pins of the oracle's time stepping, MGRIT and learned-network restatement.

* Heat: per grid and per sine mode, N backward-Euler steps scale the mode by
  rho^N with rho = 1 / (1 + dt * sum_i (4/h_i^2) sin^2(k_i pi h_i / 2)); the
  combined solution approaches exp(-d pi^2 t) prod sin(pi x_i).
* OU: the Gaussian law of the process (Sec. 4.4, Eq. "sde_analytical_solution",
  with mean e^{-theta t} m and variance s^2 e^{-2 theta t} +
  sigma^2 (1 - e^{-2 theta t}) / (2 theta)), first-order convergence, positivity.
* MGRIT (Alg. 2): converged MGRIT equals sequential stepping (Eq.
  "space_time_solution" has a unique solution); with FCF relaxation each cycle
  makes two more C-points exact, so ceil(Nc/2) cycles reproduce the
  sequential result for any coarse propagator; with Phi_coarse = Phi^m the
  coarse correction is exact and the second cycle sees a zero residual.
* Network: central finite differences of the loss, and closed-form special
  cases (all-zero weights give the identity map).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_22156_gb300 import workloads as W


def _nodes(P, g):
    l = P.levels[g]
    axes = [P.lo[i] + (P.hi[i] - P.lo[i]) * np.arange(1, 2 ** l[i]) / 2 ** l[i] for i in range(P.d)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.ravel() for m in mesh], axis=1)


def _problem(wl, n=None):
    return oracle.Problem(wl.d, n or wl.n, wl.L0, wl.op, wl.lo, wl.hi, wl.theta, wl.sigma, wl.vamp)


def _heat_discrete_closed_form(P, modes, dt, nsteps):
    out = np.zeros(P.n_total)
    for g in range(P.G):
        x = _nodes(P, g)
        h = (P.hi - P.lo) / 2.0 ** P.levels[g]
        for amp, k in modes:
            k = np.asarray(k, dtype=float)
            lam = np.sum(4.0 / h ** 2 * np.sin(k * np.pi * h / 2) ** 2)
            out[P.grid_slice(g)] += amp * (1 + dt * lam) ** (-nsteps) * np.prod(np.sin(np.pi * k * x), axis=1)
    return out


@pytest.mark.parametrize("k", [1, 2])
def test_heat_sequential_discrete_closed_form(k):
    wl = W.workload(k)
    n = wl.n if k == 1 else 5
    P = _problem(wl, n)
    u0 = P.initial(wl.ic_kind, wl.ic_params)
    steps = wl.nsteps if k == 1 else 32
    uT = P.sequential(u0, wl.dt, steps, rtol=1e-15)
    K = int(wl.ic_params[0])
    modes = [(wl.ic_params[1 + m * (wl.d + 1)], wl.ic_params[2 + m * (wl.d + 1): 1 + (m + 1) * (wl.d + 1)])
             for m in range(K)]
    ref = _heat_discrete_closed_form(P, modes, wl.dt, steps)
    np.testing.assert_allclose(uT, ref, rtol=0, atol=1e-12)


def test_heat_combined_against_continuous_solution():
    wl = W.workload(1)
    errs = []
    for n, steps in ((5, 64), (7, 256)):
        P = _problem(wl, n)
        u0 = P.initial(wl.ic_kind, wl.ic_params)
        uT = P.sequential(u0, wl.t1 / steps, steps, rtol=1e-13)
        pts = W.eval_points(2, wl.lo, wl.hi, n_uniform=2000, n_diag=33, seed=5)
        ref = math.exp(-2 * math.pi ** 2 * wl.t1) * np.prod(np.sin(np.pi * pts), axis=1)
        errs.append(np.linalg.norm(P.combine(uT, pts) - ref) / np.linalg.norm(ref))
    # backward Euler (first order in dt) plus the combination error (Sec. 2.2.1)
    assert errs[0] < 0.06 and errs[1] < errs[0] / 2.5, errs


def test_ou_gaussian_law_first_order_and_positivity():
    theta, sigma, m0, s0, T = 1.0, 1.0, 1.0, 0.5, 0.5
    errs = []
    for n in (7, 8, 9):
        P = oracle.Problem(1, n, 1, W.OP_OU, [-6.0], [6.0], theta, sigma)
        u0 = P.initial(W.IC_GAUSS, W.gauss_params([m0], [s0]))
        steps = 2 ** (n - 2)
        uT = P.sequential(u0, T / steps, steps, rtol=1e-14)
        x = _nodes(P, 0)[:, 0]
        mean = math.exp(-theta * T) * m0
        var = s0 ** 2 * math.exp(-2 * theta * T) + sigma ** 2 * (1 - math.exp(-2 * theta * T)) / (2 * theta)
        ref = np.exp(-0.5 * (x - mean) ** 2 / var) / math.sqrt(2 * math.pi * var)
        errs.append(np.linalg.norm(uT - ref) / np.linalg.norm(ref))
        assert np.all(uT >= 0.0)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 0.02 and np.all(rates > 0.8), (errs, rates)


def _mgrit_case(k, n=None, nsteps=None):
    wl = W.workload(k)
    P = _problem(wl, n)
    u0 = P.initial(wl.ic_kind, wl.ic_params)
    N = nsteps or wl.nsteps
    dt = (wl.t1 - wl.t0) / N
    return wl, P, u0, N, dt


def test_mgrit_converged_equals_sequential():
    wl, P, u0, N, dt = _mgrit_case(1)
    seq = P.sequential(u0, dt, N, rtol=1e-15)
    uT, its, hist, st = P.mgrit(u0, dt, N, wl.m, 2, tol=1e-13, maxit=50, rtol=1e-15)
    assert np.all(its < 16)           # converged before the FCF exactness bound
    np.testing.assert_allclose(uT, seq, rtol=0, atol=1e-11)
    # residual histories decrease monotonically until round-off
    for g in range(P.G):
        h = hist[g, :its[g]]
        assert np.all(np.diff(np.log10(h[h > 1e-12])) < 0)


def test_mgrit_fcf_exactness_after_half_nc_cycles():
    wl = W.workload(1)
    P = _problem(wl)
    u0 = W.random_vector(5, P.n_total)          # rough data: slow enough to see
    m, dt = wl.m, wl.dt
    for k in (1, 2):
        # Nc = 2k coarse intervals: k FCF cycles reproduce sequential stepping
        N = m * 2 * k
        seq = P.sequential(u0, dt, N, rtol=1e-15)
        uT, its, hist, st = P.mgrit(u0, dt, N, m, 2, tol=0.0, maxit=k, rtol=1e-15, check=False)
        assert np.all(its == k)
        np.testing.assert_allclose(uT, seq, rtol=0, atol=1e-13)
        # Nc = 2k + 2: the last C-point is not yet exact after k cycles
        N = m * (2 * k + 2)
        seq = P.sequential(u0, dt, N, rtol=1e-15)
        uT, *_ = P.mgrit(u0, dt, N, m, 2, tol=0.0, maxit=k, rtol=1e-15, check=False)
        assert np.max(np.abs(uT - seq)) > 1e-8


def test_mgrit_f_relaxation_exactness_after_nc_cycles():
    # F-relaxation carries exactness one coarse interval per cycle (FCF: two),
    # for any coarse propagator
    wl = W.workload(1)
    P = _problem(wl)
    u0 = W.random_vector(5, P.n_total)
    m, dt = wl.m, wl.dt
    for k in (1, 2, 3):
        N = m * k
        seq = P.sequential(u0, dt, N, rtol=1e-15)
        uT, its, hist, st = P.mgrit(u0, dt, N, m, 2, tol=0.0, maxit=k, rtol=1e-15, check=False, relax="F")
        assert np.all(its == k)
        np.testing.assert_allclose(uT, seq, rtol=0, atol=1e-13)
        # Nc = k + 1: not yet exact after k F cycles (FCF would be)
        N = m * (k + 1)
        seq = P.sequential(u0, dt, N, rtol=1e-15)
        uT, *_ = P.mgrit(u0, dt, N, m, 2, tol=0.0, maxit=k, rtol=1e-15, check=False, relax="F")
        assert np.max(np.abs(uT - seq)) > 1e-8
    # converged F-relaxation MGRIT is sequential stepping, also with three levels
    wl, P, u0, N, dt = _mgrit_case(2, n=4, nsteps=64)
    seq = P.sequential(u0, dt, N, rtol=1e-15)
    for levels, m in ((2, 8), (3, 4)):
        uT, its, hist, st = P.mgrit(u0, dt, N, m, levels, tol=1e-13, maxit=60, rtol=1e-15, relax="F")
        np.testing.assert_allclose(uT, seq, rtol=0, atol=1e-11)


def test_mgrit_coarse_sweep_initial_guess():
    # with Phi_c = Phi^m the initial coarse sweep is already the sequential
    # solution at every C-point: the first cycle sees no residual
    wl, P, u0, N, dt = _mgrit_case(1)
    seq = P.sequential(u0, dt, N, rtol=1e-15)
    uT, its, hist, st = P.mgrit(u0, dt, N, wl.m, 2, tol=0.0, maxit=1, coarse_kind=W.COARSE_EXACT,
                                rtol=1e-15, check=False, init=True)
    assert np.all(hist[:, 0] < 1e-13 * max(1.0, np.abs(u0).max()))
    np.testing.assert_allclose(uT, seq, rtol=0, atol=1e-12)
    # with the implicit coarse step it changes the iterates, not the fixed
    # point, and converges in no more cycles than the plain start
    for relax in ("FCF", "F"):
        a, its_a, *_ = P.mgrit(u0, dt, N, wl.m, 2, tol=1e-12, maxit=60, rtol=1e-15, relax=relax)
        b, its_b, *_ = P.mgrit(u0, dt, N, wl.m, 2, tol=1e-12, maxit=60, rtol=1e-15, relax=relax, init=True)
        np.testing.assert_allclose(b, seq, rtol=0, atol=1e-10)
        assert its_b.max() <= its_a.max()


def test_mgrit_exact_coarse_propagator_one_cycle():
    wl, P, u0, N, dt = _mgrit_case(1)
    uT, its, hist, st = P.mgrit(u0, dt, N, wl.m, 2, tol=0.0, maxit=3, coarse_kind=W.COARSE_EXACT,
                                rtol=1e-15, check=False)
    seq = P.sequential(u0, dt, N, rtol=1e-15)
    assert np.all(hist[:, 1] < 1e-13 * max(1.0, np.abs(u0).max()))
    np.testing.assert_allclose(uT, seq, rtol=0, atol=1e-12)


def test_mgrit_three_level_and_ou_bicgstab():
    # three levels on a small d = 3 heat problem: 64 steps, m = 4 -> 16 -> 4
    wl, P, u0, N, dt = _mgrit_case(2, n=4, nsteps=64)
    seq = P.sequential(u0, dt, N, rtol=1e-15)
    uT, its, hist, st = P.mgrit(u0, dt, N, 4, 3, tol=1e-13, maxit=40, rtol=1e-15)
    np.testing.assert_allclose(uT, seq, rtol=0, atol=1e-11)
    assert np.all(its < 16)
    # drift operator (BiCGStab inside Phi)
    wl, P, u0, N, dt = _mgrit_case(3, n=3, nsteps=64)
    seq = P.sequential(u0, dt, N, rtol=1e-15)
    uT, its, hist, st = P.mgrit(u0, dt, N, wl.m, 2, tol=1e-14, maxit=40, rtol=1e-15)
    np.testing.assert_allclose(uT, seq, rtol=0, atol=1e-12)


def test_net_gradient_finite_differences_and_identity():
    P = oracle.Problem(2, 3, 1, W.OP_VARHEAT, vamp=0.5)
    npar = P.net_param_count()
    assert npar == 16 * 3 * 5 + 16 + 2 * (16 * 17 * 5 + 16) + (1 * 17 * 5 + 1)
    theta = 0.2 * W.normal(21, npar)
    u = W.random_vector(22, 2 * P.n_total)
    y = W.random_vector(23, 2 * P.n_total)
    dT = 0.01
    loss, grad = P.net_loss_grad(dT, theta, u, y)
    eps = 1e-6
    idx = np.unique(np.concatenate([np.arange(0, npar, 97), [npar - 1, npar - 2, 16 * 3 * 5]]))
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        lp, _ = P.net_loss_grad(dT, tp, u, y)
        lm, _ = P.net_loss_grad(dT, tm, u, y)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, grad[k])
    # zero parameters: identity; only the last bias: constant shift
    z = np.zeros(npar)
    np.testing.assert_array_equal(P.net_forward(dT, z, u), u)
    z[-1] = 0.25
    # output bias b: u + sigma * b per grid, sigma = RMS of the grid's state
    out = P.net_forward(dT, z, u)
    for b in range(2):
        for g in range(P.G):
            sl = slice(b * P.n_total + P.offsets[g], b * P.n_total + P.offsets[g + 1])
            sigma = np.sqrt(np.mean(u[sl] ** 2))
            np.testing.assert_allclose(out[sl], u[sl] + 0.25 * sigma, atol=1e-15)
    # scale equivariance: N(alpha u) = alpha N(u) for alpha > 0
    np.testing.assert_allclose(P.net_forward(dT, theta, 3.0 * u), 3.0 * P.net_forward(dT, theta, u), rtol=1e-12)
    # the loss of the identity map against y is sum ||u - y||^2 / ||y||^2
    l0, _ = P.net_loss_grad(dT, np.zeros(npar), u, y)
    ref = 0.0
    for b in range(2):
        for g in range(P.G):
            sl = slice(b * P.n_total + P.offsets[g], b * P.n_total + P.offsets[g + 1])
            ref += np.sum((u[sl] - y[sl]) ** 2) / np.sum(y[sl] ** 2)
    assert abs(l0 - ref) < 1e-12 * ref
