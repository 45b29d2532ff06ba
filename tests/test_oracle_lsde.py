"""Pins of the oracle's linear-SDE Fokker-Planck operator (Sec. 4.4, Eqs.
"sde", "sde_fokker_planck", "sde_analytical_solution"): dX = A X dt + sigma dW
with a full drift matrix A and H = 2 sigma D sigma^T, so that
  u_t = -sum_i d_i((A x)_i u) + (1/2) sum_ij H_ij d_i d_j u.

  - with A = -theta I and H = sigma^2 I it is the diagonal (OU) operator;
  - on a normal density with a full covariance its nodal values approach the
    analytic operator, written out in numpy from the density's derivatives
    (d_i p = -p g_i, d_i d_j p = p (g_i g_j - Cinv_ij), g = Cinv (x - M)),
    at first order in h (donor-cell drift);
  - with the central drift flux (the paper's second-order finite differences)
    the same comparison converges at second order, and the symmetric part of
    the drift operator is trace(A) times the identity (the face fluxes are
    skew, only the divergence of the velocity field, trace A, is left);
  - the flux form and the four-point mixed stencil conserve mass away from
    the boundary;
  - a normal initial density evolves towards the closed-form normal law of
    the SDE, mean e^{At} M and covariance e^{At} C e^{A^T t} + int_0^t e^{As}
    H e^{A^T s} ds (computed with scipy), the error shrinking with the level
    and the step;
  - BiCGStab solves the non-symmetric backward-Euler system like a dense
    direct solve.
"""
import numpy as np
import pytest

import oracle
from paper_2509_22156_gb300 import workloads as W

scipy_linalg = pytest.importorskip("scipy.linalg")
integrate = pytest.importorskip("scipy.integrate")

A2 = np.array([[-0.4, 1.0], [-1.0, -0.3]])
H2 = np.array([[0.3, 0.1], [0.1, 0.5]])


def gauss_params(M, C):
    return np.concatenate([np.asarray(M, float), np.asarray(C, float).ravel()])


def node_coords(O, g):
    shape = tuple(int(2 ** l - 1) for l in O.levels[g])
    idx = np.indices(shape).reshape(len(shape), -1).T
    h = (O.hi - O.lo) / 2.0 ** O.levels[g]
    return O.lo + (idx + 1) * h


def gauss(x, M, C):
    Ci = np.linalg.inv(C)
    z = x - M
    q = np.einsum("ni,ij,nj->n", z, Ci, z)
    return np.exp(-0.5 * q) / np.sqrt((2 * np.pi) ** len(M) * np.linalg.det(C))


def analytic_L(x, M, C, A, H):
    Ci = np.linalg.inv(C)
    p = gauss(x, M, C)
    g = (x - M) @ Ci.T
    Ax = x @ A.T
    drift = p * (np.trace(A) - np.sum(Ax * g, axis=1))
    diff = 0.5 * p * (np.einsum("ni,ij,nj->n", g, H, g) - np.trace(H @ Ci))
    return drift - diff


def test_diagonal_drift_reduces_to_the_ou_operator():
    for d in (2, 3):
        Ou = oracle.Problem(d, 5, 1, W.OP_OU, lo=[-6.0] * d, hi=[6.0] * d, theta=0.7, sigma=1.3)
        Ls = oracle.Problem(d, 5, 1, oracle.OP_LSDE, lo=[-6.0] * d, hi=[6.0] * d,
                            drift=-0.7 * np.eye(d), diffusion=1.3 ** 2 * np.eye(d))
        p = W.random_vector(5, Ou.n_total)
        # (equal up to the rounding of A_ii (x + h/2) against A_ii x + A_ii h/2)
        np.testing.assert_allclose(Ls.apply(0.01, p), Ou.apply(0.01, p), rtol=0, atol=1e-15)


def test_gaussian_initial_value_matches_the_density():
    M, C = np.array([0.5, -0.3]), np.array([[0.6, 0.2], [0.2, 0.4]])
    O = oracle.Problem(2, 6, 1, oracle.OP_LSDE, lo=[-5.0] * 2, hi=[5.0] * 2, drift=A2, diffusion=H2)
    u = O.initial(4, gauss_params(M, C))
    for g in range(O.G):
        np.testing.assert_allclose(u[O.grid_slice(g)], gauss(node_coords(O, g), M, C), rtol=1e-13, atol=1e-300)


def test_operator_is_first_order_consistent_on_a_full_covariance_gaussian():
    M, C = np.array([0.4, -0.2]), np.array([[0.5, 0.2], [0.2, 0.4]])
    errs = []
    for lev in (5, 6, 7):
        # one isotropic grid of level lev: d = 2, combination level 2 lev - 1, L0 = lev
        O = oracle.Problem(2, 2 * lev - 1, lev, oracle.OP_LSDE, lo=[-4.0] * 2, hi=[4.0] * 2, drift=A2,
                           diffusion=H2)
        g = [k for k in range(O.G) if tuple(O.levels[k]) == (lev, lev)][0]
        x = node_coords(O, g)
        p = O.initial(4, gauss_params(M, C))
        dt = 1.0
        Lp = (O.apply(dt, p) - p)[O.grid_slice(g)] / dt
        ref = analytic_L(x, M, C, A2, H2)
        errs.append(np.abs(Lp - ref).max() / np.abs(ref).max())
    # measured 0.48, 0.26, 0.13: first order
    assert errs[0] / errs[1] > 1.6 and errs[1] / errs[2] > 1.6, errs
    assert errs[2] < 0.2, errs


def test_central_drift_is_second_order_consistent_on_a_full_covariance_gaussian():
    M, C = np.array([0.4, -0.2]), np.array([[0.5, 0.2], [0.2, 0.4]])
    errs = []
    for lev in (5, 6, 7):
        O = oracle.Problem(2, 2 * lev - 1, lev, oracle.OP_LSDE, lo=[-4.0] * 2, hi=[4.0] * 2, drift=A2,
                           diffusion=H2, central=True)
        g = [k for k in range(O.G) if tuple(O.levels[k]) == (lev, lev)][0]
        p = O.initial(4, gauss_params(M, C))
        Lp = (O.apply(1.0, p) - p)[O.grid_slice(g)]
        ref = analytic_L(node_coords(O, g), M, C, A2, H2)
        errs.append(np.abs(Lp - ref).max() / np.abs(ref).max())
    # measured 0.060, 0.016, 0.0040: second order
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
    assert errs[2] < 0.005, errs


@pytest.mark.parametrize("central", [False, True])
def test_symmetric_part_of_the_central_drift_is_the_trace(central):
    # (I + dt L) assembled column by column on every grid of a small problem,
    # drift only: M + M^T - 2 I = dt (L + L^T) = dt trace(A) I for the central
    # flux; the donor-cell flux adds numerical diffusion, which this detects
    A = np.array([[-0.4, 1.0], [-1.0, -0.3]])
    dt = 0.1
    O = oracle.Problem(2, 4, 1, oracle.OP_LSDE, lo=[-3.0] * 2, hi=[3.0] * 2, drift=A, diffusion=np.zeros((2, 2)),
                       central=central)
    worst = 0.0
    for g in range(O.G):
        sl = O.grid_slice(g)
        n = sl.stop - sl.start
        Mx = np.zeros((n, n))
        for k in range(n):
            e = np.zeros(O.n_total)
            e[sl.start + k] = 1.0
            Mx[:, k] = O.apply(dt, e)[sl]
        S = (Mx + Mx.T - 2.0 * np.eye(n)) / dt
        worst = max(worst, float(np.abs(S - np.trace(A) * np.eye(n)).max()))
    if central:
        assert worst < 1e-13
    else:
        assert worst > 1.0


@pytest.mark.parametrize("central", [False, True])
def test_mass_is_conserved_away_from_the_boundary(central):
    M, C = np.array([0.3, 0.1, -0.2]), np.array([[0.4, 0.1, 0.0], [0.1, 0.5, 0.1], [0.0, 0.1, 0.3]])
    A3 = np.array([[-0.5, 0.3, 0.0], [-0.2, -0.4, 0.6], [0.1, -0.6, -0.3]])
    H3 = np.array([[0.4, 0.1, 0.0], [0.1, 0.3, 0.05], [0.0, 0.05, 0.2]])
    # a box wide enough that the density is negligible at the boundary nodes
    O = oracle.Problem(3, 8, 3, oracle.OP_LSDE, lo=[-9.0] * 3, hi=[9.0] * 3, drift=A3, diffusion=H3,
                       central=central)
    p = O.initial(4, gauss_params(M, C))
    q = O.apply(0.01, p)
    for g in range(O.G):
        sl = O.grid_slice(g)
        assert abs(np.sum(q[sl] - p[sl])) <= 1e-9 * np.sum(p[sl])


def law(t, M, C, A, H):
    E = scipy_linalg.expm(A * t)
    integrand = lambda s: (scipy_linalg.expm(A * s) @ H @ scipy_linalg.expm(A * s).T).ravel()
    Q = integrate.quad_vec(integrand, 0.0, t, epsabs=1e-13, epsrel=1e-12)[0].reshape(A.shape)
    return E @ M, E @ C @ E.T + Q


def test_backward_euler_approaches_the_closed_form_law():
    M, C = np.array([1.0, 1.0]), np.array([[0.25, 0.0], [0.0, 0.25]])
    T = 0.5
    Mt, Ct = law(T, M, C, A2, H2)
    pts = W.eval_points(2, [-3.0, -3.0], [4.0, 4.0], n_uniform=3000, n_diag=0)
    ref = gauss(pts, Mt, Ct)
    errs = {}
    for central in (False, True):
        errs[central] = []
        for n, N in ((6, 16), (7, 64), (8, 256)):
            O = oracle.Problem(2, n, 3, oracle.OP_LSDE, lo=[-6.0] * 2, hi=[6.0] * 2, drift=A2, diffusion=H2,
                               central=central)
            u = O.sequential(O.initial(4, gauss_params(M, C)), T / N, N, rtol=1e-13)
            errs[central].append(np.linalg.norm(O.combine(u, pts) - ref) / np.linalg.norm(ref))
    up, ce = errs[False], errs[True]
    # donor cell, measured 0.50, 0.31, 0.19: its drift and backward Euler are
    # first order, the combination second order
    assert up[0] / up[1] > 1.4 and up[1] / up[2] > 1.4 and up[2] < 0.25, up
    # central, measured 0.36, 0.17, 0.078: below the donor cell at every level
    assert ce[0] / ce[1] > 1.8 and ce[1] / ce[2] > 1.8 and ce[2] < 0.1, ce
    assert all(c < u for c, u in zip(ce, up)), errs


def test_bicgstab_matches_a_dense_solve():
    O = oracle.Problem(2, 5, 1, oracle.OP_LSDE, lo=[-4.0] * 2, hi=[4.0] * 2, drift=A2, diffusion=H2)
    b = W.random_vector(6, O.n_total)
    x = O.phi(0.3, b, rtol=1e-15)
    for g in range(O.G):
        sl = O.grid_slice(g)
        np.testing.assert_allclose(x[sl], O.dense_solve(g, 0.3, b[sl]), rtol=0, atol=1e-12 * np.abs(b).max())
