"""Pins of the oracle's operators, Krylov solvers and backward-Euler steps.

* Heat: sin(k pi x) is an eigenvector of the 1-D second difference with
  eigenvalue (4/h^2) sin^2(k pi h / 2), so (I + dt L) acts on a product of
  sines by an exactly known factor, and BE steps decay it by its inverse.
* The matrix probed from the stencil equals the Kronecker-sum assembly of
  the 1-D operators (catches stride, ordering and boundary mistakes).
* Consistency with the continuous operators: second order for the
  (variable-coefficient) diffusion, first order for the upwinded drift.
* OU drift: discrete mass conservation away from the boundary, M-matrix sign
  pattern; variable coefficient: symmetry, reduction to heat at amplitude 0.
* CG / BiCGStab against a dense direct solve on tiny grids.
"""
import numpy as np
import pytest

import oracle
from paper_2509_22156_gb300 import workloads as W


def _node_axes(P, g):
    l = P.levels[g]
    return [P.lo[i] + (P.hi[i] - P.lo[i]) * np.arange(1, 2 ** l[i]) / 2 ** l[i] for i in range(P.d)]


def _nodes(P, g):
    mesh = np.meshgrid(*_node_axes(P, g), indexing="ij")
    return np.stack([m.ravel() for m in mesh], axis=1)


def _probe(P, g, dt):
    """Dense matrix of (I + dt L) on grid g, probed column by column."""
    sl = P.grid_slice(g)
    n = sl.stop - sl.start
    A = np.zeros((n, n))
    e = np.zeros(P.n_total)
    for k in range(n):
        e[:] = 0
        e[sl.start + k] = 1
        A[:, k] = P.apply(dt, e)[sl]
    return A


@pytest.mark.parametrize("d,n", [(2, 5), (3, 4), (4, 3)])
def test_heat_eigenfunctions(d, n):
    P = oracle.Problem(d, n)
    dt = 0.013
    rng_k = [1, 2, 3, 1, 2, 1]
    u = np.zeros(P.n_total)
    ref = np.zeros(P.n_total)
    for g in range(P.G):
        x = _nodes(P, g)
        k = np.array(rng_k[:d])
        v = np.prod(np.sin(np.pi * k * x), axis=1)
        h = 1.0 / 2.0 ** P.levels[g]
        lam = np.sum(4.0 / h ** 2 * np.sin(k * np.pi * h / 2) ** 2)
        u[P.grid_slice(g)] = v
        ref[P.grid_slice(g)] = (1 + dt * lam) * v
    np.testing.assert_allclose(P.apply(dt, u), ref, rtol=0, atol=1e-11 * np.max(np.abs(ref)))
    # one backward-Euler step divides by the same factor
    out = P.phi(dt, ref, rtol=1e-15)
    np.testing.assert_allclose(out, u, rtol=0, atol=1e-12)


def _oned(op, N, h, x, dt, theta=1.0, sigma=1.0):
    """1-D pieces of the Kronecker-sum assembly (zero Dirichlet values)."""
    T = (2 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)) / h ** 2
    if op == W.OP_HEAT:
        return T
    # donor-cell flux difference: F_{j+1/2} = v+ p_j + v- p_{j+1}, v = -theta x
    D = np.zeros((N, N))
    for j in range(N):
        vp = -theta * (x[j] + h / 2)
        vm = -theta * (x[j] - h / 2)
        D[j, j] += max(vp, 0) / h - min(vm, 0) / h
        if j + 1 < N:
            D[j, j + 1] += min(vp, 0) / h
        if j - 1 >= 0:
            D[j, j - 1] -= max(vm, 0) / h
    return D + 0.5 * sigma ** 2 * T


@pytest.mark.parametrize("op,lo,hi", [(W.OP_HEAT, 0.0, 1.0), (W.OP_OU, -6.0, 6.0), (W.OP_OU, -1.0, 3.0)])
def test_stencil_equals_kronecker_assembly(op, lo, hi):
    d = 3
    P = oracle.Problem(d, 4, 1, op, [lo] * d, [hi] * d, theta=0.7, sigma=1.3)
    dt = 0.01
    for g in range(P.G):
        axes = _node_axes(P, g)
        Ns = [len(a) for a in axes]
        hs = [(hi - lo) / 2 ** P.levels[g][i] for i in range(d)]
        n = int(np.prod(Ns))
        L = np.zeros((n, n))
        for i in range(d):
            term = np.array([[1.0]])
            for k in range(d):
                blk = _oned(op, Ns[k], hs[k], axes[k], dt, 0.7, 1.3) if k == i else np.eye(Ns[k])
                term = np.kron(term, blk)
            L += term
        A = np.eye(n) + dt * L
        np.testing.assert_allclose(_probe(P, g, dt), A, rtol=0, atol=1e-12 * np.abs(A).max())


def _gauss(x, mean, std):
    return np.prod(np.exp(-0.5 * ((x - mean) / std) ** 2) / (std * np.sqrt(2 * np.pi)), axis=1)


def _ou_L_exact(x, mean, std, theta, sigma):
    """L p = -sum_i d_i(theta x_i p) - (sigma^2/2) Laplace p for a product Gaussian."""
    p = _gauss(x, mean, std)
    z = (x - mean) / std ** 2
    dp = -z * p[:, None]
    d2p = (z ** 2 - 1.0 / std ** 2) * p[:, None]
    return -np.sum(theta * p[:, None] + theta * x * dp, axis=1) - 0.5 * sigma ** 2 * np.sum(d2p, axis=1)


def test_ou_consistency_first_order():
    # grid (k, k) belongs to the d = 2 problem at level 2k-1 (layer w = 0)
    errs = []
    mean, std, theta, sigma = np.array([1.0, -0.5]), np.array([0.7, 0.6]), 1.0, 1.0
    for k in (6, 7, 8):
        P = oracle.Problem(2, 2 * k - 1, 1, W.OP_OU, [-6, -6], [6, 6], theta, sigma)
        g = [i for i in range(P.G) if tuple(P.levels[i]) == (k, k)][0]
        x = _nodes(P, g)
        p = np.zeros(P.n_total)
        p[P.grid_slice(g)] = _gauss(x, mean, std)
        dt = 1.0
        Lh = (P.apply(dt, p) - p)[P.grid_slice(g)] / dt
        errs.append(np.max(np.abs(Lh - _ou_L_exact(x, mean, std, theta, sigma))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 0.8) and np.all(rates < 1.3), (errs, rates)
    # a flipped drift sign would leave an O(1) error
    assert errs[-1] < 0.1 * np.max(np.abs(_ou_L_exact(x, mean, std, theta, sigma)))


def test_ou_mass_conservation_and_m_matrix():
    P = oracle.Problem(2, 5, 1, W.OP_OU, [-6, -6], [6, 6], 1.0, 1.0)
    dt = 0.05
    rng = W.uniform(7, P.n_total)
    for g in range(P.G):
        sl = P.grid_slice(g)
        N = [2 ** l - 1 for l in P.levels[g]]
        p = np.zeros(P.n_total)
        blk = rng[sl].reshape(N).copy()
        # mass away from the boundary: zero the two outermost node layers
        blk[:2, :] = 0
        blk[-2:, :] = 0
        blk[:, :2] = 0
        blk[:, -2:] = 0
        p[sl] = blk.ravel()
        q = P.apply(dt, p)
        assert abs(q[sl].sum() - p[sl].sum()) < 1e-12 * max(1.0, p[sl].sum())
        A = _probe(P, g, dt)
        off = A - np.diag(np.diag(A))
        assert np.all(off <= 1e-15) and np.all(np.diag(A) > 0)


def _varcoef_exact(x, amp):
    s1, c1 = np.sin(2 * np.pi * x[:, 0]), np.cos(2 * np.pi * x[:, 0])
    s2, c2 = np.sin(2 * np.pi * x[:, 1]), np.cos(2 * np.pi * x[:, 1])
    s3, c3 = np.sin(2 * np.pi * x[:, 2]), np.cos(2 * np.pi * x[:, 2])
    a = 1 + amp * s1 * c2 * s3
    da = [amp * 2 * np.pi * c1 * c2 * s3, -amp * 2 * np.pi * s1 * s2 * s3, amp * 2 * np.pi * s1 * c2 * c3]
    u = np.prod(np.sin(np.pi * x), axis=1)
    du = [np.pi * np.cos(np.pi * x[:, i]) * np.prod(np.sin(np.pi * np.delete(x, i, axis=1)), axis=1)
          for i in range(3)]
    d2u = -np.pi ** 2 * u
    div = sum(da[i] * du[i] for i in range(3)) + 3 * a * d2u
    return u, -div  # L u = -div(a grad u)


def test_varheat_consistency_second_order_symmetry_and_reduction():
    errs = []
    for k in (4, 5, 6):
        # grid (k, k, k) is on layer w = 0 of the d = 3 problem at level 3k - 2
        P = oracle.Problem(3, 3 * k - 2, k, W.OP_VARHEAT, vamp=0.5)
        g = [i for i in range(P.G) if tuple(P.levels[i]) == (k, k, k)][0]
        x = _nodes(P, g)
        uex, Lex = _varcoef_exact(x, 0.5)
        p = np.zeros(P.n_total)
        p[P.grid_slice(g)] = uex
        Lh = (P.apply(1.0, p) - p)[P.grid_slice(g)]
        errs.append(np.max(np.abs(Lh - Lex)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.7), (errs, rates)
    # symmetric operator, equal to heat at amplitude zero
    Pv = oracle.Problem(3, 3, 1, W.OP_VARHEAT, vamp=0.5)
    P0 = oracle.Problem(3, 3, 1, W.OP_VARHEAT, vamp=0.0)
    Ph = oracle.Problem(3, 3, 1, W.OP_HEAT)
    for g in range(Pv.G):
        A = _probe(Pv, g, 0.02)
        np.testing.assert_allclose(A, A.T, atol=1e-13)
        np.testing.assert_allclose(_probe(P0, g, 0.02), _probe(Ph, g, 0.02), atol=1e-13)


@pytest.mark.parametrize("op,lo,hi", [(W.OP_HEAT, 0, 1), (W.OP_VARHEAT, 0, 1), (W.OP_OU, -6, 6)])
def test_krylov_matches_dense_solve(op, lo, hi):
    d = 3
    P = oracle.Problem(d, 4, 1, op, [lo] * d, [hi] * d)
    dt = 0.02 if op != W.OP_OU else 0.2
    b = W.random_vector(11, P.n_total)
    x, its = P.phi(dt, b, rtol=1e-15, return_iters=True)
    assert np.all(its > 0)
    for g in range(P.G):
        sl = P.grid_slice(g)
        A = _probe(P, g, dt)
        ref = np.linalg.solve(A, b[sl])
        np.testing.assert_allclose(x[sl], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        np.testing.assert_allclose(P.dense_solve(g, dt, b[sl]), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_phi_with_forcing():
    P = oracle.Problem(2, 4)
    dt = 0.01
    u = W.random_vector(3, P.n_total)
    f = W.random_vector(4, P.n_total)
    out = P.phi(dt, u, f, rtol=1e-15)
    np.testing.assert_allclose(P.apply(dt, out), u + dt * f, atol=1e-13)
