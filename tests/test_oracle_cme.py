"""Pins of the oracle's chemical-master-equation operator in Fokker-Planck
form (Sec. 4.3, Eqs. "cme", "cme_fp") for the toggle-switch networks of
Tables "toggle_switch_2d" / "toggle_switch_3d": species i is produced at rate
a_i = p_i / (s_i + y_i^b_i), y_i the total of the other species, and degraded
at rate g_i x_i, so
  u_t = sum_i [-d_i((a_i - g_i x_i) u) + (1/2) d_i^2((a_i + g_i x_i) u)].

  - on a normal density the nodal values of the discrete operator approach
    the analytic operator, differentiated symbolically by sympy from the
    equation above: second order with the central drift flux, first order
    with the donor cell;
  - both fluxes and the second difference of D u conserve mass away from the
    boundary;
  - with b = 0 the network is an immigration-death process (constant
    production a = p / (s + 1)); the moments of the Fokker-Planck equation
    then close: mean' = a - g mean, var' = a + g mean - 2 g var, and the
    backward-Euler solution's moments follow them;
  - BiCGStab solves the backward-Euler system like a dense direct solve.
"""
import numpy as np
import pytest

import oracle

sympy = pytest.importorskip("sympy")

# the paper's rates scaled to a smaller box: production 3 / (110 + y^2),
# degradation 0.01 x (the paper: 3e3 / (1.1e4 + y^2), 1e-3 x on [0, 399]^2)
RATES = (3.0, 110.0, 2.0, 0.01)


def node_coords(O, g):
    shape = tuple(int(2 ** l - 1) for l in O.levels[g])
    idx = np.indices(shape).reshape(len(shape), -1).T
    h = (O.hi - O.lo) / 2.0 ** O.levels[g]
    return O.lo + (idx + 1) * h


def gauss_params(M, C):
    return np.concatenate([np.asarray(M, float), np.asarray(C, float).ravel()])


def analytic_L(d, M, C, rates):
    """L u = -(right-hand side of Eq. "cme_fp") for the toggle network on the
    normal density N(M, C), as a numpy function of node coordinates."""
    p, s, b, g = rates
    xs = sympy.symbols(f"x0:{d}", real=True)
    X = sympy.Matrix(xs)
    Mv = sympy.Matrix([sympy.nsimplify(m) for m in M])
    Ci = sympy.Matrix(np.linalg.inv(C).tolist())
    z = X - Mv
    u = sympy.exp(-(z.T * Ci * z)[0] / 2) / sympy.sqrt((2 * sympy.pi) ** d * float(np.linalg.det(C)))
    Lu = 0
    for i in range(d):
        y = sum(xs[k] for k in range(d) if k != i)
        a = p / (s + y ** b)
        v, D = a - g * xs[i], a + g * xs[i]
        Lu += sympy.diff(v * u, xs[i]) - sympy.Rational(1, 2) * sympy.diff(D * u, xs[i], 2)
    f = sympy.lambdify(xs, Lu, "numpy")
    return lambda x: np.asarray(f(*[x[:, i] for i in range(d)]), dtype=float)


@pytest.mark.parametrize("central,order", [(True, 2), (False, 1)])
def test_operator_consistency_order_on_a_normal_density(central, order):
    d = 2
    M, C = np.array([15.0, 21.0]), np.array([[16.0, 4.0], [4.0, 12.0]])
    ref_L = analytic_L(d, M, C, RATES)
    errs = []
    for lev in (5, 6, 7):
        O = oracle.Problem(d, 2 * lev - 1, lev, oracle.OP_CME, lo=[0.0] * d, hi=[40.0] * d, cme=RATES,
                           central=central)
        g = [k for k in range(O.G) if tuple(O.levels[k]) == (lev, lev)][0]
        p = O.initial(4, gauss_params(M, C))
        Lp = (O.apply(1.0, p) - p)[O.grid_slice(g)]
        ref = ref_L(node_coords(O, g))
        errs.append(np.abs(Lp - ref).max() / np.abs(ref).max())
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    # measured: central 0.058, 0.015, 0.0037; donor cell 0.42, 0.22, 0.11
    if order == 2:
        assert min(ratios) > 3.5 and errs[2] < 0.01, errs
    else:
        assert min(ratios) > 1.7 and max(ratios) < 2.5, errs


@pytest.mark.parametrize("central", [False, True])
def test_mass_is_conserved_away_from_the_boundary(central):
    d = 3
    # mean in the middle: 7 standard deviations from the first node of the
    # coarsest axes (h = 7.5), so that no mass leaves through the boundary
    M, C = np.array([30.0, 32.0, 28.0]), np.diag([9.0, 12.0, 8.0])
    O = oracle.Problem(d, 8, 3, oracle.OP_CME, lo=[0.0] * d, hi=[60.0] * d, cme=RATES, central=central)
    p = O.initial(4, gauss_params(M, C))
    q = O.apply(0.5, p)
    for g in range(O.G):
        sl = O.grid_slice(g)
        # (measured at most 3.5e-10 relative: the central flux through the
        # boundary faces of the coarsest axes; a non-telescoping stencil
        # would leak about 1e-3)
        assert abs(np.sum(q[sl] - p[sl])) <= 1e-8 * np.sum(p[sl])


def test_immigration_death_moments_follow_their_closed_form():
    # d = 1: one species, constant production a = p / (s + 1) (y = 0, b = 0)
    p_, s_, g_ = 4.0, 1.0, 0.05
    a = p_ / (s_ + 1.0)
    M0, V0, T, N = 20.0, 4.0, 10.0, 1000
    O = oracle.Problem(1, 11, 1, oracle.OP_CME, lo=[0.0], hi=[100.0], cme=(p_, s_, 0.0, g_), central=True)
    u = O.sequential(O.initial(4, [M0, V0]), T / N, N, rtol=1e-14)
    x = node_coords(O, 0)[:, 0]
    mass = u.sum()
    mean = (x * u).sum() / mass
    var = ((x - mean) ** 2 * u).sum() / mass
    mt = a / g_ + (M0 - a / g_) * np.exp(-g_ * T)
    # var' = a + g mean - 2 g var with mean(t) above, solved in closed form
    c = a / g_
    vt = (V0 * np.exp(-2 * g_ * T) + (a + g_ * c) / (2 * g_) * (1 - np.exp(-2 * g_ * T))
          + (M0 - c) * (np.exp(-g_ * T) - np.exp(-2 * g_ * T)))
    assert abs(mass * 100.0 / 2 ** 11 - 1.0) < 1e-9
    # measured: mean 5.4e-5, variance 1.5e-3 relative (backward Euler,
    # dt = 0.01; a diffusion factor 1 instead of 1/2 would double the
    # stationary variance)
    assert abs(mean - mt) / mt < 2e-4, (mean, mt)
    assert abs(var - vt) / vt < 4e-3, (var, vt)


@pytest.mark.parametrize("central", [False, True])
def test_bicgstab_matches_a_dense_solve(central):
    O = oracle.Problem(2, 5, 1, oracle.OP_CME, lo=[0.0] * 2, hi=[40.0] * 2, cme=RATES, central=central)
    rng = np.random.default_rng(6)
    b = rng.standard_normal(O.n_total)
    x = O.phi(40.0, b, rtol=1e-15)
    for g in range(O.G):
        sl = O.grid_slice(g)
        np.testing.assert_allclose(x[sl], O.dense_solve(g, 40.0, b[sl]), rtol=0, atol=1e-12 * np.abs(b).max())
