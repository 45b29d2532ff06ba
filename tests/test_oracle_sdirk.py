"""Pins of the oracle's higher-order coarse propagators, applied on every
coarse level of the MGRIT hierarchy; neither is in the paper, whose coarse
propagator is backward Euler with dT = m dt (Sec. 3.3.1):
coarse kind 3, the L-stable, stiffly accurate two-stage SDIRK scheme of order
2 with gamma = 1 - 1/sqrt 2; coarse kind 4, the extrapolated backward Euler
2 BE(dT/2)^2 - BE(dT) (order 2, A-stable).

* Discrete eigenmodes: on a heat grid the product sine mode with discrete
  eigenvalue lambda is scaled by R(-lambda dT), R(z) = (1 + (1 - 2 gamma) z)
  / (1 - gamma z)^2 for SDIRK, 2 / (1 - z/2)^2 - 1 / (1 - z) for the
  extrapolated step, at level 1 (dT = m dt) and level 2 (dT = m^2 dt);
  backward Euler by 1 / (1 + lambda dT).
* Order: against the exact decay exp(-lambda dT) the one-step error falls by
  about 2^3 when dT halves (local error of a second-order scheme); a slip to
  first order falls by 2^2.
* L-stability: stiff modes (lambda dT >> 1) are damped to near zero.
* MGRIT: the fixed point is the sequential backward-Euler solution whatever the
  coarse propagator; FCF exactness after ceil(Nc / 2) cycles holds with it, and
  on smooth heat data both need fewer cycles than the coarse backward Euler.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_22156_gb300 import workloads as W

GAMMA = 1.0 - 1.0 / math.sqrt(2.0)


def R_sdirk(z):
    return (1.0 + (1.0 - 2.0 * GAMMA) * z) / (1.0 - GAMMA * z) ** 2


def R_ext(z):
    return 2.0 / (1.0 - 0.5 * z) ** 2 - 1.0 / (1.0 - z)


def _nodes(P, g):
    l = P.levels[g]
    axes = [P.lo[i] + (P.hi[i] - P.lo[i]) * np.arange(1, 2 ** l[i]) / 2 ** l[i] for i in range(P.d)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.ravel() for m in mesh], axis=1)


def _mode(P, k):
    """Per grid: the product sine mode k and its discrete eigenvalue."""
    u = np.zeros(P.n_total)
    lam = np.zeros(P.G)
    for g in range(P.G):
        x = _nodes(P, g)
        h = (P.hi - P.lo) / 2.0 ** P.levels[g]
        kk = np.asarray(k, dtype=float)
        lam[g] = np.sum(4.0 / h ** 2 * np.sin(kk * np.pi * h / 2) ** 2)
        u[P.grid_slice(g)] = np.prod(np.sin(np.pi * kk * x), axis=1)
    return u, lam


def _heat(d=2, n=5):
    return oracle.Problem(d, n, 1, W.OP_HEAT, [0.0] * d, [1.0] * d)


@pytest.mark.parametrize("level", [1, 2])
@pytest.mark.parametrize("k", [(1, 1), (3, 2)])
def test_sdirk_and_backward_euler_scale_eigenmodes_by_their_stability_functions(level, k):
    P = _heat()
    u, lam = _mode(P, k)
    dt, m = 1e-3, 4
    dT = dt * m ** level
    got = P.coarse_step(u, dt, m, level=level, coarse_kind=3)
    ext = P.coarse_step(u, dt, m, level=level, coarse_kind=4)
    be = P.coarse_step(u, dt, m, level=level, coarse_kind=0)
    for g in range(P.G):
        sl = P.grid_slice(g)
        if not np.any(u[sl]):
            continue
        np.testing.assert_allclose(got[sl], R_sdirk(-lam[g] * dT) * u[sl], rtol=0, atol=1e-12)
        np.testing.assert_allclose(ext[sl], R_ext(-lam[g] * dT) * u[sl], rtol=0, atol=1e-12)
        np.testing.assert_allclose(be[sl], u[sl] / (1.0 + lam[g] * dT), rtol=0, atol=1e-12)


@pytest.mark.parametrize("kind", [3, 4])
def test_coarse_schemes_are_second_order_against_the_exact_decay(kind):
    P = _heat()
    u, lam = _mode(P, (1, 1))
    g = int(np.argmax(lam))  # the finest grid's smooth-mode eigenvalue
    sl = P.grid_slice(g)
    errs = []
    for dT in (0.01, 0.005, 0.0025):
        out = P.coarse_step(u, dT, 1, level=1, coarse_kind=kind)
        errs.append(np.max(np.abs(out[sl] - math.exp(-lam[g] * dT) * u[sl])))
    for a, b in zip(errs, errs[1:]):
        assert 6.0 < a / b < 9.0, errs


@pytest.mark.parametrize("kind", [3, 4])
def test_coarse_schemes_damp_stiff_modes(kind):
    P = _heat(1, 8)  # one grid of 255 nodes
    u, lam = _mode(P, (200,))
    dt, m = 1e-2, 16
    out = P.coarse_step(u, dt, m, level=1, coarse_kind=kind)
    z = -lam[0] * dt * m
    assert lam[0] * dt * m > 1e4
    R = R_sdirk(z) if kind == 3 else R_ext(z)
    np.testing.assert_allclose(out, R * u, rtol=0, atol=1e-11)  # |R(z)| ~ 1e-4 here
    assert np.max(np.abs(out)) < 1e-3 * np.max(np.abs(u))


def test_mgrit_with_higher_order_coarse_propagators_keeps_the_fixed_point():
    wl = W.workload(1)
    P = oracle.Problem(wl.d, wl.n, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = W.random_vector(5, P.n_total)
    m, dt = wl.m, wl.dt
    # FCF exactness does not depend on the coarse propagator
    N = m * 4
    seq = P.sequential(u0, dt, N, rtol=1e-15)
    for kind in (3, 4):
        uT, its, *_ = P.mgrit(u0, dt, N, m, 2, tol=0.0, maxit=2, coarse_kind=kind, rtol=1e-15, check=False)
        np.testing.assert_allclose(uT, seq, rtol=0, atol=1e-13)
    # converged two- and three-level MGRIT (F and FCF) is sequential stepping
    wl2 = W.workload(2)
    P2 = oracle.Problem(wl2.d, 4, wl2.L0, wl2.op, wl2.lo, wl2.hi)
    u2 = P2.initial(wl2.ic_kind, wl2.ic_params)
    N2, dt2 = 64, 0.05 / 64
    seq2 = P2.sequential(u2, dt2, N2, rtol=1e-15)
    for kind in (3, 4):
        for levels, mm, relax in ((2, 8, "F"), (3, 4, "F"), (3, 4, "FCF")):
            uT2, *_ = P2.mgrit(u2, dt2, N2, mm, levels, tol=1e-13, maxit=60, coarse_kind=kind, rtol=1e-15,
                               relax=relax, init=True)
            np.testing.assert_allclose(uT2, seq2, rtol=0, atol=1e-11)


def test_mgrit_with_higher_order_coarse_needs_fewer_cycles_on_smooth_heat_data():
    wl = W.workload(5)
    P = oracle.Problem(wl.d, 6, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = P.initial(wl.ic_kind, wl.ic_params)
    cyc = {}
    for kind in (0, 3, 4):
        _, its, *_ = P.mgrit(u0, wl.dt, wl.nsteps, wl.m, wl.levels, tol=1e-9, maxit=30, coarse_kind=kind,
                             rtol=1e-12, relax="F", init=True)
        cyc[kind] = int(its.max())
    assert cyc[3] < cyc[0] and cyc[4] < cyc[0], cyc


def test_extrapolated_initial_sweep_lowers_every_residual_and_keeps_the_fixed_point():
    """init = 2: the initial coarse sweep with the extrapolated step, the cycles
    with the coarse backward Euler: the same fixed point, and on smooth heat
    data a first residual an order of magnitude below the plain sweep's."""
    wl = W.workload(2)
    P = oracle.Problem(wl.d, 6, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = P.initial(wl.ic_kind, wl.ic_params)
    seq = P.sequential(u0, wl.dt, wl.nsteps, rtol=1e-14)
    res = {}
    for init in (1, 2):
        uT, its, hist, _ = P.mgrit(u0, wl.dt, wl.nsteps, wl.m, 2, tol=1e-12, maxit=40, coarse_kind=0, rtol=1e-14,
                                   relax="F", init=init)
        np.testing.assert_allclose(uT, seq, rtol=0, atol=1e-10)
        res[init] = np.nanmax(hist[:, 0])
    assert res[2] < 0.2 * res[1], res


def test_f_relaxation_on_every_level_keeps_the_fixed_point():
    """relax "F_ALL": F-relaxation also on the middle level of three levels;
    converged MGRIT is still sequential stepping (also after the extrapolated
    initial sweep), and the middle level's relaxation does change the iterates
    (the second cycle's residuals differ from those with FCF there)."""
    wl = W.workload(2)
    P = oracle.Problem(wl.d, 4, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = P.initial(wl.ic_kind, wl.ic_params)
    N, dt = 64, 0.05 / 64
    seq = P.sequential(u0, dt, N, rtol=1e-15)
    for init in (1, 2):
        uT, its, *_ = P.mgrit(u0, dt, N, 4, 3, tol=1e-13, maxit=80, rtol=1e-15, relax="F_ALL", init=init)
        np.testing.assert_allclose(uT, seq, rtol=0, atol=1e-11)
    # the middle level's relaxation changes the iterates, not the two-level exactness
    _, its_f, hist_f, _ = P.mgrit(u0, dt, N, 4, 3, tol=0.0, maxit=2, rtol=1e-15, relax="F", check=False)
    _, its_a, hist_a, _ = P.mgrit(u0, dt, N, 4, 3, tol=0.0, maxit=2, rtol=1e-15, relax="F_ALL", check=False)
    assert np.any(np.abs(hist_f[:, 1] - hist_a[:, 1]) > 0)
