"""Pins of the oracle's forcing path, per-grid time partitions and the
manufactured solution of the heat experiment (Sec. 4.2, Eq. "heat_equation";
Sec. 2.2.1 for subproblem-specific time partitions).

  - u* and its forcing f = du*/dt - Laplace u*: u* against its formula
    evaluated in numpy, f against central finite differences of that numpy
    u* in t and x (second order, step 1e-4);
  - backward Euler with a forcing that is a discrete eigenvector: on every
    grid the solution stays a multiple of the mode and its amplitude follows
    a_n = rho (a_{n-1} + dt c_n), rho = 1 / (1 + dt sum_i 4 sin^2(k pi h_i / 2)
    / h_i^2), exactly; with tmul substeps per step each substep uses the
    step's forcing and dt / tmul;
  - MGRIT with forcing and per-grid partitions converges to the sequential
    solution of the same discretization (Alg. 2's fixed point);
  - the combined solution of the heat experiment approaches u*(T) as the
    level and the number of steps grow (backward Euler O(dt), combination
    O(h^2 log)).
"""
import numpy as np
import pytest

import oracle
from paper_2509_22156_gb300 import workloads as W


def node_coords(O, g):
    shape = tuple(int(2 ** l - 1) for l in O.levels[g])
    idx = np.indices(shape).reshape(len(shape), -1).T
    h = (O.hi - O.lo) / 2.0 ** O.levels[g]
    return O.lo + (idx + 1) * h


def u_star(x, t, lo, hi):
    xi = (x - lo) / (hi - lo)
    return np.sqrt(np.sum(x * x, axis=1) + t * t) * np.exp(-t) * np.prod(np.sin(np.pi * xi), axis=1)


@pytest.mark.parametrize("t", [0.05, 0.7])
def test_manufactured_solution_and_forcing(t):
    d = 3
    O = oracle.Problem(d, 4, 1, W.OP_HEAT)
    u = O.initial(2, [t])
    f = O.initial(3, [t])
    dl = 1e-4
    for g in range(O.G):
        x = node_coords(O, g)
        sl = O.grid_slice(g)
        np.testing.assert_allclose(u[sl], u_star(x, t, O.lo, O.hi), rtol=0, atol=1e-15)
        ut = (u_star(x, t + dl, O.lo, O.hi) - u_star(x, t - dl, O.lo, O.hi)) / (2 * dl)
        lap = np.zeros(x.shape[0])
        for i in range(d):
            e = np.zeros(d)
            e[i] = dl
            lap += (u_star(x + e, t, O.lo, O.hi) - 2 * u_star(x, t, O.lo, O.hi) + u_star(x - e, t, O.lo, O.hi)) / dl ** 2
        np.testing.assert_allclose(f[sl], ut - lap, rtol=0, atol=2e-5 * max(1.0, np.abs(f[sl]).max()))


def _mode(O, k):
    return O.initial(0, W.sine_modes(O.d, [(1.0, [k] * O.d)]))


def _rho(O, g, dt, k):
    h = (O.hi - O.lo) / 2.0 ** O.levels[g]
    return 1.0 / (1.0 + dt * np.sum(4.0 * np.sin(k * np.pi * h / 2.0) ** 2 / h ** 2))


@pytest.mark.parametrize("with_tmul", [False, True])
def test_forced_eigenmode_follows_the_scalar_recurrence(with_tmul):
    O = oracle.Problem(2, 5, 1, W.OP_HEAT)
    k, N, dt = 1, 12, 0.01
    phi = _mode(O, k)
    c = np.cos(np.arange(1, N + 1) * 0.7) + 0.3
    F = np.concatenate([cn * phi for cn in c])
    a0 = 0.8
    tmul = (1 + np.arange(O.G) % 3).astype(np.int32) if with_tmul else None
    out = O.sequential(a0 * phi, dt, N, rtol=1e-15, forcing=F, tmul=tmul)
    for g in range(O.G):
        tm = int(tmul[g]) if with_tmul else 1
        rho = _rho(O, g, dt / tm, k)
        a = a0
        for n in range(N):
            for _ in range(tm):
                a = rho * (a + dt / tm * c[n])
        sl = O.grid_slice(g)
        np.testing.assert_allclose(out[sl], a * phi[sl], rtol=0, atol=1e-12)


@pytest.mark.parametrize("levels,relax", [(2, "F"), (2, "FCF"), (3, "F")])
def test_mgrit_with_forcing_and_partitions_converges_to_sequential(levels, relax):
    O = oracle.Problem(3, 4, 1, W.OP_HEAT)
    N, m, T = 32, 4, 0.2
    dt = T / N
    u0 = O.initial(2, [0.0])
    F = np.concatenate([O.initial(3, [(n + 1) * dt]) for n in range(N)])
    tmul = (1 + (np.arange(O.G) % 2) * 3).astype(np.int32)  # 1 or 4 steps per common step
    seq = O.sequential(u0, dt, N, rtol=1e-15, forcing=F, tmul=tmul)
    uT, its, _, st = O.mgrit(u0, dt, N, m, levels, tol=1e-13, maxit=60, rtol=1e-15, relax=relax, init=True,
                             forcing=F, tmul=tmul)
    np.testing.assert_allclose(uT, seq, rtol=0, atol=1e-11)
    # the partitions matter: a uniform one gives a different discrete solution
    seq1 = O.sequential(u0, dt, N, rtol=1e-15, forcing=F)
    assert np.abs(seq1 - seq).max() > 1e-5


def test_heat_experiment_approaches_the_manufactured_solution():
    T = 0.1
    errs = []
    for n, N in ((4, 16), (5, 64), (6, 256)):
        O = oracle.Problem(2, n, 1, W.OP_HEAT)
        dt = T / N
        F = np.concatenate([O.initial(3, [(k + 1) * dt]) for k in range(N)])
        uT = O.sequential(O.initial(2, [0.0]), dt, N, rtol=1e-13, forcing=F)
        pts = W.eval_points(2, [0.0] * 2, [1.0] * 2, n_uniform=2000, n_diag=0)
        got = O.combine(uT, pts)
        ref = u_star(pts, T, np.zeros(2), np.ones(2))
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[2] > 2.5 and errs[2] < 0.02, errs
