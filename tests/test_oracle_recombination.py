"""Pins of the oracle's recombination (Sec. 2.2.2, Eqs. "recombination_operator"
and "overall_combination_operator"): hierarchization of every grid, the
node-wise combination of the surpluses over the grids that share a node, and
dehierarchization.

The pins do not go through the oracle's transforms:
  - a piecewise d-linear hat function of the hierarchical basis, sampled at a
    grid's nodes (the hat evaluated in numpy), hierarchizes to a single unit
    surplus at its own node;
  - the recombined value at every node of every grid equals the combined
    solution sum_l c_l I_l[u_l] evaluated there by the interpolation code of
    the combination sum, which is pinned on its own by the interpolation
    property (the projection of the combined function onto a grid's nodal
    space is its nodal interpolant, because a hierarchical hat of a finer
    level vanishes at every coarser node);
  - a function of the sparse-grid space sampled on every grid is left
    unchanged (the combination coefficients of the grids containing one
    hierarchical increment sum to one);
  - Q is a projection, and H^-1 H is the identity.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2509_22156_gb300 import workloads as W


def node_coords(O, g):
    shape = tuple(int(2 ** l - 1) for l in O.levels[g])
    idx = np.indices(shape).reshape(len(shape), -1).T
    h = (O.hi - O.lo) / 2.0 ** O.levels[g]
    return O.lo + (idx + 1) * h


def hat(O, lam, p, x):
    """Hierarchical hat of level lam and position p (node at (2p + 1) 2^-lam
    of the box along every axis), evaluated at points x."""
    centre = O.lo + (2 * np.asarray(p) + 1) * (O.hi - O.lo) / 2.0 ** np.asarray(lam)
    width = (O.hi - O.lo) / 2.0 ** np.asarray(lam)
    return np.prod(np.maximum(0.0, 1.0 - np.abs(x - centre) / width), axis=1)


CASES = [(2, 5, 1), (3, 4, 1), (3, 5, 2), (4, 4, 1)]


@pytest.mark.parametrize("d,n,L0", CASES)
def test_hierarchize_is_inverted_by_dehierarchize(d, n, L0):
    O = oracle.Problem(d, n, L0, W.OP_HEAT)
    u = W.random_vector(3, O.n_total)
    np.testing.assert_allclose(O.hierarchize(O.hierarchize(u), inverse=True), u, rtol=0, atol=1e-14)
    np.testing.assert_allclose(O.hierarchize(O.hierarchize(u, inverse=True)), u, rtol=0, atol=1e-14)


@pytest.mark.parametrize("d,n,L0", CASES)
def test_hat_function_has_one_unit_surplus(d, n, L0):
    O = oracle.Problem(d, n, L0, W.OP_HEAT, lo=[-1.0] * d, hi=[2.0] * d)
    rng = np.random.default_rng(5)
    for g in range(O.G):
        lev = O.levels[g]
        x = node_coords(O, g)
        for _ in range(4):
            lam = np.array([rng.integers(1, l + 1) for l in lev])
            p = np.array([rng.integers(0, 2 ** (k - 1)) for k in lam])
            u = np.zeros(O.n_total)
            u[O.grid_slice(g)] = hat(O, lam, p, x)
            s = O.hierarchize(u)[O.grid_slice(g)]
            # the hat's node on this grid: 1-based index (2p+1) 2^(l - lam)
            J = (2 * p + 1) * 2 ** (lev - lam)
            shape = tuple(int(2 ** l - 1) for l in lev)
            j = np.ravel_multi_index(tuple(J - 1), shape)
            ref = np.zeros(s.size)
            ref[j] = 1.0
            np.testing.assert_allclose(s, ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("d,n,L0", CASES)
def test_recombination_equals_combined_solution_at_every_node(d, n, L0):
    O = oracle.Problem(d, n, L0, W.OP_HEAT)
    u = W.random_vector(7, O.n_total)
    q = O.recombine(u)
    for g in range(O.G):
        ref = O.combine(u, node_coords(O, g))
        np.testing.assert_allclose(q[O.grid_slice(g)], ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("d,n,L0", CASES)
def test_recombination_fixes_sparse_grid_functions_and_is_a_projection(d, n, L0):
    O = oracle.Problem(d, n, L0, W.OP_HEAT)
    # a random function of the sparse-grid space: hats of every increment
    # lam <= l of some grid, random positions and amplitudes
    rng = np.random.default_rng(9)
    lams = set()
    for g in range(O.G):
        for lam in itertools.product(*[range(1, l + 1) for l in O.levels[g]]):
            lams.add(lam)
    terms = []
    for lam in sorted(lams):
        p = [int(rng.integers(0, 2 ** (k - 1))) for k in lam]
        terms.append((np.array(lam), np.array(p), rng.normal()))
    u = np.zeros(O.n_total)
    for g in range(O.G):
        x = node_coords(O, g)
        u[O.grid_slice(g)] = sum(a * hat(O, lam, p, x) for lam, p, a in terms)
    q = O.recombine(u)
    np.testing.assert_allclose(q, u, rtol=0, atol=1e-12)
    # projection: Q Q v = Q v for a vector outside the sparse-grid space
    v = W.random_vector(11, O.n_total)
    qv = O.recombine(v)
    np.testing.assert_allclose(O.recombine(qv), qv, rtol=0, atol=1e-13)
    assert np.linalg.norm(qv - v) > 1e-3 * np.linalg.norm(v)
