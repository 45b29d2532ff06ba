"""Pins of the oracle's grid set and combination (no GPU).

* Process counts printed in the paper (Table 1 and Secs. 4.3-4.4) fix the
  grid set, the level bounds, 2^l - 1 interior nodes per axis and l >= L0.
* Stars and bars: there are C(s-1, d-1) multi-indices l >= 1 with |l|_1 = s.
* The combination of nodal interpolants of a function is its sparse-grid
  interpolant, which equals the function at every sparse-grid node
  (Sec. 2.2.2: combination in the hierarchical basis).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2509_22156_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "process_counts.txt")


def _golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    return rows


@pytest.mark.parametrize("row", _golden_rows())
def test_process_counts_match_paper(row):
    d, L, L0, S, Pt, total = row
    lev, _ = oracle.enumerate_grids(d, L, L0)
    sizes = [oracle.grid_points(l) for l in lev]
    procs = sum(-(-s // (1 << S)) for s in sizes)
    assert procs * Pt == total


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_grid_count_stars_and_bars_and_coefficients(d, n):
    lev, lay = oracle.enumerate_grids(d, n, 1)
    for w in range(d):
        s = n + d - 1 - w
        expect = math.comb(s - 1, d - 1) if s >= d else 0
        got = int(np.sum(lay == w))
        assert got == expect
        assert np.all(lev[lay == w].sum(axis=1) == s)
    assert np.all(lev >= 1)
    # the grids of each layer are distinct
    assert len({tuple(l) for l in lev}) == len(lev)
    # coefficients (-1)^w C(d-1, w): their sum over all grids is 1 whenever
    # every layer is populated (inclusion-exclusion over the hyperbolic cross)
    P = oracle.Problem(d, n, 1)
    if n >= 1:
        assert abs(P.coef.sum() - 1.0) < 1e-12
    for g in range(P.G):
        w = lay[g]
        assert P.coef[g] == (-1) ** w * math.comb(d - 1, w)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_workload_sizes(k):
    wl = W.workload(k)
    lev, _ = oracle.enumerate_grids(wl.d, wl.n, wl.L0)
    P = oracle.Problem(wl.d, wl.n, wl.L0) if k != 5 else None
    sizes = np.prod((1 << lev.astype(np.int64)) - 1, axis=1)
    expect = {1: (9, 273), 2: (109, 73915), 3: (195, 32259), 4: (85, 27109), 5: (4921, 11876081)}[k]
    assert (len(lev), int(sizes.sum())) == expect
    if P is not None:
        assert P.n_total == expect[1]
        assert abs(P.coef.sum() - 1.0) < 1e-12


def _node_coords(P, g):
    """Interior node coordinates of grid g, C order with the last axis fastest."""
    l = P.levels[g]
    axes = [P.lo[i] + (P.hi[i] - P.lo[i]) * np.arange(1, 2 ** l[i]) / 2 ** l[i] for i in range(P.d)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.ravel() for m in mesh], axis=1)


def _bump(x, lo, hi):
    """A smooth function vanishing on the boundary of the box."""
    t = (x - lo) / (hi - lo)
    v = np.prod(t * (1 - t), axis=1)
    return v * (1.0 + 0.3 * np.sin(3.1 * x[:, 0]) + 0.2 * np.cos(2.3 * x.sum(axis=1)))


@pytest.mark.parametrize("d,n", [(1, 4), (2, 4), (2, 6), (3, 4), (4, 3)])
def test_combination_interpolates_at_sparse_grid_nodes(d, n):
    lo, hi = np.full(d, -0.5), np.full(d, 1.5)
    P = oracle.Problem(d, n, 1, lo=lo, hi=hi)
    u = np.empty(P.n_total)
    nodes = []
    for g in range(P.G):
        x = _node_coords(P, g)
        u[P.grid_slice(g)] = _bump(x, lo, hi)
        nodes.append(x)
    nodes = np.unique(np.concatenate(nodes), axis=0)
    out = P.combine(u, nodes)
    np.testing.assert_allclose(out, _bump(nodes, lo, hi), rtol=0, atol=1e-13)
    # away from the nodes the sparse-grid interpolant differs from the function
    pts = W.eval_points(d, lo, hi, n_uniform=64, n_diag=0, seed=3)
    assert np.max(np.abs(P.combine(u, pts) - _bump(pts, lo, hi))) > 1e-6


def test_single_grid_interpolation_is_multilinear():
    P = oracle.Problem(2, 3, 1)
    g = 2
    x = _node_coords(P, g)
    u = 0.3 + 0.7 * x[:, 0] - 0.2 * x[:, 1] + 0.5 * x[:, 0] * x[:, 1]
    # inside the convex hull of the interior nodes a bilinear function is reproduced
    l = P.levels[g]
    h = 1.0 / 2 ** l
    pts = np.stack([np.linspace(h[0], 1 - h[0], 11), np.linspace(1 - h[1], h[1], 11)], axis=1)
    val = P.interp(g, u, pts)
    ref = 0.3 + 0.7 * pts[:, 0] - 0.2 * pts[:, 1] + 0.5 * pts[:, 0] * pts[:, 1]
    np.testing.assert_allclose(val, ref, atol=1e-14)


@pytest.mark.parametrize("k", [1, 3, 4])
def test_initial_values_at_nodes(k):
    wl = W.workload(k)
    P = oracle.Problem(wl.d, wl.n, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = P.initial(wl.ic_kind, wl.ic_params)
    for g in [0, P.G // 2, P.G - 1]:
        x = _node_coords(P, g)
        if wl.ic_kind == W.IC_SINES:
            K = int(wl.ic_params[0])
            ref = np.zeros(len(x))
            for m in range(K):
                blk = wl.ic_params[1 + m * (wl.d + 1): 1 + (m + 1) * (wl.d + 1)]
                ref += blk[0] * np.prod(np.sin(np.pi * blk[1:] * (x - P.lo) / (P.hi - P.lo)), axis=1)
        else:
            mean, std = wl.ic_params[:wl.d], wl.ic_params[wl.d:]
            ref = np.prod(np.exp(-0.5 * ((x - mean) / std) ** 2) / (std * np.sqrt(2 * np.pi)), axis=1)
        np.testing.assert_allclose(u0[P.grid_slice(g)], ref, rtol=1e-14, atol=1e-300)


def test_splitmix64_reference_values():
    # SplitMix64 from seed 0: published first outputs of the generator
    z = W.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
