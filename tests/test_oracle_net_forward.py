"""Pins of the oracle's network forward pass (the learned coarse propagator).

The network is not in the paper; its definition is the architecture this
library fixes for the learned coarse step of MGRIT (Sec. 3.3.1 replaces the
coarse propagator): four layers of width-5 convolutions along every axis of
the grid with ONE weight set shared by all axes and the per-axis results
summed, channels (u / sigma, a(x), s_i) -> 16 -> 16 -> 16 -> 1, ReLU on the
hidden layers, taps outside the grid read zero (homogeneous Dirichlet
values), s_i = 1 / (1 + 4 dT / h_i^2) a constant channel of axis i, sigma the
RMS of the grid's state, output u + sigma * h4.

Each test below chooses parameters for which the output has a closed form
that does not go through the oracle's loops: a single nonzero tap (the output
is the input shifted by t - 2 along every axis, summed over the axes, with
zeros past both ends), the s channel alone (the in-range indicator of the tap
weighted by each axis' own s_i), the coefficient channel alone, and one
hidden channel behind a bias and ReLU.  A slip in the tap direction, the
padding, the axis loop, the channel layout or the s formula changes one of
these closed forms.
"""
import numpy as np
import pytest

import oracle
from paper_2509_22156_gb300 import workloads as W

CIN = (3, 17, 17, 17)
COUT = (16, 16, 16, 1)
NW = 5


def offsets():
    """Offsets of W_k[o][c][t] (Cout x Cin x 5) and b_k in the parameter block."""
    wo, bo, s = [], [], 0
    for k in range(4):
        wo.append(s)
        s += COUT[k] * CIN[k] * NW
        bo.append(s)
        s += COUT[k]
    return wo, bo, s


def widx(k, o, c, t):
    wo, _, _ = offsets()
    return wo[k] + (o * CIN[k] + c) * NW + t


def bidx(k, o):
    _, bo, _ = offsets()
    return bo[k] + o


def pass_through(theta, d, first_layer=1, ch=0):
    """Layers first_layer..3 copy channel `ch` (then channel 0) unchanged: the
    centre tap 1/d summed over the d axes is the identity on a node."""
    for k in range(first_layer, 4):
        theta[widx(k, 0, ch if k == first_layer else 0, 2)] = 1.0 / d


def shift_sum(v, shape, off):
    """sum_i of v shifted by `off` along axis i (value at node c is
    v[c + off e_i]), zero where c + off e_i leaves the grid."""
    v = v.reshape(shape)
    out = np.zeros(shape)
    for i, n in enumerate(shape):
        src = [slice(None)] * len(shape)
        dst = [slice(None)] * len(shape)
        if off >= 0:
            if off >= n:
                continue
            dst[i] = slice(0, n - off)
            src[i] = slice(off, n)
        else:
            if -off >= n:
                continue
            dst[i] = slice(-off, n)
            src[i] = slice(0, n + off)
        out[tuple(dst)] += v[tuple(src)]
    return out.ravel()


def in_range_weighted(shape, off, w):
    """sum_i w_i * [0 <= c_i + off < N_i] at every node c."""
    idx = np.indices(shape)
    out = np.zeros(shape)
    for i, n in enumerate(shape):
        out += w[i] * ((idx[i] + off >= 0) & (idx[i] + off < n))
    return out.ravel()


def grid_shape(P, g):
    return tuple(int(2 ** l - 1) for l in P.levels[g])


def node_coords(P, g):
    shape = grid_shape(P, g)
    idx = np.indices(shape).reshape(len(shape), -1).T
    h = (P.hi - P.lo) / 2.0 ** P.levels[g]
    return P.lo + (idx + 1) * h


def problem(op=W.OP_HEAT, d=2, n=4):
    # d = 2, level 4: grids (1,4) (2,3) (3,2) (4,1) (1,3) (2,2) (3,1), so every
    # tap reaches past an end on some axis and the axes differ in h
    return oracle.Problem(d, n, 1, op, lo=[0.0] * d, hi=[1.0] * d, vamp=0.5)


def positive_state(P, seed):
    return 0.5 + W.uniform(seed, P.n_total)


@pytest.mark.parametrize("t", range(NW))
def test_single_tap_shifts_the_input_along_every_axis(t):
    P = problem()
    _, _, npar = offsets()
    theta = np.zeros(npar)
    theta[widx(0, 0, 0, t)] = 1.0
    pass_through(theta, P.d)
    u = positive_state(P, 31 + t)
    out = P.net_forward(0.01, theta, u)
    for g in range(P.G):
        sl = P.grid_slice(g)
        ug = u[sl]
        # u + sigma * sum_i shift(u / sigma) = u + sum_i shift(u)
        ref = ug + shift_sum(ug, grid_shape(P, g), t - 2)
        np.testing.assert_allclose(out[sl], ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("t", range(NW))
def test_s_channel_enters_once_per_axis_with_its_own_width(t):
    P = problem()
    _, _, npar = offsets()
    dT = 0.003
    theta = np.zeros(npar)
    theta[widx(0, 0, CIN[0] - 1, t)] = 1.0
    pass_through(theta, P.d)
    u = positive_state(P, 41 + t)
    out = P.net_forward(dT, theta, u)
    for g in range(P.G):
        sl = P.grid_slice(g)
        h = 1.0 / 2.0 ** P.levels[g]
        s = 1.0 / (1.0 + 4.0 * dT / h ** 2)
        sigma = np.sqrt(np.mean(u[sl] ** 2))
        ref = u[sl] + sigma * in_range_weighted(grid_shape(P, g), t - 2, s)
        np.testing.assert_allclose(out[sl], ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("t", [0, 3])
def test_coefficient_channel_is_a_at_the_nodes(t):
    P = problem(W.OP_VARHEAT)
    _, _, npar = offsets()
    theta = np.zeros(npar)
    theta[widx(0, 0, 1, t)] = 1.0
    pass_through(theta, P.d)
    u = positive_state(P, 51 + t)
    out = P.net_forward(0.01, theta, u)
    for g in range(P.G):
        sl = P.grid_slice(g)
        x = node_coords(P, g)
        a = 1.0 + 0.5 * np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1])
        sigma = np.sqrt(np.mean(u[sl] ** 2))
        ref = u[sl] + sigma * shift_sum(a, grid_shape(P, g), t - 2)
        np.testing.assert_allclose(out[sl], ref, rtol=0, atol=1e-13)
    # the constant-coefficient operators feed ones
    Ph = problem(W.OP_HEAT)
    u = positive_state(Ph, 59)
    out = Ph.net_forward(0.01, theta, u)
    for g in range(Ph.G):
        sl = Ph.grid_slice(g)
        sigma = np.sqrt(np.mean(u[sl] ** 2))
        ones = np.ones(sl.stop - sl.start)
        np.testing.assert_allclose(out[sl], u[sl] + sigma * shift_sum(ones, grid_shape(Ph, g), t - 2),
                                   rtol=0, atol=1e-13)


def test_hidden_channel_bias_relu_and_layout():
    """Layer 0 writes ReLU(u / sigma - beta) into hidden channel 3 (centre tap
    1/d, bias -beta); layer 1 reads channel 3 through tap t = 4 only; layers 2
    and 3 pass channel 0 through.  The output is u + sigma * sum_i shift_{+2,i}
    (ReLU(u / sigma - beta)), which needs the [o][c][t] weight layout of the
    hidden layers, the bias of the right channel and the ReLU."""
    P = problem(d=3, n=4)
    _, _, npar = offsets()
    beta = 0.3
    theta = np.zeros(npar)
    theta[widx(0, 3, 0, 2)] = 1.0 / P.d
    theta[bidx(0, 3)] = -beta
    theta[widx(1, 0, 3, 4)] = 1.0
    theta[widx(2, 0, 0, 2)] = 1.0 / P.d
    theta[widx(3, 0, 0, 2)] = 1.0 / P.d
    u = W.random_vector(61, P.n_total)  # both signs: the ReLU matters
    out = P.net_forward(0.01, theta, u)
    for g in range(P.G):
        sl = P.grid_slice(g)
        sigma = np.sqrt(np.mean(u[sl] ** 2))
        h = np.maximum(u[sl] / sigma - beta, 0.0)
        ref = u[sl] + sigma * shift_sum(h, grid_shape(P, g), 2)
        np.testing.assert_allclose(out[sl], ref, rtol=0, atol=1e-13)
    # the last layer's bias adds sigma * b, the output channel of layer 3 is 0
    theta2 = np.zeros(npar)
    theta2[bidx(3, 0)] = -0.75
    out = P.net_forward(0.01, theta2, u)
    for g in range(P.G):
        sl = P.grid_slice(g)
        sigma = np.sqrt(np.mean(u[sl] ** 2))
        np.testing.assert_allclose(out[sl], u[sl] - 0.75 * sigma, rtol=0, atol=1e-14)


def _numpy_forward(P, g, dT, theta, ug, a):
    """The network written with array shifts (independent of the oracle's
    node loop): per layer pre[o] = b[o] + sum_i sum_t sum_c W[o, c, t]
    shift_{t-2, i}(z_c), z = (hidden or input channels, then the s channel of
    axis i as a constant field)."""
    shape = grid_shape(P, g)
    n = ug.size
    h = 1.0 / 2.0 ** P.levels[g]
    s = 1.0 / (1.0 + 4.0 * dT / h ** 2)
    sigma = np.sqrt(np.mean(ug ** 2))
    z = np.stack([ug / sigma, a])
    wo, bo, _ = offsets()
    for k in range(4):
        Wk = theta[wo[k]:wo[k] + COUT[k] * CIN[k] * NW].reshape(COUT[k], CIN[k], NW)
        pre = np.repeat(theta[bo[k]:bo[k] + COUT[k]][:, None], n, axis=1)
        for i in range(P.d):
            zi = np.concatenate([z, np.full((1, n), s[i])])
            for t in range(NW):
                sh = np.stack([_shift_axis(zc, shape, i, t - 2) for zc in zi])
                pre += Wk[:, :, t] @ sh
        z = np.maximum(pre, 0.0) if k < 3 else pre
    return ug + sigma * z[0]


def _shift_axis(v, shape, i, off):
    v = v.reshape(shape)
    out = np.zeros(shape)
    n = shape[i]
    src = [slice(None)] * len(shape)
    dst = [slice(None)] * len(shape)
    if abs(off) < n:
        if off >= 0:
            dst[i], src[i] = slice(0, n - off), slice(off, n)
        else:
            dst[i], src[i] = slice(-off, n), slice(0, n + off)
        out[tuple(dst)] = v[tuple(src)]
    return out.ravel()


def test_random_network_matches_array_restatement():
    P = problem(W.OP_VARHEAT)
    _, _, npar = offsets()
    theta = 0.3 * W.normal(71, npar)
    u = W.random_vector(72, P.n_total)
    dT = 0.004
    out = P.net_forward(dT, theta, u)
    for g in range(P.G):
        sl = P.grid_slice(g)
        x = node_coords(P, g)
        a = 1.0 + 0.5 * np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1])
        ref = _numpy_forward(P, g, dT, theta, u[sl], a)
        scale = max(1.0, float(np.abs(ref).max()))
        np.testing.assert_allclose(out[sl], ref, rtol=0, atol=1e-13 * scale)
