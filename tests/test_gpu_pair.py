"""GPU parity of the pair precision form (PIT_PREC_MIXED_PAIR): FP32 Krylov
inside a refinement whose state and residual are FP32 pairs, against the CPU
oracle (FP64, Krylov to 1e-15) on the same seeded inputs.

Tolerance: relative L2 1e-9 per grid, as for the FP64-refinement form; the
refinement stops at the same residual rule and the residual is formed to about
1e-14 relative, so the pair form reaches the tolerance like the FP64 form."""
import numpy as np
import pytest

import oracle
from paper_2509_22156_gb300 import binding as B
from paper_2509_22156_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PAIR = B.PIT_PREC_MIXED_PAIR


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_22156_gb300 import build
    build.build()
    B.load()
    torch.cuda.set_device(0)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def opts(rtol=1e-12, ir_maxit=30):
    return B.solve_opts(PAIR, rtol=rtol, maxit=20000, inner_rtol=1e-5, ir_maxit=ir_maxit)


HEAT = {
    # name: (d, n, L0, lo, hi, dt, operator)
    "heat1d": (1, 9, 1, [0.0], [1.0], 0.01, W.OP_HEAT),
    "heat2d": (2, 5, 1, [0.0] * 2, [1.0] * 2, 0.1 / 64, W.OP_HEAT),
    "heat3d": (3, 6, 1, [0.0] * 3, [1.0] * 3, 0.05 / 1024, W.OP_HEAT),
    "heat3d_l0": (3, 7, 2, [0.0] * 3, [1.0] * 3, 0.05 / 256, W.OP_HEAT),
    "heat6d": (6, 4, 1, [0.0] * 6, [1.0] * 6, 0.02 / 512, W.OP_HEAT),
    "varheat2d": (2, 6, 1, [0.0] * 2, [1.0] * 2, 0.1 / 256, W.OP_VARHEAT),
    "varheat3d": (3, 5, 1, [0.0] * 3, [1.0] * 3, 0.1 / 2048, W.OP_VARHEAT),
    "varheat4d": (4, 4, 1, [0.0] * 4, [1.0] * 4, 0.05 / 256, W.OP_VARHEAT),
}


def per_grid(P, got, ref, nb, tol):
    for b in range(nb):
        for g in range(P.G):
            sl = slice(b * P.n_total + P.offsets[g], b * P.n_total + P.offsets[g + 1])
            assert rel(got[sl], ref[sl]) < tol, (b, g, P.levels[g])


@pytest.mark.parametrize("name", list(HEAT))
def test_pair_phi_batch_matches_oracle(name):
    d, n, L0, lo, hi, dt, op = HEAT[name]
    P = B.Problem(d, n, L0, op, lo, hi)
    O = oracle.Problem(d, n, L0, op, lo, hi)
    nb = 4
    u = W.random_vector(222, nb * P.n_total)
    f = W.random_vector(223, nb * P.n_total)
    out = torch.empty(nb * P.n_total, dtype=torch.float64, device="cuda")
    st = P.phi_batch(dt, cuda(u), out, opts())
    assert st.n_items == nb * P.G and st.n_failed == 0 and st.max_refine >= 1
    per_grid(P, host(out), O.phi(dt, u, rtol=1e-15), nb, 1e-9)
    # with a forcing term, in place
    x = cuda(u)
    P.phi_batch(dt, x, x, opts(), f=cuda(f))
    per_grid(P, host(x), O.phi(dt, u, f, rtol=1e-15), nb, 1e-9)


@pytest.mark.parametrize("d, n, dt", [(2, 6, 0.1), (3, 6, 0.01), (3, 5, 0.2), (4, 5, 0.05)])
@pytest.mark.parametrize("op", [W.OP_HEAT, W.OP_VARHEAT])
def test_pair_stiff_anisotropic_steps_match_oracle(d, n, dt, op):
    # large steps (dt / h^2 up to 100) on anisotropic grids (heat: with the
    # line preconditioner): the differences of neighbours are formed exactly
    # from the pairs, so the stiff stencil does not amplify the rounding
    P = B.Problem(d, n, 1, op)
    O = oracle.Problem(d, n, 1, op)
    nb = 2
    u = W.random_vector(616 + d, nb * P.n_total)
    out = torch.empty(nb * P.n_total, dtype=torch.float64, device="cuda")
    st = P.phi_batch(dt, cuda(u), out, opts(ir_maxit=40))
    assert st.n_failed == 0
    per_grid(P, host(out), O.phi(dt, u, rtol=1e-15), nb, 1e-9)
    u0 = W.random_vector(717 + d, P.n_total)
    uT = np.empty(P.n_total)
    P.sequential_solve(u0, dt, 5, uT, opts(ir_maxit=40))
    assert rel(uT, O.sequential(u0, dt, 5, rtol=1e-15)) < 1e-9


def test_pair_sequential_matches_oracle_workload1():
    wl = W.workload(1)
    P = B.Problem(wl.d, wl.n, wl.L0, wl.op, wl.lo, wl.hi)
    O = oracle.Problem(wl.d, wl.n, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = O.initial(wl.ic_kind, wl.ic_params)
    uT = np.empty(P.n_total)
    P.sequential_solve(u0, wl.dt, wl.nsteps, uT, opts(rtol=1e-13))
    assert rel(uT, O.sequential(u0, wl.dt, wl.nsteps, rtol=1e-15)) < 1e-9


def test_pair_long_run_tracks_the_fp64_form():
    # 1024 steps of the heat3d workload at level 6: the pairs' rounding
    # (about 2^-48 per update) does not accumulate visibly
    wl = W.workload(2)
    P = B.Problem(wl.d, 6, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    P.sample_initial(wl.ic_kind, wl.ic_params, u0)
    a = torch.empty_like(u0)
    b = torch.empty_like(u0)
    P.sequential_solve(u0, wl.dt, wl.nsteps, a, B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13, maxit=20000))
    P.sequential_solve(u0, wl.dt, wl.nsteps, b, opts(rtol=1e-13))
    assert rel(host(b), host(a)) < 1e-11


@pytest.mark.parametrize("scale", [1e-120, 1e-30, 1e30, 1e120])
@pytest.mark.parametrize("op", [W.OP_HEAT, W.OP_VARHEAT])
def test_pair_steps_scale_with_the_state(scale, op):
    # Phi is linear; the pairs hold the state scaled by a power of two
    P = B.Problem(3, 6, 1, op)
    O = oracle.Problem(3, 6, 1, op)
    dt = 0.05 / 1024
    u0 = W.random_vector(313, P.n_total)
    ref = O.sequential(u0, dt, 6, rtol=1e-15)
    uT = np.empty(P.n_total)
    P.sequential_solve(u0 * scale, dt, 6, uT, opts())
    assert np.all(np.isfinite(uT))
    assert rel(uT / scale, ref) < 1e-9


def test_pair_rescales_a_fading_state():
    # 40 large steps: the state fades by about 2^-40 (its squared norm leaves
    # the kept range [2^-20, 2^20] several times), which the kernel follows
    # with exact power-of-two rescaling of the pairs
    P = B.Problem(2, 5, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(2, 5, 1, W.OP_HEAT)
    dt = 0.05
    u0 = W.random_vector(414, P.n_total)
    ref = O.sequential(u0, dt, 40, rtol=1e-15)
    uT = np.empty(P.n_total)
    P.sequential_solve(u0, dt, 40, uT, opts())
    assert np.linalg.norm(ref) < 1e-11 * np.linalg.norm(u0)
    assert rel(uT, ref) < 1e-9


MG = {
    # name: (workload, n, nsteps, m, levels, relax)
    "w1_fcf": (1, 5, 64, 4, 2, B.PIT_RELAX_FCF),
    "w2_f": (2, 5, 128, 8, 2, B.PIT_RELAX_F),
    "w2_3lev": (2, 4, 64, 4, 3, B.PIT_RELAX_FCF),
    "w5_f": (5, 3, 64, 4, 3, B.PIT_RELAX_F),
    "w4_f": (4, 4, 128, 8, 2, B.PIT_RELAX_F),
    "w4_fcf": (4, 4, 128, 8, 2, B.PIT_RELAX_FCF),
}


@pytest.mark.parametrize("name", list(MG))
def test_pair_mgrit_matches_oracle(name):
    k, n, N, m, lev, relax = MG[name]
    wl = W.workload(k)
    P = B.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi, vamp=wl.vamp)
    O = oracle.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi, vamp=wl.vamp)
    u0 = O.initial(wl.ic_kind, wl.ic_params)
    tol = 1e-10 * np.abs(u0).max()
    fine = B.solve_opts(PAIR, rtol=1e-13, maxit=50000, inner_rtol=1e-4, ir_maxit=40)
    o = B.mgrit_opts(wl.t0, wl.t1, N, m, lev, tol=tol, maxit=40, fine=fine, relax=relax)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    st = P.mgrit_solve(cuda(u0), o, uT)
    assert st.n_converged == P.G
    seq = O.sequential(u0, (wl.t1 - wl.t0) / N, N, rtol=1e-15)
    assert rel(host(uT), seq) < 1e-8


def test_pair_mgrit_lanes_and_coarse_fp32_solves():
    # the chosen configuration of the heat workloads: F relaxation in the pair
    # form, FP32 coarse correction solves, initial coarse sweep, six lanes
    wl = W.workload(2)
    P = B.Problem(wl.d, 6, wl.L0, wl.op, wl.lo, wl.hi)
    O = oracle.Problem(wl.d, 6, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = O.initial(wl.ic_kind, wl.ic_params)
    N, m = 256, 16
    fine = B.solve_opts(PAIR, rtol=1e-12, maxit=4000, inner_rtol=1e-5, ir_maxit=12)
    crs = B.solve_opts(B.PIT_PREC_FP32, rtol=1e-2, maxit=4000)
    tol = 1e-10 * np.abs(u0).max()
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    res = []
    for lanes in (1, 6):
        o = B.mgrit_opts(wl.t0, wl.t1, N, m, 2, tol=tol, maxit=40, fine=fine, crs=crs, relax=B.PIT_RELAX_F,
                         lanes=lanes, init=True)
        st = P.mgrit_solve(cuda(u0), o, uT)
        assert st.n_converged == P.G
        res.append(host(uT).copy())
    # lanes only change which grids share a launch: bitwise the same result
    assert np.array_equal(res[0], res[1])
    seq = O.sequential(u0, (wl.t1 - wl.t0) / N, N, rtol=1e-15)
    assert rel(res[0], seq) < 1e-8


def test_pair_large_grids_keep_their_pairs_in_global_memory():
    # grids with 8001 nodes exceed the on-chip state: their pairs live in
    # global memory (the Krylov vectors stay on chip), beside the on-chip items
    P = B.Problem(2, 12, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(2, 12, 1, W.OP_HEAT)
    assert int(np.diff(P.offsets).max()) == 127 * 63
    dt = 1e-4
    nb = 2
    u = W.random_vector(525, nb * P.n_total)
    out = torch.empty(nb * P.n_total, dtype=torch.float64, device="cuda")
    st = P.phi_batch(dt, cuda(u), out, opts())
    assert st.n_items == nb * P.G and st.n_failed == 0
    per_grid(P, host(out), O.phi(dt, u, rtol=1e-15), nb, 1e-9)
    # several steps in one launch, with a state scaled far outside FP32 (a
    # smaller step: with dt / h^2 = 419 on the finest axis a random state
    # puts the pair residual's floor, about 2^-48 x 4 dt / h^2, near 1e-12)
    u0 = W.random_vector(526, P.n_total)
    uT = np.empty(P.n_total)
    P.sequential_solve(u0 * 1e-60, 1e-6, 6, uT, opts())
    assert rel(uT * 1e60, O.sequential(u0, 1e-6, 6, rtol=1e-15)) < 1e-9
    # MGRIT over both classes, F relaxation with FP32 coarse solves; Krylov
    # 1e-10 as for the FP64-refinement form on these stiff grids
    u0 = O.initial(W.IC_SINES, W.sine_modes(2, [(1.0, [1, 1]), (0.3, [2, 3])]))
    N, m = 32, 4
    tol = 1e-9 * np.abs(u0).max()
    fine = B.solve_opts(PAIR, rtol=1e-10, maxit=20000, inner_rtol=1e-5, ir_maxit=30)
    crs = B.solve_opts(B.PIT_PREC_FP32, rtol=1e-2, maxit=20000)
    o = B.mgrit_opts(0.0, N * dt, N, m, 2, tol=tol, maxit=60, fine=fine, crs=crs, relax=B.PIT_RELAX_F)
    uTd = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    stm = P.mgrit_solve(cuda(u0), o, uTd)
    assert stm.n_converged == P.G
    assert rel(host(uTd), O.sequential(u0, dt, N, rtol=1e-15)) < 1e-8


def test_pair_rejects_other_operators_and_reports_errors():
    P = B.Problem(4, 3, 1, B.PIT_OP_OU, [-6.0] * 4, [6.0] * 4)
    u = cuda(W.random_vector(8, P.n_total))
    with pytest.raises(B.PitError) as e:
        P.phi_batch(1e-3, u, torch.empty_like(u), opts())
    assert e.value.status == B.PIT_ERR_UNSUPPORTED
    H = B.Problem(3, 5, 1, B.PIT_OP_HEAT)
    u = cuda(W.random_vector(9, H.n_total))
    out = torch.empty_like(u)
    with pytest.raises(B.PitError) as e:
        H.phi_batch(1e-2, u, out, B.solve_opts(PAIR, rtol=1e-14, maxit=1, inner_rtol=1e-5, ir_maxit=1))
    assert e.value.status == B.PIT_ERR_NOCONV
    bad = u.clone()
    bad[5] = float("nan")
    with pytest.raises(B.PitError) as e:
        H.phi_batch(1e-2, bad, out, opts())
    assert e.value.status == B.PIT_ERR_NONFINITE
    H.phi_batch(1e-2, u, out, opts())  # the context is still usable
