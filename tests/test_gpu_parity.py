"""GPU parity: libpit (through its C ABI) against the CPU oracle, element by
element on the same seeded inputs.

Tolerances (relative L2 per vector unless stated):
  FP64 path vs FP64 oracle       1e-10 (both Krylov solves run to 1e-13 or
                                 tighter, so their difference is ~kappa*1e-13)
  mixed path vs FP64 oracle      1e-6 required; the FP64 refinement reaches
                                 the same 1e-12 target, checked at 1e-9
  stencil, initial values,       1e-13 (same formulas, different rounding order)
  combination sum
"""
import numpy as np
import pytest

import oracle
from paper_2509_22156_gb300 import binding as B
from paper_2509_22156_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


CASES = {
    # name: (d, n, L0, op, lo, hi, dt)
    "heat2d": (2, 5, 1, W.OP_HEAT, [0.0] * 2, [1.0] * 2, 0.1 / 64),
    "heat3d": (3, 6, 1, W.OP_HEAT, [0.0] * 3, [1.0] * 3, 0.05 / 1024),
    "heat6d": (6, 4, 1, W.OP_HEAT, [0.0] * 6, [1.0] * 6, 0.02 / 512),
    "varheat3d": (3, 5, 1, W.OP_VARHEAT, [0.0] * 3, [1.0] * 3, 0.1 / 2048),
    "ou4d": (4, 4, 1, W.OP_OU, [-6.0] * 4, [6.0] * 4, 1.0 / 512),
    "ou2d_l0": (2, 7, 2, W.OP_OU, [-6.0] * 2, [6.0] * 2, 1.0 / 64),
}


def pair(name):
    d, n, L0, op, lo, hi, dt = CASES[name]
    P = B.Problem(d, n, L0, op, lo, hi)
    O = oracle.Problem(d, n, L0, op, lo, hi)
    return P, O, dt


@pytest.mark.parametrize("name", list(CASES))
def test_grid_table_matches_oracle(name):
    P, O, _ = pair(name)
    assert (P.G, P.n_total) == (O.G, O.n_total)
    np.testing.assert_array_equal(P.levels, O.levels)
    np.testing.assert_array_equal(P.coef, O.coef)
    np.testing.assert_array_equal(P.offsets, O.offsets)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_initial_values_match_oracle(k):
    wl = W.workload(k)
    n = min(wl.n, 6)
    P = B.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    O = oracle.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    u = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    P.sample_initial(wl.ic_kind, wl.ic_params, u)
    ref = O.initial(wl.ic_kind, wl.ic_params)
    assert rel(host(u), ref) < 1e-14
    # host output buffer path
    uh = np.empty(P.n_total)
    P.sample_initial(wl.ic_kind, wl.ic_params, uh)
    np.testing.assert_array_equal(uh, host(u))


@pytest.mark.parametrize("name", list(CASES))
def test_apply_matches_oracle(name):
    P, O, dt = pair(name)
    nb = 3
    p = W.random_vector(101, nb * P.n_total)
    q = torch.empty(nb * P.n_total, dtype=torch.float64, device="cuda")
    P.apply(dt, cuda(p), q)
    ref = O.apply(dt, p)
    assert rel(host(q), ref) < 1e-13


@pytest.mark.parametrize("prec", [B.PIT_PREC_FP64, B.PIT_PREC_MIXED])
@pytest.mark.parametrize("name", list(CASES))
def test_phi_batch_matches_oracle(name, prec):
    P, O, dt = pair(name)
    nb = 4
    u = W.random_vector(202, nb * P.n_total)
    out = torch.empty(nb * P.n_total, dtype=torch.float64, device="cuda")
    opts = B.solve_opts(prec, rtol=1e-12, maxit=20000, inner_rtol=1e-4, ir_maxit=30)
    st = P.phi_batch(dt, cuda(u), out, opts)
    assert st.n_items == nb * P.G and st.n_failed == 0
    ref = O.phi(dt, u, rtol=1e-15)
    got = host(out)
    for b in range(nb):
        for g in range(P.G):
            sl = slice(b * P.n_total + P.offsets[g], b * P.n_total + P.offsets[g + 1])
            assert rel(got[sl], ref[sl]) < (1e-10 if prec == B.PIT_PREC_FP64 else 1e-9), (b, g)
    if prec == B.PIT_PREC_MIXED:
        assert st.max_refine >= 1


@pytest.mark.parametrize("name", list(CASES))
def test_phi_batch_fp32_form_matches_oracle(name):
    # FP32 Krylov on the scaled FP32 state: accuracy set by rtol and FP32
    # rounding (relative 1e-6 asked, 1e-4 allowed), with a forcing term
    P, O, dt = pair(name)
    nb = 3
    u = W.random_vector(212, nb * P.n_total)
    f = W.random_vector(213, nb * P.n_total)
    out = torch.empty(nb * P.n_total, dtype=torch.float64, device="cuda")
    st = P.phi_batch(dt, cuda(u), out, B.solve_opts(B.PIT_PREC_FP32, rtol=1e-6, maxit=20000), f=cuda(f))
    assert st.n_items == nb * P.G and st.n_failed == 0
    ref = O.phi(dt, u, f, rtol=1e-15)
    got = host(out)
    for b in range(nb):
        for g in range(P.G):
            sl = slice(b * P.n_total + P.offsets[g], b * P.n_total + P.offsets[g + 1])
            assert rel(got[sl], ref[sl]) < 1e-4, (b, g)


@pytest.mark.parametrize("scale", [1e-100, 1e-20, 1e20, 1e100])
def test_fp32_form_scales_with_the_state(scale):
    P, O, dt = pair("varheat3d")
    u0 = W.random_vector(304, P.n_total)
    ref = O.sequential(u0, dt, 4, rtol=1e-15)
    uT = np.empty(P.n_total)
    P.sequential_solve(u0 * scale, dt, 4, uT, B.solve_opts(B.PIT_PREC_FP32, rtol=1e-6))
    assert np.all(np.isfinite(uT))
    assert rel(uT / scale, ref) < 1e-4


@pytest.mark.parametrize("d, n, dt", [(2, 6, 0.1), (3, 6, 0.01), (3, 5, 0.2), (4, 5, 0.05)])
@pytest.mark.parametrize("prec", [B.PIT_PREC_MIXED, B.PIT_PREC_FP32])
@pytest.mark.parametrize("op", [B.PIT_OP_HEAT, B.PIT_OP_VARHEAT])
def test_stiff_anisotropic_heat_steps_match_oracle(d, n, dt, prec, op):
    # large steps on grids whose finest axis is at least twice as fine as the
    # others: the FP32 Krylov solves of the (variable-coefficient) heat
    # operator use the line preconditioner along that axis there; the solution
    # is the same
    P = B.Problem(d, n, 1, op)
    O = oracle.Problem(d, n, 1, op)
    nb = 2
    u = W.random_vector(606 + d, nb * P.n_total)
    out = torch.empty(nb * P.n_total, dtype=torch.float64, device="cuda")
    rtol = 1e-12 if prec == B.PIT_PREC_MIXED else 1e-6
    st = P.phi_batch(dt, cuda(u), out, B.solve_opts(prec, rtol=rtol, maxit=20000, inner_rtol=1e-5, ir_maxit=40))
    assert st.n_failed == 0
    ref = O.phi(dt, u, rtol=1e-15)
    got = host(out)
    # the FP32 form stops at a relative residual of 1e-6, so its error can
    # reach cond(A) x 1e-6, up to several hundred x 1e-6 at these step sizes
    tol = 1e-9 if prec == B.PIT_PREC_MIXED else 2e-3
    for b in range(nb):
        for g in range(P.G):
            sl = slice(b * P.n_total + P.offsets[g], b * P.n_total + P.offsets[g + 1])
            assert rel(got[sl], ref[sl]) < tol, (b, g, P.levels[g])
    # several steps in one launch (carried residual, preconditioner reused)
    u0 = W.random_vector(707 + d, P.n_total)
    uT = np.empty(P.n_total)
    P.sequential_solve(u0, dt, 5, uT, B.solve_opts(prec, rtol=rtol, maxit=20000, inner_rtol=1e-5, ir_maxit=40))
    assert rel(uT, O.sequential(u0, dt, 5, rtol=1e-15)) < tol


def test_stiff_heat_mgrit_with_preconditioned_sweeps():
    # coarse steps of 1/40 on level-5 grids in d = 3: the FP32 coarse
    # correction sweep runs preconditioned on the anisotropic grids; MGRIT
    # still reaches the oracle's fixed point
    d, n, N, m, T = 3, 5, 64, 8, 0.2
    P = B.Problem(d, n, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(d, n, 1, W.OP_HEAT)
    u0 = O.initial(W.IC_SINES, W.sine_modes(d, [(1.0, [1, 1, 1]), (0.5, [1, 2, 3])]))
    fine = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-13, maxit=50000, inner_rtol=1e-5, ir_maxit=40)
    crs = B.solve_opts(B.PIT_PREC_FP32, rtol=1e-2, maxit=50000)
    tol = 1e-12 * np.abs(u0).max()
    opts = B.mgrit_opts(0.0, T, N, m, 2, tol=tol, maxit=60, fine=fine, crs=crs, relax=B.PIT_RELAX_F)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    st = P.mgrit_solve(cuda(u0), opts, uT)
    seq = O.sequential(u0, T / N, N, rtol=1e-15)
    assert st.n_converged == P.G
    assert rel(host(uT), seq) < 1e-9


def test_phi_in_place_forcing_and_empty_batch():
    P, O, dt = pair("heat3d")
    u = W.random_vector(5, 2 * P.n_total)
    f = W.random_vector(6, 2 * P.n_total)
    x = cuda(u)
    opts = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13)
    P.phi_batch(dt, x, x, opts, f=cuda(f))   # in place, with forcing
    assert rel(host(x), O.phi(dt, u, f, rtol=1e-15)) < 1e-10
    st = P.phi_batch(dt, x, x, opts, n_batch=0)
    assert st is not None


def test_phi_reports_nonconvergence_and_nonfinite():
    P, O, dt = pair("heat3d")
    u = cuda(W.random_vector(7, P.n_total))
    out = torch.empty_like(u)
    with pytest.raises(B.PitError) as e:
        P.phi_batch(dt, u, out, B.solve_opts(B.PIT_PREC_FP64, rtol=1e-14, maxit=1))
    assert e.value.status == B.PIT_ERR_NOCONV
    bad = u.clone()
    bad[3] = float("nan")
    with pytest.raises(B.PitError) as e:
        P.phi_batch(dt, bad, out, B.solve_opts(B.PIT_PREC_FP64))
    assert e.value.status == B.PIT_ERR_NONFINITE
    with pytest.raises(B.PitError) as e:
        P.phi_batch(dt, bad, out, B.solve_opts(B.PIT_PREC_MIXED))
    assert e.value.status == B.PIT_ERR_NONFINITE
    # the context is still usable
    P.phi_batch(dt, u, out, B.solve_opts(B.PIT_PREC_FP64))


@pytest.mark.parametrize("prec", [B.PIT_PREC_FP64, B.PIT_PREC_MIXED])
def test_sequential_matches_oracle_workload1(prec):
    wl = W.workload(1)
    P = B.Problem(wl.d, wl.n, wl.L0, wl.op, wl.lo, wl.hi)
    O = oracle.Problem(wl.d, wl.n, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = O.initial(wl.ic_kind, wl.ic_params)
    uT = np.empty(P.n_total)
    P.sequential_solve(u0, wl.dt, wl.nsteps, uT, B.solve_opts(prec, rtol=1e-13, ir_maxit=30))
    ref = O.sequential(u0, wl.dt, wl.nsteps, rtol=1e-15)
    assert rel(uT, ref) < (1e-10 if prec == B.PIT_PREC_FP64 else 1e-9)


@pytest.mark.parametrize("name", ["varheat3d", "ou4d"])
@pytest.mark.parametrize("scale", [1e-120, 1e-30, 1e30, 1e120])
def test_mixed_steps_scale_with_the_state(name, scale):
    # Phi is linear: Phi^k(s u) = s Phi^k(u).  The mixed form keeps its FP32
    # copies in range by power-of-two scaling, so states far outside the FP32
    # range give the same relative accuracy as states of unit size.
    P, O, dt = pair(name)
    u0 = W.random_vector(303, P.n_total)
    ref = O.sequential(u0, dt, 6, rtol=1e-15)
    uT = np.empty(P.n_total)
    P.sequential_solve(u0 * scale, dt, 6, uT, B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-12, ir_maxit=30))
    assert np.all(np.isfinite(uT))
    assert rel(uT / scale, ref) < 1e-9


MG_CASES = {
    # name: (workload, n, nsteps, m, levels, coarse)
    "w1": (1, 5, 64, 4, 2, B.PIT_COARSE_IMPLICIT),
    "w1_exact": (1, 5, 64, 4, 2, B.PIT_COARSE_EXACT),
    "w2_small": (2, 5, 128, 8, 2, B.PIT_COARSE_IMPLICIT),
    "w2_3lev": (2, 4, 64, 4, 3, B.PIT_COARSE_IMPLICIT),
    "w3_small": (3, 3, 64, 8, 2, B.PIT_COARSE_IMPLICIT),
    "w4_small": (4, 4, 128, 8, 2, B.PIT_COARSE_IMPLICIT),
    "w5_small": (5, 3, 64, 4, 3, B.PIT_COARSE_IMPLICIT),
}


@pytest.mark.parametrize("prec", [B.PIT_PREC_FP64, B.PIT_PREC_MIXED])
@pytest.mark.parametrize("name", list(MG_CASES))
def test_mgrit_matches_oracle(name, prec):
    k, n, N, m, lev, coarse = MG_CASES[name]
    wl = W.workload(k)
    P = B.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    O = oracle.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = O.initial(wl.ic_kind, wl.ic_params)
    tol = 1e-10 * np.abs(u0).max()
    fine = B.solve_opts(prec, rtol=1e-13, maxit=50000, inner_rtol=1e-4, ir_maxit=40)
    opts = B.mgrit_opts(wl.t0, wl.t1, N, m, lev, tol=tol, maxit=40, coarse=coarse, fine=fine)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    st = P.mgrit_solve(cuda(u0), opts, uT)
    dt = (wl.t1 - wl.t0) / N
    ref, its, hist, _ = O.mgrit(u0, dt, N, m, lev, tol=tol, maxit=40, coarse_kind=coarse, rtol=1e-15)
    got = host(uT)
    assert rel(got, ref) < (1e-10 if prec == B.PIT_PREC_FP64 else 1e-9)
    assert st.n_converged == P.G
    # same number of cycles as the oracle on the slowest grid (converged-grid
    # masking follows the per-grid stopping rule); the GPU solves the linear
    # coarse problem for the correction, the oracle in the FAS form of Alg. 2
    # (equal in exact arithmetic), so a residual at the tolerance may tip one
    # cycle either way
    assert abs(st.max_cycles - int(its.max())) <= 1
    # and the fixed point is the sequential solution
    seq = O.sequential(u0, dt, N, rtol=1e-15)
    assert rel(got, seq) < 1e-7


F_CASES = ["w1", "w2_small", "w2_3lev", "w3_small", "w4_small", "w5_small"]


@pytest.mark.parametrize("fas", [False, True])
@pytest.mark.parametrize("prec", [B.PIT_PREC_FP64, B.PIT_PREC_MIXED])
@pytest.mark.parametrize("name", F_CASES)
def test_mgrit_f_relaxation_matches_oracle(name, prec, fas):
    k, n, N, m, lev, coarse = MG_CASES[name]
    wl = W.workload(k)
    P = B.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    O = oracle.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = O.initial(wl.ic_kind, wl.ic_params)
    tol = 1e-10 * np.abs(u0).max()
    fine = B.solve_opts(prec, rtol=1e-13, maxit=50000, inner_rtol=1e-4, ir_maxit=40)
    opts = B.mgrit_opts(wl.t0, wl.t1, N, m, lev, tol=tol, maxit=60, coarse=coarse, fine=fine, fas=fas,
                        relax=B.PIT_RELAX_F)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    st = P.mgrit_solve(cuda(u0), opts, uT)
    dt = (wl.t1 - wl.t0) / N
    ref, its, hist, _ = O.mgrit(u0, dt, N, m, lev, tol=tol, maxit=60, coarse_kind=coarse, rtol=1e-15, relax="F")
    got = host(uT)
    assert rel(got, ref) < (1e-10 if prec == B.PIT_PREC_FP64 else 1e-9)
    assert st.n_converged == P.G
    assert abs(st.max_cycles - int(its.max())) <= 1
    seq = O.sequential(u0, dt, N, rtol=1e-15)
    assert rel(got, seq) < 1e-7


@pytest.mark.parametrize("name", ["w2_small", "w2_3lev", "w3_small", "w5_small"])
@pytest.mark.parametrize("relax", [B.PIT_RELAX_FCF, B.PIT_RELAX_F])
def test_mgrit_lanes_give_identical_results(name, relax):
    # grids are independent until the combination (Alg. 3): running them in
    # concurrent lanes changes neither the per-grid arithmetic nor the cycle
    # counts, so every lane count gives the bitwise same result
    k, n, N, m, lev, coarse = MG_CASES[name]
    wl = W.workload(k)
    P = B.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    O = oracle.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = cuda(O.initial(wl.ic_kind, wl.ic_params))
    tol = 1e-10 * float(u0.abs().max())
    fine = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-12, maxit=50000, inner_rtol=1e-5, ir_maxit=40)
    crs = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-2, maxit=50000, inner_rtol=1e-5, ir_maxit=40)
    res = {}
    for lanes in (1, 2, 3, P.G):
        opts = B.mgrit_opts(wl.t0, wl.t1, N, m, lev, tol=tol, maxit=60, coarse=coarse, fine=fine, crs=crs,
                            relax=relax, lanes=lanes)
        uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
        st = P.mgrit_solve(u0, opts, uT)
        res[lanes] = (host(uT), st.max_cycles, [st.res_hist[i] for i in range(st.max_cycles)])
    for lanes in (2, 3, P.G):
        np.testing.assert_array_equal(res[lanes][0], res[1][0])
        assert res[lanes][1] == res[1][1]
        assert res[lanes][2] == res[1][2]
    dt = (wl.t1 - wl.t0) / N
    seq = O.sequential(host(u0), dt, N, rtol=1e-15)
    assert rel(res[1][0], seq) < 1e-7


@pytest.mark.parametrize("name", ["w1", "w2_small", "w3_small", "w4_small", "w3_full"])
@pytest.mark.parametrize("relax", [B.PIT_RELAX_FCF, B.PIT_RELAX_F])
def test_mgrit_fp32_coarse_correction_solves(name, relax):
    # the correction equation only needs the coarse tolerance: FP32 coarse
    # solves reach the same fixed point in (about) the same number of cycles
    if name == "w3_full":
        # the drift workload at its full size and tolerance (BiCGStab in FP32,
        # residuals spanning many orders of magnitude across the intervals)
        wl = W.workload(3)
        k, n, N, m, lev = 3, wl.n, wl.nsteps, wl.m, 2
    else:
        k, n, N, m, lev, coarse = MG_CASES[name]
        wl = W.workload(k)
    P = B.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    O = oracle.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = O.initial(wl.ic_kind, wl.ic_params)
    tol = 1e-10 * np.abs(u0).max()
    fine = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-13, maxit=50000, inner_rtol=1e-5, ir_maxit=40)
    res = {}
    for cp in (B.PIT_PREC_MIXED, B.PIT_PREC_FP32):
        crs = B.solve_opts(cp, rtol=1e-2, maxit=50000, inner_rtol=1e-5, ir_maxit=40)
        opts = B.mgrit_opts(wl.t0, wl.t1, N, m, lev, tol=tol, maxit=60, fine=fine, crs=crs, relax=relax)
        uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
        st = P.mgrit_solve(cuda(u0), opts, uT)
        res[cp] = (host(uT), st.max_cycles)
    dt = (wl.t1 - wl.t0) / N
    seq = O.sequential(u0, dt, N, rtol=1e-15)
    assert rel(res[B.PIT_PREC_FP32][0], seq) < 1e-8
    assert abs(res[B.PIT_PREC_FP32][1] - res[B.PIT_PREC_MIXED][1]) <= 1


@pytest.mark.parametrize("name", ["w1", "w2_small", "w2_3lev", "w3_small", "w5_small"])
@pytest.mark.parametrize("relax", [B.PIT_RELAX_FCF, B.PIT_RELAX_F])
def test_mgrit_coarse_sweep_initial_guess_matches_oracle(name, relax):
    k, n, N, m, lev, coarse = MG_CASES[name]
    wl = W.workload(k)
    P = B.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    O = oracle.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = O.initial(wl.ic_kind, wl.ic_params)
    tol = 1e-10 * np.abs(u0).max()
    fine = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13, maxit=50000)
    opts = B.mgrit_opts(wl.t0, wl.t1, N, m, lev, tol=tol, maxit=60, coarse=coarse, fine=fine, relax=relax,
                        init=True)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    st = P.mgrit_solve(cuda(u0), opts, uT)
    dt = (wl.t1 - wl.t0) / N
    ref, its, hist, _ = O.mgrit(u0, dt, N, m, lev, tol=tol, maxit=60, coarse_kind=coarse, rtol=1e-15,
                                relax="F" if relax == B.PIT_RELAX_F else "FCF", init=True)
    got = host(uT)
    assert rel(got, ref) < 1e-10
    assert abs(st.max_cycles - int(its.max())) <= 1
    assert rel(got, O.sequential(u0, dt, N, rtol=1e-15)) < 1e-7


def test_mgrit_exact_coarse_sweep_start_is_converged():
    # with Phi_c = Phi^m the initial sweep is sequential stepping at the
    # C-points: the first cycle's residual is at round-off level
    k, n, N, m, lev, _ = MG_CASES["w1"]
    wl = W.workload(k)
    P = B.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = W.random_vector(9, P.n_total)
    fine = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-14, maxit=50000)
    opts = B.mgrit_opts(wl.t0, wl.t1, N, m, 2, tol=1e-9, maxit=5, coarse=B.PIT_COARSE_EXACT, fine=fine, init=True)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    st = P.mgrit_solve(cuda(u0), opts, uT)
    assert st.max_cycles == 1 and st.res_hist[0] < 1e-9


@pytest.mark.parametrize("kc", [1, 2, 3])
def test_mgrit_f_relaxation_exact_after_nc_cycles(kc):
    # kc F-relaxation cycles on Nc = kc coarse intervals reproduce sequential
    # stepping for any coarse propagator (exactness moves one interval per cycle)
    wl = W.workload(1)
    P = B.Problem(wl.d, wl.n, wl.L0, wl.op, wl.lo, wl.hi)
    O = oracle.Problem(wl.d, wl.n, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = W.random_vector(5, P.n_total)
    m, dt = wl.m, wl.dt
    N = m * kc
    fine = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-14, maxit=50000)
    opts = B.mgrit_opts(0.0, dt * N, N, m, 2, tol=0.0, maxit=kc, fine=fine, relax=B.PIT_RELAX_F)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    st, rc = P.mgrit_solve(cuda(u0), opts, uT, check=False)
    assert rc in (0, B.PIT_ERR_NOCONV) and st.max_cycles == kc
    seq = O.sequential(u0, dt, N, rtol=1e-15)
    assert np.max(np.abs(host(uT) - seq)) < 1e-11


@pytest.mark.parametrize("name", ["heat2d", "heat3d", "ou2d_l0", "heat6d"])
def test_combine_matches_oracle(name):
    P, O, _ = pair(name)
    d = P.d
    lo, hi = CASES[name][4], CASES[name][5]
    u = W.random_vector(303, P.n_total)
    pts = W.eval_points(d, lo, hi, n_uniform=4096, n_diag=65, seed=9)
    out = torch.empty(pts.shape[0], dtype=torch.float64, device="cuda")
    P.combine(cuda(u), cuda(pts), out)
    ref = O.combine(u, pts)
    assert rel(host(out), ref) < 1e-13
    # host pointers: the library stages them
    outh = np.empty(pts.shape[0])
    P.combine(u, pts, outh)
    assert rel(outh, ref) < 1e-13
    # empty point set
    P.combine(u, pts[:0].copy(), outh[:0].copy())


@pytest.mark.parametrize("n_uniform", [1, 200, 20000, 90000])
def test_combine_grid_chunks_match_oracle(n_uniform):
    # the sum splits the grids into chunks when the points alone fill few
    # SMs (one chunk for 90,000 points, several below); every split gives the
    # oracle's values
    P, O, _ = pair("heat6d")
    lo, hi = CASES["heat6d"][4], CASES["heat6d"][5]
    u = W.random_vector(808, P.n_total)
    pts = W.eval_points(6, lo, hi, n_uniform=n_uniform, n_diag=5, seed=11)
    out = torch.empty(pts.shape[0], dtype=torch.float64, device="cuda")
    P.combine(cuda(u), cuda(pts), out)
    assert rel(host(out), O.combine(u, pts)) < 1e-13


def test_large_grids_keep_their_state_in_global_memory():
    """d = 2, level 12: grids (6, 7) and (7, 6) hold 8001 nodes, more than the
    shared-memory solver state allows; the mixed form keeps their FP64 state,
    the FP64 form its state and Krylov vectors in global memory, and both run
    them beside the other grids."""
    P = B.Problem(2, 12, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(2, 12, 1, W.OP_HEAT)
    assert int(np.diff(P.offsets).max()) == 127 * 63
    dt = 1e-4
    nb = 2
    u = W.random_vector(505, nb * P.n_total)
    out = torch.empty(nb * P.n_total, dtype=torch.float64, device="cuda")
    opts = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-12, maxit=20000, inner_rtol=1e-5, ir_maxit=30)
    st = P.phi_batch(dt, cuda(u), out, opts)
    assert st.n_items == nb * P.G and st.n_failed == 0
    ref = O.phi(dt, u, rtol=1e-15)
    got = host(out)
    for b in range(nb):
        for g in range(P.G):
            sl = slice(b * P.n_total + P.offsets[g], b * P.n_total + P.offsets[g + 1])
            assert rel(got[sl], ref[sl]) < 1e-9, (b, g)
    st = P.phi_batch(dt, cuda(u), out, B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13, maxit=20000))
    assert st.n_items == nb * P.G and st.n_failed == 0
    got = host(out)
    for b in range(nb):
        for g in range(P.G):
            sl = slice(b * P.n_total + P.offsets[g], b * P.n_total + P.offsets[g + 1])
            assert rel(got[sl], ref[sl]) < 1e-10, (b, g)
    # MGRIT over both classes.  The coarse systems have dT/h^2 up to 6700, so a
    # true FP64 residual cannot go much below 1e-12 relative: Krylov 1e-10.
    u0 = O.initial(W.IC_SINES, W.sine_modes(2, [(1.0, [1, 1]), (0.3, [2, 3])]))
    N, m = 32, 4
    tol = 1e-9 * np.abs(u0).max()
    mo = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-10, maxit=20000, inner_rtol=1e-5, ir_maxit=30)
    mopts = B.mgrit_opts(0.0, N * dt, N, m, 2, tol=tol, maxit=40, fine=mo)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    P.mgrit_solve(cuda(u0), mopts, uT)
    seq = O.sequential(u0, dt, N, rtol=1e-15)
    assert rel(host(uT), seq) < 1e-7
    # the paper's form (FP64 Krylov, FAS, FCF) over both classes
    fo = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-10, maxit=20000)
    fopts = B.mgrit_opts(0.0, N * dt, N, m, 2, tol=tol, maxit=40, fine=fo, fas=True)
    P.mgrit_solve(cuda(u0), fopts, uT)
    assert rel(host(uT), seq) < 1e-7
