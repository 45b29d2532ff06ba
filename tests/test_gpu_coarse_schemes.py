"""GPU parity of MGRIT with the higher-order coarse propagators, options beside
the paper's coarse backward Euler (Sec. 3.3.1) with the same fixed point:
PIT_COARSE_SDIRK2 (every coarse level steps with the L-stable two-stage SDIRK
scheme of order 2, gamma = 1 - 1/sqrt 2; oracle coarse kind 3) and
PIT_COARSE_EXTRAP (the extrapolated backward Euler 2 BE(dT/2)^2 - BE(dT);
oracle coarse kind 4).  Against the oracle's MGRIT with the same coarse
propagator (exact solves): the same result (1e-9 relative L2 with the
refinement form) and the same number of cycles within one, and the fixed
point is the oracle's sequential solution.  FP32 coarse solves change the
iterates, not the fixed point.
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
    # name: (workload, n, nsteps, m, levels)
    "w1": (1, 5, 64, 4, 2),
    "w2_small": (2, 5, 128, 8, 2),
    "w2_3lev": (2, 4, 64, 4, 3),
    "w3_small": (3, 3, 64, 8, 2),
    "w4_small": (4, 4, 128, 8, 2),
    "w5_small": (5, 3, 64, 4, 3),
}


def setup(name):
    k, n, N, m, lev = CASES[name]
    wl = W.workload(k)
    P = B.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    O = oracle.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = O.initial(wl.ic_kind, wl.ic_params)
    return wl, P, O, u0, N, m, lev


ORACLE_KIND = {B.PIT_COARSE_SDIRK2: 3, B.PIT_COARSE_EXTRAP: 4}
HEAT_CASES = ["w1", "w2_small", "w2_3lev", "w4_small", "w5_small"]  # constant and variable coefficient


@pytest.mark.parametrize("relax", [B.PIT_RELAX_FCF, B.PIT_RELAX_F])
@pytest.mark.parametrize("name,coarse", [(c, B.PIT_COARSE_SDIRK2) for c in CASES] +
                         [(c, B.PIT_COARSE_EXTRAP) for c in HEAT_CASES])
def test_higher_order_coarse_mgrit_matches_oracle(name, coarse, relax):
    wl, P, O, u0, N, m, lev = setup(name)
    tol = 1e-10 * np.abs(u0).max()
    so = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-13, maxit=50000, inner_rtol=1e-4, ir_maxit=40)
    opts = B.mgrit_opts(wl.t0, wl.t1, N, m, lev, tol=tol, maxit=60, coarse=coarse, fine=so, crs=so,
                        relax=relax, init=True)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    st = P.mgrit_solve(cuda(u0), opts, uT)
    dt = (wl.t1 - wl.t0) / N
    ref, its, hist, _ = O.mgrit(u0, dt, N, m, lev, tol=tol, maxit=60, coarse_kind=ORACLE_KIND[coarse], rtol=1e-15,
                                relax="F" if relax == B.PIT_RELAX_F else "FCF", init=True)
    got = host(uT)
    assert st.n_converged == P.G
    assert rel(got, ref) < 1e-9
    assert abs(st.max_cycles - int(its.max())) <= 1
    assert rel(got, O.sequential(u0, dt, N, rtol=1e-15)) < 1e-7


@pytest.mark.parametrize("name,coarse,init", [("w2_small", B.PIT_COARSE_SDIRK2, 1), ("w3_small", B.PIT_COARSE_SDIRK2, 1),
                                              ("w4_small", B.PIT_COARSE_SDIRK2, 1), ("w2_small", B.PIT_COARSE_EXTRAP, 1),
                                              ("w2_small", B.PIT_COARSE_IMPLICIT, 2),
                                              ("w2_3lev", B.PIT_COARSE_EXTRAP, 2), ("w1", B.PIT_COARSE_EXTRAP, 2),
                                              ("w4_small", B.PIT_COARSE_EXTRAP, 2)])
def test_higher_order_coarse_with_fp32_coarse_solves_reaches_the_sequential_solution(name, coarse, init):
    wl, P, O, u0, N, m, lev = setup(name)
    tol = 1e-10 * np.abs(u0).max()
    fine = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-13, maxit=50000, inner_rtol=1e-4, ir_maxit=40)
    crs = B.solve_opts(B.PIT_PREC_FP32, rtol=1e-5, maxit=50000)
    opts = B.mgrit_opts(wl.t0, wl.t1, N, m, lev, tol=tol, maxit=60, coarse=coarse, fine=fine, crs=crs,
                        relax=B.PIT_RELAX_F, init=init)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    st = P.mgrit_solve(cuda(u0), opts, uT)
    assert st.n_converged == P.G
    dt = (wl.t1 - wl.t0) / N
    assert rel(host(uT), O.sequential(u0, dt, N, rtol=1e-15)) < 1e-8


def test_higher_order_coarse_needs_fewer_cycles_on_smooth_heat_data():
    wl, P, O, u0, N, m, lev = setup("w5_small")
    P = B.Problem(wl.d, 5, wl.L0, wl.op, wl.lo, wl.hi)
    O = oracle.Problem(wl.d, 5, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = cuda(O.initial(wl.ic_kind, wl.ic_params))
    so = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-12, maxit=50000, inner_rtol=1e-6, ir_maxit=40)
    uT = torch.empty_like(u0)
    cyc = {}
    for coarse in (B.PIT_COARSE_IMPLICIT, B.PIT_COARSE_SDIRK2, B.PIT_COARSE_EXTRAP):
        opts = B.mgrit_opts(wl.t0, wl.t1, wl.nsteps, wl.m, wl.levels, tol=1e-9, maxit=60, coarse=coarse, fine=so,
                            crs=so, relax=B.PIT_RELAX_F, init=True)
        cyc[coarse] = P.mgrit_solve(u0, opts, uT).max_cycles
    assert cyc[B.PIT_COARSE_SDIRK2] < cyc[B.PIT_COARSE_IMPLICIT], cyc
    assert cyc[B.PIT_COARSE_EXTRAP] < cyc[B.PIT_COARSE_IMPLICIT], cyc


def test_higher_order_coarse_rejects_unsupported_forms():
    wl, P, O, u0, N, m, lev = setup("w2_small")
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    bad = [(B.PIT_COARSE_SDIRK2, B.PIT_PREC_FP64), (B.PIT_COARSE_SDIRK2, B.PIT_PREC_MIXED_PAIR),
           (B.PIT_COARSE_EXTRAP, B.PIT_PREC_FP64), (B.PIT_COARSE_EXTRAP, B.PIT_PREC_MIXED_PAIR)]
    for coarse, prec in bad:
        so = B.solve_opts(prec, rtol=1e-10, maxit=50000, inner_rtol=1e-4, ir_maxit=40)
        opts = B.mgrit_opts(wl.t0, wl.t1, N, m, lev, tol=1e-8, maxit=10, coarse=coarse, crs=so)
        with pytest.raises(B.PitError, match="UNSUPPORTED"):
            P.mgrit_solve(cuda(u0), opts, uT)
    # the extrapolated coarse step is built for the heat operator only
    wl, P, O, u0, N, m, lev = setup("w3_small")
    so = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-10, maxit=50000, inner_rtol=1e-4, ir_maxit=40)
    opts = B.mgrit_opts(wl.t0, wl.t1, N, m, lev, tol=1e-8, maxit=10, coarse=B.PIT_COARSE_EXTRAP, crs=so)
    with pytest.raises(B.PitError, match="UNSUPPORTED"):
        P.mgrit_solve(cuda(u0), opts, torch.empty(P.n_total, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("name", ["w2_small", "w2_3lev", "w4_small", "w5_small"])
def test_extrapolated_initial_sweep_matches_oracle(name):
    """init = 2: the initial sweep with the extrapolated step, the cycles with
    the coarse backward Euler; against the oracle's MGRIT with the same start."""
    wl, P, O, u0, N, m, lev = setup(name)
    tol = 1e-10 * np.abs(u0).max()
    so = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-13, maxit=50000, inner_rtol=1e-4, ir_maxit=40)
    opts = B.mgrit_opts(wl.t0, wl.t1, N, m, lev, tol=tol, maxit=60, coarse=B.PIT_COARSE_IMPLICIT, fine=so, crs=so,
                        relax=B.PIT_RELAX_F, init=2)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    st = P.mgrit_solve(cuda(u0), opts, uT)
    dt = (wl.t1 - wl.t0) / N
    ref, its, hist, _ = O.mgrit(u0, dt, N, m, lev, tol=tol, maxit=60, coarse_kind=0, rtol=1e-15, relax="F", init=2)
    assert st.n_converged == P.G
    assert rel(host(uT), ref) < 1e-9
    assert abs(st.max_cycles - int(its.max())) <= 1
    assert st.res_hist[0] < 1.5 * float(np.nanmax(hist[:, 0])) + 1e-300


def test_extrapolated_initial_sweep_rejects_unsupported_forms():
    wl, P, O, u0, N, m, lev = setup("w2_small")
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    crs = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-2, maxit=50000)
    opts = B.mgrit_opts(wl.t0, wl.t1, N, m, lev, tol=1e-8, maxit=10, crs=crs, init=2)
    with pytest.raises(B.PitError, match="UNSUPPORTED"):
        P.mgrit_solve(cuda(u0), opts, uT)


@pytest.mark.parametrize("name", ["w2_3lev", "w5_small"])
@pytest.mark.parametrize("init", [1, 2])
def test_f_relaxation_on_every_level_matches_oracle(name, init):
    """PIT_RELAX_F_ALL: F-relaxation on the middle level of three levels too,
    against the oracle's MGRIT with the same relaxation."""
    wl, P, O, u0, N, m, lev = setup(name)
    tol = 1e-10 * np.abs(u0).max()
    so = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-13, maxit=50000, inner_rtol=1e-4, ir_maxit=40)
    opts = B.mgrit_opts(wl.t0, wl.t1, N, m, lev, tol=tol, maxit=80, fine=so, crs=so, relax=B.PIT_RELAX_F_ALL,
                        init=init)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    st = P.mgrit_solve(cuda(u0), opts, uT)
    dt = (wl.t1 - wl.t0) / N
    ref, its, hist, _ = O.mgrit(u0, dt, N, m, lev, tol=tol, maxit=80, coarse_kind=0, rtol=1e-15, relax="F_ALL",
                                init=init)
    assert st.n_converged == P.G
    assert rel(host(uT), ref) < 1e-9
    assert abs(st.max_cycles - int(its.max())) <= 1
    assert rel(host(uT), O.sequential(u0, dt, N, rtol=1e-15)) < 1e-7
