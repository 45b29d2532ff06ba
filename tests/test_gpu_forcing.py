"""GPU parity of the forcing path, the per-grid time partitions and the heat
experiment with its manufactured solution (Sec. 4.2, Eq. "heat_equation";
Sec. 2.2.1; Alg. 3 with recombination) against the oracle.

Tolerances (relative L2 over the packed state): FP64 path 1e-10, FP32 Krylov
in FP64 or FP32-pair refinement 1e-9 (both sides solve every step to 1e-13
relative and MGRIT to a residual of 1e-13 of the state); the manufactured
solution and its forcing 1e-13 (same formula, different rounding order).
"""
import numpy as np
import pytest

import oracle
from paper_2509_22156_gb300 import binding as B
from paper_2509_22156_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PRECS = [(B.PIT_PREC_FP64, 1e-10), (B.PIT_PREC_MIXED, 1e-9), (B.PIT_PREC_MIXED_PAIR, 1e-9)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_22156_gb300 import build
    build.build()
    B.load()
    torch.cuda.set_device(0)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def forcing(P, O, dt, N):
    """f_n = f(x, t_n), n = 1..N, on the GPU and on the oracle."""
    F = torch.empty(N * P.n_total, dtype=torch.float64, device="cuda")
    for n in range(N):
        P.sample_initial(3, [(n + 1) * dt], F[n * P.n_total:(n + 1) * P.n_total])
    Fo = np.concatenate([O.initial(3, [(n + 1) * dt]) for n in range(N)])
    return F, Fo


@pytest.mark.parametrize("d", [2, 3, 6])
def test_manufactured_solution_and_forcing_match_oracle(d):
    n = {2: 6, 3: 5, 6: 4}[d]
    P = B.Problem(d, n, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(d, n, 1, W.OP_HEAT)
    u = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    for kind in (2, 3):
        for t in (0.0, 0.3):
            P.sample_initial(kind, [t], u)
            ref = O.initial(kind, [t])
            assert rel(u.cpu().numpy(), ref) < 1e-13, (kind, t)
    P.close()


@pytest.mark.parametrize("prec,tol", PRECS)
def test_sequential_with_forcing_and_partitions_matches_oracle(prec, tol):
    P = B.Problem(3, 5, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(3, 5, 1, W.OP_HEAT)
    N, T = 24, 0.1
    dt = T / N
    F, Fo = forcing(P, O, dt, N)
    u0 = O.initial(2, [0.0])
    tmul = (1 + (np.arange(P.G) % 3)).astype(np.int32)
    opts = B.solve_opts(prec, rtol=1e-13, maxit=5000, inner_rtol=1e-5, ir_maxit=40)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    for tm in (None, tmul):
        ref = O.sequential(u0, dt, N, rtol=1e-15, forcing=Fo, tmul=tm)
        P.sequential_solve_forced(torch.from_numpy(u0).cuda(), dt, N, uT, opts, forcing=F, tmul=tm)
        assert rel(uT.cpu().numpy(), ref) < tol
    P.close()


@pytest.mark.parametrize("prec,tol", PRECS)
@pytest.mark.parametrize("levels,relax", [(2, B.PIT_RELAX_F), (2, B.PIT_RELAX_FCF), (3, B.PIT_RELAX_F)])
def test_mgrit_with_forcing_matches_oracle_sequential(prec, tol, levels, relax):
    P = B.Problem(3, 5, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(3, 5, 1, W.OP_HEAT)
    N, m, T = 64, 4, 0.1
    dt = T / N
    F, Fo = forcing(P, O, dt, N)
    u0 = O.initial(2, [0.0])
    ref = O.sequential(u0, dt, N, rtol=1e-15, forcing=Fo)
    fine = B.solve_opts(prec, rtol=1e-13, maxit=5000, inner_rtol=1e-5, ir_maxit=40)
    crs = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13, maxit=5000)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    for fas in (False, True):
        opts = B.mgrit_opts(0.0, T, N, m, levels, tol=1e-13 * np.abs(ref).max(), maxit=64, fine=fine, crs=crs,
                            relax=relax, init=True, fas=fas, forcing=F)
        st = P.mgrit_solve(torch.from_numpy(u0).cuda(), opts, uT)
        assert st.n_converged == P.G
        assert rel(uT.cpu().numpy(), ref) < tol, fas
    P.close()


@pytest.mark.parametrize("prec,tol", PRECS)
def test_mgrit_with_per_grid_partitions_and_forcing_matches_oracle(prec, tol):
    """Grids with 1, 2 or 4 steps per fine step: three lanes, each with its
    own fine step and the common coarse step; MGRIT must reach the oracle's
    sequential solution of the same partitions."""
    P = B.Problem(3, 5, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(3, 5, 1, W.OP_HEAT)
    N, m, T = 32, 4, 0.1
    dt = T / N
    F, Fo = forcing(P, O, dt, N)
    u0 = O.initial(2, [0.0])
    tmul = np.array([1, 2, 4], dtype=np.int32)[np.arange(P.G) % 3]
    ref = O.sequential(u0, dt, N, rtol=1e-15, forcing=Fo, tmul=tmul)
    ref_o, _, _, _ = O.mgrit(u0, dt, N, m, 2, tol=1e-13, maxit=64, rtol=1e-15, relax="F", init=True,
                             forcing=Fo, tmul=tmul)
    fine = B.solve_opts(prec, rtol=1e-13, maxit=5000, inner_rtol=1e-5, ir_maxit=40)
    crs = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13, maxit=5000)
    opts = B.mgrit_opts(0.0, T, N, m, 2, tol=1e-13 * np.abs(ref).max(), maxit=64, fine=fine, crs=crs,
                        relax=B.PIT_RELAX_F, init=True, forcing=F, tmul=tmul)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    st = P.mgrit_solve(torch.from_numpy(u0).cuda(), opts, uT)
    assert st.n_converged == P.G
    got = uT.cpu().numpy()
    assert rel(got, ref) < tol
    assert rel(got, ref_o) < tol
    # the FAS form cannot run the partitions as lanes
    bad = B.mgrit_opts(0.0, T, N, m, 2, tol=1e-10, fine=fine, crs=crs, fas=True, forcing=F, tmul=tmul)
    with pytest.raises(B.PitError) as e:
        P.mgrit_solve(torch.from_numpy(u0).cuda(), bad, uT)
    assert e.value.status == B.PIT_ERR_UNSUPPORTED
    P.close()


def test_heat_experiment_with_recombination_matches_oracle_and_approaches_u_star():
    """The heat experiment (Sec. 4.2): u0 = u*(., 0), forcing from u*, s = 4
    recombination steps (Alg. 3), MGRIT per grid with F-relaxation; against
    the oracle's time-sequential combination method (Alg. 1) step by step,
    and against u*(T) at the evaluation points."""
    d, n, N, m, s, T = 3, 6, 64, 4, 4, 0.1
    dt = T / N
    P = B.Problem(d, n, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(d, n, 1, W.OP_HEAT)
    F, Fo = forcing(P, O, dt, N)
    u0 = O.initial(2, [0.0])
    ref = u0.copy()
    for k in range(s):
        ref = O.recombine(ref)
        lo, hi = k * (N // s) * O.n_total, (k + 1) * (N // s) * O.n_total
        ref = O.sequential(ref, dt, N // s, rtol=1e-15, forcing=Fo[lo:hi])
    fine = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-13, maxit=5000, inner_rtol=1e-5, ir_maxit=40)
    crs = B.solve_opts(B.PIT_PREC_FP32, rtol=1e-2, maxit=5000)
    opts = B.mgrit_opts(0.0, T, N, m, 2, tol=1e-13 * np.abs(ref).max(), maxit=64, fine=fine, crs=crs,
                        relax=B.PIT_RELAX_F, init=True, recomb=s, forcing=F)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    P.mgrit_solve(torch.from_numpy(u0).cuda(), opts, uT)
    assert rel(uT.cpu().numpy(), ref) < 1e-9
    pts = W.eval_points(d, [0.0] * d, [1.0] * d, n_uniform=4096, n_diag=33)
    out = np.empty(pts.shape[0])
    P.combine(uT, pts, out)
    x = pts
    ustar = np.sqrt(np.sum(x * x, axis=1) + T * T) * np.exp(-T) * np.prod(np.sin(np.pi * x), axis=1)
    err = rel(out, ustar)
    assert err < 0.01, err  # discretisation error (backward Euler, level-6 combination): 2.3e-3
    P.close()
