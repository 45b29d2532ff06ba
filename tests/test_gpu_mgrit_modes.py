"""GPU tests of the MGRIT variants and solver options beside the default cycle: the
residual mode of Sec. 4.4.1 (inexact fine solves inside F-relaxation, the
space-time residual of the backward-Euler equation at the C-points, coarse
problem (I + dT L) e_j = e_{j-1} + rho_j) against the oracle's sequential
solution.

With exact fine solves (relative 1e-13) residual mode has the sequential
solution as its fixed point; its coarse correction divides a stiff mode's
residual by the coarse operator, not the fine one, so those modes converge
slowly and the test stops at a space-time residual of 1e-9 of the state and
bounds the error by 1e-6.  With a fixed two Krylov iterations per fine step
(the paper's tuned run) the F-points are inexact, so the result is an
approximation whose error against the sequential solution is bounded here by
1e-2 and printed.
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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def heat_case(forced):
    d, n, N, m, T = 3, 5, 64, 8, 0.1
    dt = T / N
    P = B.Problem(d, n, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(d, n, 1, W.OP_HEAT)
    F = Fo = None
    if forced:
        F = torch.empty(N * P.n_total, dtype=torch.float64, device="cuda")
        for k in range(N):
            P.sample_initial(3, [(k + 1) * dt], F[k * P.n_total:(k + 1) * P.n_total])
        Fo = np.concatenate([O.initial(3, [(k + 1) * dt]) for k in range(N)])
        u0 = O.initial(2, [0.0])
    else:
        wl = W.workload(2)
        u0 = O.initial(wl.ic_kind, wl.ic_params)
    ref = O.sequential(u0, dt, N, rtol=1e-15, forcing=Fo)
    return P, O, u0, ref, F, (N, m, T)


@pytest.mark.parametrize("forced", [False, True])
def test_residual_mode_with_exact_solves_reaches_the_sequential_solution(forced):
    P, O, u0, ref, F, (N, m, T) = heat_case(forced)
    fine = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13, maxit=5000)
    crs = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13, maxit=5000)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    opts = B.mgrit_opts(0.0, T, N, m, 2, tol=1e-9 * np.abs(ref).max(), maxit=200, fine=fine, crs=crs,
                        relax=B.PIT_RELAX_F, init=True, forcing=F, residual=True)
    st = P.mgrit_solve(torch.from_numpy(u0).cuda(), opts, uT)
    assert st.n_converged == P.G
    err = rel(uT.cpu().numpy(), ref)
    print(f"residual mode, exact solves: {st.max_cycles} cycles, "
          f"residuals {[f'{st.res_hist[i]:.1e}' for i in range(min(st.max_cycles, 12))]}, error {err:.2e}")
    assert err < 1e-6
    P.close()


@pytest.mark.parametrize("prec", [B.PIT_PREC_FP64, B.PIT_PREC_MIXED])
def test_residual_mode_with_two_krylov_iterations(prec, capsys):
    P, O, u0, ref, F, (N, m, T) = heat_case(True)
    fine = B.solve_opts(prec, rtol=0.0, maxit=2, inner_rtol=1e-5, ir_maxit=1)
    crs = B.solve_opts(B.PIT_PREC_FP32, rtol=1e-2, maxit=5000)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    tol = 1e-7 * np.abs(ref).max()
    opts = B.mgrit_opts(0.0, T, N, m, 2, tol=tol, maxit=200, fine=fine, crs=crs, relax=B.PIT_RELAX_F, init=True,
                        forcing=F, residual=True)
    st = P.mgrit_solve(torch.from_numpy(u0).cuda(), opts, uT)
    assert st.n_converged == P.G
    err = rel(uT.cpu().numpy(), ref)
    with capsys.disabled():
        print(f"\nresidual mode, 2 Krylov iterations per fine step ({'FP64' if prec == 0 else 'refinement'}): "
              f"{st.max_cycles} cycles, error vs sequential {err:.2e}")
    assert err < 1e-2
    # the same options without residual mode are exact-solve options that do
    # not converge: hitting the caps is a failure there
    bad = B.mgrit_opts(0.0, T, N, m, 2, tol=tol, maxit=4, fine=fine, crs=crs, relax=B.PIT_RELAX_F, forcing=F)
    st2, rc = P.mgrit_solve(torch.from_numpy(u0).cuda(), bad, uT, check=False)
    assert rc != 0
    P.close()


def test_residual_mode_rejects_unsupported_combinations():
    P, O, u0, ref, F, (N, m, T) = heat_case(False)
    fine = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13, maxit=5000)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    for kw in (dict(relax=B.PIT_RELAX_FCF), dict(relax=B.PIT_RELAX_F, fas=True)):
        opts = B.mgrit_opts(0.0, T, N, m, 2, tol=1e-10, fine=fine, residual=True, **kw)
        with pytest.raises(B.PitError) as e:
            P.mgrit_solve(torch.from_numpy(u0).cuda(), opts, uT)
        assert e.value.status == B.PIT_ERR_UNSUPPORTED
    P.close()


# Preconditioners of the Krylov solves (Sec. 4.1 preconditions CG and
# BiCGStab; on one GPU: Jacobi scaling of the FP32 correction solves, the line
# preconditioner of the heat operator, or none): the solution must not change
# (the FP64 refinement decides the accuracy), only the iteration counts.
PC_CASES = {
    "varheat3d": (3, 5, 1, W.OP_VARHEAT, [0.0] * 3, [1.0] * 3, 0.1 / 2048 * 32),
    "ou4d": (4, 4, 1, W.OP_OU, [-6.0] * 4, [6.0] * 4, 1.0 / 512 * 8),
    "ou2d_l0": (2, 7, 2, W.OP_OU, [-6.0] * 2, [6.0] * 2, 1.0 / 64),
}


@pytest.mark.parametrize("prec", [B.PIT_PREC_MIXED, B.PIT_PREC_MIXED_PAIR])
@pytest.mark.parametrize("name", list(PC_CASES))
def test_jacobi_preconditioned_steps_match_oracle(name, prec, capsys):
    d, n, L0, op, lo, hi, dt = PC_CASES[name]
    if op == W.OP_OU and prec == B.PIT_PREC_MIXED_PAIR:
        pytest.skip("the pair form is for the symmetric operators")
    P = B.Problem(d, n, L0, op, lo, hi)
    O = oracle.Problem(d, n, L0, op, lo, hi)
    nb = 4
    u = W.random_vector(501, nb * P.n_total)
    ref = O.phi(dt, u, rtol=1e-15)
    its = {}
    for pc in (B.PIT_PRECOND_NONE, B.PIT_PRECOND_JACOBI):
        out = torch.empty(nb * P.n_total, dtype=torch.float64, device="cuda")
        opts = B.solve_opts(prec, rtol=1e-12, maxit=20000, inner_rtol=1e-4, ir_maxit=30, precond=pc)
        st = P.phi_batch(dt, torch.from_numpy(u).cuda(), out, opts)
        assert st.n_failed == 0
        its[pc] = st.sum_iters
        got = out.cpu().numpy()
        for b in range(nb):
            for g in range(P.G):
                sl = slice(b * P.n_total + P.offsets[g], b * P.n_total + P.offsets[g + 1])
                assert rel(got[sl], ref[sl]) < 1e-9, (pc, b, g)
    with capsys.disabled():
        print(f"\n{name} prec {prec}: Krylov iterations without / with Jacobi {its[1]} / {its[2]}")
    P.close()


def test_line_preconditioner_can_be_switched_off():
    """The heat operator's line preconditioner (default) and none give the
    same step; the preconditioned solve takes fewer iterations on the
    anisotropic grids at a stiff step."""
    P = B.Problem(3, 7, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(3, 7, 1, W.OP_HEAT)
    dt = 0.05 / 1024 * 16
    u = W.random_vector(502, P.n_total)
    ref = O.phi(dt, u, rtol=1e-15)
    its = {}
    for pc in (B.PIT_PRECOND_DEFAULT, B.PIT_PRECOND_NONE):
        out = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
        st = P.phi_batch(dt, torch.from_numpy(u).cuda(), out,
                         B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-12, maxit=20000, inner_rtol=1e-4, ir_maxit=30,
                                      precond=pc))
        its[pc] = st.sum_iters
        assert rel(out.cpu().numpy(), ref) < 1e-9
    assert its[B.PIT_PRECOND_DEFAULT] < its[B.PIT_PRECOND_NONE]
    P.close()
