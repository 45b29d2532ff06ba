"""GPU parity of the recombination (Sec. 2.2.2, Eq. "overall_combination_operator")
and of CTMGRIT^loc with s recombination steps (Alg. 3) against the oracle.

pit_recombine runs the same arithmetic as the oracle in the same order
(surpluses parent by parent, axis by axis; the coefficient-weighted surpluses
summed over the grids in ascending order), so the tolerance is 1e-13 relative.
MGRIT with recombination must reach the oracle's time-sequential combination
method (Alg. 1): u <- Q u, then the interval's backward-Euler steps, s times;
the FP64 path within 1e-10 and the FP64-refinement path within 1e-9 (both
solve to 1e-13 relative, MGRIT to a residual of 1e-13 |u0|).
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


RCASES = [(1, 6, 1), (2, 6, 1), (3, 5, 1), (3, 6, 2), (4, 5, 1), (6, 5, 1), (6, 8, 1)]


@pytest.mark.parametrize("d,n,L0", RCASES)
def test_recombine_matches_oracle(d, n, L0):
    P = B.Problem(d, n, L0, B.PIT_OP_HEAT)
    O = oracle.Problem(d, n, L0, W.OP_HEAT)
    u = W.random_vector(100 + d, P.n_total)
    ud = torch.from_numpy(u).cuda()
    out = torch.empty_like(ud)
    P.recombine(ud, out)
    q = O.recombine(u) if O.n_total < 200000 else None
    got = out.cpu().numpy()
    if q is None:
        # large case: the projection property and a sample of nodes against
        # the oracle's combined solution at their coordinates
        again = torch.empty_like(ud)
        P.recombine(out, again)
        # (each node sums up to G coefficient-weighted surpluses with |c| up to
        # C(d-1, (d-1)/2) = 10 at d = 6, so rounding grows past 1e-13; measured
        # 6.4e-12 at d = 6, level 8, 1,709 grids)
        assert rel(again.cpu().numpy(), got) < 1e-10
        rng = np.random.default_rng(3)
        for g in rng.choice(O.G, 8, replace=False):
            shape = tuple(int(2 ** l - 1) for l in O.levels[g])
            idx = np.indices(shape).reshape(d, -1).T
            pick = rng.choice(idx.shape[0], min(64, idx.shape[0]), replace=False)
            x = O.lo + (idx[pick] + 1) * (O.hi - O.lo) / 2.0 ** O.levels[g]
            ref = O.combine(u, x)
            np.testing.assert_allclose(got[O.grid_slice(g)][pick], ref, rtol=0,
                                       atol=1e-10 * max(1.0, float(np.abs(got).max())))
    else:
        assert rel(got, q) < 1e-13
    # in place
    P.recombine(ud, ud)
    torch.cuda.synchronize()
    assert rel(ud.cpu().numpy(), got) < 1e-15
    P.close()


@pytest.mark.parametrize("prec,tolerance", [(B.PIT_PREC_FP64, 1e-10), (B.PIT_PREC_MIXED, 1e-9),
                                            (B.PIT_PREC_MIXED_PAIR, 1e-9)])
@pytest.mark.parametrize("s", [1, 4])
def test_mgrit_with_recombination_matches_sequential_combination_method(prec, tolerance, s):
    d, n, N, m = 3, 5, 64, 4
    T = 0.05
    dt = T / N
    P = B.Problem(d, n, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(d, n, 1, W.OP_HEAT)
    wl = W.workload(2)
    u0 = O.initial(wl.ic_kind, wl.ic_params)
    ref = u0.copy()
    for _ in range(s):
        ref = O.recombine(ref)
        ref = O.sequential(ref, dt, N // s, rtol=1e-15)
    fine = B.solve_opts(prec, rtol=1e-13, maxit=5000, inner_rtol=1e-5, ir_maxit=40)
    crs = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13, maxit=5000)
    opts = B.mgrit_opts(0.0, T, N, m, 2, tol=1e-13 * np.abs(u0).max(), maxit=64, fine=fine, crs=crs,
                        relax=B.PIT_RELAX_F, init=True, recomb=s)
    u0d = torch.from_numpy(u0).cuda()
    uT = torch.empty_like(u0d)
    st = P.mgrit_solve(u0d, opts, uT)
    assert st.n_converged == P.G
    assert rel(uT.cpu().numpy(), ref) < tolerance
    # three levels with recombination: the interval holds N / s = 16 steps = m^2
    if s == 4:
        opts3 = B.mgrit_opts(0.0, T, N, m, 3, tol=1e-13 * np.abs(u0).max(), maxit=64, fine=fine, crs=crs,
                             relax=B.PIT_RELAX_F, recomb=s)
        P.mgrit_solve(u0d, opts3, uT)
        assert rel(uT.cpu().numpy(), ref) < tolerance
    P.close()


def test_recombination_changes_the_anisotropic_solution_and_rejects_bad_step_counts():
    """With s > 1 the grids are coupled at every recombination step: the
    result differs from s = 0 (no recombination) by more than the solver
    tolerance on this anisotropic heat problem; a step count that the
    intervals do not divide is refused."""
    d, n, N, m = 2, 6, 64, 4
    P = B.Problem(d, n, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(d, n, 1, W.OP_HEAT)
    u0 = O.initial(W.IC_SINES, W.sine_modes(2, [(1.0, [1, 1]), (0.5, [5, 2])]))
    fine = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13, maxit=5000)
    u0d = torch.from_numpy(u0).cuda()
    a, b = torch.empty_like(u0d), torch.empty_like(u0d)
    P.mgrit_solve(u0d, B.mgrit_opts(0.0, 0.1, N, m, 2, tol=1e-12, fine=fine, recomb=0), a)
    P.mgrit_solve(u0d, B.mgrit_opts(0.0, 0.1, N, m, 2, tol=1e-12, fine=fine, recomb=8), b)
    assert rel(b.cpu().numpy(), a.cpu().numpy()) > 1e-6
    with pytest.raises(B.PitError) as e:
        P.mgrit_solve(u0d, B.mgrit_opts(0.0, 0.1, N, m, 2, tol=1e-12, fine=fine, recomb=32), b)
    assert e.value.status == B.PIT_ERR_INVALID_ARG
    P.close()


@pytest.mark.parametrize("prec,tolerance", [(B.PIT_PREC_FP64, 1e-10), (B.PIT_PREC_MIXED, 1e-9)])
@pytest.mark.parametrize("r", [2, 8])
def test_global_mgrit_matches_combination_method_recombined_every_r_steps(prec, tolerance, r):
    """Global MGRIT (Sec. 3.4): the propagator of r fine steps is Phi^r o Q,
    so every grid is recombined every r steps inside MGRIT; the fixed point
    is Alg. 1 with a recombination step every r fine steps (computed by the
    oracle step by step), here with the heat experiment's forcing."""
    d, n, N, m, T = 3, 5, 64, 8, 0.1
    dt = T / N
    P = B.Problem(d, n, 1, B.PIT_OP_HEAT)
    O = oracle.Problem(d, n, 1, W.OP_HEAT)
    F = torch.empty(N * P.n_total, dtype=torch.float64, device="cuda")
    for k in range(N):
        P.sample_initial(3, [(k + 1) * dt], F[k * P.n_total:(k + 1) * P.n_total])
    Fo = np.concatenate([O.initial(3, [(k + 1) * dt]) for k in range(N)])
    u0 = O.initial(2, [0.0])
    ref = u0.copy()
    for k in range(N // r):
        ref = O.recombine(ref)
        ref = O.sequential(ref, dt, r, rtol=1e-15, forcing=Fo[k * r * O.n_total:(k + 1) * r * O.n_total])
    fine = B.solve_opts(prec, rtol=1e-13, maxit=5000, inner_rtol=1e-5, ir_maxit=40)
    crs = B.solve_opts(B.PIT_PREC_FP32, rtol=1e-2, maxit=5000)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    opts = B.mgrit_opts(0.0, T, N, m, 2, tol=1e-13 * np.abs(ref).max(), maxit=64, fine=fine, crs=crs,
                        relax=B.PIT_RELAX_F, init=True, forcing=F, global_every=r)
    st = P.mgrit_solve(torch.from_numpy(u0).cuda(), opts, uT)
    assert st.n_converged == P.G and st.max_cycles >= 2
    assert rel(uT.cpu().numpy(), ref) < tolerance
    # r must divide m
    with pytest.raises(B.PitError) as e:
        P.mgrit_solve(torch.from_numpy(u0).cuda(),
                      B.mgrit_opts(0.0, T, N, m, 2, tol=1e-10, fine=fine, crs=crs, relax=B.PIT_RELAX_F,
                                   global_every=3), uT)
    assert e.value.status == B.PIT_ERR_INVALID_ARG
    P.close()
