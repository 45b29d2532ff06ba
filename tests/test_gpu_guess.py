"""GPU parity of the refinement form's initial guesses (PIT_GUESS_PREVIOUS and
PIT_GUESS_EXTRAPOLATE, the latter the default): both must reach the oracle's
backward-Euler steps to the same tolerance as every mixed-form test (1e-9
relative L2 per grid against the FP64 oracle, both solved to 1e-12 or
tighter), on shared-memory and global-memory grids, with every operator, and
the extrapolated guess must need fewer FP64 refinement passes on smooth
solutions.  The guess changes the iterate a solve starts from, never the
stopping rule, so the fixed point of MGRIT is unchanged too.
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


GUESSES = [B.PIT_GUESS_PREVIOUS, B.PIT_GUESS_EXTRAPOLATE]

CASES = {
    # name: (d, n, L0, op, lo, hi, dt, nsteps, initial value (smooth or seeded random))
    "heat3d": (3, 6, 1, W.OP_HEAT, [0.0] * 3, [1.0] * 3, 0.05 / 1024, 24, "smooth"),
    "heat6d": (6, 4, 1, W.OP_HEAT, [0.0] * 6, [1.0] * 6, 0.02 / 512, 12, "smooth"),
    "varheat3d": (3, 5, 1, W.OP_VARHEAT, [0.0] * 3, [1.0] * 3, 0.1 / 2048, 16, "random"),
    "ou4d": (4, 4, 1, W.OP_OU, [-6.0] * 4, [6.0] * 4, 1.0 / 512, 12, "smooth"),
    "heat2d_global": (2, 12, 1, W.OP_HEAT, [0.0] * 2, [1.0] * 2, 1e-4, 10, "random"),
}


def initial(O, kind, d, op):
    if kind == "random":
        return W.random_vector(909, O.n_total)
    if op == W.OP_OU:
        wl = W.workload(3)
        return O.initial(wl.ic_kind, wl.ic_params)
    return O.initial(W.IC_SINES, W.sine_modes(d, [(1.0, [1] * d), (0.1, [3] * d)]))


@pytest.mark.parametrize("guess", GUESSES)
@pytest.mark.parametrize("name", list(CASES))
def test_sequential_steps_match_oracle_with_either_guess(name, guess):
    d, n, L0, op, lo, hi, dt, N, kind = CASES[name]
    P = B.Problem(d, n, L0, op, lo, hi)
    O = oracle.Problem(d, n, L0, op, lo, hi)
    u0 = initial(O, kind, d, op)
    ref = O.sequential(u0, dt, N, rtol=1e-15)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    opts = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-12, maxit=20000, inner_rtol=1e-6, ir_maxit=30, guess=guess)
    st = P.sequential_solve(cuda(u0), dt, N, uT, opts)
    assert st.n_failed == 0
    got = host(uT)
    for g in range(P.G):
        sl = slice(P.offsets[g], P.offsets[g + 1])
        assert rel(got[sl], ref[sl]) < 1e-9, (name, g)


@pytest.mark.parametrize("name", ["heat3d", "heat6d"])
def test_extrapolated_guess_needs_fewer_refinement_passes(name, capsys):
    """Smooth heat solutions: the extrapolated guess starts each step about
    (dt lambda)^2 |x| from its solution instead of dt lambda |x|, so one FP32
    correction mostly suffices where the previous state needed two."""
    d, n, L0, op, lo, hi, dt, N, kind = CASES[name]
    P = B.Problem(d, n, L0, op, lo, hi)
    O = oracle.Problem(d, n, L0, op, lo, hi)
    u0 = cuda(initial(O, kind, d, op))
    uT = torch.empty_like(u0)
    passes = {}
    for guess in GUESSES:
        opts = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-11, maxit=20000, inner_rtol=1e-6, ir_maxit=30, guess=guess)
        P.profile_enable(True)
        P.sequential_solve(u0, dt, N, uT, opts)
        prof = P.profile_read()
        P.profile_enable(False)
        passes[guess] = sum(prof.point_passes_f) / max(1, sum(prof.point_steps_f))
    with capsys.disabled():
        print(f"\n{name}: FP64 passes per node-step, previous {passes[B.PIT_GUESS_PREVIOUS]:.3f}, "
              f"extrapolated {passes[B.PIT_GUESS_EXTRAPOLATE]:.3f}")
    assert passes[B.PIT_GUESS_EXTRAPOLATE] < 0.8 * passes[B.PIT_GUESS_PREVIOUS]


@pytest.mark.parametrize("guess", GUESSES)
def test_mgrit_fixed_point_is_unchanged_by_the_guess(guess):
    """F-relaxation MGRIT with refinement fine solves converges to the
    oracle's sequential solution with either guess."""
    wl = W.workload(2)
    n, N, m = 5, 128, 8
    P = B.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    O = oracle.Problem(wl.d, n, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = O.initial(wl.ic_kind, wl.ic_params)
    dt = 0.05 / N
    fine = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-12, maxit=20000, inner_rtol=1e-6, ir_maxit=30, guess=guess)
    crs = B.solve_opts(B.PIT_PREC_FP32, rtol=1e-2, maxit=20000)
    mo = B.mgrit_opts(0.0, N * dt, N, m, 2, tol=1e-11, maxit=40, fine=fine, crs=crs, relax=B.PIT_RELAX_F)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    st = P.mgrit_solve(cuda(u0), mo, uT)
    assert st.n_converged == P.G
    assert rel(host(uT), O.sequential(u0, dt, N, rtol=1e-15)) < 1e-9
