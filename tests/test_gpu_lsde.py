"""GPU parity of the linear-SDE Fokker-Planck operator (Sec. 4.4, Eqs. "sde",
"sde_fokker_planck"): full drift matrix A, H = 2 sigma D sigma^T with
off-diagonal entries (mixed-derivative stencil), BiCGStab inside every
backward-Euler step, against the oracle; every case with the donor-cell and
with the central (second-order) drift flux.

Tolerances (relative L2): stencil and initial density 1e-13 (same formulas,
different rounding order); backward-Euler batches and MGRIT 1e-10 in FP64,
1e-9 with FP32 Krylov in FP64 refinement (both sides solve to 1e-13 or
tighter); the FP32 form 1e-4.
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


# (d, n, L0, A, H, box half-width): the two-dimensional linear oscillator of
# Sec. 4.4.1 (omega_0 = 1, xi = 0.05, sigma = (0, 1)^T, D = 0.1), a rotated
# three-dimensional system and a four-dimensional one with coupled diffusion
OSC_A = np.array([[0.0, 1.0], [-1.0, -0.1]])
OSC_H = np.array([[0.0, 0.0], [0.0, 0.2]])
A3 = np.array([[-0.5, 0.3, 0.0], [-0.2, -0.4, 0.6], [0.1, -0.6, -0.3]])
H3 = np.array([[0.4, 0.1, 0.0], [0.1, 0.3, 0.05], [0.0, 0.05, 0.2]])
A4 = -0.5 * np.eye(4) + 0.3 * np.diag(np.ones(3), 1) - 0.3 * np.diag(np.ones(3), -1)
H4 = 0.3 * np.eye(4) + 0.08 * (np.ones((4, 4)) - np.eye(4))
CASES = {"osc2d": (2, 6, 2, OSC_A, OSC_H, 10.0), "sde3d": (3, 5, 1, A3, H3, 5.0), "sde4d": (4, 5, 1, A4, H4, 5.0)}


def pair(name, central=False):
    d, n, L0, A, H, w = CASES[name]
    lo, hi = [-w] * d, [w] * d
    P = B.Problem(d, n, L0, B.PIT_OP_LSDE, lo, hi, drift=A, diffusion=H,
                  drift_scheme=B.PIT_DRIFT_CENTRAL if central else B.PIT_DRIFT_UPWIND)
    O = oracle.Problem(d, n, L0, oracle.OP_LSDE, lo, hi, drift=A, diffusion=H, central=central)
    return P, O


SCHEMES = pytest.mark.parametrize("central", [False, True], ids=["upwind", "central"])


def gauss_params(d):
    M = np.linspace(0.5, 1.0, d)
    C = 0.3 * np.eye(d) + 0.05 * (np.ones((d, d)) - np.eye(d))
    return np.concatenate([M, C.ravel()])


@SCHEMES
@pytest.mark.parametrize("name", list(CASES))
def test_stencil_and_initial_density_match_oracle(name, central):
    P, O = pair(name, central)
    nb = 2
    p = W.random_vector(31, nb * P.n_total)
    q = torch.empty(nb * P.n_total, dtype=torch.float64, device="cuda")
    P.apply(0.01, torch.from_numpy(p).cuda(), q)
    assert rel(q.cpu().numpy(), O.apply(0.01, p)) < 1e-13
    u = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    prm = gauss_params(P.d)
    P.sample_initial(4, prm, u)
    assert rel(u.cpu().numpy(), O.initial(4, prm)) < 1e-13
    P.close()


@pytest.mark.parametrize("prec,tol", [(B.PIT_PREC_FP64, 1e-10), (B.PIT_PREC_MIXED, 1e-9), (B.PIT_PREC_FP32, 1e-4)])
@pytest.mark.parametrize("name", list(CASES))
@SCHEMES
def test_phi_batch_matches_oracle(name, prec, tol, central):
    P, O = pair(name, central)
    nb, dt = 3, 0.02
    u = W.random_vector(41, nb * P.n_total)
    out = torch.empty(nb * P.n_total, dtype=torch.float64, device="cuda")
    opts = B.solve_opts(prec, rtol=1e-13 if prec != B.PIT_PREC_FP32 else 1e-6, maxit=20000, inner_rtol=1e-4,
                        ir_maxit=30)
    st = P.phi_batch(dt, torch.from_numpy(u).cuda(), out, opts)
    assert st.n_failed == 0
    ref = O.phi(dt, u, rtol=1e-15)
    got = out.cpu().numpy()
    for b in range(nb):
        for g in range(P.G):
            sl = slice(b * P.n_total + P.offsets[g], b * P.n_total + P.offsets[g + 1])
            assert rel(got[sl], ref[sl]) < tol, (b, g)
    P.close()


@pytest.mark.parametrize("prec,tol", [(B.PIT_PREC_FP64, 1e-10), (B.PIT_PREC_MIXED, 1e-9)])
@pytest.mark.parametrize("name", ["osc2d", "sde3d"])
@SCHEMES
def test_mgrit_matches_oracle_sequential(name, prec, tol, central):
    P, O = pair(name, central)
    N, m, T = 64, 8, 0.5
    dt = T / N
    u0 = O.initial(4, gauss_params(P.d))
    ref = O.sequential(u0, dt, N, rtol=1e-15)
    fine = B.solve_opts(prec, rtol=1e-13, maxit=20000, inner_rtol=1e-5, ir_maxit=40)
    crs = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13, maxit=20000)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    for relax, fas in ((B.PIT_RELAX_F, False), (B.PIT_RELAX_FCF, True)):
        opts = B.mgrit_opts(0.0, T, N, m, 2, tol=1e-13 * np.abs(ref).max(), maxit=64, fine=fine, crs=crs,
                            relax=relax, init=True, fas=fas)
        st = P.mgrit_solve(torch.from_numpy(u0).cuda(), opts, uT)
        assert st.n_converged == P.G
        assert rel(uT.cpu().numpy(), ref) < tol, (relax, fas)
    P.close()


def test_pair_form_is_refused_for_the_drift_operator():
    P, _ = pair("sde3d")
    x = torch.zeros(P.n_total, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PitError) as e:
        P.phi_batch(0.01, x, torch.empty_like(x), B.solve_opts(B.PIT_PREC_MIXED_PAIR, inner_rtol=1e-4))
    assert e.value.status == B.PIT_ERR_UNSUPPORTED
    P.close()


@SCHEMES
def test_large_grids_in_the_fp64_global_state_class_match_oracle(central):
    """Grids too large for the on-chip solve (here up to 8,001 nodes, the
    oscillator at level 12, L0 = 5) run the FP64 form's global-state variant,
    which keeps x, the Krylov vectors and the coefficient table in global
    memory; steps and MGRIT against the oracle."""
    d, n, L0, w = 2, 12, 5, 10.0
    P = B.Problem(d, n, L0, B.PIT_OP_LSDE, [-w] * d, [w] * d, drift=OSC_A, diffusion=OSC_H,
                  drift_scheme=B.PIT_DRIFT_CENTRAL if central else B.PIT_DRIFT_UPWIND)
    O = oracle.Problem(d, n, L0, oracle.OP_LSDE, [-w] * d, [w] * d, drift=OSC_A, diffusion=OSC_H, central=central)
    assert max(O.offsets[g + 1] - O.offsets[g] for g in range(O.G)) == 8001
    nb, dt = 2, 0.01
    u = W.random_vector(51, nb * P.n_total)
    out = torch.empty(nb * P.n_total, dtype=torch.float64, device="cuda")
    st = P.phi_batch(dt, torch.from_numpy(u).cuda(), out, B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13, maxit=20000))
    assert st.n_failed == 0
    assert rel(out.cpu().numpy(), O.phi(dt, u, rtol=1e-15)) < 1e-10
    # MGRIT in FP64 on the oscillator's normal initial law
    N, m, T = 64, 8, 0.5
    u0 = O.initial(4, np.concatenate([[5.0, 5.0], np.diag([1 / 9.0, 1 / 9.0]).ravel()]))
    ref = O.sequential(u0, T / N, N, rtol=1e-15)
    fine = B.solve_opts(B.PIT_PREC_FP64, rtol=1e-13, maxit=20000)
    uT = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    opts = B.mgrit_opts(0.0, T, N, m, 2, tol=1e-12 * np.abs(ref).max(), maxit=64, fine=fine, crs=fine,
                        relax=B.PIT_RELAX_F, init=True)
    st = P.mgrit_solve(torch.from_numpy(u0).cuda(), opts, uT)
    assert st.n_converged == P.G
    assert rel(uT.cpu().numpy(), ref) < 1e-10
    P.close()
