"""Profiling counters of the C ABI: timed calls, device time and kernel
launches per kernel family, read back after an MGRIT solve and a combination
sum."""
import numpy as np
import pytest

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


def test_profile_counts_calls_and_kernels():
    wl = W.workload(2)
    P = B.Problem(wl.d, 6, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    P.sample_initial(wl.ic_kind, wl.ic_params, u0)
    uT = torch.empty_like(u0)
    fine = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-11, maxit=4000, inner_rtol=1e-5, ir_maxit=12)
    opts = B.mgrit_opts(wl.t0, wl.t1, 256, 16, 2, tol=1e-9, maxit=20, fine=fine, relax=B.PIT_RELAX_F)
    P.mgrit_solve(u0, opts, uT)  # first call plans and tunes the launch shapes
    pts = torch.from_numpy(np.random.default_rng(3).uniform(0.0, 1.0, (500, wl.d))).cuda()
    out = torch.empty(500, dtype=torch.float64, device="cuda")

    P.profile_enable(True)
    st = P.mgrit_solve(u0, opts, uT)
    P.combine(uT, pts, out)
    pr = P.profile_read()
    P.profile_enable(False)

    assert st.max_cycles >= 1
    # relaxation and sweeps: at least one kernel per timed call, one per
    # shared-memory bucket the call splits into
    for f in (0, 1):
        assert pr.launches[f] > 0
        assert pr.kernels[f] >= pr.launches[f]
        assert pr.ms[f] > 0.0
    # the combination sum is one call: one kernel, or two when it splits the
    # grids into chunks whose partial sums a second kernel adds
    assert pr.launches[2] == 1 and pr.kernels[2] in (1, 2)
    assert pr.phi_items > 0 and pr.point_steps > 0

    # disabled profiling records nothing; enabling again starts from zero
    P.mgrit_solve(u0, opts, uT)
    P.profile_enable(True)
    pr2 = P.profile_read()
    P.profile_enable(False)
    assert sum(pr2.launches) == 0 and sum(pr2.kernels) == 0


def test_profile_splits_work_counters_by_family():
    wl = W.workload(2)
    P = B.Problem(wl.d, 5, wl.L0, wl.op, wl.lo, wl.hi)
    u0 = torch.empty(P.n_total, dtype=torch.float64, device="cuda")
    P.sample_initial(wl.ic_kind, wl.ic_params, u0)
    uT = torch.empty_like(u0)
    fine = B.solve_opts(B.PIT_PREC_MIXED_PAIR, rtol=1e-11, maxit=4000, inner_rtol=1e-5, ir_maxit=12)
    crs = B.solve_opts(B.PIT_PREC_FP32, rtol=1e-2, maxit=4000)
    opts = B.mgrit_opts(wl.t0, wl.t1, 256, 16, 2, tol=1e-9, maxit=20, fine=fine, crs=crs, relax=B.PIT_RELAX_F)
    P.mgrit_solve(u0, opts, uT)
    P.profile_enable(True)
    P.mgrit_solve(u0, opts, uT)
    pr = P.profile_read()
    P.profile_enable(False)
    assert pr.point_iters_f[0] + pr.point_iters_f[1] == pr.point_iters
    assert pr.point_passes_f[0] + pr.point_passes_f[1] == pr.point_passes
    assert pr.point_steps_f[0] + pr.point_steps_f[1] == pr.point_steps
    # relaxation in the pair refinement: residual passes; FP32 coarse sweeps: none
    assert pr.point_passes_f[0] > 0 and pr.point_passes_f[1] == 0
    assert pr.point_iters_f[1] > 0
