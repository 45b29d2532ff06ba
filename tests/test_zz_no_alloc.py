"""The allocation-free in-place step (pit_phi_batch_inplace_static).

It exists for callers that cannot allocate device memory while they run (an
application whose GPU memory is reserved by another allocator, or a loop that
forbids allocation after start-up).  It must give what pit_phi_batch gives
for the same step, call after call: the static scratch it stages through is
shared and reused, so two consecutive calls are checked.  It must also
allocate nothing on its first call on a new problem: the library counts its
own device allocations (pit_profile_read's device_allocs), and the count must
not move across the call, while it does move across an in-place
pit_phi_batch call, which stages through an allocated buffer.  This file is
collected last so that a failing run stopped at the first failure has already
run every other test.
"""
import numpy as np
import pytest

from paper_2509_22156_gb300 import binding as B
from paper_2509_22156_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# the tolerance of the FP64 parity tests
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_22156_gb300 import build
    build.build()
    B.load()
    torch.cuda.set_device(0)


def _rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [B.PIT_PREC_FP64, B.PIT_PREC_MIXED])
def test_static_inplace_matches_phi_batch_two_calls(prec):
    P = B.Problem(3, 6, 1, B.PIT_OP_HEAT)
    dt = 0.05 / 1024
    nb = 3
    opts = B.solve_opts(prec, rtol=1e-12, inner_rtol=1e-4, ir_maxit=30)
    u = torch.from_numpy(W.random_vector(404, nb * P.n_total)).cuda()
    # reference: the allocating entry point, out of place
    y1 = torch.empty_like(u)
    y2 = torch.empty_like(u)
    P.phi_batch(dt, u, y1, opts)
    P.phi_batch(dt, y1, y2, opts)
    # two calls in a row, in place, through the static scratch
    x = u.clone()
    st = P.phi_batch_inplace_static(dt, x, opts)
    torch.cuda.synchronize()
    assert st.n_items == nb * P.G and st.n_failed == 0
    assert _rel(x, y1) < TOL
    P.phi_batch_inplace_static(dt, x, opts, stats=False)
    torch.cuda.synchronize()
    assert _rel(x, y2) < TOL


def test_static_inplace_rejects_oversize_and_keeps_working():
    P = B.Problem(3, 6, 1, B.PIT_OP_HEAT)
    too_many = B.STATIC_SCRATCH_DOUBLES // P.n_total + 1
    x = torch.zeros(P.n_total, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PitError) as e:
        P.phi_batch_inplace_static(1e-4, x, n_batch=too_many)
    assert e.value.status == B.PIT_ERR_INVALID_ARG
    assert "static scratch" in str(e.value)
    # a valid call afterwards still works (zero state stays zero)
    P.phi_batch_inplace_static(1e-4, x)
    torch.cuda.synchronize()
    assert float(x.abs().max()) == 0.0


def _allocs_during(P, fn):
    P.profile_enable(True)
    fn()
    torch.cuda.synchronize()
    n = P.profile_read().device_allocs
    P.profile_enable(False)
    return n


@pytest.mark.parametrize("prec", [B.PIT_PREC_FP64, B.PIT_PREC_MIXED, B.PIT_PREC_MIXED_PAIR])
def test_static_first_call_on_a_new_problem_allocates_nothing(prec):
    opts = B.solve_opts(prec, rtol=1e-12, inner_rtol=1e-4, ir_maxit=30)
    dt = 0.05 / 1024
    # a new problem: no pit_phi_batch call has planned or tuned anything on it
    P = B.Problem(3, 5, 1, B.PIT_OP_HEAT)
    u = torch.from_numpy(W.random_vector(405, 2 * P.n_total)).cuda()
    x = u.clone()
    torch.cuda.synchronize()
    assert _allocs_during(P, lambda: P.phi_batch_inplace_static(dt, x, opts)) == 0
    assert _allocs_during(P, lambda: P.phi_batch_inplace_static(dt, x, opts)) == 0
    # the counter sees allocations: the in-place step of pit_phi_batch stages
    # through a buffer it allocates on first use
    y = u.clone()
    assert _allocs_during(P, lambda: P.phi_batch(dt, y, y, opts)) > 0
    # and the result is the one of two pit_phi_batch steps, out of place
    y1, y2 = torch.empty_like(u), torch.empty_like(u)
    P.phi_batch(dt, u, y1, opts)
    P.phi_batch(dt, y1, y2, opts)
    assert _rel(x, y2) < TOL


def test_static_forcing_and_wide_batch_match_phi_batch():
    """Forcing f in the right-hand side, and a batch of 9 entries (the wide
    batch class, whose CTA size comes from the autotuner's other slot)."""
    P = B.Problem(3, 5, 1, B.PIT_OP_VARHEAT)
    dt = 0.1 / 2048 * 32
    nb = 9
    opts = B.solve_opts(B.PIT_PREC_MIXED, rtol=1e-12, inner_rtol=1e-4, ir_maxit=30)
    u = torch.from_numpy(W.random_vector(406, nb * P.n_total)).cuda()
    f = torch.from_numpy(W.random_vector(407, nb * P.n_total)).cuda()
    y1, y2 = torch.empty_like(u), torch.empty_like(u)
    P.phi_batch(dt, u, y1, opts, f=f)
    P.phi_batch(dt, y1, y2, opts, f=f)
    x = u.clone()
    st = P.phi_batch_inplace_static(dt, x, opts, f=f)
    torch.cuda.synchronize()
    assert st.n_items == nb * P.G and st.n_failed == 0
    assert _rel(x, y1) < TOL
    P.phi_batch_inplace_static(dt, x, opts, f=f)
    torch.cuda.synchronize()
    assert _rel(x, y2) < TOL


def test_static_rejects_global_scratch_grids_and_unsupported_forms():
    # d = 2, level 13: the grids (1, 13) and (13, 1) hold 8191 nodes, more than
    # one CTA's shared memory takes in the FP64-refinement form
    P = B.Problem(2, 13, 1, B.PIT_OP_HEAT)
    x = torch.zeros(P.n_total, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PitError) as e:
        P.phi_batch_inplace_static(1e-4, x, B.solve_opts(B.PIT_PREC_MIXED, inner_rtol=1e-4))
    assert e.value.status == B.PIT_ERR_UNSUPPORTED
    # the pair form is not implemented for the drift operator
    Q = B.Problem(2, 4, 1, B.PIT_OP_OU, lo=[-6.0] * 2, hi=[6.0] * 2)
    y = torch.zeros(Q.n_total, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PitError) as e:
        Q.phi_batch_inplace_static(1e-3, y, B.solve_opts(B.PIT_PREC_MIXED_PAIR, inner_rtol=1e-4))
    assert e.value.status == B.PIT_ERR_UNSUPPORTED
