"""Host-side checks of the benchmark's per-workload MGRIT configuration (no
GPU): the options each measured form hands to the library.  The extrapolated
initial sweep (init 2) needs the heat operators and refinement or FP32
coarse solves; a form without them must fall back to the plain sweep rather
than be refused at run time, and the oracle legs must use the same coarse
step as the GPU arm."""
import pytest

import bench
from paper_2509_22156_gb300 import binding as B
from paper_2509_22156_gb300 import workloads as W


def setup(k, **kw):
    wl = W.workload(k)
    wl.extra["k"] = k
    chosen, fp64, mixed, plain = bench.solver_setup(wl, B, relax=B.PIT_RELAX_F, **kw)
    return wl, chosen, fp64


def test_headline_uses_the_refinement_form_and_the_extrapolated_sweep():
    wl, chosen, fp64 = setup(5)
    assert chosen.fine.prec == B.PIT_PREC_MIXED and chosen.crs.prec == B.PIT_PREC_MIXED
    assert chosen.init == 2 and chosen.levels == 3
    assert chosen.tol == bench.MGRIT_TOL_BY_WORKLOAD[5] and chosen.fine.rtol == bench.KRYLOV_RTOL_BY_WORKLOAD[5]
    assert chosen.fine.guess == B.PIT_GUESS_DEFAULT  # extrapolated guess of every refinement step
    # the paper's form: FP64 Krylov, FAS, FCF, no initial sweep
    assert fp64.fine.prec == B.PIT_PREC_FP64 and fp64.fas == 1 and fp64.init == 0 and fp64.relax == B.PIT_RELAX_FCF


def test_extrapolated_sweep_falls_back_where_it_is_not_built():
    # the pair-refinement comparison form: pair coarse solves, plain sweep
    wl, chosen, _ = setup(5, coarse=B.PIT_COARSE_IMPLICIT, fine_prec=B.PIT_PREC_MIXED_PAIR)
    assert chosen.init == 1
    # heat3d_n9 keeps the plain sweep (measured faster); ou4d_n7 has a drift operator
    for k in (2, 3):
        wl, chosen, _ = setup(k)
        assert chosen.init == 1, k


def test_variable_coefficient_workload_takes_the_extrapolated_steps():
    wl, chosen, _ = setup(4)
    assert chosen.init == 2 and chosen.crs.prec == B.PIT_PREC_FP32
    assert bench.COARSE_FALLBACK_BY_WORKLOAD[4] == B.PIT_COARSE_EXTRAP
    assert bench.ORACLE_COARSE_KIND[B.PIT_COARSE_EXTRAP] == 4
    assert bench.ORACLE_COARSE_KIND[B.PIT_COARSE_LEARNED] == 0  # a rejected network falls back to BE


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_every_workload_has_consistent_tolerances(k):
    wl, chosen, fp64 = setup(k)
    assert 0.0 < chosen.tol < 1e-6
    assert 0.0 < chosen.fine.rtol <= 1e-10
    assert wl.nsteps % (wl.m ** (wl.levels - 1)) == 0
