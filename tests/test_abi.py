"""The C-ABI library builds, loads and exports every symbol include/*.h declares
(no compute calls: this runs without a GPU)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pit_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2509_22156_gb300 import build as B
    B.build()
    from paper_2509_22156_gb300 import binding
    return binding.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("pit_problem_create", "pit_phi_batch", "pit_combine", "pit_mgrit_solve"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2509_22156_gb300 import binding
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(pit_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)
    # the binding wraps the same names
    assert set(binding.EXPORTED) <= set(_declared())


def test_creation_without_a_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    from paper_2509_22156_gb300 import binding as B
    with pytest.raises(B.PitError) as e:
        B.Problem(2, 5)
    assert e.value.status == B.PIT_ERR_CUDA


def test_invalid_descriptions_rejected_before_any_device_use(lib):
    from paper_2509_22156_gb300 import binding as B
    import ctypes
    bad = [dict(d=7, n=5), dict(d=0, n=5), dict(d=2, n=3, L0=4), dict(d=2, n=5, L0=0)]
    for kw in bad:
        desc = B.pit_problem_desc()
        desc.d, desc.level_n, desc.level0, desc.op = kw["d"], kw["n"], kw.get("L0", 1), 0
        for i in range(6):
            desc.lo[i], desc.hi[i] = 0.0, 1.0
        h = ctypes.c_void_p()
        rc = lib.pit_problem_create(ctypes.byref(desc), None, ctypes.byref(h))
        assert rc == B.PIT_ERR_INVALID_ARG, kw
        assert b"" != lib.pit_last_error()
    desc = B.pit_problem_desc()
    desc.d, desc.level_n, desc.level0, desc.op = 2, 5, 1, 0
    desc.lo[0], desc.hi[0], desc.lo[1], desc.hi[1] = 0.0, 1.0, 1.0, 1.0  # empty box on axis 1
    h = ctypes.c_void_p()
    assert lib.pit_problem_create(ctypes.byref(desc), None, ctypes.byref(h)) == B.PIT_ERR_INVALID_ARG
    # drift schemes: unknown value, and the central flux on an operator without it
    for op, scheme in ((B.PIT_OP_LSDE, 2), (B.PIT_OP_LSDE, -1), (B.PIT_OP_HEAT, B.PIT_DRIFT_CENTRAL),
                       (B.PIT_OP_OU, B.PIT_DRIFT_CENTRAL)):
        desc = B.pit_problem_desc()
        desc.d, desc.level_n, desc.level0, desc.op = 2, 5, 1, op
        for i in range(2):
            desc.lo[i], desc.hi[i] = -1.0, 1.0
        desc.drift_scheme = scheme
        assert lib.pit_problem_create(ctypes.byref(desc), None, ctypes.byref(h)) == B.PIT_ERR_INVALID_ARG, (op, scheme)
    # CME rates: finite, production and degradation >= 0, saturation > 0, box in x >= 0
    good = (3.0, 110.0, 2.0, 0.01)
    for rates, lo in (((3.0, 0.0, 2.0, 0.01), 0.0), ((-3.0, 110.0, 2.0, 0.01), 0.0),
                      ((3.0, 110.0, 2.0, -0.01), 0.0), ((3.0, 110.0, float("inf"), 0.01), 0.0), (good, -1.0)):
        desc = B.pit_problem_desc()
        desc.d, desc.level_n, desc.level0, desc.op = 2, 5, 1, B.PIT_OP_CME
        for i in range(2):
            desc.lo[i], desc.hi[i] = lo, 60.0
            desc.cme_prod[i], desc.cme_sat[i], desc.cme_exp[i], desc.cme_deg[i] = rates
        assert lib.pit_problem_create(ctypes.byref(desc), None, ctypes.byref(h)) == B.PIT_ERR_INVALID_ARG, rates
