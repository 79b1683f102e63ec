"""The C ABI library builds, loads and exports what include/shearsim.h declares;
host-side argument checks answer without touching a GPU."""
import ctypes
import math
import subprocess

import numpy as np
import pytest

import oracle
import paper_1808_06381_gb300 as ss
from paper_1808_06381_gb300 import build as ss_build


@pytest.fixture(scope="module")
def lib():
    ss_build.build()
    return ss.load()


def test_library_exports_every_declared_symbol(lib):
    declared = ss.declared_symbols()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", ss.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for name in declared:
        getattr(lib, name)


def test_library_is_built_for_sm_103a_only(lib):
    """Every translation unit is compiled with exactly one -gencode, for sm_103a (the GPU side
    checks the architecture the device actually runs: tests/test_gpu_build.py)."""
    assert ss_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert not any("gencode" in f or "arch" in f for f in ss_build.NVCC_FLAGS)


def _params(**kw):
    p = ss.sp_params()
    p.n = kw.get("n", 100)
    for a in range(3):
        p.L[a] = kw.get("L", 4.0)
    p.rc, p.alpha, p.eps, p.zeta, p.kT = 1.0, 4.0, 1.0, 1.0, 1.0
    p.kappa, p.dt, p.seed = 1.0, 0.01, 1
    p.precision, p.warm_start = kw.get("precision", 0), 0
    p.cg_tol, p.cg_max_iter, p.device = 1e-8, 100, kw.get("device", 0)
    for k, v in kw.items():
        if hasattr(p, k) and k not in ("L",):
            setattr(p, k, v)
    return p


@pytest.mark.parametrize("kw,code", [
    (dict(n=1), ss.SP_ERR_INVALID_ARG),
    (dict(L=1.5), ss.SP_ERR_BOX_TOO_SMALL),
    (dict(dt=0.0), ss.SP_ERR_INVALID_ARG),
    (dict(zeta=-1.0), ss.SP_ERR_INVALID_ARG),
    (dict(precision=7), ss.SP_ERR_INVALID_ARG),
    (dict(cg_tol=0.0), ss.SP_ERR_INVALID_ARG),
])
def test_invalid_parameters_are_rejected_on_the_host(lib, kw, code):
    p = _params(**kw)
    h = ctypes.c_void_p()
    assert lib.sp_sim_create(ctypes.byref(p), None, ctypes.byref(h)) == code
    assert not h.value
    assert len(lib.sp_last_error(None)) > 0


def test_missing_device_is_reported(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = _params()
    h = ctypes.c_void_p()
    assert lib.sp_sim_create(ctypes.byref(p), None, ctypes.byref(h)) == ss.SP_ERR_NO_DEVICE


def test_null_handles_are_safe(lib):
    assert lib.sp_sim_destroy(None) == 0
    assert lib.sp_build_neighbors(None) == ss.SP_ERR_INVALID_ARG
    assert lib.sp_step(None, 1, None) == ss.SP_ERR_INVALID_ARG


def test_kappa_conversion_matches_the_oracle(lib):
    for kt in (0.005, 0.05, 0.5):
        assert abs(ss.kappa_from_kappa_tau(kt) - oracle.kappa_from_kappa_tau(kt)) < 1e-15 * kt * 10
    assert abs(ss.kappa_from_kappa_tau(0.5) - 0.5 * 2 * math.log(20.0)) < 1e-12
    assert math.isnan(lib.sp_kappa_from_kappa_tau(0.5, 1.0, 1.0, 0.0))
