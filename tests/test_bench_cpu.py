"""bench.py's roofline bookkeeping, on the CPU.

The measured DRAM traffic is reported only for the kernel, workload and regime
(burn-in steps) it was captured in; algorithmic bytes follow the per-particle
rule; kernel names match the tile configurations the library reports.
"""
import pytest

import bench

RESIDENT = {"gathers_in_flight": 4, "blocks_per_sm": 1, "pipelined": False, "block_threads": 512,
            "resident": True, "matrix_free": False}
STREAMING = {"gathers_in_flight": 6, "blocks_per_sm": 1, "pipelined": False, "block_threads": 1024,
             "resident": False, "matrix_free": False}
MATRIX_FREE = {"gathers_in_flight": 4, "blocks_per_sm": 3, "pipelined": False, "block_threads": 256,
               "resident": False, "matrix_free": True}


def test_traffic_only_for_the_captured_regime():
    # the on-chip solve was captured in the timed steps after the 1,000-step burn-in
    t = bench.profiled_traffic("mixed-n262144", RESIDENT, 1000)
    assert t is not None and 1e8 < t < 1e9
    assert bench.profiled_traffic("mixed-n262144", RESIDENT, 0) is None         # from the uniform start
    assert bench.profiled_traffic("mixed-n262144-kt0.05", RESIDENT, 1000) is None   # another workload
    assert bench.profiled_traffic("mixed-n262144", STREAMING, 1000) is None     # another kernel
    assert bench.profiled_traffic("mixed-n262144", None, 1000) is None


def test_kernel_names_follow_the_configuration():
    assert bench.solver_kernel_name(RESIDENT) == "k32_cg_resident<512,4>"
    assert bench.solver_kernel_name(dict(RESIDENT, block_threads=1024)) == "k32_cg_resident<1024,2>"
    assert bench.solver_kernel_name(STREAMING) == "k32_cg_persistent<6,1,0,1024>"
    assert bench.solver_kernel_name(MATRIX_FREE) == "k32_cg_persistent<4,3,0,256,1>"
    # the large workload's captures are keyed by these names
    for tune in (STREAMING, MATRIX_FREE):
        assert bench.solver_kernel_name(tune) in bench.LARGE_PROFILED_TRAFFIC


def test_algorithmic_bytes_rule():
    n, iters = 262144, 54
    assert bench.plan_algorithmic_bytes(n, iters, "mixed") == pytest.approx(280.0 * n * iters)
    assert bench.plan_algorithmic_bytes(n, iters, "fp64") == pytest.approx(450.0 * n * iters)
    # the detailed count adds the replacements' and the initial residual's bytes
    base = bench.persistent_algorithmic_bytes(n, 18 * n, iters, 2)
    assert bench.persistent_algorithmic_bytes(n, 18 * n, iters, 2, init=True) > base > 0
