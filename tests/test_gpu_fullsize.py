"""The benchmark's own solves, certified by the oracle at full size.

The default benchmark line steps N = 262,144 particles (density 3, alpha = 4,
dt = 0.01) with the mixed-precision solver to ||b - A v|| <= 1e-8 ||b||, each
step warm-started from the previous velocities.  The solver's own stopping
test uses its double-float copy of the system.  Here every step's velocities
are checked against the system the FP64 CPU oracle assembles for the same
positions, offset and step (its own cell-list pair search and its own
normals): the oracle's residual ||b - A v|| / ||b|| must be <= 1e-8 and agree
with the residual the GPU reports.  Both shear rates of that workload
(kappa tau = 0.5 and 0.05), the on-chip solver (the benchmark's choice), the
streaming one, and the streaming one with the matrix-free SpMV.
"""
import numpy as np
import pytest

import oracle
import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu

RESIDENT_CONFIG = 9   # k32_cg_resident<512, 4>, the autotuner's choice at this size
MATRIX_FREE_CONFIG = 11   # the streaming solve with the matrix-free SpMV


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ss.load()


@pytest.mark.parametrize("workload,config", [(synth.PRECISION, RESIDENT_CONFIG), (synth.PRECISION, 0),
                                             (synth.PRECISION_LOW_SHEAR, RESIDENT_CONFIG),
                                             (synth.PRECISION, MATRIX_FREE_CONFIG)])
def test_benchmark_steps_meet_the_tolerance_on_the_oracle_system(workload, config):
    w = workload
    pos = synth.uniform_positions(w.n, w.L, w.seed)
    kappa = ss.kappa_from_kappa_tau(w.kappa_tau)
    sim = ss.Simulation(w.n, w.L, kappa, alpha=w.alpha, eps=w.eps, zeta=w.zeta, kT=w.kT, dt=w.dt, rc=w.rc,
                        seed=w.seed, precision="mixed", warm_start="prev", cg_tol=w.tol, cg_max_iter=2000,
                        positions=pos)
    tune = sim.set_solver_config(config)
    assert tune["resident"] == (config == RESIDENT_CONFIG)
    assert tune["matrix_free"] == (config == MATRIX_FREE_CONFIG)
    p = oracle.Params.from_workload(w)
    sim.step(2)   # the warm start then comes from real previous velocities
    for _ in range(3):
        x0 = sim.get_positions()
        delta0, step0 = sim.state()
        info = sim.step(1)
        assert info["status"] == 0 and info["host_driven"] == 0
        v = sim.get_velocities()
        pairs = oracle.neighbors(p, x0, delta0, "cells")
        sysr = oracle.assemble(p, x0, pairs, oracle.noise(p.seed, step0, np.arange(p.n)), delta0)
        res = np.linalg.norm(sysr.b - sysr.matvec(v)) / np.linalg.norm(sysr.b)
        assert res <= w.tol, (res, info["last_residual"])
        # the GPU's double-float residual and the oracle's FP64 one differ by the
        # double-float system's rounding (~1e-12 relative), far inside the tolerance
        assert abs(res - info["last_residual"]) <= 1e-3 * w.tol, (res, info["last_residual"])
    sim.close()
