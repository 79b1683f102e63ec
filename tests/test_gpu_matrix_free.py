"""Matrix-free SpMV of the streaming mixed solver (tile configurations 10 and 11).

The inner iteration recomputes each pair weight w_ij = exp(-|R_ij|^2 / 2 lambda^2)
(§Method) in FP32 from the positions in 32-bit fixed point, and reads only
the columns of the pair list; the residual replacements still use the
assembled double-float weights.  So a matrix-free solve must meet the same
tolerance on the same system, in about the same number of iterations as the
stored-weight streaming solve (configuration 0), and its velocities must agree
with those to cond x tol.  A weight taken at the wrong periodic or sheared
image would make the inner operator disagree with the assembled one and stall
the replacements: the offsets below put the Lees-Edwards image shift at a
quarter, near half, and near the whole of L_x, where the wrapped fixed-point
differences must still give the pair's own image.  The oracle's FP64 system
certifies the velocities.
"""
import numpy as np
import pytest

import oracle
import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu

MF_CONFIGS = (10, 11)


def _sim(n, seed, kappa_tau=0.5, tol=1e-8, warm="none"):
    L = (synth.box_length(n),) * 3
    pos = synth.uniform_positions(n, L, seed)
    kappa = ss.kappa_from_kappa_tau(kappa_tau)
    return ss.Simulation(n, L, kappa, alpha=4.0, eps=1.0, zeta=1.0, kT=1.0, dt=0.01, rc=1.0, seed=seed,
                         precision="mixed", warm_start=warm, cg_tol=tol, cg_max_iter=2000, positions=pos)


@pytest.mark.parametrize("config", MF_CONFIGS)
def test_matrix_free_configs_are_described(config):
    s = _sim(4096, 5)
    info = s.set_solver_config(config)
    assert info["matrix_free"] and not info["resident"]
    assert not s.set_solver_config(0)["matrix_free"]
    s.close()


@pytest.mark.parametrize("config", MF_CONFIGS)
@pytest.mark.parametrize("delta_frac", [0.0, 0.25, 0.4999, 0.9999])
def test_matrix_free_solve_matches_stored_weights_and_oracle(config, delta_frac):
    n, seed = 20000, 41
    a, b = _sim(n, seed), _sim(n, seed)
    L = synth.box_length(n)
    pos = synth.uniform_positions(n, (L,) * 3, seed + 1)
    delta = delta_frac * L
    for s in (a, b):
        s.set_positions(pos, delta)
    assert a.set_solver_config(config)["matrix_free"]
    b.set_solver_config(0)
    for s in (a, b):
        s.build_neighbors()
        s.assemble()
    ia, ib = a.solve_velocities(), b.solve_velocities()
    assert ia["status"] == 0 and ib["status"] == 0
    assert ia["residual"] <= 1e-8 and ib["residual"] <= 1e-8
    # same system, same start: the recomputed weights (~3e-7 relative) change
    # the iteration count by rounding-level amounts only
    assert abs(ia["iterations"] - ib["iterations"]) <= 3, (ia, ib)
    va, vb = a.get_velocities(), b.get_velocities()
    assert np.abs(va - vb).max() <= 1e-6 * np.abs(vb).max()
    # the oracle's FP64 system of the same positions, offset and step
    p = oracle.Params(n=n, L=(L,) * 3, kappa=oracle.kappa_from_kappa_tau(0.5), alpha=4.0, eps=1.0, zeta=1.0, kT=1.0,
                      dt=0.01, rc=1.0, seed=seed)
    _, step0 = a.state()
    pairs = oracle.neighbors(p, pos, delta, "cells")
    sysr = oracle.assemble(p, pos, pairs, oracle.noise(p.seed, step0, np.arange(n)), delta)
    res = np.linalg.norm(sysr.b - sysr.matvec(va)) / np.linalg.norm(sysr.b)
    assert res <= 1e-8, res
    a.close()
    b.close()


@pytest.mark.parametrize("config", MF_CONFIGS)
def test_matrix_free_steps_follow_the_stored_weight_steps(config):
    """Warm-started steps (the offset advancing with the shear) stay together."""
    n, seed = 32768, 7
    a, b = _sim(n, seed, kappa_tau=5.0, warm="prev"), _sim(n, seed, kappa_tau=5.0, warm="prev")
    a.set_solver_config(config)
    b.set_solver_config(0)
    for _ in range(4):
        ia, ib = a.step(1), b.step(1)
        assert ia["status"] == 0 and ib["status"] == 0
        assert ia["last_residual"] <= 1e-8
        assert abs(ia["cg_iterations"] - ib["cg_iterations"]) <= 3, (ia, ib)
        va, vb = a.get_velocities(), b.get_velocities()
        assert np.abs(va - vb).max() <= 1e-6 * np.abs(vb).max()
    assert a.state()[0] != 0.0
    a.close()
    b.close()
