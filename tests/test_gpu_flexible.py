"""Flexible CG (sp_solve_flexible) with Jacobi and with the learned network as preconditioner.

With Jacobi at every iteration FCG(1) is Jacobi-PCG in exact arithmetic: its iteration
count and solution match sp_solve_velocities (FP64, same start).  With the network applied
to the residual every k iterations the preconditioner changes between iterations; the
solve must still reach the tolerance, certified by the oracle's own FP64 system."""
import numpy as np
import pytest

import oracle
import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ss.load()


def _fp64_system(n, seed):
    L = synth.box_length(n)
    pos = synth.uniform_positions(n, (L, L, L), seed)
    kappa = ss.kappa_from_kappa_tau(0.5)
    sim = ss.Simulation(n, (L, L, L), kappa, seed=seed, cg_tol=TOL, cg_max_iter=3000, positions=pos,
                        precision="fp64", warm_start="none")
    delta = 0.3 * L
    sim.set_positions(pos, delta)
    sim.build_neighbors()
    sim.assemble()
    p = oracle.Params(n=n, L=(L, L, L), kappa=kappa, seed=seed)
    sysr = oracle.assemble(p, pos, sim.neighbors(), oracle.noise(seed, 0, np.arange(n)), delta)
    return sim, sysr


def _oracle_residual(sysr, v):
    return np.linalg.norm(sysr.b - sysr.matvec(v)) / np.linalg.norm(sysr.b)


def test_flexible_cg_with_jacobi_is_pcg():
    sim, sysr = _fp64_system(12000, 31)
    a = sim.solve_velocities()
    v_pcg = sim.get_velocities()
    b = sim.solve_flexible(0)
    v_fcg = sim.get_velocities()
    assert a["status"] == 0 and b["status"] == 0
    assert b["residual"] <= TOL and abs(b["iterations"] - a["iterations"]) <= 2, (a, b)
    assert np.abs(v_fcg - v_pcg).max() <= 1e-8 * np.abs(v_pcg).max()
    assert _oracle_residual(sysr, v_fcg) <= TOL * (1 + 1e-3)
    sim.close()


def _train_prior_free_network(n=20000, steps=40):
    """Weights of a network trained with its previous-velocity feature 0 (readout started at the
    Jacobi guess b / A_ii), on the solves of a mixed-precision trajectory."""
    L = synth.box_length(n)
    pos = synth.uniform_positions(n, (L, L, L), 41)
    sim = ss.Simulation(n, (L, L, L), ss.kappa_from_kappa_tau(0.5), seed=41, cg_tol=1e-8, positions=pos,
                        precision="mixed", warm_start="prev")
    sim.step(3)
    sim.mpnn_enable(seed=2)
    sim.mpnn_set_prior(False)
    w = sim.mpnn_weights()
    o = len(w) - 11
    w[o + 8], w[o + 9] = 1.0, 0.0
    sim.mpnn_set_weights(w)
    for _ in range(steps):
        info = sim.step(1)
        assert info["status"] == 0
        sim.mpnn_train_step(lr=2e-3)
    w = sim.mpnn_weights()
    sim.close()
    return w


def test_flexible_cg_with_the_network_as_preconditioner():
    weights = _train_prior_free_network()
    sim, sysr = _fp64_system(12000, 32)
    jac = sim.solve_flexible(0)
    sim.mpnn_enable(weights=weights)
    sim.mpnn_set_prior(False)
    its = {0: jac["iterations"]}
    for every in (1, 2, 4):
        info = sim.solve_flexible(every)
        v = sim.get_velocities()
        assert info["status"] == 0 and info["residual"] <= TOL, (every, info)
        assert _oracle_residual(sysr, v) <= TOL * (1 + 1e-3), every
        its[every] = info["iterations"]
    print("FCG iterations by net_every:", its)
    sim.close()


def test_flexible_cg_rejects_mixed_precision_and_missing_network():
    n = 3000
    L = synth.box_length(n)
    pos = synth.uniform_positions(n, (L, L, L), 5)
    for prec, every in (("mixed", 0), ("fp64", 2)):
        sim = ss.Simulation(n, (L, L, L), 1.0, seed=5, positions=pos, precision=prec)
        sim.build_neighbors()
        sim.assemble()
        with pytest.raises(ss.ShearsimError) as e:
            sim.solve_flexible(every)
        assert e.value.code == ss.SP_ERR_INVALID_ARG
        sim.close()
