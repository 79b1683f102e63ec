"""Learned warm start on the GPU against its FP64 oracle (oracle/mpnn.py).

BF16 tolerance: weights and the MLP's inputs and activations are rounded to
BF16 (relative 2^-9) before each tensor-core product with FP32 accumulation;
through three layers this leaves about 1 % relative error on the guess and a
few per cent on the gradients, so the bounds are 3e-2 (guess) and 8e-2
(gradient, relative L2 per weight tensor)."""
import numpy as np
import pytest

import oracle
from oracle import mpnn
import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu


def _weights(seed):
    W = mpnn.init_weights(seed)
    W.o = np.random.Generator(np.random.PCG64(seed + 1)).normal(0, 0.6, W.o.shape)
    return W


def _solved_sim(n, seed, precision="fp64"):
    L = synth.box_length(n)
    pos = synth.uniform_positions(n, (L, L, L), seed)
    sim = ss.Simulation(n, (L, L, L), ss.kappa_from_kappa_tau(0.5), seed=seed, cg_tol=1e-12, positions=pos,
                        precision=precision, warm_start="prev", cg_max_iter=5000)
    sim.set_positions(pos, 0.3 * L)
    sim.build_neighbors()
    sim.assemble()
    sim.solve_velocities()
    return sim


def test_forward_matches_oracle():
    n = 3000
    sim = _solved_sim(n, 5)
    W = _weights(3)
    sim.mpnn_enable(weights=W.flat().astype(np.float32))
    vprev = sim.get_velocities()            # the network reads the current velocities as vprev
    sim.set_step(1)                          # fresh noise: b differs from the one solved
    sim.assemble()
    diag, b, pairs, w = sim.system()
    guess = sim.mpnn_forward()
    ref, _ = mpnn.forward(mpnn.Weights.unflat(W.flat().astype(np.float32)), n, 4.0, pairs, w, diag, b, vprev)
    rel = np.linalg.norm(guess - ref) / np.linalg.norm(ref)
    assert rel < 3e-2, rel
    sim.close()


def test_gradients_match_oracle():
    n = 3000
    sim = _solved_sim(n, 7)
    W = _weights(11)
    Wf = W.flat().astype(np.float32)
    sim.mpnn_enable(weights=Wf)
    vprev = sim.get_velocities()
    sim.set_step(1)
    sim.assemble()
    diag, b, pairs, w = sim.system()
    sim.mpnn_forward()
    sim.solve_velocities()
    vstar = sim.get_velocities()
    loss, grad = sim.mpnn_train_step(lr=0.0, want_grad=True)
    rloss, rg = mpnn.loss_and_grad(mpnn.Weights.unflat(Wf), n, 4.0, pairs, w, diag, b, vprev, vstar)
    assert abs(loss - rloss) <= 3e-2 * rloss, (loss, rloss)
    g = mpnn.Weights.unflat(grad)
    for name in ("W1", "W2", "W3", "o"):
        a, r = getattr(g, name), getattr(rg, name)
        rel = np.linalg.norm(a - r) / np.linalg.norm(r)
        assert rel < 8e-2, (name, rel)
    # lr = 0 leaves the weights unchanged
    assert np.array_equal(sim.mpnn_weights(), Wf)
    sim.close()


def test_online_training_lowers_the_loss_and_keeps_cg_exact():
    """Train on the systems the simulation generates (one Adam step per time step);
    CG still reaches the tolerance from the network's guess."""
    n, steps = 20000, 40
    L = synth.box_length(n)
    pos = synth.uniform_positions(n, (L, L, L), 13)
    sim = ss.Simulation(n, (L, L, L), ss.kappa_from_kappa_tau(0.5), seed=13, cg_tol=1e-8, positions=pos,
                        precision="mixed", warm_start="prev")
    sim.step(3)
    sim.mpnn_enable(seed=1)
    losses, iters = [], []
    for _ in range(steps):
        info = sim.step(1)
        assert info["status"] == 0 and info["last_residual"] <= 1e-8
        iters.append(info["cg_iterations"])
        losses.append(sim.mpnn_train_step(lr=2e-3))
    assert np.mean(losses[-10:]) < 0.8 * np.mean(losses[:5]), (losses[:5], losses[-10:])
    sim.close()


def test_adam_steps_match_the_oracle_element_by_element():
    """Two GPU Adam steps on the FP32 masters against oracle/mpnn.py's adam_step, fed the
    same gradients (the GPU's), after a gradient-only call that must not count as a step."""
    n, lr = 3000, 2e-3
    sim = _solved_sim(n, 17, precision="mixed")
    W = _weights(21)
    w = W.flat().astype(np.float32)
    sim.mpnn_enable(weights=w)
    sim.step(1)
    sim.mpnn_train_step(lr=0.0)   # gradient only
    assert np.array_equal(sim.mpnn_weights(), w)
    m = np.zeros(w.shape)
    v = np.zeros(w.shape)
    for t in (1, 2):
        sim.step(1)
        _, g = sim.mpnn_train_step(lr=lr, want_grad=True)
        got = sim.mpnn_weights()
        ref, m, v = mpnn.adam_step(mpnn.Weights.unflat(w.astype(np.float64)),
                                   mpnn.Weights.unflat(g.astype(np.float64)), m, v, t, lr)
        ref = ref.flat()
        # FP32 masters and moments: the update lr m^/(sqrt(v^) + eps) to ~1e-6 relative, the
        # stored weight to its FP32 rounding
        err = np.abs(got - ref)
        assert np.all(err <= 2e-7 * np.maximum(np.abs(ref), 1.0) + 1e-5 * lr), (t, err.max())
        w = got
    sim.close()


def _train_on_streamed_solves(seeds, steps_per_seed, lr=2e-3):
    """Online training on the precision workload's dynamics (N = 262,144, kappa tau 0.5): one Adam
    step per time step, the weights carried from one seed's trajectory to the next."""
    w = synth.PRECISION
    weights = None
    for sd in seeds:
        pos = synth.uniform_positions(w.n, w.L, sd)
        sim = ss.Simulation(w.n, w.L, ss.kappa_from_kappa_tau(w.kappa_tau), seed=sd, cg_tol=w.tol, positions=pos,
                            precision="mixed", warm_start="prev")
        sim.step(3)
        sim.mpnn_enable(seed=1, weights=weights)
        for _ in range(steps_per_seed):
            info = sim.step(1)
            assert info["status"] == 0 and info["last_residual"] <= w.tol
            sim.mpnn_train_step(lr=lr)
        weights = sim.mpnn_weights()
        sim.close()
    return weights


def test_trained_network_cuts_cg_iterations():
    """The network trained on streamed solves of three seeds, then run on a held-out seed: CG
    iterations per step to the same 1e-8 with its guess, with a cold start (v0 = 0) and with the
    previous velocities, from the same state after a common burn-in."""
    w = synth.PRECISION
    weights = _train_on_streamed_solves([101, 102, 103], 40)
    held_out = 104
    pos = synth.uniform_positions(w.n, w.L, held_out)
    kappa = ss.kappa_from_kappa_tau(w.kappa_tau)
    iters = {}
    for mode in ("learned", "prev", "none"):
        sim = ss.Simulation(w.n, w.L, kappa, seed=held_out, cg_tol=w.tol, positions=pos, precision="mixed",
                            warm_start="none" if mode == "none" else "prev")
        sim.step(5)
        if mode == "learned":
            sim.mpnn_enable(weights=weights)
        its = []
        for _ in range(20):
            info = sim.step(1)
            assert info["status"] == 0 and info["last_residual"] <= w.tol
            its.append(info["cg_iterations"])
        iters[mode] = float(np.mean(its))
        sim.close()
    print("CG iterations per step:", iters)
    assert iters["learned"] < iters["none"] - 1.0, iters
    assert iters["learned"] < iters["prev"], iters
