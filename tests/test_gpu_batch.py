"""Batches of replicas (one graph per step, one cooperative solve launch) against
the same replicas advanced one by one."""
import numpy as np
import pytest

import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu

REPLICAS = [(2000, 0.01), (3500, 0.05), (6000, 0.2), (9000, 0.5), (15000, 1.0)]


def _replicas(tol=1e-10):
    out = []
    for k, (n, kt) in enumerate(REPLICAS):
        L = synth.box_length(n)
        out.append(dict(n=n, L=(L, L, L), kappa=ss.kappa_from_kappa_tau(kt), seed=900 + k, cg_tol=tol,
                        cg_max_iter=2000, precision="mixed", warm_start="prev"))
    return out


def _positions():
    return [synth.uniform_positions(n, (synth.box_length(n),) * 3, 77 + k) for k, (n, _) in enumerate(REPLICAS)]


def test_batch_matches_individual_runs():
    reps = _replicas()
    pos = _positions()
    steps = 3
    batch = ss.Batch(reps, positions=pos)
    infos = batch.step(steps)
    assert batch.blocks().min() >= 1
    for k, kw in enumerate(reps):
        assert infos[k]["status"] == 0 and infos[k]["steps_done"] == steps
        assert infos[k]["last_residual"] <= kw["cg_tol"]
        got = batch.sim(k).get_positions()
        delta, step = batch.sim(k).state()
        assert step == steps
        with ss.Simulation(positions=pos[k], **kw) as sim:
            sim.step(steps)
            ref = sim.get_positions()
            d_ref, _ = sim.state()
        L = kw["L"][0]
        d = got - ref
        d -= np.round(d / L) * L
        assert np.abs(d).max() < 1e-8, (k, np.abs(d).max())
        assert abs(delta - d_ref) < 1e-12
    batch.close()


def test_batch_is_deterministic():
    outs = []
    for _ in range(2):
        batch = ss.Batch(_replicas(1e-8), positions=_positions())
        batch.step(2)
        outs.append([batch.sim(k).get_positions() for k in range(len(REPLICAS))])
        batch.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_batch_follows_the_oracle():
    """Each replica of a batch, stepped by the FP64 CPU oracle from the same positions with its own
    seed, shear rate and box: the positions after the steps agree to the solve tolerance."""
    import oracle
    reps = _replicas(1e-10)
    pos = _positions()
    steps = 3
    batch = ss.Batch(reps, positions=pos)
    infos = batch.step(steps)
    for k, kw in enumerate(reps):
        assert infos[k]["status"] == 0 and infos[k]["steps_done"] == steps
        p = oracle.Params(n=kw["n"], L=kw["L"], kappa=kw["kappa"], seed=kw["seed"])
        opos, od = pos[k], 0.0
        for s in range(steps):
            r = oracle.step(p, opos, od, s, tol=1e-13)
            opos, od = r.pos, r.delta
        got = batch.sim(k).get_positions()
        delta, _ = batch.sim(k).state()
        L = kw["L"][0]
        d = got - opos
        d -= np.round(d / L) * L
        # per step |v_gpu - v| <= ~cond * 1e-10 * max|v| (cond ~ 22, max|v| ~ 60), times dt = 0.01
        assert np.abs(d).max() < 1e-9 * steps, (k, np.abs(d).max())
        assert abs(delta - od) < 1e-12
    batch.close()


def test_batch_with_a_replica_at_the_largest_ensemble_size():
    """A replica of 131,072 particles (the ensemble's upper end) beside a small one, against the
    single-system path."""
    sizes = [(131072, 0.3), (8192, 0.01)]
    reps, pos = [], []
    for k, (n, kt) in enumerate(sizes):
        L = synth.box_length(n)
        reps.append(dict(n=n, L=(L, L, L), kappa=ss.kappa_from_kappa_tau(kt), seed=950 + k, cg_tol=1e-10,
                         cg_max_iter=2000, precision="mixed", warm_start="prev"))
        pos.append(synth.uniform_positions(n, (L, L, L), 500 + k))
    steps = 2
    batch = ss.Batch(reps, positions=pos)
    infos = batch.step(steps)
    for k, kw in enumerate(reps):
        assert infos[k]["status"] == 0 and infos[k]["steps_done"] == steps
        got = batch.sim(k).get_positions()
        with ss.Simulation(positions=pos[k], **kw) as sim:
            sim.step(steps)
            ref = sim.get_positions()
        L = kw["L"][0]
        d = got - ref
        d -= np.round(d / L) * L
        assert np.abs(d).max() < 1e-9 * steps, (k, np.abs(d).max())
    batch.close()


def test_batch_autotune_keeps_the_state_and_the_results():
    """sp_batch_autotune times every tile configuration of the batched solver, leaves the
    replicas' state unchanged, and the tuned batch still matches the replicas stepped alone."""
    reps = _replicas(1e-10)
    pos = _positions()
    batch = ss.Batch(reps, positions=pos)
    batch.step(1)
    before = [(batch.sim(k).get_positions(), batch.sim(k).state()) for k in range(len(reps))]
    tune = batch.autotune(trials=2)
    assert 0 <= tune["config"] < tune["num_configs"] and tune["ms"][tune["config"]] > 0
    assert sum(1 for t in tune["ms"] if t > 0) >= 2
    for k in range(len(reps)):
        after = batch.sim(k).get_positions(), batch.sim(k).state()
        assert np.array_equal(before[k][0], after[0]) and before[k][1] == after[1]
    steps = 2
    infos = batch.step(steps)
    for k, kw in enumerate(reps):
        assert infos[k]["status"] == 0 and infos[k]["steps_done"] == steps
        with ss.Simulation(positions=pos[k], **kw) as sim:
            sim.step(1 + steps)
            ref = sim.get_positions()
        L = kw["L"][0]
        d = batch.sim(k).get_positions() - ref
        d -= np.round(d / L) * L
        assert np.abs(d).max() < 1e-8, (k, np.abs(d).max())
    for cfg in range(tune["num_configs"]):   # every configuration steps correctly
        batch.set_config(cfg)
        infos = batch.step(1)
        assert all(x["status"] == 0 and x["last_residual"] <= 1e-10 for x in infos), cfg
    batch.close()
