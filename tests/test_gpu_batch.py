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
