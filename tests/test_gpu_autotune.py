"""Autotuning of the persistent solver's tile configuration (sp_autotune).

Every configuration runs the same iteration with the same per-row arithmetic;
only the grouping of the dot products' block partial sums (hence their
rounding, ~1e-13 relative) depends on the block count.  So a tuned simulation
must step like an untuned one to rounding, and tuning must leave positions,
step counter and warm start unchanged.
"""
import numpy as np
import pytest

import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu


def _sim(n=32768, precision="mixed", seed=97):
    L = (synth.box_length(n),) * 3
    pos = synth.uniform_positions(n, L, seed)
    kappa = ss.kappa_from_kappa_tau(0.5)
    return ss.Simulation(n, L, kappa, alpha=4.0, eps=1.0, zeta=1.0, kT=1.0, dt=0.01, rc=1.0, seed=seed,
                         precision=precision, warm_start="prev", cg_tol=1e-8, cg_max_iter=2000, positions=pos)


def test_autotune_keeps_results(monkeypatch):
    monkeypatch.delenv("SHEARSIM_TUNE_CACHE", raising=False)
    a, b = _sim(), _sim()
    a.step(2)
    b.step(2)
    before = a.get_positions()
    st_before = a.state()
    info = a.autotune(trials=1)
    assert 0 <= info["config"] < len(info["ms"])
    assert all(t > 0 for t in info["ms"])
    assert info["ms"][info["config"]] == min(info["ms"])
    assert not info["from_cache"]
    assert np.array_equal(a.get_positions(), before)
    assert a.state() == st_before
    a.step(3)
    b.step(3)
    L = synth.box_length(32768)
    d = a.get_positions() - b.get_positions()
    d -= np.round(d / L) * L
    # each step's velocities agree within cond * tol (solves to 1e-8): |dx| <= 3 dt |dv| ~ 1e-6
    assert np.abs(d).max() < 1e-5
    va, vb = a.get_velocities(), b.get_velocities()
    # both solved to 1e-8 relative residual: velocities agree within cond * tol
    assert np.abs(va - vb).max() <= 1e-6 * np.abs(vb).max()
    a.close()
    b.close()


def test_autotune_cache_and_fp64(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SHEARSIM_TUNE_CACHE", str(cache))
    a = _sim(n=16384)
    first = a.autotune(trials=1)
    assert cache.exists() and cache.read_text().strip()
    b = _sim(n=16384)
    second = b.autotune(trials=1)
    assert second["from_cache"] and second["config"] == first["config"]
    c = _sim(n=4096, precision="fp64")
    none = c.autotune(trials=1)
    assert none["config"] == 0 and all(t == 0 for t in none["ms"])
    for s in (a, b, c):
        s.close()
