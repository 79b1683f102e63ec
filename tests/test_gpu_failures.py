"""Failure paths of the C ABI, injected on the host (no GPU fault, trap or hang).

- positions that are NaN or outside the box, given through sp_set_positions or
  sp_step_host, are caught by the device-side check of the gather and return
  SP_ERR_INVALID_ARG, with no step taken;
- a NaN in the injected thermal normals (sp_set_noise) makes the solve return
  SP_ERR_NONFINITE;
- a wait limit far below one grid barrier (sp_set_wait_limit) makes the
  persistent solver's bounded barrier wait give up: SP_ERR_TIMEOUT;
and in every case the same simulation steps correctly afterwards.
"""
import numpy as np
import pytest

import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ss.load()


def _sim(n, precision="fp64", seed=3, warm_start="none"):
    L = synth.box_length(n)
    pos = synth.uniform_positions(n, (L, L, L), seed)
    sim = ss.Simulation(n, (L, L, L), ss.kappa_from_kappa_tau(0.5), seed=seed, cg_tol=1e-8, positions=pos,
                        precision=precision, warm_start=warm_start)
    return sim, pos, L


@pytest.mark.parametrize("bad", [np.nan, -1e-3, "L", np.inf])
def test_set_positions_rejects_bad_coordinates_and_recovers(bad):
    sim, pos, L = _sim(1500)
    wrong = pos.copy()
    wrong[777, 1] = L if bad == "L" else bad
    with pytest.raises(ss.ShearsimError) as e:
        sim.set_positions(wrong, 0.0)
    assert e.value.code == ss.SP_ERR_INVALID_ARG
    sim.set_positions(pos, 0.0)
    info = sim.step(2)
    assert info["status"] == 0 and info["steps_done"] == 2
    ref, pr, _ = _sim(1500)
    ref.step(2)
    assert np.array_equal(sim.get_positions(), ref.get_positions())
    sim.close()
    ref.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_host_rejects_bad_coordinates_without_stepping(precision):
    sim, pos, L = _sim(2000, precision)
    wrong = pos.copy()
    wrong[5, 2] = np.nan
    out = np.empty_like(pos)
    info = sim.step_host(wrong, 0.0, 3, out, raise_on_error=False)
    assert info["status"] == ss.SP_ERR_INVALID_ARG, info
    assert info["steps_done"] == 0
    assert sim.state()[1] == 0   # the step counter did not move
    info = sim.step_host(pos, 0.0, 3, out)
    assert info["status"] == 0 and info["steps_done"] == 3
    ref, _, _ = _sim(2000, precision)
    ref.step(3)
    assert np.array_equal(out, ref.get_positions())
    sim.close()
    ref.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nan_in_the_noise_returns_nonfinite_and_recovers(precision):
    n = 2500
    sim, pos, L = _sim(n, precision)
    xi = np.random.default_rng(1).standard_normal((n, 3))
    xi[123, 0] = np.nan
    sim.set_noise(xi)
    info = sim.step(1, raise_on_error=False)
    assert info["status"] == ss.SP_ERR_NONFINITE, info
    assert info["steps_done"] == 0
    sim.set_noise(None)
    info = sim.step(2)
    assert info["status"] == 0 and info["steps_done"] == 2
    assert np.isfinite(sim.get_positions()).all()
    sim.close()


RESIDENT_CONFIG = 9   # the on-chip solver k32_cg_resident<512, 4> (sp_set_solver_config)


@pytest.mark.parametrize("n,config", [(20000, RESIDENT_CONFIG), (20000, 0), (400000, 0)])
def test_barrier_wait_limit_returns_timeout_and_recovers(n, config):
    """The on-chip and the streaming persistent solvers give up a grid-barrier wait at the limit."""
    sim, pos, L = _sim(n, "mixed")
    ref, _, _ = _sim(n, "mixed")
    for s in (sim, ref):
        assert s.set_solver_config(config)["resident"] == (config == RESIDENT_CONFIG)
    sim.set_wait_limit(1e-9)
    info = sim.step(1, raise_on_error=False)
    assert info["status"] == ss.SP_ERR_TIMEOUT, info
    assert info["steps_done"] == 0
    sim.set_wait_limit(2.0)
    info = sim.step(2)
    assert info["status"] == 0 and info["steps_done"] == 2
    ref.step(2)
    assert np.array_equal(sim.get_positions(), ref.get_positions())
    with pytest.raises(ss.ShearsimError):
        sim.set_wait_limit(0.0)
    sim.close()
    ref.close()
