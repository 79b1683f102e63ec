"""sp_step_host: host positions in, steps, host positions out in one call.

The call runs the same graph as sp_step between the copies that
sp_set_positions and sp_get_positions make, so a trajectory stepped through
it is bit-identical to one stepped through the three calls, whatever the
number of steps per call and when the output aliases the input.
"""
import numpy as np
import pytest

import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu


def _sim(n, pos, precision):
    L = (synth.box_length(n),) * 3
    kappa = ss.kappa_from_kappa_tau(0.5)
    return ss.Simulation(n, L, kappa, seed=11, cg_tol=1e-8, positions=pos, warm_start="prev", precision=precision)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_host_stepping_matches_the_three_calls(precision):
    n = 20000
    L = (synth.box_length(n),) * 3
    pos0 = synth.uniform_positions(n, L, 5)
    delta0 = 0.3 * L[0]
    a, b, c = _sim(n, pos0, precision), _sim(n, pos0, precision), _sim(n, pos0, precision)
    pa, da = pos0.copy(), delta0
    for _ in range(3):
        a.set_positions(pa, da)
        da = a.step(1)["delta"]
        pa = a.get_positions()
    bufs = [pos0.copy(), np.empty_like(pos0)]
    db = delta0
    for k in range(3):
        info = b.step_host(bufs[k & 1], db, 1, bufs[(k + 1) & 1])
        assert info["status"] == 0 and info["steps_done"] == 1
        db = info["delta"]
    pb = bufs[1]
    pc = pos0.copy()   # three steps in one call, output over the input
    info = c.step_host(pc, delta0, 3, pc)
    assert info["steps_done"] == 3
    assert np.array_equal(pa, pb) and da == db
    assert np.array_equal(pa, pc) and da == info["delta"]
    assert a.state() == b.state() == c.state()
    for s in (a, b, c):
        s.close()


def test_host_stepping_rejects_bad_offsets():
    n = 1000
    L = (synth.box_length(n),) * 3
    pos = synth.uniform_positions(n, L, 2)
    s = _sim(n, pos, "mixed")
    with pytest.raises(ss.ShearsimError):
        s.step_host(pos, L[0], 1, pos.copy())
    s.close()
