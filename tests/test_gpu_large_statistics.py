"""The large-scale workload (N = 4,194,304, mixed precision) against the FP64 GPU path at
N = 262,144, statistically: same density, alpha = 4, kappa tau = 0.5, dt = 0.01, both from a
uniform start over the same time window.  The shear stress is intensive and S(q) depends on
|q| and direction only, so their block averages (stress) and shell averages (S) must agree
within the statistical errors of the two runs (the FP64 path at N = 262,144 is the one the
oracle pins step by step; the large run's own steps are the mixed solver's)."""
import numpy as np
import pytest

import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu

SHELLS = [(0.5, 1.0), (1.0, 1.6), (1.6, 2.4)]


def _run(w, precision, steps, every, grid, nk):
    pos = synth.uniform_positions(w.n, w.L, w.seed)
    sim = ss.Simulation(w.n, w.L, ss.kappa_from_kappa_tau(w.kappa_tau), seed=w.seed, precision=precision,
                        warm_start="prev", cg_tol=1e-8, cg_max_iter=2000, positions=pos)
    sim.step(100)   # one time unit (~6 tau) from the uniform start, the same for both sizes
    stress, shells = [], [[] for _ in SHELLS]
    for k in range(steps):
        info = sim.step(1)
        assert info["status"] == 0 and info["last_residual"] <= 1e-8
        stress.append(info["stress_xy"])
        if k % every == every - 1:
            S, qx, qy = sim.structure_factor(nk, nk, grid=grid)
            qa = np.hypot(qx, qy).ravel()
            S = S.ravel()
            for j, (a, b) in enumerate(SHELLS):
                sel = (qa >= a) & (qa < b)
                shells[j].append(S[sel].mean())
    sim.close()
    return np.array(stress), np.array(shells)


def _blocks(x, nb):
    x = np.asarray(x)
    m = len(x) // nb * nb
    b = x[:m].reshape(nb, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nb)


def test_large_mixed_run_matches_fp64_statistics_at_262144():
    small = synth.PRECISION
    large = synth.LARGE
    kmax = lambda L: int(np.ceil(SHELLS[-1][1] * L / (2 * np.pi)))
    st_s, sq_s = _run(small, "fp64", 240, 20, 0, kmax(small.L[0]))
    st_l, sq_l = _run(large, "mixed", 240, 20, 256, kmax(large.L[0]))
    ms, es = _blocks(st_s, 6)
    ml, el = _blocks(st_l, 6)
    assert abs(ms - ml) <= 3 * np.hypot(es, el), (ms, es, ml, el)
    assert ml > 3 * el   # the pairs' friction stress opposes the imposed flow in the large run too
    for j in range(len(SHELLS)):
        a, ea = _blocks(sq_s[j], 4)
        b, eb = _blocks(sq_l[j], 4)
        assert abs(a - b) <= 3 * np.hypot(ea, eb) + 0.02 * a, (SHELLS[j], a, ea, b, eb)
