"""xi = p(A) g ~ A^(1/2) g (FDT-consistent noise) on the GPU against the oracle.

Both sides evaluate the same degree-K Chebyshev interpolant of sqrt on
[1, Gershgorin max] by the same three-term recurrence, each on its own
assembled matrix: FP64 entries agree to ~1e-14, and the recurrence (|T_k| <= 1
on the spectrum) keeps the difference near K times that, so the FP64 path
must agree to 1e-11 relative; the mixed path's double-float entries agree to
~1e-12, so 1e-9 there.
"""
import numpy as np
import pytest

import oracle
import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu


def _setup(n, seed, precision, alpha=4.0, delta_frac=0.3):
    L = synth.box_length(n)
    pos = synth.uniform_positions(n, (L, L, L), seed)
    kappa = ss.kappa_from_kappa_tau(0.5)
    sim = ss.Simulation(n, (L, L, L), kappa, alpha=alpha, seed=seed, positions=pos, precision=precision,
                        warm_start="none", cg_tol=1e-12 if precision == "fp64" else 1e-8, cg_max_iter=5000)
    delta = delta_frac * L
    sim.set_positions(pos, delta)
    sim.build_neighbors()
    sim.assemble()
    p = oracle.Params(n=n, L=(L, L, L), kappa=kappa, alpha=alpha, seed=seed)
    pairs = oracle.neighbors(p, pos, delta)
    sysr = oracle.assemble(p, pos, pairs, np.zeros((n, 3)), delta)
    return sim, p, pos, delta, pairs, sysr


@pytest.mark.parametrize("precision,n,degree,tol", [("fp64", 3000, 24, 1e-11), ("fp64", 777, 5, 1e-11),
                                                    ("mixed", 3000, 24, 1e-9)])
def test_sqrt_apply_matches_the_oracle(precision, n, degree, tol):
    sim, p, pos, delta, pairs, sysr = _setup(n, n + 3, precision)
    g = np.random.default_rng(n).standard_normal((n, 3))
    xi, lmax = sim.sqrt_apply(g, degree)
    ref, lref = oracle.sqrt_apply(sysr, g, degree)
    sim.close()
    assert lmax == pytest.approx(lref, rel=1e-12)
    assert np.abs(xi - ref).max() <= tol * np.abs(ref).max()


def test_uncoupled_system_returns_g_and_bad_arguments_raise():
    sim, p, pos, delta, pairs, sysr = _setup(500, 4, "fp64", alpha=0.0)
    g = np.random.default_rng(1).standard_normal((500, 3))
    xi, lmax = sim.sqrt_apply(g, 8)
    assert lmax == 1.0 and np.array_equal(xi, g)
    for deg in (0, 5000):
        with pytest.raises(ss.ShearsimError):
            sim.sqrt_apply(g, deg)
    sim.close()


def test_fdt_step_through_the_api_matches_the_oracle():
    """Build and assemble, correlate the step's noise as A^(1/2) g, inject it,
    assemble again and solve: the velocities are the oracle's for the same
    injected noise."""
    n = 2000
    sim, p, pos, delta, pairs, sysr = _setup(n, 9, "fp64")
    g = oracle.noise(p.seed, 0, np.arange(n))
    xi, _ = sim.sqrt_apply(g, 32)
    sim.set_noise(xi)
    sim.assemble()
    assert sim.solve_velocities()["status"] == 0
    v = sim.get_velocities()
    sim.close()
    xi_ref, _ = oracle.sqrt_apply(sysr, g, 32)
    ref, _, _ = oracle.pcg(oracle.assemble(p, pos, pairs, xi_ref, delta), 1e-13)
    assert np.abs(v - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("precision,tol,pos_tol", [("fp64", 1e-13, 1e-10), ("mixed", 1e-11, 1e-9)])
def test_fdt_steps_follow_the_oracle(precision, tol, pos_tol):
    """sp_step with A^(1/2)-correlated noise against the oracle's step whose
    normals are the oracle's p(A) g for the same step (two steps: the second
    uses the first's positions, offset and step counter)."""
    n, steps, degree = 1500, 2, 24
    L = synth.box_length(n)
    seed = 31
    pos = synth.uniform_positions(n, (L, L, L), seed)
    kappa = ss.kappa_from_kappa_tau(0.5)
    sim = ss.Simulation(n, (L, L, L), kappa, seed=seed, positions=pos, precision=precision, warm_start="prev",
                        cg_tol=tol, cg_max_iter=5000)
    sim.set_fdt_noise(degree)
    info = sim.step(steps)
    assert info["status"] == 0
    gpos = sim.get_positions()
    sim.close()
    p = oracle.Params(n=n, L=(L, L, L), kappa=kappa, seed=seed)
    opos, od = pos, 0.0
    for s in range(steps):
        sysr = oracle.assemble(p, opos, oracle.neighbors(p, opos, od), np.zeros((n, 3)), od)
        xi, _ = oracle.sqrt_apply(sysr, oracle.noise(seed, s, np.arange(n)), degree)
        r = oracle.step(p, opos, od, s, xi=xi, tol=1e-13)
        opos, od = r.pos, r.delta
    d = gpos - opos
    d -= np.round(d / L) * L
    assert np.abs(d).max() < pos_tol * steps


def test_fdt_off_again_is_the_paper_noise():
    n = 1200
    L = synth.box_length(n)
    outs = []
    for toggle in (False, True):
        pos = synth.uniform_positions(n, (L, L, L), 5)
        sim = ss.Simulation(n, (L, L, L), ss.kappa_from_kappa_tau(0.5), seed=5, positions=pos, warm_start="prev")
        if toggle:
            sim.set_fdt_noise(16)
            sim.set_fdt_noise(0)
        sim.step(2)
        outs.append(sim.get_positions())
        sim.close()
    assert np.array_equal(outs[0], outs[1])
