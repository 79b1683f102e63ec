"""Long-run statistics of the GPU path against what the physics fixes.

- Zero shear, no friction coupling (alpha = kappa = 0), eps = 1: overdamped
  Langevin dynamics of the Gaussian-core pair potential U = 0.1 kT w(r) of
  Eq. exvol (truncated and shifted at r_c).  Its equilibrium structure factor
  follows the random-phase approximation S(q) = 1 / (1 + rho beta U(q)), very
  accurate for this weak potential (beta U <= 0.1); the comparison pins the
  noise amplitude against the force (both enter S(q)).
- eps = 0 as well: free diffusion, mean squared displacement 6 kT t / zeta.
- Sheared runs (kappa tau = 0.5, alpha = 4): block-averaged shear stress and
  S(q) of the mixed-precision solver agree with the FP64 solver within their
  statistical errors.
"""
import numpy as np
import pytest

import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu

LAMBDA2 = 1.0 / (2.0 * np.log(20.0))   # r_c = 1: w(r_c) = 0.05


def _sim(n, seed, kappa_tau, alpha, eps, precision="mixed", tol=1e-8):
    L = (synth.box_length(n),) * 3
    pos = synth.uniform_positions(n, L, seed)
    kappa = ss.kappa_from_kappa_tau(kappa_tau) if kappa_tau > 0 else 0.0
    return ss.Simulation(n, L, kappa, alpha=alpha, eps=eps, zeta=1.0, kT=1.0, dt=0.01, rc=1.0, seed=seed,
                         precision=precision, warm_start="prev", cg_tol=tol, cg_max_iter=2000, positions=pos), L


def _rpa(q, rho):
    """1 / (1 + rho beta U(q)), U(q) the 3-d transform of 0.1 (w - 0.05) inside r_c."""
    from scipy.integrate import quad
    def u(r):
        return 0.1 * (np.exp(-r * r / (2 * LAMBDA2)) - 0.05)
    uq = np.array([4 * np.pi * quad(lambda r: u(r) * r * r * np.sinc(qq * r / np.pi), 0.0, 1.0)[0] for qq in q])
    return 1.0 / (1.0 + rho * uq)


def _blocks(x, nb):
    x = np.asarray(x)
    m = len(x) // nb * nb
    b = x[:m].reshape(nb, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nb)


def test_zero_shear_structure_factor_follows_rpa():
    n = 4096
    sim, L = _sim(n, 811, 0.0, 0.0, 1.0)
    sim.step(1000)                              # ~4 relaxation times of the slowest density mode
    shells = [(0.5, 1.0), (1.0, 1.6), (1.6, 2.4), (2.4, 3.4)]
    samples = [[] for _ in shells]
    qmid = np.zeros(len(shells))
    for _ in range(320):
        sim.step(25)
        S, qx, qy = sim.structure_factor(6, 6, grid=0)
        qa = np.hypot(qx, qy).ravel()
        S = S.ravel()
        for k, (a, b) in enumerate(shells):
            sel = (qa >= a) & (qa < b)
            samples[k].append(S[sel].mean())
            qmid[k] = qa[sel].mean()
    sim.close()
    rpa = _rpa(qmid, n / L[0] ** 3)
    for k in range(len(shells)):
        m, err = _blocks(samples[k], 10)
        assert abs(m - rpa[k]) <= 3 * err + 0.02 * rpa[k], (shells[k], m, err, rpa[k])
    # the structure is visibly depleted at small q (S(0.75) ~ 0.77): the force is on
    assert _blocks(samples[0], 10)[0] < 0.9


def test_free_diffusion_einstein():
    n = 8192
    sim, _ = _sim(n, 813, 0.0, 0.0, 0.0)
    steps, dt = 100, 0.01
    disp = np.zeros((n, 3))
    for _ in range(steps):
        sim.step(1)
        disp += sim.get_velocities() * dt
    sim.close()
    msd = (disp ** 2).sum(axis=1)
    t = steps * dt
    # 6 kT t / zeta; per-particle MSD is 2 t chi^2_3-distributed: sd = sqrt(6)(2t)/sqrt(n)
    assert abs(msd.mean() - 6 * t) <= 4 * np.sqrt(6) * 2 * t / np.sqrt(n)


def test_sheared_mixed_matches_fp64_statistics():
    n = 4096
    runs = {}
    for prec in ("mixed", "fp64"):
        sim, _ = _sim(n, 817, 0.5, 4.0, 1.0, precision=prec)
        sim.step(100)
        stress, sq = [], []
        for k in range(600):
            sim.step(1)
            stress.append(sim.stress_xy())
            if k % 50 == 49:
                S, qx, qy = sim.structure_factor(4, 4, grid=0)
                sq.append(S.ravel())
        sim.close()
        runs[prec] = (np.array(stress), np.array(sq))
    sm, se = _blocks(runs["mixed"][0], 6)
    fm, fe = _blocks(runs["fp64"][0], 6)
    assert abs(sm - fm) <= 3 * np.hypot(se, fe) + 1e-12, (sm, se, fm, fe)
    assert sm > 3 * se    # the friction stress of the pairs opposes the imposed flow
    qm = runs["mixed"][1].mean(axis=0)
    qf = runs["fp64"][1].mean(axis=0)
    qe = np.hypot(runs["mixed"][1].std(axis=0), runs["fp64"][1].std(axis=0)) / np.sqrt(len(runs["mixed"][1]))
    ok = np.isfinite(qm) & (qe > 0)
    assert np.all(np.abs(qm - qf)[ok] <= 4 * qe[ok] + 1e-9)
