"""The velocity cross-correlation (Fig. vv) on the GPU against the oracle.

Counts must agree exactly (pairs near a bin edge, the cut-off or an image
boundary are decided with the definition's FP64 operations).  Each product
enters its bin rounded to a fixed point of 2^-20 of the largest FP32 |u|^2
(at most 2^-20 max|u|^2 per pair) after FP32 rounding of u and of the
product (at most 5 2^-24 |u_c||u_c'|): per bin |sum - oracle| <=
count 2^-19 max|u|^2.  <|u|^2> is an FP64 sum in another order (1e-13).
"""
import numpy as np
import pytest

import oracle
import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu


def _check(got, ref_sums, ref_counts, ref_vsq, u2max):
    assert np.array_equal(got["counts"], ref_counts)
    tol = ref_counts * 2.0 ** -19 * u2max + 1e-12
    assert np.all(np.abs(got["sums"] - ref_sums) <= tol), np.abs(got["sums"] - ref_sums).max()
    assert got["vsq"] == pytest.approx(ref_vsq, rel=1e-13, abs=1e-300)


def _u2max(pos, v, kappa, Ly):
    u = v.copy()
    u[:, 0] -= kappa * (pos[:, 1] - 0.5 * Ly)
    return float((u * u).sum(1).max())


@pytest.mark.parametrize("n,nbins,rmax", [(3000, 40, 2.5), (257, 7, 3.1), (2, 5, 4.0), (1, 3, 1.0)])
def test_random_configurations_match_the_oracle(n, nbins, rmax):
    """Several tiles with a ragged last one, one tile plus one particle, a single pair, no pair."""
    L = (7.3, 6.1, 5.2)
    rng = np.random.default_rng(n)
    pos = rng.random((n, 3)) * np.asarray(L)
    v = rng.standard_normal((n, 3))
    delta, kappa = 2.71, 0.35
    p = oracle.Params(n=n, L=L, kappa=kappa)
    rs, rc, rv = oracle.velocity_correlation(p, pos, delta, v, nbins, rmax)
    got = ss.velocity_correlation(pos, v, L, delta, kappa, nbins, rmax)
    _check(got, rs, rc, rv, _u2max(pos, v, kappa, L[1]))
    assert got["pairs"] == n * (n - 1) // 2


def test_lattice_puts_many_pairs_on_bin_edges_and_image_ties(monkeypatch):
    """A simple cubic lattice of spacing 0.5 in a box of 10 x 8 x 6 spacings:
    distances 0.5 sqrt(m) fall on the edges of bins of width 0.25, and pairs
    half a box apart tie between two images; a tiny initial list forces its
    growth."""
    monkeypatch.setenv("SHEARSIM_VCORR_BAND_CAP", "16")
    g = np.stack(np.meshgrid(np.arange(10), np.arange(8), np.arange(6), indexing="ij"), -1).reshape(-1, 3)
    pos = 0.5 * g.astype(np.float64)
    L = (5.0, 4.0, 3.0)
    n = pos.shape[0]
    v = np.random.default_rng(5).standard_normal((n, 3))
    for delta in (0.0, 1.5):
        p = oracle.Params(n=n, L=L, kappa=0.0)
        rs, rc, rv = oracle.velocity_correlation(p, pos, delta, v, 12, 3.0)
        got = ss.velocity_correlation(pos, v, L, delta, 0.0, 12, 3.0)
        assert got["boundary_pairs"] > 16
        _check(got, rs, rc, rv, _u2max(pos, v, 0.0, L[1]))


def test_uniform_velocity_gives_correlation_one():
    L = (6.0, 5.0, 4.0)
    rng = np.random.default_rng(9)
    pos = rng.random((1000, 3)) * np.asarray(L)
    v = np.tile([0.5, -0.25, 1.0], (1000, 1))
    got = ss.velocity_correlation(pos, v, L, 0.7, 0.0, 16, 2.0)
    ok = got["counts"] > 0
    assert np.allclose(got["correlation"][ok], 1.0, rtol=0, atol=2.0 ** -18)


def test_invalid_arguments():
    L = (6.0, 5.0, 4.0)
    pos = np.full((4, 3), 1.0)
    v = np.zeros((4, 3))
    for nbins, rmax in ((0, 1.0), (1025, 1.0), (8, 0.0), (8, -1.0)):
        with pytest.raises(ss.ShearsimError):
            ss.velocity_correlation(pos, v, L, 0.0, 0.0, nbins, rmax)
    bad = pos.copy()
    bad[2, 1] = 5.0   # y = L_y is outside [0, L_y)
    with pytest.raises(ss.ShearsimError):
        ss.velocity_correlation(bad, v, L, 0.0, 0.0, 8, 1.0)
    with pytest.raises(ss.ShearsimError):
        ss.velocity_correlation(pos, v, L, 6.0, 0.0, 8, 1.0)   # delta = L_x


@pytest.mark.parametrize("kappa_tau", [0.0, 0.5])
def test_paper_box_after_steps_matches_the_oracle(kappa_tau):
    """The paper's box (87.6 x 43.6 x 22 lambda^3, 17,191 particles) after a few
    steps, from the simulation's own positions and velocities."""
    w = synth.PAPER_BOX_VV
    kappa = ss.kappa_from_kappa_tau(kappa_tau)
    pos0 = synth.uniform_positions(w.n, w.L, w.seed)
    sim = ss.Simulation(w.n, w.L, kappa, seed=w.seed, precision="mixed", warm_start="prev", cg_tol=w.tol,
                        positions=pos0)
    assert sim.step(3)["status"] == 0
    nbins, rmax = 120, 12.25
    got = sim.velocity_correlation(nbins, rmax)
    pos, v = sim.get_positions(), sim.get_velocities()
    delta = sim.state()[0]
    sim.close()
    p = oracle.Params(n=w.n, L=w.L, kappa=kappa)
    rs, rc, rv = oracle.velocity_correlation(p, pos, delta, v, nbins, rmax)
    _check(got, rs, rc, rv, _u2max(pos, v, kappa, w.L[1]))
    # the friction coupling correlates neighbours: positive at contact
    assert got["correlation"][:8][got["counts"][:8] > 0].mean() > 0.0
