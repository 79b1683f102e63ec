"""Pins of the oracle's velocity cross-correlation (§Results, Fig. vv) against
things other than itself: closed forms (uniform and purely affine velocity
fields), a k-d tree's periodic pair search (scipy, at delta = 0), brute force
over explicit Lees-Edwards images (delta != 0), and hand-placed pairs."""
import math

import numpy as np
import pytest

import oracle

scipy_spatial = pytest.importorskip("scipy.spatial")


def _random(n, L, seed):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * np.asarray(L)
    v = rng.standard_normal((n, 3))
    return pos, v


def test_uniform_velocity_gives_correlation_one():
    L = (6.0, 5.0, 4.0)
    pos, _ = _random(300, L, 1)
    v = np.tile([0.3, -1.2, 0.7], (300, 1))
    p = oracle.Params(n=300, L=L, kappa=0.0)
    sums, counts, vsq = oracle.velocity_correlation(p, pos, 1.3, v, 16, 2.0)
    u2 = 0.3 * 0.3 + 1.2 * 1.2 + 0.7 * 0.7
    assert vsq == pytest.approx(u2, rel=1e-14)
    assert counts.sum() > 1000
    assert np.allclose(sums, counts * u2, rtol=1e-12, atol=0)


def test_affine_flow_is_subtracted():
    """v = kappa (y - L_y/2) x is the imposed flow itself: u = 0 everywhere."""
    L = (6.0, 5.0, 4.0)
    pos, _ = _random(200, L, 2)
    kappa = 0.37
    v = np.zeros((200, 3))
    v[:, 0] = kappa * (pos[:, 1] - 0.5 * L[1])
    p = oracle.Params(n=200, L=L, kappa=kappa)
    sums, counts, vsq = oracle.velocity_correlation(p, pos, 2.1, v, 8, 2.0)
    assert vsq == 0.0 and np.all(sums == 0.0) and counts.sum() > 0
    # the same field with the opposite sign is not the flow: u = -2 v
    v[:, 0] *= -1.0
    _, _, vsq2 = oracle.velocity_correlation(p, pos, 2.1, v, 8, 2.0)
    assert vsq2 == pytest.approx(4.0 * np.mean(v[:, 0] ** 2), rel=1e-12)


def test_counts_and_sums_match_a_kd_tree_at_zero_shift():
    L = (7.0, 6.0, 5.0)
    n = 1500
    pos, v = _random(n, L, 3)
    nbins, rmax = 20, 2.4
    p = oracle.Params(n=n, L=L, kappa=0.0)
    sums, counts, vsq = oracle.velocity_correlation(p, pos, 0.0, v, nbins, rmax)
    tree = scipy_spatial.cKDTree(pos, boxsize=L)
    dm = tree.sparse_distance_matrix(tree, rmax, output_type="coo_matrix")
    keep = dm.row < dm.col
    keep &= dm.data < rmax
    i, j, r = dm.row[keep], dm.col[keep], dm.data[keep]
    k = np.minimum(np.floor(r * (nbins / rmax)).astype(np.int64), nbins - 1)
    assert np.array_equal(np.bincount(k, minlength=nbins), counts)
    dots = np.einsum("ij,ij->i", v[i], v[j])
    ref = np.bincount(k, weights=dots, minlength=nbins)
    assert np.allclose(sums, ref, rtol=0, atol=1e-10 * np.abs(dots).sum())
    assert vsq == pytest.approx(np.mean(np.einsum("ij,ij->i", v, v)), rel=1e-13)


def test_lees_edwards_images_by_brute_force():
    """delta != 0: every pair's shortest separation over the explicit images
    (j + (a L_x + b delta, b L_y, c L_z)); below half the shortest edge the
    minimum image is unique, so the binned counts and sums agree."""
    L = (7.0, 6.0, 5.0)
    n, delta, kappa = 700, 2.35, 0.2
    pos, v = _random(n, L, 4)
    nbins, rmax = 12, 0.45 * min(L)
    p = oracle.Params(n=n, L=L, kappa=kappa)
    sums, counts, _ = oracle.velocity_correlation(p, pos, delta, v, nbins, rmax)
    shifts = np.array([(a * L[0] + b * delta, b * L[1], c * L[2])
                       for a in range(-2, 3) for b in (-1, 0, 1) for c in (-1, 0, 1)])
    u = v.copy()
    u[:, 0] -= kappa * (pos[:, 1] - 0.5 * L[1])
    ref_c = np.zeros(nbins, dtype=np.int64)
    ref_s = np.zeros(nbins)
    for a in range(n - 1):
        d = pos[a] - (pos[a + 1:, None, :] + shifts[None, :, :])
        r = np.sqrt((d * d).sum(-1)).min(axis=1)
        m = r < rmax
        k = np.floor(r[m] * (nbins / rmax)).astype(np.int64)
        ref_c += np.bincount(k, minlength=nbins)
        ref_s += np.bincount(k, weights=u[a + 1:][m] @ u[a], minlength=nbins)
    assert np.array_equal(ref_c, counts)
    assert np.allclose(sums, ref_s, rtol=1e-12, atol=1e-12)


def test_hand_placed_pairs():
    L = (10.0, 8.0, 6.0)
    delta = 3.0
    p = oracle.Params(n=2, L=L, kappa=0.0)
    v = np.array([[1.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    # an exact bin edge: |R| = 0.5 with bins of width 0.25 is the first entry of bin 2
    pos = np.array([[1.0, 1.0, 1.0], [1.5, 1.0, 1.0]])
    sums, counts, _ = oracle.velocity_correlation(p, pos, delta, v, 4, 1.0)
    assert counts.tolist() == [0, 0, 1, 0] and sums[2] == 2.0
    # across the sheared boundary: the image of j one box down sits at
    # (x_j - delta, y_j - L_y), 0.3 behind and 0.2 below i
    pos = np.array([[4.0, 0.1, 2.0], [4.0 + delta + 0.3, L[1] - 0.1, 2.0]])
    sums, counts, _ = oracle.velocity_correlation(p, pos, delta, v, 10, 1.0)
    r = math.sqrt(0.3 ** 2 + 0.2 ** 2)
    assert counts.sum() == 1 and counts[int(r * 10)] == 1
    # the unsheared image (x_j, y_j - L_y) would be delta + 0.3 away: nothing in range
    pos[1, 0] = 4.0 + 0.3
    _, counts, _ = oracle.velocity_correlation(p, pos, delta, v, 10, 1.0)
    assert counts.sum() == 0
    # one particle: no pairs
    p1 = oracle.Params(n=1, L=L, kappa=0.0)
    sums, counts, vsq = oracle.velocity_correlation(p1, pos[:1], delta, v[:1], 3, 1.0)
    assert counts.sum() == 0 and vsq == 1.0
