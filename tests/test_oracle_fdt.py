"""Pins of the oracle's A^(1/2) g (FDT-consistent noise, a ranked next row)
against exact linear algebra: the eigen-decomposition of small systems
(numpy.linalg.eigh), eigenvectors mapped to sqrt(lambda) times themselves,
the identity for an uncoupled system, the square of the operator against A,
and the interpolant's own bound from the tail of a high-degree expansion."""
import numpy as np
import pytest

import oracle


def _system(n, seed, alpha=4.0):
    L = (n / 3.0) ** (1.0 / 3.0)
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * L
    p = oracle.Params(n=n, L=(L, L, L), kappa=0.0, alpha=alpha, seed=seed)
    pairs = oracle.neighbors(p, pos, 0.0)
    return oracle.assemble(p, pos, pairs, np.zeros((n, 3)), 0.0)


def _tail_bound(lmax, degree):
    """Twice the sum of the Chebyshev coefficients beyond the degree (from an
    8x higher-degree interpolant): a bound of max |sqrt - p| on [1, lmax]."""
    c = oracle.chebyshev_sqrt_coeffs(1.0, lmax, 8 * degree)
    return 2.0 * np.abs(c[degree + 1:]).sum()


@pytest.mark.parametrize("degree", [8, 24])
def test_matches_the_eigen_decomposition(degree):
    sys = _system(120, 1)
    A = sys.dense()
    lam, V = np.linalg.eigh(A)
    assert lam.min() > 1.0 - 1e-12 and lam.max() <= oracle.gershgorin_max(sys) + 1e-12
    g = np.random.default_rng(2).standard_normal((sys.n, 3))
    xi, lmax = oracle.sqrt_apply(sys, g, degree)
    exact = V @ (np.sqrt(lam)[:, None] * (V.T @ g))
    err = np.linalg.norm(xi - exact, axis=0) / np.linalg.norm(g, axis=0)
    assert np.all(err <= 1.01 * _tail_bound(lmax, degree) + 1e-13), (err, _tail_bound(lmax, degree))


def test_eigenvectors_scale_by_the_root():
    sys = _system(80, 3)
    lam, V = np.linalg.eigh(sys.dense())
    g = np.stack([V[:, 0], V[:, -1], V[:, 40]], axis=1)
    xi, lmax = oracle.sqrt_apply(sys, g, 40)
    for c, k in enumerate((0, -1, 40)):
        assert np.allclose(xi[:, c], np.sqrt(lam[k]) * V[:, k], atol=2 * _tail_bound(lmax, 40) + 1e-12)


def test_uncoupled_system_is_the_identity():
    sys = _system(60, 4, alpha=0.0)
    g = np.random.default_rng(5).standard_normal((sys.n, 3))
    xi, lmax = oracle.sqrt_apply(sys, g, 16)
    assert lmax == 1.0 and np.array_equal(xi, g)


def test_square_is_A():
    sys = _system(150, 6)
    g = np.random.default_rng(7).standard_normal((sys.n, 3))
    xi, lmax = oracle.sqrt_apply(sys, g, 48)
    xi2, _ = oracle.sqrt_apply(sys, xi, 48)
    Ag = sys.matvec(g)
    tb = _tail_bound(lmax, 48)
    # |p(A)^2 - A| <= 2 sqrt(lmax) tb + tb^2 on the spectrum
    assert np.linalg.norm(xi2 - Ag) <= (2 * np.sqrt(lmax) * tb + tb * tb) * np.linalg.norm(g) + 1e-10
