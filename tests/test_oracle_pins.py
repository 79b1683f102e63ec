"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form (the two-particle time delay of Eq. timedelay, the exact Couette flow of
a lattice, Bragg peaks of a sheared lattice, the Einstein relation), an
invariant of Eq. algebra (symmetry, zero row sums, positive definiteness,
cancelling pair terms), brute force written independently with explicit
periodic images, or a library routine (numpy's Philox4x64-10 and
numpy.linalg.solve, scipy's normal distribution).
"""
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle
import synth

LAMBDA2 = 1.0 / (2.0 * math.log(20.0))
LAM = math.sqrt(LAMBDA2)


def _images(p, delta):
    """All lattice translations of a sheared periodic box within one box in every direction."""
    out = []
    for m in (-1, 0, 1):
        for a in (-2, -1, 0, 1, 2):
            for c in (-1, 0, 1):
                out.append((a * p.L[0] + m * delta, m * p.L[1], c * p.L[2], m))
    return np.array(out)


def _explicit_pairs(p, pos, delta):
    """Brute force over explicit Lees-Edwards images: (i, j, d_min, m) for |d| < r_c."""
    imgs = _images(p, delta)
    res = {}
    for i in range(p.n):
        d = pos[i][None, None, :] - (pos[None, :, :] + imgs[:, None, :3])  # [img, j, 3]
        r2 = (d ** 2).sum(-1)
        k = r2.argmin(0)
        r2min = r2[k, np.arange(p.n)]
        for j in np.nonzero(r2min < p.rc ** 2)[0]:
            if j > i:
                res[(i, int(j))] = (d[k[j], j], imgs[k[j], 3])
    return res


# ---------------------------------------------------------------- generator


def test_philox_matches_numpy_reference_generator():
    """or_philox4x64_10 equals numpy's independent Philox4x64-10 (which
    increments its counter before each block, hence ctr - 1)."""
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(20):
        key = rng.integers(0, 2 ** 64, size=2, dtype=np.uint64)
        ctr = rng.integers(1, 2 ** 64, size=4, dtype=np.uint64)
        ref = np.random.Philox(key=key, counter=np.array([ctr[0] - np.uint64(1), ctr[1], ctr[2], ctr[3]],
                                                          dtype=np.uint64)).random_raw(4)
        assert np.array_equal(oracle.philox4x64_10(ctr, key), np.asarray(ref, dtype=np.uint64))
    # carry across the low word
    key = np.array([7, 9], dtype=np.uint64)
    ref = np.random.Philox(key=key, counter=np.array([2 ** 64 - 1, 4, 0, 0], dtype=np.uint64)).random_raw(4)
    assert np.array_equal(oracle.philox4x64_10(np.array([0, 5, 0, 0], dtype=np.uint64), key),
                          np.asarray(ref, dtype=np.uint64))


def test_noise_is_standard_normal_and_counter_keyed():
    ids = np.arange(40000)
    xi = oracle.noise(123, 7, ids)
    for a in range(3):
        ks = stats.kstest(xi[:, a], "norm")
        assert ks.pvalue > 1e-3, (a, ks)
    c = np.corrcoef(xi.T)
    assert np.abs(c - np.eye(3)).max() < 0.03
    # a different step, seed or id gives independent draws; the same ones repeat exactly
    assert np.array_equal(xi[5:9], oracle.noise(123, 7, ids[5:9]))
    other = oracle.noise(123, 8, ids)
    assert abs(np.corrcoef(xi[:, 0], other[:, 0])[0, 1]) < 0.03
    other = oracle.noise(124, 7, ids)
    assert abs(np.corrcoef(xi[:, 0], other[:, 0])[0, 1]) < 0.03


# ------------------------------------------------------ Lees-Edwards geometry


def test_min_image_matches_explicit_sheared_images():
    rng = np.random.Generator(np.random.PCG64(11))
    p = oracle.Params(n=2, L=(5.0, 4.0, 3.5), kappa=1.0)
    imgs = _images(p, 0.0)
    for _ in range(3000):
        delta = rng.uniform(0, p.L[0])
        imgs = _images(p, delta)
        ri = rng.uniform(0, 1, 3) * p.L
        rj = rng.uniform(0, 1, 3) * p.L
        d, n = oracle.min_image(p, delta, ri, rj)
        # d is one of the image separations, with the vertical image index n
        cand = ri[None, :] - (rj[None, :] + imgs[:, :3])
        k = np.argmin(((cand - d) ** 2).sum(-1))
        assert np.allclose(cand[k], d, atol=1e-12) and imgs[k, 3] == n
        assert abs(d[1]) <= p.L[1] / 2 + 1e-12 and abs(d[0]) <= p.L[0] / 2 + 1e-12
        assert abs(d[2]) <= p.L[2] / 2 + 1e-12
        # and it is the nearest image whenever some image is within r_c
        r2 = (cand ** 2).sum(-1)
        if r2.min() < 1.0:
            assert abs((d ** 2).sum() - r2.min()) < 1e-12


@pytest.mark.parametrize("n,delta", [(60, 0.0), (150, 1.37), (300, 2.9)])
def test_neighbors_brute_equals_explicit_images(n, delta):
    L = synth.box_length(n)
    p = oracle.Params(n=n, L=(L, L, L), kappa=1.0)
    pos = synth.uniform_positions(n, p.L, 100 + n)
    got = {tuple(x) for x in oracle.neighbors(p, pos, delta % L, method="brute")}
    ref = _explicit_pairs(p, pos, delta % L)
    assert got == set(ref.keys())


@pytest.mark.parametrize("n,seed", [(3000, 1), (6000, 2)])
def test_neighbors_cell_list_equals_brute_force(n, seed):
    L = synth.box_length(n)
    p = oracle.Params(n=n, L=(L, 0.93 * L, 1.07 * L), kappa=1.0)
    pos = synth.uniform_positions(n, p.L, seed)
    # put particles on cell faces and on the box faces too
    pos[:50, 1] = 0.0
    pos[50:100, 1] = np.nextafter(p.L[1], 0)
    pos[100:150, 0] = np.floor(pos[100:150, 0])
    for delta in (0.0, 0.5 * p.L[0], 0.123456789, p.L[0] - 1e-9):
        a = oracle.neighbors(p, pos, delta, method="brute")
        b = oracle.neighbors(p, pos, delta, method="cells")
        assert np.array_equal(a, b)


# ------------------------------------------------------------ Eq. algebra


def _random_system(n, seed, delta=0.7, kappa_tau=0.5, **kw):
    L = synth.box_length(n)
    p = oracle.Params(n=n, L=(L, L, L), kappa=oracle.kappa_from_kappa_tau(kappa_tau), seed=seed, **kw)
    pos = synth.uniform_positions(n, p.L, seed)
    pairs = oracle.neighbors(p, pos, delta)
    xi = oracle.noise(seed, 0, np.arange(n))
    return p, pos, oracle.assemble(p, pos, pairs, xi, delta), xi


@pytest.mark.parametrize("n,seed", [(24, 1), (48, 2), (64, 3), (500, 4)])
def test_matrix_symmetric_zero_row_sums_and_spd(n, seed):
    p, pos, sys, _ = _random_system(n, seed)
    A = sys.dense()
    assert np.array_equal(A, A.T)
    assert np.abs((A - np.eye(n)).sum(1)).max() < 1e-12
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= 1.0 - 1e-12          # I + alpha L_w with L_w a graph Laplacian
    ev_lap = np.linalg.eigvalsh(A - np.eye(n))
    assert ev_lap.min() > -1e-12            # positive semidefinite, and
    assert abs(ev_lap.min()) < 1e-10        # singular (the constant vector)


@pytest.mark.parametrize("n,delta", [(64, 0.0), (400, 2.1)])
def test_weights_are_the_truncated_gaussian_of_explicit_distances(n, delta):
    L = synth.box_length(n)
    p = oracle.Params(n=n, L=(L, L, L), kappa=2.0)
    pos = synth.uniform_positions(n, p.L, 3 + n)
    pairs = oracle.neighbors(p, pos, delta)
    sys = oracle.assemble(p, pos, pairs, None, delta)
    ref = _explicit_pairs(p, pos, delta)
    for k, (i, j) in enumerate(pairs):
        d, m = ref[(int(i), int(j))]
        assert abs(sys.w[k] - math.exp(-(d ** 2).sum() / (2 * LAMBDA2))) < 1e-13 * sys.w[k]
    assert sys.w.min() > 0.05 - 1e-15       # "truncate the weights below 5 %"
    # and the cut sits at r_c: the weakest kept pairs are just above 5 %
    assert sys.w.min() < 0.06


def test_excluded_volume_force_is_minus_gradient_of_gaussian_core():
    """Eq. exvol is the force of U = eps (v/lambda^3) kT exp(-R^2/2 lambda^2), v/lambda^3 = 0.1:
    two particles, no noise, no friction, no shear; v = F/zeta must equal -dU/dR (central differences)."""
    p = oracle.Params(n=2, L=(6.0, 6.0, 6.0), kappa=0.0, alpha=0.0, eps=1.0, kT=1.3, zeta=0.7)
    rng = np.random.Generator(np.random.PCG64(2))
    for _ in range(20):
        ri = rng.uniform(2, 4, 3)
        rj = ri + rng.uniform(-0.55, 0.55, 3)
        pos = np.array([ri, rj])
        pairs = oracle.neighbors(p, pos, 0.0)
        sys = oracle.assemble(p, pos, pairs, None, 0.0)
        v, _, _ = oracle.pcg(sys, 1e-14)

        def U(x):
            return 1.0 * 0.1 * p.kT * math.exp(-((x - rj) ** 2).sum() / (2 * LAMBDA2))
        h = 1e-6
        grad = np.array([(U(ri + h * e) - U(ri - h * e)) / (2 * h) for e in np.eye(3)])
        assert np.allclose(v[0] * p.zeta, -grad, rtol=1e-7, atol=1e-9)
        assert np.allclose(v[1], -v[0], atol=1e-14)


@pytest.mark.parametrize("n,seed,delta", [(64, 5, 0.0), (1000, 6, 3.3), (4096, 7, 9.9)])
def test_momentum_bookkeeping(n, seed, delta):
    """Pair terms cancel in the total: sum_i v_i = sum_i (noise_i + shear_i)/zeta."""
    p, pos, sys, xi = _random_system(n, seed, delta=delta % synth.box_length(n))
    v, it, res = oracle.pcg(sys, 1e-13)
    amp = math.sqrt(2 * p.zeta * p.kT / p.dt)
    expect = (amp * xi).sum(0) / p.zeta
    expect[0] += p.kappa * (pos[:, 1] - p.L[1] / 2).sum()
    scale = np.abs(v).sum()
    assert np.allclose(v.sum(0), expect, atol=1e-11 * scale)
    assert np.allclose(sys.b.sum(0), expect, atol=1e-12 * np.abs(sys.b).sum())


@pytest.mark.parametrize("n,seed", [(24, 8), (40, 9), (64, 10)])
def test_dense_cholesky_pcg_and_library_solve_agree(n, seed):
    p, pos, sys, _ = _random_system(n, seed)
    x_chol = oracle.dense_solve(sys)
    x_lib = np.linalg.solve(sys.dense(), sys.b)
    x_cg, it, res = oracle.pcg(sys, 1e-14)
    scale = np.abs(x_lib).max()
    assert np.abs(x_chol - x_lib).max() <= 1e-13 * scale
    assert np.abs(x_cg - x_lib).max() <= 1e-12 * scale
    assert res <= 1e-14


def test_pcg_error_decreases_monotonically_in_energy_norm():
    p, pos, sys, _ = _random_system(64, 12)
    A = sys.dense()
    x_star = np.linalg.solve(A, sys.b)
    errs = []
    for k in range(1, 30):
        x, it, _ = oracle.pcg(sys, 0.0, max_iter=k)
        e = x - x_star
        errs.append(float(np.einsum("ia,ij,ja->", e, A, e)))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:]))


# ----------------------------------------------------------- closed forms


def _two_particle_crossing_time(dt, kappa=10.0, alpha=4.0, x0=-1.5, x1=1.5):
    """Run the oracle's time step on two particles a height lambda apart."""
    L = 12.0
    p = oracle.Params(n=2, L=(L, L, L), kappa=kappa, alpha=alpha, eps=0.0, kT=0.0, dt=dt)
    y = LAM
    pos = np.array([[6.0 + x0 / 2, 6.0 + y / 2, 6.0], [6.0 - x0 / 2, 6.0 - y / 2, 6.0]])
    delta, t, sep = 0.0, 0.0, x0
    while sep < x1:
        r = oracle.step(p, pos, delta, 0)
        pos, delta = r.pos, r.delta
        d, _ = oracle.min_image(p, delta, pos[0], pos[1])
        assert abs(d[1] - y) < 1e-12 and abs(r.v[0, 1]) < 1e-14
        new = d[0]
        if new >= x1:
            t += dt * (x1 - sep) / (new - sep)
        else:
            t += dt
        sep = new
    return t


def test_two_particle_time_delay_closed_form():
    """Eq. timedelay with the 5 % truncation: for |dx| < x_c = sqrt(r_c^2 - y^2) the
    separation obeys d(dx)/dt = kappa y / (1 + 2 alpha w); outside it kappa y."""
    kappa, alpha, x0, x1, y = 10.0, 4.0, -1.5, 1.5, LAM
    xc = math.sqrt(1.0 - y * y)
    erf_term = special.erf(xc / (LAM * math.sqrt(2))) - special.erf(-xc / (LAM * math.sqrt(2)))
    t_exact = ((x1 - x0) + math.sqrt(2 * math.pi) * alpha * LAM * math.exp(-y * y / (2 * LAMBDA2)) * erf_term) / (kappa * y)
    errs = []
    for dt in (4e-3, 2e-3, 1e-3):
        errs.append(abs(_two_particle_crossing_time(dt, kappa, alpha, x0, x1) - t_exact))
    # first order in time: the error shrinks with dt, and is small at the smallest dt
    assert errs[2] < errs[0]
    assert errs[2] / t_exact < 2e-3
    # the entangled crossing takes about 2.6x longer than the free one (the delay of Fig. trafficjam)
    assert t_exact / ((x1 - x0) / (kappa * y)) > 2.0


@pytest.mark.parametrize("alpha,eps,kappa", [(4.0, 1.0, 3.0), (0.5, 0.0, 1.0), (10.0, 2.0, -2.0)])
def test_lattice_moves_in_exact_couette_flow(alpha, eps, kappa):
    """A simple cubic lattice (spacing below r_c, delta = 0) without noise: all neighbour
    sums vanish by symmetry, so v = kappa (y - L_y/2) x exactly, boundary images included."""
    a, m = 0.6, 6
    p = oracle.Params(n=m ** 3, L=(a * m,) * 3, kappa=kappa, alpha=alpha, eps=eps, kT=0.0)
    pos = synth.lattice_positions(m, a, offset=(0.1, 0.2, 0.3))
    r = oracle.step(p, pos, 0.0, 0)
    expect = np.zeros_like(r.v)
    expect[:, 0] = kappa * (pos[:, 1] - p.L[1] / 2)
    assert np.abs(r.v - expect).max() < 1e-11
    assert r.system.pairs.shape[0] == p.n * 18 // 2


def test_free_diffusion_einstein_relation():
    """alpha = eps = kappa = 0: mean square displacement 6 kT t / zeta (noise of Eq. F)."""
    n, steps = 2000, 40
    L = synth.box_length(n)
    p = oracle.Params(n=n, L=(L, L, L), kappa=0.0, alpha=0.0, eps=0.0, kT=1.0, zeta=2.0, seed=77)
    pos = synth.uniform_positions(n, p.L, 3)
    disp = np.zeros((n, 3))
    delta = 0.0
    for s in range(steps):
        r = oracle.step(p, pos, delta, s)
        disp += r.v * p.dt
        pos, delta = r.pos, r.delta
    t = steps * p.dt
    msd = (disp ** 2).sum(1).mean()
    expect = 6 * p.kT * t / p.zeta
    sigma = math.sqrt(6.0) * (2 * p.kT * t / p.zeta) / math.sqrt(n)
    assert abs(msd - expect) < 4 * sigma


def test_integrate_lands_on_an_image_of_the_unwrapped_position():
    n = 500
    L = synth.box_length(n)
    p = oracle.Params(n=n, L=(L, 1.1 * L, L), kappa=5.0, dt=0.05)
    pos = synth.uniform_positions(n, p.L, 9)
    rng = np.random.Generator(np.random.PCG64(1))
    v = rng.normal(0, 20, (n, 3))
    delta = 1.7
    new, dnew = oracle.integrate(p, pos, v, delta)
    assert abs(dnew - (delta + p.kappa * p.L[1] * p.dt) % p.L[0]) < 1e-12
    assert (new >= 0).all() and (new < np.array(p.L)).all()
    imgs = _images(p, dnew)
    un = pos + v * p.dt
    for i in range(n):
        cand = un[i][None, :] - (new[i][None, :] + imgs[:, :3])
        assert ((cand ** 2).sum(-1)).min() < 1e-20


# -------------------------------------------------------- structure factor


def test_structure_factor_bragg_peaks_of_sheared_lattice():
    m, a = 5, 0.8
    Lb = m * a
    p = oracle.Params(n=m ** 3, L=(Lb, Lb, Lb), kappa=1.0)
    base = synth.lattice_positions(m, a, offset=(0.05, 0.1, 0.2))
    for gamma in (0.0, 0.37, 1.9):
        pos = base.copy()
        pos[:, 0] = (pos[:, 0] + gamma * pos[:, 1]) % Lb
        delta = (gamma * Lb) % Lb
        ks = np.array([[m, 0], [0, m], [m, m], [2 * m, -m], [1, 0], [0, 2], [3, 1], [m, 1]])
        S, qx, qy = oracle.structure_factor(p, pos, delta, ks)
        assert np.allclose(S[:4], p.n, rtol=1e-10)
        assert np.all(S[4:] < 1e-20)
        # the sheared reciprocal lattice: q . (delta, L_y) is a multiple of 2 pi
        assert np.allclose((qx * delta + qy * Lb) / (2 * np.pi), np.round((qx * delta + qy * Lb) / (2 * np.pi)))


def test_structure_factor_of_ideal_gas_is_one():
    n = 3000
    L = synth.box_length(n)
    p = oracle.Params(n=n, L=(L, L, L), kappa=1.0)
    pos = synth.uniform_positions(n, p.L, 21)
    ks = np.array([(kx, ky) for kx in range(-10, 11) for ky in range(1, 11)])
    S, _, _ = oracle.structure_factor(p, pos, 1.234, ks)
    assert abs(S.mean() - 1.0) < 4.0 / math.sqrt(len(ks))


# ------------------------------------------------------------------ stress


def test_stress_of_lattice_in_couette_flow_is_the_friction_viscosity():
    """Friction only (eps = 0), exact Couette flow of a lattice: every pair carries
    f_x = -zeta alpha w kappa y_ij, so sigma_xy = kappa zeta alpha sum_{i<j} w y_ij^2 / V,
    summed here over the lattice's neighbour shell by hand."""
    a, m, alpha, zeta, kappa = 0.6, 6, 4.0, 1.5, 2.0
    p = oracle.Params(n=m ** 3, L=(a * m,) * 3, kappa=kappa, alpha=alpha, eps=0.0, kT=0.0, zeta=zeta)
    pos = synth.lattice_positions(m, a)
    r = oracle.step(p, pos, 0.0, 0)
    s = oracle.stress_xy(p, pos, 0.0, r.system.pairs, r.v)
    # per particle: 2 neighbours at (0, +-a, 0) and 8 at (+-a, +-a, 0) / (0, +-a, +-a) carry y^2 = a^2
    shell = 2 * math.exp(-a * a / (2 * LAMBDA2)) + 8 * math.exp(-2 * a * a / (2 * LAMBDA2))
    expect = kappa * zeta * alpha * (p.n * shell / 2) * a * a / (p.L[0] ** 3)
    assert s > 0 and abs(s - expect) < 1e-10 * expect


def test_excluded_volume_stress_is_affine_strain_derivative_of_energy():
    """For the conservative part, -(1/V) sum y_ij f_ij,x equals (1/V) dU/dgamma under the
    affine shear x -> x + gamma y of every pair separation (central differences of the
    Gaussian-core energy), with zero velocities and zero shear so that friction vanishes."""
    n = 300
    L = synth.box_length(n)
    p = oracle.Params(n=n, L=(L, L, L), kappa=0.0, alpha=4.0, eps=1.0, kT=1.0)
    pos = synth.uniform_positions(n, p.L, 31)
    delta = 0.9
    pairs = oracle.neighbors(p, pos, delta)
    d = np.array([oracle.min_image(p, delta, pos[i], pos[j])[0] for i, j in pairs])

    def energy(g):
        dd = d.copy()
        dd[:, 0] += g * dd[:, 1]
        return (0.1 * p.kT * np.exp(-(dd ** 2).sum(1) / (2 * LAMBDA2))).sum()
    h = 1e-6
    expect = (energy(h) - energy(-h)) / (2 * h) / (L ** 3)
    got = oracle.stress_xy(p, pos, delta, pairs, np.zeros((n, 3)))
    assert abs(got - expect) < 1e-7 * max(abs(expect), 1e-3)
