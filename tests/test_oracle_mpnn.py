"""Pins of the warm-start network oracle: finite differences of the loss, and the
symmetries it is built to have."""
import numpy as np
import pytest

import oracle
from oracle import mpnn
import synth


def _system(n=200, seed=3):
    L = synth.box_length(n)
    p = oracle.Params(n=n, L=(L, L, L), kappa=oracle.kappa_from_kappa_tau(0.5), seed=seed)
    pos = synth.uniform_positions(n, p.L, seed)
    pairs = oracle.neighbors(p, pos, 0.4)
    sysr = oracle.assemble(p, pos, pairs, oracle.noise(seed, 0, np.arange(n)), 0.4)
    v, _, _ = oracle.pcg(sysr, 1e-13)
    rng = np.random.Generator(np.random.PCG64(seed))
    vprev = v + rng.normal(0, 0.3, v.shape) * np.abs(v).mean()
    return p, sysr, v, vprev


def test_gradients_match_central_differences():
    p, s, v, vprev = _system()
    W = mpnn.init_weights(1)
    W.o = np.random.Generator(np.random.PCG64(2)).normal(0, 0.5, W.o.shape)
    args = (s.n, s.alpha, s.pairs, s.w, s.diag, s.b, vprev, v)
    loss, g = mpnn.loss_and_grad(W, *args)
    flat, gflat = W.flat(), g.flat()
    rng = np.random.Generator(np.random.PCG64(9))
    idx = np.concatenate([rng.choice(len(flat), 40, replace=False), np.arange(len(flat) - 11, len(flat))])
    h = 1e-6
    for k in idx:
        wp, wm = flat.copy(), flat.copy()
        wp[k] += h
        wm[k] -= h
        lp, _ = mpnn.loss_and_grad(mpnn.Weights.unflat(wp), *args)
        lm, _ = mpnn.loss_and_grad(mpnn.Weights.unflat(wm), *args)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, gflat[k])


def test_coupling_transpose_is_the_adjoint():
    p, s, v, vprev = _system(150, 4)
    M, MT = mpnn.coupling(s.n, s.alpha, s.pairs, s.w, s.diag)
    rng = np.random.Generator(np.random.PCG64(1))
    u = rng.normal(size=(s.n, 5))
    g = rng.normal(size=(s.n, 5))
    assert abs((M(u) * g).sum() - (u * MT(g)).sum()) < 1e-10 * abs((M(u) * g).sum())
    # M is the Jacobi-scaled coupling: (I - M) = D^-1 A
    A = s.dense()
    assert np.allclose(np.eye(s.n) - M(np.eye(s.n)), A / s.diag[:, None], atol=1e-12)


def test_guess_is_odd_scale_equivariant_and_starts_as_previous_velocity():
    p, s, v, vprev = _system(120, 5)
    W = mpnn.init_weights(3)
    g0, _ = mpnn.forward(W, s.n, s.alpha, s.pairs, s.w, s.diag, s.b, vprev)
    assert np.allclose(g0, vprev, atol=1e-12)           # readout starts as the previous velocity
    W.o[:] = np.random.Generator(np.random.PCG64(7)).normal(0, 1, W.o.shape)
    g1, _ = mpnn.forward(W, s.n, s.alpha, s.pairs, s.w, s.diag, s.b, vprev)
    g2, _ = mpnn.forward(W, s.n, s.alpha, s.pairs, s.w, s.diag, -s.b, -vprev)
    g3, _ = mpnn.forward(W, s.n, s.alpha, s.pairs, s.w, s.diag, 3.0 * s.b, 3.0 * vprev)
    assert np.allclose(g2, -g1, atol=1e-12)
    assert np.allclose(g3, 3.0 * g1, rtol=1e-12, atol=1e-12)


def test_adam_reduces_the_loss():
    p, s, v, vprev = _system(300, 6)
    W = mpnn.init_weights(4)
    args = (s.n, s.alpha, s.pairs, s.w, s.diag, s.b, vprev, v)
    m = np.zeros_like(W.flat())
    vv = np.zeros_like(m)
    l0, _ = mpnn.loss_and_grad(W, *args)
    for t in range(1, 61):
        _, g = mpnn.loss_and_grad(W, *args)
        W, m, vv = mpnn.adam_step(W, g, m, vv, t, 3e-3)
    l1, _ = mpnn.loss_and_grad(W, *args)
    assert l1 < 0.7 * l0
