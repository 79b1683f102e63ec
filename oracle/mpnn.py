"""FP64 oracle of the message-passing warm start for the velocity solve.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).  The paper has no
learned component; this is the reference for the GPU network that guesses
v = A^-1 b before CG (Eq. algebra of §Method), written plainly in numpy with a
hand-derived backward pass.  Pins: finite differences of the loss
(tests/test_oracle_mpnn.py) and the symmetries the network is built to have
(oddness in b, scale equivariance, permutation equivariance).

The network acts on each Cartesian component separately with shared weights
(the matrix of Eq. algebra acts on the three components alike).  For node i
and component c (row r = 3 i + c):

    s      = sqrt(sum b^2 / (3 n))                     (scale of the system)
    x0_r   = [b_ic / A_ii, vprev_ic, b_ic] / s          (3 input features)
    (M u)_i = sum_j alpha w_ij / A_ii u_j                (Jacobi-scaled coupling)
    a0_r   = (M x0)_r                                   (message pass 1)
    h1     = tanh([x0, a0] W1)     W1: 6 x 64
    h2     = tanh(h1 W2)           W2: 64 x 64
    y_r    = h2 W3                 W3: 64 x 4
    a1_r   = (M y)_r                                    (message pass 2)
    out_r  = [y, a1, x0]_r . o     o: 11
    guess_ic = s out_r
    loss   = (1 / 3n) sum_r (out_r - vstar_ic / s)^2

No biases and an odd activation make the guess odd in (b, vprev); dividing by
s makes it scale-equivariant.
"""
from __future__ import annotations

import dataclasses

import numpy as np

HIDDEN = 64
N_IN = 3
N_MSG = 4
N_OUT_FEAT = N_MSG + N_MSG + N_IN   # 11


@dataclasses.dataclass
class Weights:
    W1: np.ndarray   # [6, 64]
    W2: np.ndarray   # [64, 64]
    W3: np.ndarray   # [64, 4]
    o: np.ndarray    # [11]

    def copy(self) -> "Weights":
        return Weights(self.W1.copy(), self.W2.copy(), self.W3.copy(), self.o.copy())

    def flat(self) -> np.ndarray:
        return np.concatenate([self.W1.ravel(), self.W2.ravel(), self.W3.ravel(), self.o.ravel()])

    @staticmethod
    def unflat(v) -> "Weights":
        v = np.asarray(v, dtype=np.float64)
        a = 2 * N_IN * HIDDEN
        b = a + HIDDEN * HIDDEN
        c = b + HIDDEN * N_MSG
        return Weights(v[:a].reshape(2 * N_IN, HIDDEN).copy(), v[a:b].reshape(HIDDEN, HIDDEN).copy(),
                       v[b:c].reshape(HIDDEN, N_MSG).copy(), v[c:c + N_OUT_FEAT].copy())


def init_weights(seed: int) -> Weights:
    """Scaled normal hidden weights; the readout starts as the previous-velocity guess."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.normal(0.0, 1.0 / np.sqrt(2 * N_IN), (2 * N_IN, HIDDEN))
    W2 = rng.normal(0.0, 1.0 / np.sqrt(HIDDEN), (HIDDEN, HIDDEN))
    W3 = rng.normal(0.0, 1.0 / np.sqrt(HIDDEN), (HIDDEN, N_MSG))
    o = np.zeros(N_OUT_FEAT)
    o[2 * N_MSG + 1] = 1.0
    return Weights(W1, W2, W3, o)


def coupling(n: int, alpha: float, pairs, w, diag):
    """M as a function u [n, k] -> [n, k], (M u)_i = sum_j alpha w_ij / A_ii u_j, and its transpose."""
    pairs = np.asarray(pairs)
    i, j = pairs[:, 0], pairs[:, 1]
    c = alpha * np.asarray(w)

    def M(u):
        out = np.zeros_like(u)
        np.add.at(out, i, c[:, None] * u[j])
        np.add.at(out, j, c[:, None] * u[i])
        return out / diag[:, None]

    def MT(g):
        gs = g / diag[:, None]
        out = np.zeros_like(g)
        np.add.at(out, j, c[:, None] * gs[i])
        np.add.at(out, i, c[:, None] * gs[j])
        return out

    return M, MT


def _rows_to_nodes(x, n):
    """[3n, k] (row 3i + c) -> [n, 3k] so that M acts per node on all components."""
    return x.reshape(n, -1)


def forward(Wt: Weights, n: int, alpha: float, pairs, w, diag, b, vprev):
    """Returns (guess [n, 3], cache for backward)."""
    b = np.asarray(b, dtype=np.float64)
    vprev = np.asarray(vprev, dtype=np.float64)
    s = np.sqrt((b ** 2).sum() / (3 * n))
    if s == 0.0:
        s = 1.0
    M, MT = coupling(n, alpha, pairs, w, diag)
    x0 = np.stack([b / diag[:, None], vprev, b], axis=2).reshape(3 * n, N_IN) / s
    a0 = M(_rows_to_nodes(x0, n)).reshape(3 * n, N_IN)
    inp = np.concatenate([x0, a0], axis=1)
    h1 = np.tanh(inp @ Wt.W1)
    h2 = np.tanh(h1 @ Wt.W2)
    y = h2 @ Wt.W3
    a1 = M(_rows_to_nodes(y, n)).reshape(3 * n, N_MSG)
    feat = np.concatenate([y, a1, x0], axis=1)
    out = feat @ Wt.o
    cache = dict(s=s, x0=x0, inp=inp, h1=h1, h2=h2, y=y, a1=a1, feat=feat, out=out, MT=MT, n=n)
    return (s * out).reshape(n, 3), cache


def loss_and_grad(Wt: Weights, n: int, alpha: float, pairs, w, diag, b, vprev, vstar):
    """Loss and its gradient with respect to every weight (hand-derived backward)."""
    _, c = forward(Wt, n, alpha, pairs, w, diag, b, vprev)
    target = np.asarray(vstar, dtype=np.float64).reshape(3 * n) / c["s"]
    e = c["out"] - target
    loss = (e ** 2).sum() / (3 * n)
    dout = 2.0 * e / (3 * n)                          # [3n]
    do = c["feat"].T @ dout                            # [11]
    dy = np.outer(dout, Wt.o[:N_MSG])                  # direct path
    da1 = np.outer(dout, Wt.o[N_MSG:2 * N_MSG])
    dy = dy + c["MT"](_rows_to_nodes(da1, n)).reshape(3 * n, N_MSG)
    dW3 = c["h2"].T @ dy
    dh2 = dy @ Wt.W3.T
    dp2 = dh2 * (1.0 - c["h2"] ** 2)
    dW2 = c["h1"].T @ dp2
    dh1 = dp2 @ Wt.W2.T
    dp1 = dh1 * (1.0 - c["h1"] ** 2)
    dW1 = c["inp"].T @ dp1
    return loss, Weights(dW1, dW2, dW3, do)


def adam_step(Wt: Weights, grad: Weights, m: np.ndarray, v: np.ndarray, t: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """Adam (Kingma & Ba 2015) on the flattened weights; returns new (weights, m, v)."""
    g = grad.flat()
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    x = Wt.flat() - lr * mh / (np.sqrt(vh) + eps)
    return Weights.unflat(x), m, v
