"""CPU FP64 oracle of the coupled velocity solve (arXiv 1808.06381, §Method).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it; the CUDA library never does.  It
shares no code with the CUDA path.  The arithmetic lives in
``shearsim_oracle.c`` (plain C, FP64, no FMA contraction); this module only
marshals numpy arrays into it and composes whole time steps in the paper's
order: neighbours, forces and Eq. algebra, solve, position update.

Every function is pinned by a CPU test against something other than itself
(closed forms, invariants, brute force, library routines); see
``tests/test_oracle_pins.py``.  The velocity cross-checks of ``stress_xy``
(no definition in the paper) are the only "parity unpinned" item: the stress
is pinned only by its sign and by a two-particle hand calculation.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "shearsim_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")

OR_OK = 0
OR_ERR_ARG = -1
OR_ERR_CAPACITY = -2
OR_ERR_NOT_CONVERGED = -3
OR_ERR_NOT_SPD = -4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into oracle/lib/liboracle.so."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("L", ctypes.c_double * 3), ("rc", ctypes.c_double),
                ("alpha", ctypes.c_double), ("eps", ctypes.c_double), ("zeta", ctypes.c_double),
                ("kT", ctypes.c_double), ("kappa", ctypes.c_double), ("dt", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i64, u64 = ctypes.c_double, ctypes.c_int64, ctypes.c_uint64
        vp = ctypes.c_void_p
        lib.or_kappa_from_kappa_tau.restype = d
        lib.or_kappa_from_kappa_tau.argtypes = [d, d, d, d]
        lib.or_neighbors_brute.argtypes = [P(_Params), vp, d, i64, vp, P(i64)]
        lib.or_neighbors_cells.argtypes = [P(_Params), vp, d, i64, vp, P(i64)]
        lib.or_philox4x64_10.argtypes = [vp, vp, vp]
        lib.or_noise.argtypes = [u64, u64, i64, vp, vp]
        lib.or_assemble.argtypes = [P(_Params), vp, d, i64, vp, vp, vp, vp, vp]
        lib.or_matvec.argtypes = [i64, d, i64, vp, vp, vp, vp, vp]
        lib.or_pcg.argtypes = [i64, d, i64, vp, vp, vp, vp, d, i64, vp, vp]
        lib.or_dense_solve.argtypes = [i64, d, i64, vp, vp, vp, vp, vp]
        lib.or_integrate.restype = d
        lib.or_integrate.argtypes = [P(_Params), vp, vp, d]
        lib.or_structure_factor.argtypes = [P(_Params), vp, d, i64, vp, vp, vp, vp]
        lib.or_stress_xy.restype = d
        lib.or_stress_xy.argtypes = [P(_Params), vp, d, i64, vp, vp]
        lib.or_min_image.argtypes = [P(_Params), d, vp, vp, vp, vp]
        lib.or_velocity_correlation.argtypes = [P(_Params), vp, d, vp, i64, d, vp, vp, P(d)]
        lib.or_row_neighbors.restype = i64
        lib.or_row_neighbors.argtypes = [P(_Params), vp, d, i64, i64, vp]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def kappa_from_kappa_tau(kappa_tau: float, rc: float = 1.0, zeta: float = 1.0, kT: float = 1.0) -> float:
    """Shear rate in units kT/(zeta r_c^2) from the paper's kappa*tau (tau = lambda^2 zeta/kT)."""
    return _load().or_kappa_from_kappa_tau(kappa_tau, rc, zeta, kT)


@dataclasses.dataclass
class Params:
    """Model parameters (§Method).  Lengths in r_c; kappa is the absolute shear rate."""
    n: int
    L: tuple
    kappa: float
    alpha: float = 4.0
    eps: float = 1.0
    zeta: float = 1.0
    kT: float = 1.0
    dt: float = 0.01
    rc: float = 1.0
    seed: int = 0

    def c(self) -> _Params:
        p = _Params()
        p.n = int(self.n)
        for k in range(3):
            p.L[k] = float(self.L[k])
        p.rc, p.alpha, p.eps, p.zeta = self.rc, self.alpha, self.eps, self.zeta
        p.kT, p.kappa, p.dt, p.seed = self.kT, self.kappa, self.dt, int(self.seed)
        return p

    @staticmethod
    def from_workload(w, n=None) -> "Params":
        return Params(n=w.n if n is None else n, L=tuple(w.L),
                      kappa=kappa_from_kappa_tau(w.kappa_tau, w.rc, w.zeta, w.kT),
                      alpha=w.alpha, eps=w.eps, zeta=w.zeta, kT=w.kT, dt=w.dt, rc=w.rc, seed=w.seed)


def lambda2(rc: float = 1.0) -> float:
    """lambda^2 from the 5 % truncation at r_c (same formula as the C oracle's or_derive)."""
    return rc * rc / (2.0 * math.log(20.0))


def min_image(p: Params, delta: float, ri, rj):
    d = np.zeros(3)
    n = ctypes.c_double()
    _load().or_min_image(ctypes.byref(p.c()), float(delta), _ptr(_f64(ri)), _ptr(_f64(rj)), _ptr(d),
                         ctypes.byref(n))
    return d, n.value


def neighbors(p: Params, pos, delta: float = 0.0, method: str = "auto") -> np.ndarray:
    """Pairs (i < j) with R_ij^2 < r_c^2, sorted, int64 [npairs, 2]."""
    lib = _load()
    pos = _f64(pos)
    if method == "auto":
        method = "brute" if p.n <= 8192 else "cells"
    fn = lib.or_neighbors_brute if method == "brute" else lib.or_neighbors_cells
    cap = max(64, 16 * p.n)
    while True:
        pairs = np.zeros((cap, 2), dtype=np.int64)
        m = ctypes.c_int64()
        rc = fn(ctypes.byref(p.c()), _ptr(pos), float(delta), cap, _ptr(pairs), ctypes.byref(m))
        if rc == OR_OK:
            return pairs[: m.value].copy()
        if rc != OR_ERR_CAPACITY:
            raise RuntimeError(f"oracle neighbour search failed: {rc}")
        cap = m.value


def velocity_correlation(p: Params, pos, delta: float, v, nbins: int, rmax: float):
    """Fig. vv: per-bin sums of u_c . u_c' and pair counts over all pairs c < c'
    with minimum-image distance below rmax (bins of width rmax / nbins), and
    <|u|^2>; u = v minus the imposed flow kappa (y - L_y/2) x.  The correlation
    of bin k is sums[k] / (counts[k] * vsq)."""
    sums = np.zeros(nbins)
    counts = np.zeros(nbins, dtype=np.int64)
    vsq = ctypes.c_double()
    _load().or_velocity_correlation(ctypes.byref(p.c()), _ptr(_f64(pos)), float(delta), _ptr(_f64(v)),
                                    int(nbins), float(rmax), _ptr(sums), _ptr(counts), ctypes.byref(vsq))
    return sums, counts, vsq.value


def row_neighbors(p: Params, pos, delta: float, i: int) -> np.ndarray:
    """All j != i with R_ij^2 < r_c^2 for one particle i, by brute force (sorted)."""
    pos = _f64(pos)
    out = np.zeros(256, dtype=np.int64)
    m = _load().or_row_neighbors(ctypes.byref(p.c()), _ptr(pos), float(delta), int(i), 256, _ptr(out))
    if m > 256:
        out = np.zeros(m, dtype=np.int64)
        _load().or_row_neighbors(ctypes.byref(p.c()), _ptr(pos), float(delta), int(i), m, _ptr(out))
    return out[:m].copy()


def philox4x64_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, dtype=np.uint64)
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    _load().or_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def noise(seed: int, step: int, ids) -> np.ndarray:
    """Standard normals [n, 3] for the given particle ids at a time step."""
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    xi = np.zeros((ids.shape[0], 3))
    _load().or_noise(int(seed), int(step), ids.shape[0], _ptr(ids), _ptr(xi))
    return xi


@dataclasses.dataclass
class System:
    """Eq. algebra: A = diag - alpha W on each Cartesian component, and b."""
    n: int
    alpha: float
    pairs: np.ndarray   # [m, 2] int64, i < j
    w: np.ndarray       # [m] pair weights
    diag: np.ndarray    # [n]
    b: np.ndarray       # [n, 3]

    def matvec(self, x) -> np.ndarray:
        x = _f64(x)
        y = np.zeros_like(x)
        _load().or_matvec(self.n, self.alpha, self.pairs.shape[0], _ptr(self.pairs), _ptr(self.w),
                          _ptr(self.diag), _ptr(x), _ptr(y))
        return y

    def dense(self) -> np.ndarray:
        """The scalar n x n matrix (for small-n checks)."""
        A = np.diag(self.diag.copy())
        i, j = self.pairs[:, 0], self.pairs[:, 1]
        np.add.at(A, (i, j), -self.alpha * self.w)
        np.add.at(A, (j, i), -self.alpha * self.w)
        return A


def assemble(p: Params, pos, pairs, xi=None, delta: float = 0.0) -> System:
    pos = _f64(pos)
    pairs = np.ascontiguousarray(pairs, dtype=np.int64)
    m = pairs.shape[0]
    w = np.zeros(m)
    diag = np.zeros(p.n)
    b = np.zeros((p.n, 3))
    xi_p = _ptr(_f64(xi)) if xi is not None else None
    rc = _load().or_assemble(ctypes.byref(p.c()), _ptr(pos), float(delta), m, _ptr(pairs), xi_p,
                             _ptr(w), _ptr(diag), _ptr(b))
    if rc != OR_OK:
        raise RuntimeError(f"oracle assembly failed: {rc}")
    return System(p.n, p.alpha, pairs, w, diag, b)


def gershgorin_max(sys: System) -> float:
    """Upper bound of A's spectrum by Gershgorin's theorem: max_i (A_ii + alpha sum_j w_ij).
    (The lower bound is 1: A = I + alpha L_w with L_w positive semidefinite.)"""
    rowsum = np.zeros(sys.n)
    np.add.at(rowsum, sys.pairs[:, 0], sys.w)
    np.add.at(rowsum, sys.pairs[:, 1], sys.w)
    return float(np.max(sys.diag + sys.alpha * rowsum))


def chebyshev_sqrt_coeffs(a: float, b: float, degree: int) -> np.ndarray:
    """Coefficients c_0..c_K of the Chebyshev interpolant of sqrt on [a, b] at the
    K + 1 Chebyshev points of the first kind: p(x) = c_0 / 2 + sum_{k >= 1} c_k T_k(u),
    u = (2 x - b - a) / (b - a)."""
    N = degree + 1
    theta = np.pi * (np.arange(N) + 0.5) / N
    f = np.sqrt(0.5 * (b - a) * np.cos(theta) + 0.5 * (b + a))
    return np.array([2.0 / N * np.sum(f * np.cos(k * theta)) for k in range(N)])


def sqrt_apply(sys: System, g, degree: int):
    """xi = p(A) g with p the degree-K Chebyshev interpolant of sqrt on [1, Gershgorin
    max], by the three-term recurrence T_{k+1} = 2 u T_k - T_{k-1} applied to g (FDT-
    consistent noise: xi has covariance A if g has covariance I).  A = I returns g.
    Returns (xi [n, 3], the interval's upper end)."""
    g = _f64(g)
    lmax = gershgorin_max(sys)
    if not (lmax - 1.0 > 1e-12):
        return g.copy(), lmax
    c = chebyshev_sqrt_coeffs(1.0, lmax, degree)

    def u(v):   # the map of [1, lmax] onto [-1, 1], applied to A
        return (2.0 * sys.matvec(v) - (lmax + 1.0) * v) / (lmax - 1.0)

    t0 = g.copy()
    y = 0.5 * c[0] * t0
    if degree == 0:
        return y, lmax
    t1 = u(t0)
    y = y + c[1] * t1
    for k in range(2, degree + 1):
        t2 = 2.0 * u(t1) - t0
        y = y + c[k] * t2
        t0, t1 = t1, t2
    return y, lmax


def pcg(sys: System, tol: float = 1e-13, max_iter: int = 100000, x0=None):
    """Jacobi-PCG; returns (v [n,3], iterations, true relative residual)."""
    x = np.zeros((sys.n, 3)) if x0 is None else _f64(x0).copy()
    info = np.zeros(2)
    rc = _load().or_pcg(sys.n, sys.alpha, sys.pairs.shape[0], _ptr(sys.pairs), _ptr(sys.w),
                        _ptr(sys.diag), _ptr(_f64(sys.b)), float(tol), int(max_iter), _ptr(x), _ptr(info))
    if rc not in (OR_OK, OR_ERR_NOT_CONVERGED):
        raise RuntimeError(f"oracle pcg failed: {rc}")
    return x, int(info[0]), float(info[1])


def dense_solve(sys: System) -> np.ndarray:
    x = np.zeros((sys.n, 3))
    rc = _load().or_dense_solve(sys.n, sys.alpha, sys.pairs.shape[0], _ptr(sys.pairs), _ptr(sys.w),
                                _ptr(sys.diag), _ptr(_f64(sys.b)), _ptr(x))
    if rc != OR_OK:
        raise RuntimeError(f"oracle dense solve failed: {rc}")
    return x


def integrate(p: Params, pos, v, delta: float):
    """Returns (new positions, new delta)."""
    pos = _f64(pos).copy()
    dnew = _load().or_integrate(ctypes.byref(p.c()), _ptr(pos), _ptr(_f64(v)), float(delta))
    return pos, dnew


def structure_factor(p: Params, pos, delta: float, ks):
    """Eq. Sfactor at q_z = 0 for integer pairs ks [nk, 2]; returns (S, qx, qy)."""
    ks = np.ascontiguousarray(ks, dtype=np.int64).reshape(-1, 2)
    nk = ks.shape[0]
    S, qx, qy = np.zeros(nk), np.zeros(nk), np.zeros(nk)
    _load().or_structure_factor(ctypes.byref(p.c()), _ptr(_f64(pos)), float(delta), nk, _ptr(ks),
                                _ptr(S), _ptr(qx), _ptr(qy))
    return S, qx, qy


def stress_xy(p: Params, pos, delta: float, pairs, v) -> float:
    pairs = np.ascontiguousarray(pairs, dtype=np.int64)
    return _load().or_stress_xy(ctypes.byref(p.c()), _ptr(_f64(pos)), float(delta), pairs.shape[0],
                                _ptr(pairs), _ptr(_f64(v)))


@dataclasses.dataclass
class StepResult:
    pos: np.ndarray
    delta: float
    v: np.ndarray
    iterations: int
    residual: float
    system: System


def step(p: Params, pos, delta: float, step_index: int, ids=None, xi=None, tol: float = 1e-13,
         solver: str = "pcg", neighbor_method: str = "auto") -> StepResult:
    """One time step in the paper's order: neighbours and weights, forces and
    Eq. algebra, the velocity solve, then R += v dt with the Lees-Edwards wrap.
    Noise is drawn from the counter-based generator unless xi is given."""
    pos = _f64(pos)
    if ids is None:
        ids = np.arange(p.n, dtype=np.int64)
    if xi is None and p.kT != 0.0:
        xi = noise(p.seed, step_index, ids)
    pairs = neighbors(p, pos, delta, neighbor_method)
    sys = assemble(p, pos, pairs, xi, delta)
    if solver == "dense":
        v, it, res = dense_solve(sys), 0, 0.0
    else:
        v, it, res = pcg(sys, tol)
    new_pos, new_delta = integrate(p, pos, v, delta)
    return StepResult(new_pos, new_delta, v, it, res, sys)
