"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only draws inputs: particle positions, box sizes and workload
descriptions.  It holds none of the method's arithmetic (no pair model, no
linear system, no solver, no units derivation), so that both sides of every
parity test can start from the same bytes without sharing any of the code
under test.

Workloads follow the paper's setting (one particle per chain, a soft liquid
near overlap density, Lees-Edwards shear in the xy plane; §Method, §Results)
at number density 3 with the truncation radius r_c = 1 as the length unit.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DENSITY = 3.0          # particles per r_c^3
SEED_BASE = 20180817   # the default seed of workload k is SEED_BASE + k


def box_length(n: int, density: float = DENSITY) -> float:
    """Edge of the cubic box that holds n particles at the given density."""
    return (n / density) ** (1.0 / 3.0)


def uniform_positions(n: int, L, seed: int) -> np.ndarray:
    """n positions drawn uniformly in [0, Lx) x [0, Ly) x [0, Lz), float64 [n, 3].

    Drawn with numpy's PCG64 so that the stream does not depend on either
    side of the comparison.
    """
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = rng.random((n, 3)) * L[None, :]
    # rng.random is in [0, 1); the product can round up to L itself.
    for d in range(3):
        col = pos[:, d]
        col[col >= L[d]] = 0.0
    return np.ascontiguousarray(pos)


def lattice_positions(m, a: float, offset=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Simple cubic lattice with m[d] sites of spacing a along axis d, float64 [n, 3]."""
    m = np.broadcast_to(np.asarray(m, dtype=np.int64), (3,))
    axes = [offset[d] + a * np.arange(m[d], dtype=np.float64) for d in range(3)]
    gx, gy, gz = np.meshgrid(*axes, indexing="ij")
    return np.ascontiguousarray(np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1))


def standard_normals(shape, seed: int) -> np.ndarray:
    """Independent N(0, 1) draws (PCG64), for injecting noise into both sides."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(rng.standard_normal(shape))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: box, particle count and model parameters.

    kappa_tau is the dimensionless shear rate of the paper's figures; each
    side converts it to a rate in its own code.
    """
    name: str
    n: int
    L: tuple
    kappa_tau: float
    steps: int
    tol: float
    seed: int
    alpha: float = 4.0
    eps: float = 1.0
    zeta: float = 1.0
    kT: float = 1.0
    dt: float = 0.01
    rc: float = 1.0


def cubic(name: str, n: int, kappa_tau: float, steps: int, tol: float, seed: int, **kw) -> Workload:
    L = box_length(n)
    return Workload(name=name, n=n, L=(L, L, L), kappa_tau=kappa_tau, steps=steps, tol=tol,
                    seed=seed, **kw)


# The five workloads of the benchmark plan: positions uniform from the seed,
# alpha = 4, eps = 1, zeta = kT = 1, dt = 0.01 (paper parameters; §Results).
PLAIN_FP64 = cubic("plain-fp64-n4096", 4096, 0.5, 200, 1e-10, SEED_BASE + 1)
PRECISION = cubic("mixed-n262144", 262144, 0.5, 2000, 1e-8, SEED_BASE + 2)
PRECISION_LOW_SHEAR = cubic("mixed-n262144-kt0.05", 262144, 0.05, 2000, 1e-8, SEED_BASE + 2)
LEARNED = cubic("learned-n262144", 262144, 0.5, 2000, 1e-8, SEED_BASE + 4)
LARGE = cubic("large-n4194304", 4194304, 0.5, 10000, 1e-8, SEED_BASE + 5)


# The paper's box for its result figures, 87.6 x 43.6 x 22 lambda^3 (§Results),
# in units of r_c (lambda = 0.408539 r_c from the 5 % truncation at r_c), at
# density 3 per r_c^3: 17,191 particles; kappa tau = 0 as for Fig. vv.
PAPER_BOX_L = (35.79, 17.81, 8.99)
PAPER_BOX_VV = Workload(name="paper-box-n17191", n=17191, L=PAPER_BOX_L, kappa_tau=0.0, steps=200, tol=1e-8,
                        seed=SEED_BASE + 6)


def batch_replicas(count: int = 64, seed: int = SEED_BASE + 3):
    """Ensemble of replicas: N log-uniform in [8192, 131072], kappa*tau log-uniform in [0.01, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.rint(np.exp(rng.uniform(math.log(8192), math.log(131072), count))).astype(np.int64)
    kts = np.exp(rng.uniform(math.log(0.01), math.log(1.0), count))
    return [cubic(f"replica-{k}", int(ns[k]), float(kts[k]), 1000, 1e-8, seed * 1000 + k)
            for k in range(count)]
