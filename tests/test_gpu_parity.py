"""CUDA path versus the CPU oracle, through the C ABI.

Tolerances (FP64 path):
  - pair lists: bit-exact (same predicate, same rounding: no contraction on either side);
  - Philox blocks: bit-exact;
  - weights, diagonal, right-hand side: 1e-14 relative (exp and the order of the
    pair sums differ by a few ulps);
  - velocities of one solve: 1e-11 relative to max |v| with both sides solved to
    1e-13 (condition number of the Jacobi-scaled matrix ~22, so the solution error
    of each side is below ~1e-12);
  - positions after k steps: 1e-10 absolute per step (v dt with v from above).
"""
import math

import numpy as np
import pytest

import oracle
import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu

KT = 0.5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ss.load()


def make(n, L, seed=1, kappa_tau=KT, delta=0.0, tol=1e-13, pos=None, **kw):
    L = tuple(L) if np.ndim(L) else (L, L, L)
    pos = synth.uniform_positions(n, L, seed) if pos is None else pos
    kw.setdefault("warm_start", "none")
    kappa = kw.pop("kappa", None)
    if kappa is None:
        kappa = ss.kappa_from_kappa_tau(kappa_tau)
    sim = ss.Simulation(n, L, kappa, seed=seed, cg_tol=tol, positions=pos, cg_max_iter=5000, **kw)
    if delta:
        sim.set_positions(pos, delta)
    okw = {k: kw[k] for k in ("alpha", "eps", "zeta", "kT", "dt") if k in kw}
    p = oracle.Params(n=n, L=L, kappa=kappa, seed=seed, **okw)
    return sim, p, pos


def pairs_equal(sim, p, pos, delta):
    got = sim.neighbors()
    ref = oracle.neighbors(p, pos, delta)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    assert np.array_equal(got, ref)
    return ref


def test_philox_bits_match_oracle():
    ids = np.arange(0, 5000, 7, dtype=np.int64)
    got = ss.philox_blocks(123456789, 42, ids)
    for k in range(0, len(ids), 37):
        ref = oracle.philox4x64_10(np.array([ids[k], 42, 0, 0], dtype=np.uint64),
                                   np.array([123456789, 0], dtype=np.uint64))
        assert np.array_equal(got[k], ref)


@pytest.mark.parametrize("n,L,delta", [
    (24, 2.0, 0.0),                     # smallest box: one cell, all pairs
    (64, 2.77, 1.3),
    (300, (7.0, 4.5, 2.6), 3.1),        # fewer than 3 cells along z only
    (500, (2.5, 9.0, 9.0), 0.7),        # fewer than 3 cells along x only
    (500, (9.0, 2.5, 9.0), 4.4),        # fewer than 3 cells along y (x scanned whole)
    (4096, synth.box_length(4096), 5.123),
    (4100, synth.box_length(4100), 11.0),   # ragged: not a multiple of any tile
])
def test_neighbor_lists_bit_exact(n, L, delta):
    sim, p, pos = make(n, L, seed=n, delta=delta)
    delta = delta % p.L[0]
    sim.build_neighbors()
    pairs_equal(sim, p, pos, delta)
    # the reported order is a permutation of the ids
    assert np.array_equal(np.sort(sim.order()), np.arange(n))
    sim.close()


def test_neighbor_lists_with_particles_on_cell_and_box_faces():
    n = 3000
    L = synth.box_length(n)
    pos = synth.uniform_positions(n, (L, L, L), 5)
    cw = L / math.floor(L)
    pos[:100, 0] = cw * np.floor(pos[:100, 0] / cw)        # on cell faces
    pos[100:200, 1] = 0.0                                    # on the sheared face
    pos[200:300, 1] = np.nextafter(L, 0)
    pos[300:400, 2] = 0.0
    pos[400:420] = pos[420:440] + np.array([0.999999, 0, 0])  # pairs right at the cut
    pos[400:420, 0] %= L
    for delta in (0.0, 0.25 * L, L - 1e-12):
        sim, p, _ = make(n, L, pos=pos, delta=delta)
        sim.build_neighbors()
        pairs_equal(sim, p, pos, delta)
        sim.close()


# FP64 assembly: exact up to rounding order (and ~2 ulp of the table-driven exponential).
# Mixed-precision path: separations, weights and pair sums in double-float from
# positions held as float pairs (2^-48 relative), so ~1e-12 relative (bound with margin).
ASSEMBLY_BOUNDS = {"fp64": (1e-14, 1e-14, 1e-13), "mixed": (2e-11, 2e-11, 2e-11)}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,delta,kappa_tau", [(64, 0.4, 0.5), (2000, 3.3, 0.05), (4096, 7.7, 0.5)])
def test_assembly_matches_oracle(n, delta, kappa_tau, precision):
    L = synth.box_length(n)
    sim, p, pos = make(n, L, seed=3 + n, kappa_tau=kappa_tau, delta=delta, precision=precision)
    sim.set_step(17)
    sim.build_neighbors()
    sim.assemble()
    diag, b, pairs, w = sim.system()
    ref_pairs = oracle.neighbors(p, pos, delta)
    assert np.array_equal(pairs, ref_pairs)
    xi = oracle.noise(p.seed, 17, np.arange(n))
    ref = oracle.assemble(p, pos, ref_pairs, xi, delta)
    bw, bd, bb = ASSEMBLY_BOUNDS[precision]
    assert np.abs(w - ref.w).max() <= bw
    assert np.abs(diag - ref.diag).max() <= bd * np.abs(ref.diag).max()
    assert np.abs(b - ref.b).max() <= bb * np.abs(ref.b).max()
    sim.close()


@pytest.mark.parametrize("n,seed", [(24, 1), (64, 2), (777, 3), (4096, 4)])
def test_single_solve_velocities(n, seed):
    L = synth.box_length(n)
    delta = 0.37 * L
    sim, p, pos = make(n, L, seed=seed, delta=delta)
    sim.build_neighbors()
    sim.assemble()
    info = sim.solve_velocities()
    assert info["status"] == 0 and info["residual"] <= 1e-13
    v = sim.get_velocities()
    sysr = oracle.assemble(p, pos, oracle.neighbors(p, pos, delta), oracle.noise(p.seed, 0, np.arange(n)), delta)
    if n <= 64:
        ref = oracle.dense_solve(sysr)
    else:
        ref, _, _ = oracle.pcg(sysr, 1e-13)
    assert np.abs(v - ref).max() <= 1e-11 * np.abs(ref).max()
    # the GPU solution satisfies the oracle's own system
    res = np.linalg.norm(sysr.b - sysr.matvec(v)) / np.linalg.norm(sysr.b)
    assert res <= 1e-12
    sim.close()


def test_steps_follow_the_oracle():
    n, steps = 1000, 5
    L = synth.box_length(n)
    sim, p, pos = make(n, L, seed=9, warm_start="prev")
    info = sim.step(steps)
    assert info["steps_done"] == steps and info["status"] == 0
    gpos = sim.get_positions()
    gv = sim.get_velocities()
    delta, step = sim.state()
    opos, od = pos, 0.0
    for s in range(steps):
        r = oracle.step(p, opos, od, s, tol=1e-13)
        opos, od, ov = r.pos, r.delta, r.v
    assert step == steps
    assert abs(delta - od) < 1e-12
    d = gpos - opos
    d -= np.round(d / L) * L
    assert np.abs(d).max() < 1e-10 * steps
    assert np.abs(gv - ov).max() <= 1e-9 * np.abs(ov).max()
    sim.close()


def test_plain_fp64_workload_follows_the_oracle_for_200_steps():
    """The plain FP64 workload in full: N = 4,096, kappa tau = 0.5, Jacobi-PCG to 1e-10 warm-started
    from the previous velocities, 200 steps in graph mode, against the oracle stepping the same
    trajectory (its solves to 1e-13).  Per step |v_gpu - v| <= ~cond * 1e-10 * max|v| (cond ~ 22 after
    Jacobi scaling), i.e. ~1e-9 in position per step of dt = 0.01."""
    w = synth.PLAIN_FP64
    pos = synth.uniform_positions(w.n, w.L, w.seed)
    kappa = ss.kappa_from_kappa_tau(w.kappa_tau)
    sim = ss.Simulation(w.n, w.L, kappa, seed=w.seed, precision="fp64", warm_start="prev", cg_tol=w.tol,
                        cg_max_iter=2000, positions=pos)
    p = oracle.Params.from_workload(w)
    opos, od = pos, 0.0
    L = w.L[0]
    done = 0
    for chunk in (50, 50, 50, 50):
        info = sim.step(chunk)
        assert info["status"] == 0 and info["steps_done"] == chunk and info["host_driven"] == 0
        assert info["last_residual"] <= w.tol
        for s in range(done, done + chunk):
            r = oracle.step(p, opos, od, s, tol=1e-13, neighbor_method="cells")
            opos, od = r.pos, r.delta
        done += chunk
        delta, step = sim.state()
        assert step == done and abs(delta - od) < 1e-11
        d = sim.get_positions() - opos
        d -= np.round(d / L) * L
        assert np.abs(d).max() < 2e-9 * done, (done, np.abs(d).max())
    assert np.abs(sim.get_velocities() - r.v).max() <= 1e-7 * np.abs(r.v).max()
    sim.close()


def test_graph_and_host_loop_modes_agree(monkeypatch):
    """The FP64 step with the two-kernel iteration as one CUDA graph (CG loop in a conditional
    WHILE node, thermal normals on the graph's side branch) and the host-driven loop give
    identical steps; the graph mode must really have captured (host_driven == 0)."""
    n = 2000
    L = synth.box_length(n)
    outs = []
    monkeypatch.setenv("SHEARSIM_PERSISTENT", "0")
    for mode in ("0", "1"):
        monkeypatch.setenv("SHEARSIM_HOST_LOOP", mode)
        sim, p, pos = make(n, L, seed=4, tol=1e-10, warm_start="prev")
        info = sim.step(3)
        assert info["host_driven"] == int(mode), (mode, info)
        outs.append((sim.get_positions(), sim.get_velocities(), info["cg_iterations"]))
        sim.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


@pytest.mark.parametrize("precision,persistent,warm", [
    ("fp64", "1", "prev"), ("fp64", "1", "none"), ("fp64", "0", "prev"), ("fp64", "0", "none"),
    ("mixed", "0", "prev"), ("mixed", "1", "prev"), ("mixed", "1", "none")])
def test_steps_and_solves_never_fall_back_to_the_host_loop(monkeypatch, capfd, precision, persistent, warm):
    """Every form of the step and of the stand-alone solve captures its CUDA graph."""
    monkeypatch.delenv("SHEARSIM_HOST_LOOP", raising=False)
    monkeypatch.setenv("SHEARSIM_PERSISTENT", persistent)
    n = 3000
    L = synth.box_length(n)
    sim, p, pos = make(n, L, seed=9, tol=1e-8, warm_start=warm, precision=precision)
    info = sim.step(2)
    assert info["host_driven"] == 0, info
    sim.build_neighbors()
    sim.assemble()
    sinfo = sim.solve_velocities()
    assert sinfo["host_driven"] == 0, sinfo
    sim.close()
    err = capfd.readouterr().err
    assert "capture failed" not in err, err


@pytest.mark.parametrize("n", [777, 4096, 60000])
def test_fp64_persistent_and_two_kernel_solvers_agree(monkeypatch, n):
    """The FP64 solve as one cooperative launch and as the two-kernel graph iteration: same
    system, both to 1e-12; velocities agree to the solve tolerance and with the oracle."""
    L = synth.box_length(n)
    res = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("SHEARSIM_PERSISTENT", flag)
        sim, p, pos = make(n, L, seed=n + 3, delta=0.37 * L, tol=1e-12)
        sim.build_neighbors()
        sim.assemble()
        info = sim.solve_velocities()
        assert info["status"] == 0 and info["residual"] <= 1e-12 and info["host_driven"] == 0
        res[flag] = (sim.get_velocities(), info["iterations"])
        sim.close()
    v1, v0 = res["1"][0], res["0"][0]
    assert np.abs(v1 - v0).max() <= 1e-10 * np.abs(v0).max()
    assert abs(res["1"][1] - res["0"][1]) <= 2


def test_runs_are_deterministic():
    n = 3000
    L = synth.box_length(n)
    res = []
    for _ in range(2):
        sim, p, pos = make(n, L, seed=6, tol=1e-8, warm_start="prev")
        sim.step(4)
        res.append(sim.get_positions())
        sim.close()
    assert np.array_equal(res[0], res[1])


def test_momentum_bookkeeping_on_gpu():
    """Pair terms cancel: sum_i v_i = sum_i (noise_i + shear_i) / zeta (no oracle involved)."""
    n = 4096
    L = synth.box_length(n)
    sim, p, pos = make(n, L, seed=12, delta=2.0, zeta=1.7, kT=0.8)
    sim.build_neighbors()
    sim.assemble()
    sim.solve_velocities()
    v = sim.get_velocities()
    amp = math.sqrt(2 * p.zeta * p.kT / p.dt)
    expect = amp * oracle.noise(p.seed, 0, np.arange(n)).sum(0) / p.zeta
    expect[0] += p.kappa * (pos[:, 1] - L / 2).sum()
    assert np.allclose(v.sum(0), expect, atol=1e-10 * np.abs(v).sum())
    sim.close()


# ------------------------------------------------------------- edge cases


def test_two_particles_minimum_box():
    pos = np.array([[0.2, 0.1, 0.3], [0.9, 1.95, 0.5]])
    sim, p, _ = make(2, 2.0, pos=pos, delta=0.6)
    sim.build_neighbors()
    sim.assemble()
    sim.solve_velocities()
    r = oracle.step(p, pos, 0.6, 0, tol=1e-14, solver="dense")
    assert np.array_equal(sim.neighbors(), r.system.pairs)
    assert np.abs(sim.get_velocities() - r.v).max() <= 1e-12 * np.abs(r.v).max()
    sim.close()


def test_no_coupling_solves_in_one_iteration():
    n = 500
    sim, p, pos = make(n, synth.box_length(n), alpha=0.0)
    sim.build_neighbors()
    sim.assemble()
    info = sim.solve_velocities()
    assert info["iterations"] <= 1
    sim.close()


def test_zero_right_hand_side_gives_zero_velocity():
    n = 400
    sim, p, pos = make(n, synth.box_length(n), kappa=0.0, kT=0.0, eps=0.0)
    sim.build_neighbors()
    sim.assemble()
    info = sim.solve_velocities()
    assert info["status"] == 0 and info["bnorm"] == 0.0
    assert np.all(sim.get_velocities() == 0.0)
    sim.close()


def test_iteration_cap_reports_not_converged_and_recovers():
    n = 2000
    L = synth.box_length(n)
    pos = synth.uniform_positions(n, (L, L, L), 2)
    sim = ss.Simulation(n, (L, L, L), 3.0, seed=2, cg_tol=1e-14, cg_max_iter=3, positions=pos)
    sim.build_neighbors()
    sim.assemble()
    info = sim.solve_velocities(raise_on_error=False)
    assert info["status"] == ss.SP_ERR_NOT_CONVERGED and info["iterations"] == 3
    st = sim.step(2, raise_on_error=False)
    assert st["status"] == ss.SP_ERR_NOT_CONVERGED and st["steps_done"] == 0
    sim.close()


def test_dense_cluster_grows_pair_storage():
    """Far more than 20 partners per particle: the pair arrays are regrown and the step retried."""
    n = 1500
    L = 10.0
    rng = np.random.Generator(np.random.PCG64(3))
    pos = rng.uniform(0.0, 2.5, (n, 3))
    sim, p, _ = make(n, L, pos=pos, tol=1e-9)
    info = sim.step(1)
    assert info["status"] == 0 and info["steps_done"] == 1
    r = oracle.step(p, pos, 0.0, 0, tol=1e-12)
    assert sim.num_pairs() == r.system.pairs.shape[0]
    assert np.abs(sim.get_velocities() - r.v).max() <= 1e-7 * np.abs(r.v).max()
    sim.close()


def test_on_chip_rows_with_many_local_entries():
    """~77 partners per row, all in the on-chip solve's one block: rows with more
    than 64 local entries keep column order in shared memory (the bank-aware order
    tracks its left-over positions in 64 bits) and the solve still meets the
    tolerance on the oracle's system."""
    n = 256
    L = 2.4   # density ~18.5: ~77 partners per particle, one block of 256 rows
    pos = synth.uniform_positions(n, (L,) * 3, 11)
    sim, p, _ = make(n, L, pos=pos, tol=1e-8, precision="mixed", delta=0.8)
    info = sim.set_solver_config(9)
    assert info["resident"]
    sim.build_neighbors()
    sim.assemble()
    res = sim.solve_velocities()
    assert res["status"] == 0 and res["offchip_blocks"] == 0, res
    pairs = pairs_equal(sim, p, pos, 0.8)
    assert pairs.shape[0] * 2 / n > 64
    sysr = oracle.assemble(p, pos, pairs, oracle.noise(p.seed, 0, np.arange(n)), 0.8)
    v = sim.get_velocities()
    assert np.linalg.norm(sysr.b - sysr.matvec(v)) / np.linalg.norm(sysr.b) <= 1e-8
    sim.close()


# ------------------------------------------------ full size (262,144 particles)


@pytest.fixture(scope="module")
def full():
    w = synth.PRECISION
    L = w.L
    pos = synth.uniform_positions(w.n, L, w.seed)
    kappa = ss.kappa_from_kappa_tau(w.kappa_tau)
    sim = ss.Simulation(w.n, L, kappa, seed=w.seed, cg_tol=1e-12, positions=pos, warm_start="none",
                        cg_max_iter=5000)
    sim.set_positions(pos, 7.25)
    sim.build_neighbors()
    sim.assemble()
    info = sim.solve_velocities()
    p = oracle.Params(n=w.n, L=L, kappa=kappa, seed=w.seed)
    yield sim, p, pos, info
    sim.close()


def test_full_size_sampled_rows(full):
    sim, p, pos, info = full
    delta = 7.25
    diag, b, pairs, w = sim.system()
    rng = np.random.Generator(np.random.PCG64(0))
    rows = rng.choice(p.n, 64, replace=False)
    xi = oracle.noise(p.seed, 0, np.arange(p.n))
    for i in rows:
        nb = oracle.row_neighbors(p, pos, delta, i)
        mine = np.sort(np.concatenate([pairs[pairs[:, 0] == i, 1], pairs[pairs[:, 1] == i, 0]]))
        assert np.array_equal(nb, mine)
        # the row of the system, from the oracle's assembly of exactly these pairs
        rp = np.stack([np.full(len(nb), i), nb], 1)
        rp = np.sort(rp, axis=1)
        ref = oracle.assemble(p, pos, rp, xi, delta)
        assert abs(diag[i] - ref.diag[i]) <= 1e-14 * ref.diag[i]
        assert np.abs(b[i] - ref.b[i]).max() <= 1e-13 * np.abs(ref.b[i]).max()


def test_full_size_velocities_against_oracle_solve(full):
    sim, p, pos, info = full
    delta = 7.25
    assert info["status"] == 0 and info["residual"] <= 1e-12
    v = sim.get_velocities()
    pairs = oracle.neighbors(p, pos, delta, method="cells")
    sysr = oracle.assemble(p, pos, pairs, oracle.noise(p.seed, 0, np.arange(p.n)), delta)
    ref, it, res = oracle.pcg(sysr, 1e-12)
    assert np.abs(v - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.linalg.norm(sysr.b - sysr.matvec(v)) <= 2e-12 * np.linalg.norm(sysr.b)


# --------------------------------------------- FP32 pre-filter of the pair search


@pytest.mark.parametrize("L,delta", [(40.0, 13.7), (111.8, 77.25)])
def test_pairs_near_the_cut_in_large_boxes(L, delta):
    """Pairs at |R|^2 = r_c^2 (1 +- 1e-5 .. 1e-7), inside the FP32 margin band, also across
    the sheared boundary: the exact predicate decides them, bit for bit as the oracle."""
    rng = np.random.Generator(np.random.PCG64(int(L)))
    n_pairs = 3000
    a = rng.uniform(0, L, (n_pairs, 3))
    a[: n_pairs // 3, 1] = rng.uniform(L - 0.5, L, n_pairs // 3)       # near the top face
    u = rng.normal(size=(n_pairs, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = 1.0 + rng.choice([-1e-5, -1e-6, -1e-7, 1e-7, 1e-6, 1e-5, 0.0], n_pairs)
    b = a + u * r[:, None]
    pos = np.concatenate([a, b])
    # b may leave the box: map it back with the sheared images
    y_over = pos[:, 1] >= L
    pos[y_over, 1] -= L
    pos[y_over, 0] -= delta
    y_under = pos[:, 1] < 0
    pos[y_under, 1] += L
    pos[y_under, 0] += delta
    pos[:, 0] %= L
    pos[:, 2] %= L
    pos[pos >= L] = 0.0
    n = pos.shape[0]
    sim, p, _ = make(n, L, pos=pos, delta=delta)
    sim.build_neighbors()
    got = sim.neighbors()
    ref = oracle.neighbors(p, pos, delta, method="cells")
    assert np.array_equal(got, ref)
    assert ref.shape[0] > n_pairs // 2
    sim.close()


# ------------------------------------------------------------ mixed precision


@pytest.mark.parametrize("n,tol,bound", [(777, 1e-10, 1e-8), (4096, 1e-10, 1e-8), (4096, 1e-8, 1e-6)])
def test_mixed_solve_meets_the_fp64_tolerance(n, tol, bound):
    """Mixed solver: FP32 inner iterations, FP64 residual replacement.  The reported
    true residual is the FP64 one and meets tol; the velocity error against the FP64
    oracle solve is within cond(A) * tol (cond ~ 22; bound stated with margin)."""
    L = synth.box_length(n)
    delta = 0.21 * L
    sim, p, pos = make(n, L, seed=n + 5, delta=delta, tol=tol, precision="mixed")
    sim.build_neighbors()
    sim.assemble()
    info = sim.solve_velocities()
    assert info["status"] == 0 and info["residual"] <= tol
    v = sim.get_velocities()
    sysr = oracle.assemble(p, pos, oracle.neighbors(p, pos, delta), oracle.noise(p.seed, 0, np.arange(n)), delta)
    ref, _, _ = oracle.pcg(sysr, 1e-13)
    assert np.abs(v - ref).max() <= bound * np.abs(ref).max()
    # the residual the solver reports is the oracle's residual of its answer, up to the
    # mixed path's assembly error (~1e-12 relative in A and b: double-float entries)
    res = np.linalg.norm(sysr.b - sysr.matvec(v)) / np.linalg.norm(sysr.b)
    assert res <= tol + 2e-11
    assert abs(res - info["residual"]) <= 1e-3 * tol + 2e-11
    sim.close()


def test_mixed_steps_follow_the_oracle():
    n, steps = 2000, 4
    L = synth.box_length(n)
    sim, p, pos = make(n, L, seed=21, warm_start="prev", tol=1e-11, precision="mixed")
    info = sim.step(steps)
    assert info["status"] == 0 and info["last_residual"] <= 1e-11
    gpos = sim.get_positions()
    opos, od = pos, 0.0
    for s in range(steps):
        r = oracle.step(p, opos, od, s, tol=1e-13)
        opos, od = r.pos, r.delta
    d = gpos - opos
    d -= np.round(d / L) * L
    assert np.abs(d).max() < 1e-9 * steps
    sim.close()


def test_mixed_full_size_against_fp64_gpu(full):
    sim64, p, pos, info64 = full
    w = synth.PRECISION
    kappa = ss.kappa_from_kappa_tau(w.kappa_tau)
    sim = ss.Simulation(w.n, w.L, kappa, seed=w.seed, cg_tol=1e-8, positions=pos, warm_start="none",
                        precision="mixed")
    sim.set_positions(pos, 7.25)
    sim.build_neighbors()
    sim.assemble()
    info = sim.solve_velocities()
    assert info["status"] == 0 and info["residual"] <= 1e-8
    v = sim.get_velocities()
    v64 = sim64.get_velocities()
    # single-solve velocity error of the mixed path vs the FP64 solve (to 1e-12): <= cond * 1e-8
    assert np.abs(v - v64).max() <= 1e-6 * np.abs(v64).max()
    sim.close()


def test_persistent_and_multikernel_mixed_solvers_agree(monkeypatch):
    """The one-launch mixed solver and the two-kernels-per-iteration one run the same
    iteration; both meet the FP64 tolerance and agree to the solve accuracy."""
    n = 20000
    L = synth.box_length(n)
    outs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("SHEARSIM_PERSISTENT", flag)
        sim, p, pos = make(n, L, seed=31, tol=1e-10, precision="mixed", delta=0.4 * L)
        sim.build_neighbors()
        sim.assemble()
        info = sim.solve_velocities()
        assert info["status"] == 0 and info["residual"] <= 1e-10, (flag, info)
        outs.append(sim.get_velocities())
        sim.close()
    assert np.abs(outs[0] - outs[1]).max() <= 2e-8 * np.abs(outs[1]).max()


def test_persistent_mixed_steps_are_deterministic():
    n = 30000
    L = synth.box_length(n)
    res = []
    for _ in range(2):
        sim, p, pos = make(n, L, seed=8, tol=1e-8, precision="mixed", warm_start="prev")
        info = sim.step(3)
        assert info["status"] == 0
        res.append(sim.get_positions())
        sim.close()
    assert np.array_equal(res[0], res[1])


# ---------------------------------------------------------- structure factor


def test_structure_factor_direct_mode_matches_oracle():
    n = 3000
    L = synth.box_length(n)
    delta = 0.31 * L
    sim, p, pos = make(n, L, seed=41, delta=delta)
    S, qx, qy = sim.structure_factor(6, 5, grid=0)
    ks = np.array([(kx, ky) for kx in range(-6, 7) for ky in range(-5, 6)])
    Sr, qxr, qyr = oracle.structure_factor(p, pos, delta, ks)
    assert np.allclose(qx.ravel(), qxr, rtol=1e-14, atol=1e-14)
    assert np.allclose(qy.ravel(), qyr, rtol=1e-14, atol=1e-14)
    assert np.allclose(S.ravel(), Sr, rtol=1e-9, atol=1e-9)
    sim.close()


def test_structure_factor_bragg_peaks_of_a_sheared_lattice_on_gpu():
    m, a = 8, 0.9
    Lb = m * a
    base = synth.lattice_positions(m, a, offset=(0.05, 0.1, 0.2))
    gamma = 0.43
    pos = base.copy()
    pos[:, 0] = (pos[:, 0] + gamma * pos[:, 1]) % Lb
    sim, p, _ = make(m ** 3, Lb, pos=pos, delta=(gamma * Lb) % Lb)
    S, qx, qy = sim.structure_factor(m, m, grid=0)
    S = S.reshape(2 * m + 1, 2 * m + 1)
    n = m ** 3
    assert abs(S[m + m, m + 0] - n) < 1e-8 * n          # (kx, ky) = (m, 0)
    assert abs(S[m + 0, m + m] - n) < 1e-8 * n          # (0, m)
    assert abs(S[m + m, m - m] - n) < 1e-8 * n          # (m, -m)
    assert S[m + 1, m + 0] < 1e-18 and S[m + 3, m + 2] < 1e-18
    sim.close()


def test_structure_factor_grid_mode_against_direct_sum():
    """CIC grid with the window divided out: the residual error is aliasing from modes
    k + G m, of relative amplitude about (k / (G - k))^2 per alias; for |k| <= G/16 the
    alias terms give a few per cent on S(q) at most (1.6 % rms estimate)."""
    n = 262144
    L = synth.box_length(n)
    sim, p, pos = make(n, L, seed=43, delta=0.27 * L, tol=1e-8, precision="mixed", warm_start="prev")
    sim.step(3)
    G, nk = 256, 16
    Sg, qxg, qyg = sim.structure_factor(nk, nk, grid=G)
    Sd, qxd, qyd = sim.structure_factor(nk, nk, grid=0)
    assert np.allclose(qxg, qxd) and np.allclose(qyg, qyd)
    mask = np.ones_like(Sd, dtype=bool)
    mask[nk, nk] = False                                # q = 0 is excluded
    rel = np.abs(Sg[mask] - Sd[mask]) / Sd[mask]
    assert np.median(rel) < 0.015, np.median(rel)
    assert np.quantile(rel, 0.95) < 0.05, np.quantile(rel, 0.95)
    assert abs(Sg[mask].mean() / Sd[mask].mean() - 1) < 0.01
    sim.close()


# ------------------------------------------------------------------- stress


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_stress_matches_oracle(precision, bound):
    """Pair-virial shear stress of the solved state: FP64 path to 1e-10 (velocities
    solved to 1e-13), mixed path to 1e-4 (FP32 separations and weights)."""
    n = 4096
    L = synth.box_length(n)
    delta = 0.6 * L
    sim, p, pos = make(n, L, seed=51, delta=delta, precision=precision, tol=1e-12)
    sim.build_neighbors()
    sim.assemble()
    sim.solve_velocities()
    got = sim.stress_xy()
    v = sim.get_velocities()
    ref = oracle.stress_xy(p, pos, delta, oracle.neighbors(p, pos, delta), v)
    assert abs(got - ref) <= bound * abs(ref), (got, ref)
    sim.close()
