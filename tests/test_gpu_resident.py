"""The on-chip configurations of the persistent mixed solver.

They run the iteration of the other configurations (Jacobi-preconditioned CG,
FP32 inner iterations, double-float dot products, FP64 residual replacement)
with each block's rows, their vectors and the matrix entries between them
kept on the SM.  Only the rounding of the FP32 sums differs (the local and the
halo entries of a row are summed in two groups), so a solve must meet the FP64
tolerance against the oracle's matrix and agree with the other configurations
to the solve accuracy (cond ~ 22 times the tolerance).  A block whose entries
do not fit in shared memory solves its rows with global gathers instead; a
reduced shared-memory budget forces that fallback on some or all blocks.
"""
import numpy as np
import pytest

import oracle
import synth

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu

KT = 0.5


def _resident_configs(sim):
    n = sim.set_solver_config(0)["num_configs"]
    out = [k for k in range(n) if sim.set_solver_config(k)["resident"]]
    sim.set_solver_config(0)
    return out


def _make(n, seed, tol, delta_frac=0.3, warm_start="none"):
    L = synth.box_length(n)
    pos = synth.uniform_positions(n, (L, L, L), seed)
    kappa = ss.kappa_from_kappa_tau(KT)
    sim = ss.Simulation(n, (L, L, L), kappa, seed=seed, cg_tol=tol, positions=pos, cg_max_iter=5000,
                        warm_start=warm_start, precision="mixed")
    delta = delta_frac * L
    sim.set_positions(pos, delta)
    p = oracle.Params(n=n, L=(L, L, L), kappa=kappa, seed=seed)
    return sim, p, pos, delta


def test_two_resident_configurations_exist():
    sim, _, _, _ = _make(1024, 3, 1e-8)
    ks = _resident_configs(sim)
    assert len(ks) == 2
    assert {sim.set_solver_config(k)["block_threads"] for k in ks} == {512, 1024}
    with pytest.raises(ss.ShearsimError):
        sim.set_solver_config(sim.set_solver_config(0)["num_configs"])
    sim.close()


@pytest.mark.parametrize("n", [300, 777, 4096, 30000])
def test_resident_solve_meets_the_fp64_tolerance(n):
    """Several blocks, a ragged last window (n not a multiple of 256) and a single block."""
    tol = 1e-10
    sim, p, pos, delta = _make(n, n + 11, tol)
    sysr = oracle.assemble(p, pos, oracle.neighbors(p, pos, delta), oracle.noise(p.seed, 0, np.arange(n)), delta)
    ref, _, _ = oracle.pcg(sysr, 1e-13)
    for k in _resident_configs(sim):
        sim.set_solver_config(k)
        sim.build_neighbors()
        sim.assemble()
        info = sim.solve_velocities()
        assert info["status"] == 0 and info["residual"] <= tol, (k, info)
        assert info["offchip_blocks"] == 0, (k, info)
        v = sim.get_velocities()
        # the reported residual is the oracle's residual of the answer, up to the
        # mixed path's assembly error (~1e-12 relative, double-float entries)
        res = np.linalg.norm(sysr.b - sysr.matvec(v)) / np.linalg.norm(sysr.b)
        assert res <= tol + 2e-11, (k, res)
        assert abs(res - info["residual"]) <= 1e-3 * tol + 2e-11
        assert np.abs(v - ref).max() <= 1e-8 * np.abs(ref).max(), k
    sim.close()


@pytest.fixture(scope="module")
def full64():
    """The full-size system (262,144 rows, seven windows per block on 152 SMs),
    solved by the FP64 path to 1e-12 (itself pinned to the oracle elsewhere)."""
    w = synth.PRECISION
    kappa = ss.kappa_from_kappa_tau(w.kappa_tau)
    pos = synth.uniform_positions(w.n, w.L, w.seed)
    sim = ss.Simulation(w.n, w.L, kappa, seed=w.seed, cg_tol=1e-12, positions=pos, warm_start="none",
                        cg_max_iter=5000)
    sim.set_positions(pos, 7.25)
    sim.build_neighbors()
    sim.assemble()
    info = sim.solve_velocities()
    assert info["status"] == 0
    v = sim.get_velocities()
    sim.close()
    return w, pos, v


def _full_mixed(w, pos):
    kappa = ss.kappa_from_kappa_tau(w.kappa_tau)
    sim = ss.Simulation(w.n, w.L, kappa, seed=w.seed, cg_tol=1e-8, positions=pos, warm_start="none",
                        precision="mixed")
    sim.set_positions(pos, 7.25)
    return sim


@pytest.mark.parametrize("smem", [None, 150 * 1024, 40 * 1024])
def test_resident_full_size_against_fp64(full64, smem, monkeypatch):
    """Full budget: every block on chip.  150 KB: some blocks fall back.  40 KB:
    every block falls back to global gathers.  All meet 1e-8 and agree with
    the FP64 solve within cond * tol."""
    w, pos, v64 = full64
    if smem is None:
        monkeypatch.delenv("SHEARSIM_RESIDENT_SMEM", raising=False)
    else:
        monkeypatch.setenv("SHEARSIM_RESIDENT_SMEM", str(smem))
    sim = _full_mixed(w, pos)
    for k in _resident_configs(sim):
        sim.set_solver_config(k)
        sim.build_neighbors()
        sim.assemble()
        info = sim.solve_velocities()
        assert info["status"] == 0 and info["residual"] <= 1e-8, (k, info)
        if smem is None:
            assert info["offchip_blocks"] == 0, (k, info)
        elif smem == 40 * 1024:
            assert info["offchip_blocks"] > 0, (k, info)
        v = sim.get_velocities()
        assert np.abs(v - v64).max() <= 1e-6 * np.abs(v64).max(), k
    sim.close()


@pytest.mark.parametrize("extra", [0, 1])
def test_resident_at_its_largest_system(extra, monkeypatch):
    """2048 rows per SM, the largest system the on-chip form takes: every block
    holds exactly eight windows (the split by entry shares at any row cannot
    keep within eight windows per block there and falls back to whole windows).
    One row more leaves the on-chip form for the streaming one.  A 40 KB
    shared-memory budget shows which form ran: only the on-chip form reports
    blocks whose entries did not fit."""
    import torch
    n = 2048 * torch.cuda.get_device_properties(0).multi_processor_count + extra
    onchip = extra == 0
    res_oracle = None
    for smem in (None, 40 * 1024):
        if smem is None:
            monkeypatch.delenv("SHEARSIM_RESIDENT_SMEM", raising=False)
        else:
            monkeypatch.setenv("SHEARSIM_RESIDENT_SMEM", str(smem))
        sim, p, pos, delta = _make(n, 19, 1e-8)
        for k in _resident_configs(sim):
            sim.set_solver_config(k)
            sim.build_neighbors()
            sim.assemble()
            info = sim.solve_velocities()
            assert info["status"] == 0 and info["residual"] <= 1e-8, (n, smem, k, info)
            assert (info["offchip_blocks"] > 0) == (onchip and smem is not None), (n, smem, k, info)
            if res_oracle is None:   # the oracle's FP64 system of the same positions, once per size
                sysr = oracle.assemble(p, pos, oracle.neighbors(p, pos, delta, "cells"),
                                       oracle.noise(p.seed, 0, np.arange(n)), delta)
                v = sim.get_velocities()
                res_oracle = np.linalg.norm(sysr.b - sysr.matvec(v)) / np.linalg.norm(sysr.b)
                assert res_oracle <= 1e-8 + 2e-11, (n, res_oracle)
        sim.close()


def test_resident_steps_are_deterministic_and_follow_config_zero():
    n = 200000
    runs = []
    for cfg in ("resident", 0):
        for _ in range(2 if cfg == "resident" else 1):
            sim, p, pos, delta = _make(n, 8, 1e-8, warm_start="prev")
            sim.set_solver_config(_resident_configs(sim)[0] if cfg == "resident" else 0)
            info = sim.step(3)
            assert info["status"] == 0
            runs.append(sim.get_positions())
            sim.close()
    assert np.array_equal(runs[0], runs[1])
    L = synth.box_length(n)
    d = runs[0] - runs[2]
    d -= np.round(d / L) * L
    # each step's velocities agree within cond * tol: |dx| <= 3 dt |dv| ~ 1e-6
    assert np.abs(d).max() < 1e-5


def test_resident_zero_rhs_gives_zero_velocities():
    """No noise, no shear, no excluded volume: b = 0 and v = 0 (the on-chip
    solve forms the initial residual itself and stops before iterating)."""
    n = 4096
    L = synth.box_length(n)
    pos = synth.uniform_positions(n, (L, L, L), 5)
    sim = ss.Simulation(n, (L, L, L), 0.0, kT=0.0, eps=0.0, seed=5, cg_tol=1e-8, positions=pos,
                        warm_start="prev", precision="mixed")
    sim.set_solver_config(_resident_configs(sim)[1])
    info = sim.step(2)
    assert info["status"] == 0 and info["cg_iterations"] == 0
    assert np.all(sim.get_velocities() == 0.0)
    sim.close()


def test_resident_start_that_meets_the_tolerance_keeps_x0():
    """A second solve of the same system from its own solution stops at once
    and returns that solution unchanged."""
    sim, p, pos, delta = _make(30000, 17, 1e-8, warm_start="prev")
    sim.set_solver_config(_resident_configs(sim)[1])
    sim.build_neighbors()
    sim.assemble()
    first = sim.solve_velocities()
    assert first["status"] == 0 and first["iterations"] > 0
    v1 = sim.get_velocities()
    again = sim.solve_velocities()
    assert again["status"] == 0 and again["iterations"] == 0 and again["residual"] <= 1e-8
    assert np.array_equal(sim.get_velocities(), v1)
    sim.close()
