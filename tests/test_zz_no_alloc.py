"""The allocation-free solve (sp_solve_csr_noalloc) against the regular solve.

sp_solve_csr_noalloc serves callers that cannot allocate device memory (a host
framework owning every device allocation, a loop that forbids allocation after
start-up): it keeps its working vectors in a fixed device array inside the
library.  Here the caller (this test) owns the system and the output in torch
tensors, and the result must match sp_solve_velocities on the same system to
the FP64 solve tolerance, on two calls in a row that share the fixed array.
"""
import numpy as np
import pytest

import synth

ss = pytest.importorskip("paper_1808_06381_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _csr(n, pairs, w):
    rows = np.concatenate([pairs[:, 0], pairs[:, 1]])
    cols = np.concatenate([pairs[:, 1], pairs[:, 0]])
    ww = np.concatenate([w, w])
    order = np.lexsort((cols, rows))
    rows, cols, ww = rows[order], cols[order], ww[order]
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr).astype(np.int32), cols.astype(np.int32), ww


def _reference_system(n, seed):
    L = synth.box_length(n)
    pos = synth.uniform_positions(n, (L, L, L), seed)
    sim = ss.Simulation(n, (L, L, L), ss.kappa_from_kappa_tau(0.5), seed=seed, cg_tol=1e-13, cg_max_iter=5000,
                        warm_start="none", positions=pos)
    sim.set_positions(pos, 0.3 * L)
    sim.build_neighbors()
    sim.assemble()
    info = sim.solve_velocities()
    assert info["status"] == 0
    diag, b, pairs, w = sim.system()
    v = sim.get_velocities()
    sim.close()
    return diag, b, pairs, w, v


def test_noalloc_solve_matches_regular_solve_twice():
    ss.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream().cuda_stream
    for call, (n, seed) in enumerate([(3000, 11), (6001, 12)]):
        diag, b, pairs, w, v_ref = _reference_system(n, seed)
        row_ptr, col, ww = _csr(n, pairs, w)
        t_rp = torch.from_numpy(row_ptr).to(dev)
        t_col = torch.from_numpy(col).to(dev)
        t_w = torch.from_numpy(ww).to(dev)
        t_diag = torch.from_numpy(diag).to(dev)
        t_b = torch.from_numpy(np.ascontiguousarray(b.T)).to(dev)          # [3][n] planes
        t_x = torch.full((3, n), float("nan"), dtype=torch.float64, device=dev)
        info = ss.solve_csr_noalloc(n, t_rp.data_ptr(), t_col.data_ptr(), t_w.data_ptr(), t_diag.data_ptr(), 4.0,
                                    t_b.data_ptr(), t_x.data_ptr(), tol=1e-13, max_iter=5000, stream=stream)
        torch.cuda.synchronize()
        assert info["status"] == 0, info
        assert info["residual"] <= 1e-13
        x = t_x.cpu().numpy().T
        assert np.abs(x - v_ref).max() <= 1e-11 * np.abs(v_ref).max(), call


def test_noalloc_rejects_oversized_systems():
    ss.load()
    n = ss.NOALLOC_MAX_ROWS + 1
    info = ss.solve_csr_noalloc(n, 1, 1, 1, 1, 4.0, 1, 1)
    assert info["status"] == ss.SP_ERR_INVALID_ARG
    assert "32768" in info["error"]
