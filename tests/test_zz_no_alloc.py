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


def test_noalloc_rejects_a_column_outside_the_system():
    """A column index >= n is refused before any gather through it (no stale or outside read)."""
    ss.load()
    dev = torch.device("cuda", 0)
    n = 64
    row_ptr = torch.tensor([0, 1] + [1] * (n - 1), dtype=torch.int32, device=dev)
    col = torch.tensor([n], dtype=torch.int32, device=dev)
    w = torch.tensor([0.5], dtype=torch.float64, device=dev)
    diag = torch.ones(n, dtype=torch.float64, device=dev)
    b = torch.ones(3, n, dtype=torch.float64, device=dev)
    x = torch.zeros(3, n, dtype=torch.float64, device=dev)
    info = ss.solve_csr_noalloc(n, row_ptr.data_ptr(), col.data_ptr(), w.data_ptr(), diag.data_ptr(), 1.0,
                                b.data_ptr(), x.data_ptr(), tol=1e-12, max_iter=100,
                                stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert info["status"] == ss.SP_ERR_INVALID_ARG, info
    assert "col" in info["error"]


def test_noalloc_refuses_a_capturing_stream():
    """The call synchronises its stream, so under stream capture it must refuse and leave the capture intact."""
    ss.load()
    dev = torch.device("cuda", 0)
    n = 16
    row_ptr = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    col = torch.zeros(1, dtype=torch.int32, device=dev)
    w = torch.zeros(1, dtype=torch.float64, device=dev)
    diag = torch.ones(n, dtype=torch.float64, device=dev)
    b = torch.ones(3, n, dtype=torch.float64, device=dev)
    x = torch.zeros(3, n, dtype=torch.float64, device=dev)
    y = torch.zeros(8, device=dev)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        info = ss.solve_csr_noalloc(n, row_ptr.data_ptr(), col.data_ptr(), w.data_ptr(), diag.data_ptr(), 1.0,
                                    b.data_ptr(), x.data_ptr(), tol=1e-12, max_iter=10,
                                    stream=torch.cuda.current_stream().cuda_stream)
        y.add_(1.0)
    g.replay()
    torch.cuda.synchronize()
    assert info["status"] == ss.SP_ERR_INVALID_ARG, info
    assert "captured" in info["error"]
    assert float(y[0]) == 1.0   # the capture stayed valid: its one op ran once, by the replay
