"""GB300 (sm_103a) coupled velocity solve of Korolkovas, arXiv 1808.06381.

Thin ctypes binding of ``libshearsim.so`` (declared in ``include/shearsim.h``):
argument marshalling only.  Every step of the method runs in the library's
CUDA kernels; there is no CPU fallback, and loading fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
LIB_PATH = os.path.join(_PKG, "lib", "libshearsim.so")
HEADER = os.path.join(_ROOT, "include", "shearsim.h")

SP_OK = 0
SP_ERR_INVALID_ARG = -1
SP_ERR_CUDA = -2
SP_ERR_NOT_CONVERGED = -3
SP_ERR_NONFINITE = -4
SP_ERR_OOM = -5
SP_ERR_BOX_TOO_SMALL = -6
SP_ERR_NO_DEVICE = -7
SP_ERR_TIMEOUT = -8
_STATUS = {0: "SP_OK", -1: "SP_ERR_INVALID_ARG", -2: "SP_ERR_CUDA", -3: "SP_ERR_NOT_CONVERGED",
           -4: "SP_ERR_NONFINITE", -5: "SP_ERR_OOM", -6: "SP_ERR_BOX_TOO_SMALL", -7: "SP_ERR_NO_DEVICE",
           -8: "SP_ERR_TIMEOUT"}

PREC = {"fp64": 0, "mixed": 1}
WARM = {"none": 0, "prev": 1}


class ShearsimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class sp_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("L", ctypes.c_double * 3), ("rc", ctypes.c_double),
                ("alpha", ctypes.c_double), ("eps", ctypes.c_double), ("zeta", ctypes.c_double),
                ("kT", ctypes.c_double), ("kappa", ctypes.c_double), ("dt", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("precision", ctypes.c_int32), ("warm_start", ctypes.c_int32),
                ("cg_tol", ctypes.c_double), ("cg_max_iter", ctypes.c_int32), ("device", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class sp_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("residual", ctypes.c_double),
                ("bnorm", ctypes.c_double), ("offchip_blocks", ctypes.c_int32), ("host_driven", ctypes.c_int32)]


class sp_step_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("max_iterations", ctypes.c_int32), ("steps_done", ctypes.c_int64),
                ("cg_iterations", ctypes.c_int64), ("last_residual", ctypes.c_double),
                ("stress_xy", ctypes.c_double), ("kernel_launches", ctypes.c_int64), ("delta", ctypes.c_double),
                ("step", ctypes.c_int64), ("host_driven", ctypes.c_int32)]


class sp_kernel_profile(ctypes.Structure):
    _fields_ = [("spmv_launches", ctypes.c_int32), ("update_launches", ctypes.c_int32),
                ("direction_launches", ctypes.c_int32), ("true_residual_launches", ctypes.c_int32),
                ("spmv_ms", ctypes.c_double), ("update_ms", ctypes.c_double), ("direction_ms", ctypes.c_double),
                ("true_residual_ms", ctypes.c_double), ("build_ms", ctypes.c_double), ("other_ms", ctypes.c_double),
                ("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("cg_iterations", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("sort_ms", ctypes.c_double), ("count_ms", ctypes.c_double),
                ("fill_ms", ctypes.c_double), ("nnz_slots", ctypes.c_int64), ("probe_reps", ctypes.c_int32),
                ("spmv_probe_ms", ctypes.c_double), ("update_probe_ms", ctypes.c_double),
                ("persistent_ms", ctypes.c_double), ("true_checks", ctypes.c_int32),
                ("persistent_blocks", ctypes.c_int32), ("init_ms", ctypes.c_double), ("stress_ms", ctypes.c_double),
                ("integrate_ms", ctypes.c_double), ("mpnn_ms", ctypes.c_double),
                ("assemble_ms", ctypes.c_double), ("persistent_init", ctypes.c_int32)]


class sp_vcorr_info(ctypes.Structure):
    _fields_ = [("pairs_ms", ctypes.c_double), ("boundary_pairs", ctypes.c_int64), ("pairs", ctypes.c_int64)]


class sp_tune_info(ctypes.Structure):
    _fields_ = [("config", ctypes.c_int32), ("gathers_in_flight", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("from_cache", ctypes.c_int32), ("num_configs", ctypes.c_int32), ("ms", ctypes.c_double * 12),
                ("pipelined", ctypes.c_int32), ("block_threads", ctypes.c_int32), ("resident", ctypes.c_int32),
                ("matrix_free", ctypes.c_int32)]


def declared_symbols() -> list:
    """Entry points declared in include/shearsim.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|int64_t|double|const char\*)\s+(sp_[a-z0-9_]+)\s*\(", text, re.M)))


_lib = None


def load(path: str = LIB_PATH):
    """Load libshearsim.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libshearsim.so is not built ({path}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(path)
    P, vp = ctypes.POINTER, ctypes.c_void_p
    i32, i64, u64, d = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sims = [("sp_sim_create", [P(sp_params), vp, P(vp)]), ("sp_sim_destroy", [vp]),
            ("sp_build_neighbors", [vp]), ("sp_assemble", [vp]),
            ("sp_solve_velocities", [vp, vp, P(sp_solve_info)]), ("sp_solve_flexible", [vp, i32, P(sp_solve_info)]), ("sp_step", [vp, i32, P(sp_step_info)]),
            ("sp_step_host", [vp, vp, ctypes.c_double, i32, vp, P(sp_step_info)]),
            ("sp_structure_factor", [vp, i32, i32, i32, vp, vp, vp]), ("sp_stress_xy", [vp, P(d)]),
            ("sp_velocity_correlation", [vp, i32, d, vp, vp, P(d), P(sp_vcorr_info)]),
            ("sp_sqrt_apply", [vp, i32, vp, vp, P(d), P(d)]), ("sp_set_fdt_noise", [vp, i32]),
            ("sp_velocity_correlation_host", [i32, i64, vp, d, d, vp, vp, i32, d, vp, vp, P(d), P(sp_vcorr_info)]),
            ("sp_get_positions", [vp, vp]), ("sp_set_positions", [vp, vp, d]), ("sp_get_velocities", [vp, vp]),
            ("sp_get_state", [vp, P(d), P(i64)]), ("sp_set_step", [vp, i64]), ("sp_get_order", [vp, vp]),
            ("sp_set_wait_limit", [vp, d]), ("sp_device_code_version", [i32, P(i32), P(i32)]),
            ("sp_get_num_pairs", [vp, P(i64)]), ("sp_get_neighbors", [vp, i64, vp, P(i64)]),
            ("sp_get_system", [vp, vp, vp, vp]), ("sp_set_noise", [vp, vp]),
            ("sp_philox_blocks", [i32, u64, u64, i64, vp, vp]),
            ("sp_normals", [i32, u64, u64, i64, vp, i32, vp]),
            ("sp_profile_step", [vp, P(sp_kernel_profile)]), ("sp_autotune", [vp, i32, P(sp_tune_info)]),
            ("sp_solve_csr_noalloc", [i32, vp, i64, vp, vp, vp, vp, d, vp, vp, d, i32, P(sp_solve_info)]),
            ("sp_batch_create", [i32, vp, vp, P(vp)]), ("sp_batch_destroy", [vp]),
            ("sp_batch_step", [vp, i32, vp]), ("sp_batch_get_sim", [vp, i32, P(vp)]),
            ("sp_batch_blocks", [vp, vp]), ("sp_batch_autotune", [vp, i32, P(sp_tune_info)]),
            ("sp_batch_set_config", [vp, i32]),
            ("sp_mpnn_enable", [vp, u64, vp]), ("sp_mpnn_disable", [vp]), ("sp_mpnn_get_weights", [vp, vp]),
            ("sp_mpnn_set_prior", [vp, i32]),
            ("sp_mpnn_set_weights", [vp, vp]), ("sp_mpnn_forward", [vp, vp]),
            ("sp_mpnn_train_step", [vp, ctypes.c_float, P(d), vp])]
    for name, args in sims:
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.sp_last_error.argtypes = [vp]
    lib.sp_last_error.restype = ctypes.c_char_p
    lib.sp_batch_last_error.argtypes = [vp]
    lib.sp_batch_last_error.restype = ctypes.c_char_p
    lib.sp_mpnn_num_params.argtypes = []
    lib.sp_mpnn_num_params.restype = ctypes.c_int
    lib.sp_kappa_from_kappa_tau.argtypes = [d, d, d, d]
    lib.sp_kappa_from_kappa_tau.restype = d
    lib.sp_state_record_bytes.argtypes = []
    lib.sp_state_record_bytes.restype = ctypes.c_int64
    _lib = lib
    return lib


def _check(rc: int, handle=None):
    if rc != SP_OK:
        msg = load().sp_last_error(handle)
        raise ShearsimError(rc, msg.decode() if msg else "")


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def device_code_version(device: int = 0) -> tuple:
    """(binary, ptx) architecture versions of the device code this library runs on `device`."""
    b, p = ctypes.c_int32(), ctypes.c_int32()
    _check(load().sp_device_code_version(int(device), ctypes.byref(b), ctypes.byref(p)))
    return b.value, p.value


def kappa_from_kappa_tau(kappa_tau: float, rc: float = 1.0, zeta: float = 1.0, kT: float = 1.0) -> float:
    return load().sp_kappa_from_kappa_tau(kappa_tau, rc, zeta, kT)


def philox_blocks(seed: int, step: int, ids, device: int = 0) -> np.ndarray:
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    out = np.zeros((ids.shape[0], 4), dtype=np.uint64)
    _check(load().sp_philox_blocks(device, seed, step, ids.shape[0], _p(ids), _p(out)))
    return out


def normals(seed: int, step: int, ids, precision: str = "mixed", device: int = 0) -> np.ndarray:
    """The thermal normals [n, 3] of particle ids at a step, as a simulation of that precision draws them."""
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    out = np.zeros((ids.shape[0], 3))
    prec = {"fp64": 0, "mixed": 1}[precision]
    _check(load().sp_normals(device, seed, step, ids.shape[0], _p(ids), prec, _p(out)))
    return out


def _vcorr_out(sums, counts, vsq, info) -> dict:
    with np.errstate(invalid="ignore", divide="ignore"):
        corr = sums / (counts * vsq)
    return {"sums": sums, "counts": counts, "vsq": vsq, "correlation": corr, "pairs_ms": info.pairs_ms,
            "boundary_pairs": info.boundary_pairs, "pairs": info.pairs}


def velocity_correlation(pos, v, L, delta: float, kappa: float, nbins: int, rmax: float, device: int = 0) -> dict:
    """Fig. vv for given positions [n, 3] (each coordinate in [0, L_a)) and velocities [n, 3]:
    per-bin sums of u_c . u_c', pair counts, <|u|^2> and their ratio (sp_velocity_correlation_host)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    Lc = np.ascontiguousarray(L, dtype=np.float64)
    sums, counts = np.zeros(nbins), np.zeros(nbins, dtype=np.int64)
    vsq = ctypes.c_double()
    info = sp_vcorr_info()
    _check(load().sp_velocity_correlation_host(device, pos.shape[0], _p(Lc), float(delta), float(kappa), _p(pos),
                                               _p(v), int(nbins), float(rmax), _p(sums), _p(counts),
                                               ctypes.byref(vsq), ctypes.byref(info)))
    return _vcorr_out(sums, counts, vsq.value, info)


NOALLOC_MAX_ROWS = 32768


def solve_csr_noalloc(n: int, row_ptr_ptr: int, col_ptr: int, w_ptr: int, diag_ptr: int, alpha: float,
                      b_ptr: int, x_ptr: int, tol: float = 1e-8, max_iter: int = 1000, device: int = 0,
                      stream=None) -> dict:
    """Allocation-free FP64 solve of (diag - alpha W) x = b for caller-owned device arrays
    given as raw pointers (CSR int32 row_ptr/col, float64 w/diag, float64 [3][n] b and x)."""
    info = sp_solve_info()
    rc = load().sp_solve_csr_noalloc(device, stream, n, row_ptr_ptr, col_ptr, w_ptr, diag_ptr, alpha, b_ptr,
                                     x_ptr, tol, max_iter, ctypes.byref(info))
    return {"status": rc, "iterations": info.iterations, "residual": info.residual, "bnorm": info.bnorm,
            "error": (load().sp_last_error(None) or b"").decode() if rc != SP_OK else ""}


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class Simulation:
    """One simulation on one GPU (see include/shearsim.h for the contract of each call)."""

    def __init__(self, n: int, L, kappa: float, alpha: float = 4.0, eps: float = 1.0, zeta: float = 1.0,
                 kT: float = 1.0, dt: float = 0.01, rc: float = 1.0, seed: int = 0, precision: str = "fp64",
                 warm_start: str = "prev", cg_tol: float = 1e-8, cg_max_iter: int = 1000, device: int = 0,
                 stream=None, positions=None, use_torch_stream: bool = True):
        lib = load()
        p = sp_params()
        p.n = int(n)
        for a in range(3):
            p.L[a] = float(L[a])
        p.rc, p.alpha, p.eps, p.zeta, p.kT, p.kappa, p.dt = rc, alpha, eps, zeta, kT, kappa, dt
        p.seed = int(seed)
        p.precision = PREC[precision]
        p.warm_start = WARM[warm_start]
        p.cg_tol = cg_tol
        p.cg_max_iter = cg_max_iter
        p.device = device
        if stream is None and use_torch_stream:
            stream = _torch_stream()
        p.stream = stream
        self.n = int(n)
        self.L = tuple(float(x) for x in L)
        self.params = p
        self._borrowed = False
        pos = None
        if positions is not None:
            pos = np.ascontiguousarray(positions, dtype=np.float64).reshape(self.n, 3)
        h = ctypes.c_void_p()
        _check(lib.sp_sim_create(ctypes.byref(p), _p(pos) if pos is not None else None, ctypes.byref(h)))
        self._h = h

    @staticmethod
    def make_params(n, L, kappa, alpha=4.0, eps=1.0, zeta=1.0, kT=1.0, dt=0.01, rc=1.0, seed=0,
                    precision="mixed", warm_start="prev", cg_tol=1e-8, cg_max_iter=1000, device=0) -> sp_params:
        p = sp_params()
        p.n = int(n)
        for a in range(3):
            p.L[a] = float(L[a])
        p.rc, p.alpha, p.eps, p.zeta, p.kT, p.kappa, p.dt = rc, alpha, eps, zeta, kT, kappa, dt
        p.seed = int(seed)
        p.precision = PREC[precision]
        p.warm_start = WARM[warm_start]
        p.cg_tol = cg_tol
        p.cg_max_iter = cg_max_iter
        p.device = device
        p.stream = None
        return p

    @classmethod
    def borrowed(cls, handle, n, L) -> "Simulation":
        """A view of a simulation owned elsewhere (a batch replica); close() does not free it."""
        self = cls.__new__(cls)
        self._h = ctypes.c_void_p(handle)
        self._borrowed = True
        self.n = int(n)
        self.L = tuple(float(x) for x in L)
        return self

    # lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value and not getattr(self, "_borrowed", False):
            load().sp_sim_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _c(self, rc):
        _check(rc, self._h)

    # the path
    def build_neighbors(self):
        self._c(load().sp_build_neighbors(self._h))

    def assemble(self):
        self._c(load().sp_assemble(self._h))

    def solve_velocities(self, v0_dev_ptr=None, raise_on_error: bool = True) -> dict:
        info = sp_solve_info()
        rc = load().sp_solve_velocities(self._h, v0_dev_ptr, ctypes.byref(info))
        if raise_on_error:
            self._c(rc)
        return {"status": rc, "iterations": info.iterations, "residual": info.residual, "bnorm": info.bnorm,
                "offchip_blocks": info.offchip_blocks, "host_driven": info.host_driven}

    def solve_flexible(self, net_every: int = 0, raise_on_error: bool = True) -> dict:
        """FCG(1) in FP64, the network as preconditioner every net_every iterations (0: Jacobi)."""
        info = sp_solve_info()
        rc = load().sp_solve_flexible(self._h, int(net_every), ctypes.byref(info))
        if raise_on_error:
            self._c(rc)
        return {"status": rc, "iterations": info.iterations, "residual": info.residual, "bnorm": info.bnorm,
                "host_driven": info.host_driven}

    def step(self, nsteps: int = 1, raise_on_error: bool = True) -> dict:
        info = sp_step_info()
        rc = load().sp_step(self._h, int(nsteps), ctypes.byref(info))
        if raise_on_error:
            self._c(rc)
        return {"status": rc, "steps_done": info.steps_done, "cg_iterations": info.cg_iterations,
                "max_iterations": info.max_iterations, "last_residual": info.last_residual,
                "stress_xy": info.stress_xy, "kernel_launches": info.kernel_launches, "delta": info.delta,
                "step": info.step, "host_driven": info.host_driven}

    def step_host(self, pos_in, delta: float, nsteps: int, pos_out, raise_on_error: bool = True) -> dict:
        """sp_step_host: host positions [n][3] (by id) and offset in, nsteps steps, positions out."""
        assert pos_in.dtype == np.float64 and pos_in.flags["C_CONTIGUOUS"] and pos_in.shape == (self.n, 3)
        assert pos_out.dtype == np.float64 and pos_out.flags["C_CONTIGUOUS"] and pos_out.shape == (self.n, 3)
        info = sp_step_info()
        rc = load().sp_step_host(self._h, _p(pos_in), float(delta), int(nsteps), _p(pos_out), ctypes.byref(info))
        if raise_on_error:
            self._c(rc)
        return {"status": rc, "steps_done": info.steps_done, "cg_iterations": info.cg_iterations,
                "max_iterations": info.max_iterations, "last_residual": info.last_residual,
                "stress_xy": info.stress_xy, "kernel_launches": info.kernel_launches, "delta": info.delta,
                "step": info.step, "host_driven": info.host_driven}

    def structure_factor(self, nkx: int, nky: int, grid: int = 256):
        m = (2 * nkx + 1) * (2 * nky + 1)
        S, qx, qy = np.zeros(m), np.zeros(m), np.zeros(m)
        self._c(load().sp_structure_factor(self._h, nkx, nky, grid, _p(S), _p(qx), _p(qy)))
        shape = (2 * nkx + 1, 2 * nky + 1)
        return S.reshape(shape), qx.reshape(shape), qy.reshape(shape)

    def profile_step(self) -> dict:
        prof = sp_kernel_profile()
        self._c(load().sp_profile_step(self._h, ctypes.byref(prof)))
        return {name: getattr(prof, name) for name, _ in sp_kernel_profile._fields_}

    def set_solver_config(self, config: int) -> dict:
        """Select a tile configuration of the persistent solver without timing (sp_set_solver_config)."""
        info = sp_tune_info()
        self._c(load().sp_set_solver_config(self._h, int(config), ctypes.byref(info)))
        return {"config": info.config, "gathers_in_flight": info.gathers_in_flight,
                "blocks_per_sm": info.blocks_per_sm, "pipelined": bool(info.pipelined),
                "block_threads": info.block_threads, "resident": bool(info.resident),
                "matrix_free": bool(info.matrix_free),
                "num_configs": info.num_configs}

    def autotune(self, trials: int = 3) -> dict:
        """Pick the persistent solver's fastest tile configuration for this system (sp_autotune)."""
        info = sp_tune_info()
        self._c(load().sp_autotune(self._h, int(trials), ctypes.byref(info)))
        return {"config": info.config, "gathers_in_flight": info.gathers_in_flight,
                "blocks_per_sm": info.blocks_per_sm, "pipelined": bool(info.pipelined),
                "block_threads": info.block_threads, "resident": bool(info.resident),
                "matrix_free": bool(info.matrix_free),
                "from_cache": bool(info.from_cache),
                "ms": [info.ms[k] for k in range(info.num_configs)]}

    # learned warm start
    def mpnn_enable(self, seed: int = 0, weights=None):
        if weights is None:
            self._c(load().sp_mpnn_enable(self._h, int(seed), None))
        else:
            w = np.ascontiguousarray(weights, dtype=np.float32)
            self._c(load().sp_mpnn_enable(self._h, int(seed), _p(w)))

    def mpnn_set_prior(self, use_vprev: bool):
        """Whether the network's previous-velocity feature is the previous velocities (True) or 0."""
        self._c(load().sp_mpnn_set_prior(self._h, 1 if use_vprev else 0))

    def mpnn_disable(self):
        self._c(load().sp_mpnn_disable(self._h))

    def mpnn_weights(self) -> np.ndarray:
        w = np.zeros(load().sp_mpnn_num_params(), dtype=np.float32)
        self._c(load().sp_mpnn_get_weights(self._h, _p(w)))
        return w

    def mpnn_set_weights(self, weights):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        self._c(load().sp_mpnn_set_weights(self._h, _p(w)))

    def mpnn_forward(self) -> np.ndarray:
        g = np.zeros((self.n, 3))
        self._c(load().sp_mpnn_forward(self._h, _p(g)))
        return g

    def mpnn_train_step(self, lr: float = 1e-3, want_grad: bool = False):
        loss = ctypes.c_double()
        grad = np.zeros(load().sp_mpnn_num_params(), dtype=np.float32) if want_grad else None
        self._c(load().sp_mpnn_train_step(self._h, float(lr), ctypes.byref(loss),
                                          _p(grad) if grad is not None else None))
        return (loss.value, grad) if want_grad else loss.value

    def sqrt_apply(self, g, degree: int = 32, timing: bool = False):
        """xi = p(A) g ~ A^(1/2) g for the assembled system (Chebyshev degree `degree` on
        [1, Gershgorin max]; sp_sqrt_apply).  g: [n, 3] in particle order.  Returns
        (xi, lambda_max), and the degree steps' device time in ms when timing is set."""
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(self.n, 3)
        xi = np.zeros_like(g)
        lmax, ms = ctypes.c_double(), ctypes.c_double()
        self._c(load().sp_sqrt_apply(self._h, int(degree), _p(g), _p(xi), ctypes.byref(lmax), ctypes.byref(ms)))
        return (xi, lmax.value, ms.value) if timing else (xi, lmax.value)

    def set_fdt_noise(self, degree: int):
        """Steps with A^(1/2)-correlated noise (Chebyshev degree `degree`; 0: independent noise)."""
        self._c(load().sp_set_fdt_noise(self._h, int(degree)))

    def velocity_correlation(self, nbins: int, rmax: float) -> dict:
        """Fig. vv on the current positions and the last solve's velocities (sp_velocity_correlation)."""
        sums, counts = np.zeros(nbins), np.zeros(nbins, dtype=np.int64)
        vsq = ctypes.c_double()
        info = sp_vcorr_info()
        self._c(load().sp_velocity_correlation(self._h, int(nbins), float(rmax), _p(sums), _p(counts),
                                               ctypes.byref(vsq), ctypes.byref(info)))
        return _vcorr_out(sums, counts, vsq.value, info)

    def stress_xy(self) -> float:
        v = ctypes.c_double()
        self._c(load().sp_stress_xy(self._h, ctypes.byref(v)))
        return v.value

    # state access
    def get_positions(self, out=None) -> np.ndarray:
        out = np.zeros((self.n, 3)) if out is None else out
        self._c(load().sp_get_positions(self._h, _p(out)))
        return out

    def set_positions(self, pos, delta: float = 0.0):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        self._c(load().sp_set_positions(self._h, _p(pos), float(delta)))

    def get_velocities(self, out=None) -> np.ndarray:
        out = np.zeros((self.n, 3)) if out is None else out
        self._c(load().sp_get_velocities(self._h, _p(out)))
        return out

    def state(self):
        d, s = ctypes.c_double(), ctypes.c_int64()
        self._c(load().sp_get_state(self._h, ctypes.byref(d), ctypes.byref(s)))
        return d.value, s.value

    def set_step(self, step: int):
        self._c(load().sp_set_step(self._h, int(step)))

    def set_wait_limit(self, seconds: float):
        """Limit of one device-side grid-barrier wait of the persistent solvers (default 2 s)."""
        self._c(load().sp_set_wait_limit(self._h, float(seconds)))

    def order(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int64)
        self._c(load().sp_get_order(self._h, _p(out)))
        return out

    def num_pairs(self) -> int:
        m = ctypes.c_int64()
        self._c(load().sp_get_num_pairs(self._h, ctypes.byref(m)))
        return m.value

    def neighbors(self) -> np.ndarray:
        """Pairs (i < j by id) sorted by (i, j)."""
        m = self.num_pairs()
        out = np.zeros((max(m, 1), 2), dtype=np.int64)
        got = ctypes.c_int64()
        self._c(load().sp_get_neighbors(self._h, m, _p(out), ctypes.byref(got)))
        pairs = out[: got.value]
        return pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]

    def system(self):
        """(diag [n], b [n, 3], pairs [m, 2] sorted, w [m]) by particle id."""
        m = self.num_pairs()
        diag, b, w = np.zeros(self.n), np.zeros((self.n, 3)), np.zeros(max(m, 1))
        out = np.zeros((max(m, 1), 2), dtype=np.int64)
        got = ctypes.c_int64()
        self._c(load().sp_get_neighbors(self._h, m, _p(out), ctypes.byref(got)))
        self._c(load().sp_get_system(self._h, _p(diag), _p(b), _p(w)))
        pairs, w = out[: got.value], w[: got.value]
        order = np.lexsort((pairs[:, 1], pairs[:, 0]))
        return diag, b, pairs[order], w[order]

    def set_noise(self, xi=None):
        if xi is None:
            self._c(load().sp_set_noise(self._h, None))
        else:
            xi = np.ascontiguousarray(xi, dtype=np.float64)
            self._c(load().sp_set_noise(self._h, _p(xi)))


class Batch:
    """Independent replicas advanced together (sp_batch_*): one graph per step with one
    cooperative launch solving every replica's velocities."""

    def __init__(self, replicas, positions=None):
        """replicas: list of dicts of Simulation.make_params arguments (precision is mixed)."""
        lib = load()
        self.R = len(replicas)
        arr = (sp_params * self.R)()
        self._shapes = []
        for k, kw in enumerate(replicas):
            kw = dict(kw)
            kw.setdefault("precision", "mixed")
            arr[k] = Simulation.make_params(**kw)
            self._shapes.append((int(kw["n"]), tuple(kw["L"])))
        self._keep = []
        pos_arr = None
        if positions is not None:
            pos_arr = (ctypes.c_void_p * self.R)()
            for k, pos in enumerate(positions):
                if pos is None:
                    pos_arr[k] = None
                else:
                    a = np.ascontiguousarray(pos, dtype=np.float64)
                    self._keep.append(a)
                    pos_arr[k] = a.ctypes.data
        h = ctypes.c_void_p()
        rc = lib.sp_batch_create(self.R, ctypes.cast(arr, ctypes.c_void_p),
                                 ctypes.cast(pos_arr, ctypes.c_void_p) if pos_arr is not None else None,
                                 ctypes.byref(h))
        if rc != SP_OK:
            raise ShearsimError(rc, (lib.sp_batch_last_error(None) or b"").decode())
        self._h = h

    def step(self, nsteps: int = 1, raise_on_error: bool = True) -> list:
        infos = (sp_step_info * self.R)()
        rc = load().sp_batch_step(self._h, int(nsteps), ctypes.cast(infos, ctypes.c_void_p))
        if raise_on_error and rc != SP_OK:
            raise ShearsimError(rc, (load().sp_batch_last_error(self._h) or b"").decode())
        return [{"status": x.status, "steps_done": x.steps_done, "cg_iterations": x.cg_iterations,
                 "max_iterations": x.max_iterations, "last_residual": x.last_residual,
                 "stress_xy": x.stress_xy, "kernel_launches": x.kernel_launches, "delta": x.delta,
                 "step": x.step} for x in infos]

    def sim(self, k: int) -> Simulation:
        h = ctypes.c_void_p()
        _check(load().sp_batch_get_sim(self._h, int(k), ctypes.byref(h)))
        n, L = self._shapes[k]
        return Simulation.borrowed(h.value, n, L)

    def blocks(self) -> np.ndarray:
        out = np.zeros(self.R, dtype=np.int32)
        _check(load().sp_batch_blocks(self._h, _p(out)))
        return out

    def autotune(self, trials: int = 2) -> dict:
        """Time the batched solver's tile configurations on the current systems; keep the fastest."""
        info = sp_tune_info()
        rc = load().sp_batch_autotune(self._h, int(trials), ctypes.byref(info))
        if rc != SP_OK:
            raise ShearsimError(rc, (load().sp_batch_last_error(self._h) or b"").decode())
        return {"config": info.config, "gathers_in_flight": info.gathers_in_flight,
                "blocks_per_sm": info.blocks_per_sm, "block_threads": info.block_threads,
                "num_configs": info.num_configs, "ms": list(info.ms)[: info.num_configs]}

    def set_config(self, config: int):
        rc = load().sp_batch_set_config(self._h, int(config))
        if rc != SP_OK:
            raise ShearsimError(rc, (load().sp_batch_last_error(self._h) or b"").decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().sp_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
