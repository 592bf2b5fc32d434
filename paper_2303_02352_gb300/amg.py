"""Thin Python binding of libamg (the C ABI declared in include/amg.h).

Argument marshalling only: every step of the setup and the solve runs in the
library's CUDA kernels.  PyTorch provides device memory and the stream.  If the
library has not been built, loading fails with an error (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_build", "libamg.so")

OK, NOT_CONVERGED = 0, 1
ERR_INVALID_ARG, ERR_NOT_SPD, ERR_BREAKDOWN, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_TOO_LARGE = -1, -2, -3, -4, -5, -6, -7
FP64, FP32, FP32_BF16FINE = 0, 1, 2
(K_SWEEP, K_RESIDUAL, K_RESTRICT, K_PROLONG, K_SPMV_DOTS, K_AXPY, K_RESTRICT_FIRST, K_SWEEP_PROLONG,
 K_SWEEP_PAIR) = range(9)

_STATUS = {0: "AMG_OK", 1: "AMG_NOT_CONVERGED", -1: "AMG_ERR_INVALID_ARG", -2: "AMG_ERR_NOT_SPD",
           -3: "AMG_ERR_BREAKDOWN", -4: "AMG_ERR_CUDA", -5: "AMG_ERR_OOM", -6: "AMG_ERR_TIMEOUT",
           -7: "AMG_ERR_TOO_LARGE"}


class AmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class amg_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


PARAM_FIELDS = ("aggr_steps", "max_levels", "coarse_size", "pre_sweeps", "post_sweeps", "coarse_sweeps",
                "precision", "true_res_every", "use_graph", "graph_batch", "num_parts", "cycle", "relax_type",
                "prolong_scale")


class amg_params(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in PARAM_FIELDS]


class amg_info_t(ctypes.Structure):
    _fields_ = [("num_levels", ctypes.c_int32), ("n", ctypes.c_int32 * 40), ("nnz", ctypes.c_int64 * 40),
                ("opc", ctypes.c_double), ("num_pairwise", ctypes.c_int32), ("setup_ms", ctypes.c_double),
                ("vcycle_bytes", ctypes.c_double), ("iteration_bytes", ctypes.c_double),
                ("vcycle_launches", ctypes.c_int32), ("iteration_launches", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("setup_match_ms", ctypes.c_double),
                ("setup_galerkin_ms", ctypes.c_double), ("bottom_level", ctypes.c_int32),
                ("tile_rows", ctypes.c_int32 * 40), ("stage_scale", ctypes.c_int32 * 40),
                ("setup_spgemm_ms", ctypes.c_double), ("last_solve_launches", ctypes.c_int32),
                ("consumer_groups", ctypes.c_int32 * 40), ("column_patterns", ctypes.c_int32 * 40),
                ("outer_patterns", ctypes.c_int32), ("column_form", ctypes.c_int32 * 40),
                ("outer_column_form", ctypes.c_int32)]


_LIB = None


def load(path: str | None = None):
    """Loads libamg.so (raises if it is missing: there is no fallback path)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or os.environ.get("AMG_LIB") or SO_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libamg.so not found at {path}: build it with paper_2303_02352_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I32, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    I32P, DP = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)
    sig = {
        "amg_params_default": (None, [ctypes.POINTER(amg_params)]),
        "amg_setup": (I32, [ctypes.POINTER(amg_csr), ctypes.POINTER(amg_params), P, ctypes.POINTER(P)]),
        "amg_pcg_solve": (I32, [P, P, P, D, I32, I32P, DP, DP]),
        "amg_pcg_solve_host": (I32, [P, P, P, D, I32, I32P, DP, DP]),
        "amg_cg_solve": (I32, [P, P, P, D, I32, I32P, DP, DP]),
        "amg_vcycle": (I32, [P, P, P]),
        "amg_spmv": (I32, [P, I32, P, P]),
        "amg_info": (I32, [P, ctypes.POINTER(amg_info_t)]),
        "amg_get_aggregates": (I32, [P, I32, P]),
        "amg_get_level_csr": (I32, [P, I32, P, P, P]),
        "amg_get_l1": (I32, [P, I32, P]),
        "amg_time_vcycle": (I32, [P, I32, DP]),
        "amg_time_kernel": (I32, [P, I32, I32, I32, DP]),
        "amg_kernel_bytes": (I32, [P, I32, I32, DP]),
        "amg_residual_norm_noalloc": (I32, [ctypes.POINTER(amg_csr), P, P, P, P, P]),
        "amg_check_bounded_wait": (I32, [I32, P]),
        "amg_spgemm": (I32, [I32, I32, I32, P, P, P, P, P, P, P, P, P, ctypes.POINTER(ctypes.c_int64), P]),
        "amg_stencil_size": (I32, [I32, I32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
        "amg_generate_stencil": (I32, [I32, I32, P, I32, P, P, P, P]),
        "amg_random_vector": (I32, [ctypes.c_int64, ctypes.c_uint64, P, P]),
        "amg_csr_times": (I32, [ctypes.POINTER(amg_csr), P, P, P]),
        "amg_features": (I32, [P, I32, P]),
        "amg_set_omega": (I32, [P, I32, P]),
        "amg_mlp_workspace_bytes": (ctypes.c_size_t, [I32]),
        "amg_mlp_forward": (I32, [I32, P, P, P, P]),
        "amg_mlp_backward": (I32, [I32, P, P, P, P, P, P]),
        "amg_adam_step": (I32, [I32, P, P, P, P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, I32, P]),
        "amg_apply_mlp": (I32, [P, P]),
        "amg_vcycle_backward": (I32, [P, P, P, P, P]),
        "amg_vcycle_loss": (I32, [P, P, I32, DP, P]),
        "amg_save": (I32, [P, ctypes.c_char_p]),
        "amg_load": (I32, [ctypes.c_char_p, ctypes.POINTER(amg_params), P, ctypes.POINTER(P)]),
        "amg_saved_params": (I32, [ctypes.c_char_p, ctypes.POINTER(amg_params)]),
        "amg_last_error": (ctypes.c_char_p, [P]),
        "amg_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def params_default(**overrides) -> amg_params:
    p = amg_params()
    load().amg_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if k not in PARAM_FIELDS:
            raise KeyError(f"unknown parameter {k}")
        setattr(p, k, int(v))
    return p


def _ptr(t) -> int:
    return t.data_ptr()


class Hierarchy:
    """An AMG hierarchy on the GPU (handle of amg_setup) and its solve phase.

    ``A``: a CSR with ``n``, ``row_ptr``, ``col_idx``, ``val`` (numpy or torch;
    copied to the GPU) or a ``torch.sparse_csr_tensor`` of float64 on CUDA.
    Keyword arguments override the fields of ``amg_params``.
    """

    def __init__(self, A, stream=None, **params):
        import torch
        self._torch = torch
        sparse = isinstance(A, torch.Tensor) and A.layout == torch.sparse_csr
        if sparse:
            if A.dim() != 2 or A.shape[0] != A.shape[1]:
                raise ValueError(f"A must be a square matrix, got shape {tuple(A.shape)}")
            if A.values().numel() >= 2 ** 31:
                raise ValueError("A has 2^31 or more stored entries (int32 indices)")
        lib = load()
        self._lib = lib
        dev = torch.device("cuda", torch.cuda.current_device())
        if sparse:
            rp = A.crow_indices().to(device=dev, dtype=torch.int32).contiguous()
            ci = A.col_indices().to(device=dev, dtype=torch.int32).contiguous()
            v = A.values().to(device=dev, dtype=torch.float64).contiguous()
            n = A.shape[0]
        else:
            def arr(x, dt_np, dt_t):  # host arrays or tensors on any device
                if isinstance(x, torch.Tensor):
                    return x.to(device=dev, dtype=dt_t).contiguous()
                return torch.as_tensor(np.asarray(x, dtype=dt_np)).to(dev)
            rp = arr(A.row_ptr, np.int32, torch.int32)
            ci = arr(A.col_idx, np.int32, torch.int32)
            v = arr(A.val, np.float64, torch.float64)
            n = int(A.n)
        self.n = n
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        csr = amg_csr(n, int(ci.numel()), _ptr(rp), _ptr(ci), _ptr(v))
        p = params_default(**params)
        self.params = {f: getattr(p, f) for f in PARAM_FIELDS}
        h = ctypes.c_void_p()
        st = lib.amg_setup(ctypes.byref(csr), ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != OK:
            raise AmgError(st, lib.amg_last_error(None).decode())
        self._h = h
        self.device = dev

    @classmethod
    def load(cls, path: str, stream=None, **params) -> "Hierarchy":
        """amg_load: a hierarchy saved with ``save``.  Keyword arguments change
        solve-phase fields of the saved parameters (sweeps, precision,
        true_res_every, use_graph, graph_batch, cycle, relax_type)."""
        import torch
        lib = load()
        self = cls.__new__(cls)
        self._torch, self._lib = torch, lib
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        bpath = os.fsencode(path)
        p = amg_params()
        st = lib.amg_saved_params(bpath, ctypes.byref(p))
        if st != OK:
            raise AmgError(st, lib.amg_last_error(None).decode())
        for k, v in params.items():
            if k not in PARAM_FIELDS:
                raise KeyError(f"unknown parameter {k}")
            setattr(p, k, int(v))
        h = ctypes.c_void_p()
        st = lib.amg_load(bpath, ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != OK:
            raise AmgError(st, lib.amg_last_error(None).decode())
        self._h = h
        self.params = {f: getattr(p, f) for f in PARAM_FIELDS}
        self.n = self.info()["n"][0]
        return self

    def save(self, path: str):
        """amg_save: writes the hierarchy to a file (``Hierarchy.load`` reads it)."""
        self._check(self._lib.amg_save(self._h, os.fsencode(path)))

    # -- lifetime -----------------------------------------------------------
    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._lib.amg_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=(OK,)):
        if st not in allow:
            raise AmgError(st, self._lib.amg_last_error(self._h).decode())
        return st

    # -- queries ------------------------------------------------------------
    def info(self) -> dict:
        inf = amg_info_t()
        self._check(self._lib.amg_info(self._h, ctypes.byref(inf)))
        L = inf.num_levels
        return {"num_levels": L, "n": list(inf.n[:L]), "nnz": list(inf.nnz[:L]), "opc": inf.opc,
                "num_pairwise": inf.num_pairwise, "setup_ms": inf.setup_ms, "vcycle_bytes": inf.vcycle_bytes,
                "iteration_bytes": inf.iteration_bytes, "vcycle_launches": inf.vcycle_launches,
                "iteration_launches": inf.iteration_launches, "precision": inf.precision,
                "setup_match_ms": inf.setup_match_ms, "setup_galerkin_ms": inf.setup_galerkin_ms,
                "bottom_level": inf.bottom_level, "tile_rows": list(inf.tile_rows[:L]),
                "stage_scale": list(inf.stage_scale[:L]), "setup_spgemm_ms": inf.setup_spgemm_ms,
                "last_solve_launches": inf.last_solve_launches, "consumer_groups": list(inf.consumer_groups[:L]),
                "column_patterns": list(inf.column_patterns[:L]), "outer_patterns": inf.outer_patterns,
                "column_form": list(inf.column_form[:L]), "outer_column_form": inf.outer_column_form}

    @property
    def num_levels(self) -> int:
        return self.info()["num_levels"]

    def aggregates(self, level: int) -> np.ndarray:
        n = self.info()["n"][level]
        out = np.zeros(n, np.int32)
        self._check(self._lib.amg_get_aggregates(self._h, level, out.ctypes.data))
        return out

    def level_csr(self, level: int):
        inf = self.info()
        n, nnz = inf["n"][level], inf["nnz"][level]
        rp, ci, v = np.zeros(n + 1, np.int32), np.zeros(nnz, np.int32), np.zeros(nnz, np.float64)
        self._check(self._lib.amg_get_level_csr(self._h, level, rp.ctypes.data, ci.ctypes.data, v.ctypes.data))
        return rp, ci, v

    def l1(self, level: int) -> np.ndarray:
        out = np.zeros(self.info()["n"][level], np.float64)
        self._check(self._lib.amg_get_l1(self._h, level, out.ctypes.data))
        return out

    # -- solve phase --------------------------------------------------------
    def _vec(self, x):
        t = self._torch
        return t.as_tensor(x, dtype=t.float64, device=self.device).contiguous()

    def pcg_solve(self, b, x0=None, tol=1e-6, maxit=1000, precond=True):
        """Alg. 1 on the GPU.  Returns dict(x, iters, hist, true_rel_res, status)."""
        t = self._torch
        b = self._vec(b)
        x = t.zeros_like(b) if x0 is None else self._vec(x0).clone()
        it = ctypes.c_int32(0)
        tr = ctypes.c_double(0.0)
        hist = np.zeros(maxit + 1)
        fn = self._lib.amg_pcg_solve if precond else self._lib.amg_cg_solve
        st = fn(self._h, _ptr(b), _ptr(x), tol, maxit, ctypes.byref(it), hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                ctypes.byref(tr))
        self._check(st, allow=(OK, NOT_CONVERGED, ERR_BREAKDOWN))
        return {"x": x, "iters": it.value, "hist": hist[: it.value + 1], "true_rel_res": tr.value, "status": st}

    def solve_into(self, b, x, tol=1e-6, maxit=1000, precond=True):
        """Alg. 1 on caller-owned device tensors (float64, contiguous); x: in u_0, out u."""
        assert b.dtype == self._torch.float64 and x.dtype == self._torch.float64
        it = ctypes.c_int32(0)
        tr = ctypes.c_double(0.0)
        fn = self._lib.amg_pcg_solve if precond else self._lib.amg_cg_solve
        st = fn(self._h, _ptr(b), _ptr(x), tol, maxit, ctypes.byref(it), None, ctypes.byref(tr))
        self._check(st, allow=(OK, NOT_CONVERGED, ERR_BREAKDOWN))
        return {"iters": it.value, "true_rel_res": tr.value, "status": st}

    def cg_solve(self, b, x0=None, tol=1e-6, maxit=1000):
        return self.pcg_solve(b, x0, tol, maxit, precond=False)

    def pcg_solve_host(self, b: np.ndarray, x: np.ndarray, tol=1e-6, maxit=1000, hist=None):
        """Alg. 1 with host vectors (copies inside the call).  x is updated in place."""
        assert b.dtype == np.float64 and x.dtype == np.float64 and b.flags.c_contiguous and x.flags.c_contiguous
        it = ctypes.c_int32(0)
        tr = ctypes.c_double(0.0)
        hp = None if hist is None else hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        st = self._lib.amg_pcg_solve_host(self._h, b.ctypes.data, x.ctypes.data, tol, maxit, ctypes.byref(it), hp,
                                          ctypes.byref(tr))
        self._check(st, allow=(OK, NOT_CONVERGED, ERR_BREAKDOWN))
        return {"iters": it.value, "true_rel_res": tr.value, "status": st}

    def vcycle(self, r):
        r = self._vec(r)
        z = self._torch.empty_like(r)
        self._check(self._lib.amg_vcycle(self._h, _ptr(r), _ptr(z)))
        return z

    def spmv(self, level, x):
        x = self._vec(x)
        y = self._torch.empty(self.info()["n"][level], dtype=self._torch.float64, device=self.device)
        self._check(self._lib.amg_spmv(self._h, level, _ptr(x), _ptr(y)))
        return y

    # -- learned damping ----------------------------------------------------
    def level_sizes(self):
        return self.info()["n"]

    def features(self, level):
        """The four row features of a level (device float32, n_k x 4)."""
        t = self._torch
        out = t.empty((self.info()["n"][level], 4), dtype=t.float32, device=self.device)
        self._check(self._lib.amg_features(self._h, level, _ptr(out)))
        return out

    def set_omega(self, level, omega=None):
        """Per-row damping of a level (device float64, n_k), None for omega = 1."""
        if omega is None:
            self._check(self._lib.amg_set_omega(self._h, level, None))
            return
        om = self._vec(omega)
        self._check(self._lib.amg_set_omega(self._h, level, _ptr(om)))

    def apply_mlp(self, w_bf16=None):
        """Features + network + damping on every level (None: back to omega = 1)."""
        self._check(self._lib.amg_apply_mlp(self._h, None if w_bf16 is None else _ptr(w_bf16)))

    def vcycle_backward(self, r, dz):
        """Adjoint of one FP64 V-cycle: (dL/dr, [dL/domega_k for every level])."""
        t = self._torch
        r, dz = self._vec(r), self._vec(dz)
        dr = t.empty_like(r)
        sizes = self.info()["n"]
        dom = [t.empty(nk, dtype=t.float64, device=self.device) for nk in sizes]
        ptrs = (ctypes.c_void_p * len(dom))(*[_ptr(d) for d in dom])
        self._check(self._lib.amg_vcycle_backward(self._h, _ptr(r), _ptr(dz), _ptr(dr), ptrs))
        return dr, dom

    def vcycle_loss(self, r0, m: int, grad: bool = True):
        """Training loss (1/m) ln(|r_m| / |r_0|), r_{t+1} = r_t - A B r_t, and, with
        grad, [dL/domega_k for every level] (device float64) from the library."""
        t = self._torch
        r0 = self._vec(r0)
        loss = ctypes.c_double(0.0)
        dom, ptrs = None, None
        if grad:
            dom = [t.empty(nk, dtype=t.float64, device=self.device) for nk in self.info()["n"]]
            ptrs = (ctypes.c_void_p * len(dom))(*[_ptr(d) for d in dom])
        self._check(self._lib.amg_vcycle_loss(self._h, _ptr(r0), int(m), ctypes.byref(loss), ptrs))
        return loss.value, dom

    # -- measurement --------------------------------------------------------
    def time_vcycle(self, reps=20) -> float:
        ms = ctypes.c_double(0.0)
        self._check(self._lib.amg_time_vcycle(self._h, reps, ctypes.byref(ms)))
        return ms.value

    def time_kernel(self, which, level=0, reps=20) -> float:
        ms = ctypes.c_double(0.0)
        self._check(self._lib.amg_time_kernel(self._h, which, level, reps, ctypes.byref(ms)))
        return ms.value

    def kernel_bytes(self, which, level=0) -> float:
        b = ctypes.c_double(0.0)
        self._check(self._lib.amg_kernel_bytes(self._h, which, level, ctypes.byref(b)))
        return b.value


def spgemm(a_row_ptr, a_col_idx, a_val, b_row_ptr, b_col_idx, b_val, ncols: int, stream=None):
    """amg_spgemm on device tensors (int32 / float64, contiguous): C = A B with
    A of len(a_row_ptr) - 1 rows, B of len(b_row_ptr) - 1 rows and ``ncols``
    columns.  Returns (row_ptr, col_idx, val) of C on the same device."""
    import torch
    lib = load()
    m, k = a_row_ptr.numel() - 1, b_row_ptr.numel() - 1
    dev = a_row_ptr.device
    s = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    crp = torch.empty(m + 1, dtype=torch.int32, device=dev)
    nnz = ctypes.c_int64(0)
    args = (m, k, int(ncols), _ptr(a_row_ptr), _ptr(a_col_idx), _ptr(a_val), _ptr(b_row_ptr), _ptr(b_col_idx),
            _ptr(b_val))
    st = lib.amg_spgemm(*args, _ptr(crp), None, None, ctypes.byref(nnz), s)
    if st != OK:
        raise AmgError(st, lib.amg_last_error(None).decode())
    cci = torch.empty(max(1, nnz.value), dtype=torch.int32, device=dev)
    cv = torch.empty(max(1, nnz.value), dtype=torch.float64, device=dev)
    st = lib.amg_spgemm(*args, _ptr(crp), _ptr(cci), _ptr(cv), ctypes.byref(nnz), s)
    if st != OK:
        raise AmgError(st, lib.amg_last_error(None).decode())
    return crp, cci[: nnz.value], cv[: nnz.value]


def _call(st, lib):
    if st != OK:
        raise AmgError(st, lib.amg_last_error(None).decode())


def generate_stencil(N: int, points: int = 7, kblock=None, block: int = 8, stream=None):
    """amg_generate_stencil: the N^3 stencil matrix (points 7 or 27) in device
    memory, as (row_ptr, col_idx, val) tensors.  kblock: the float32 values of
    the ceil(N/block)^3 coefficient blocks (host array), or None for the
    integer Poisson stencil (7 points)."""
    import torch
    lib = load()
    n, nnz = ctypes.c_int64(0), ctypes.c_int64(0)
    _call(lib.amg_stencil_size(int(N), int(points), ctypes.byref(n), ctypes.byref(nnz)), lib)
    dev = torch.device("cuda", torch.cuda.current_device())
    rp = torch.empty(n.value + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(nnz.value, dtype=torch.int32, device=dev)
    v = torch.empty(nnz.value, dtype=torch.float64, device=dev)
    kb = None if kblock is None else np.ascontiguousarray(kblock, dtype=np.float32)
    s = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    _call(lib.amg_generate_stencil(int(N), int(points), None if kb is None else kb.ctypes.data, int(block),
                                   _ptr(rp), _ptr(ci), _ptr(v), s), lib)
    return rp, ci, v


def random_vector(n: int, seed: int, stream=None):
    """amg_random_vector: x_i = 2 U_i - 1 from the SplitMix64 stream ``seed`` (device)."""
    import torch
    lib = load()
    out = torch.empty(int(n), dtype=torch.float64, device=torch.device("cuda", torch.cuda.current_device()))
    s = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    _call(lib.amg_random_vector(int(n), int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(out), s), lib)
    return out


def csr_times(rp, ci, v, x, stream=None):
    """amg_csr_times: y = A x (device), each row summed in column order."""
    import torch
    lib = load()
    y = torch.empty_like(x)
    a = amg_csr(rp.numel() - 1, ci.numel(), _ptr(rp), _ptr(ci), _ptr(v))
    s = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    _call(lib.amg_csr_times(ctypes.byref(a), _ptr(x), _ptr(y), s), lib)
    return y


def generate(name: str, stream=None):
    """A named stencil workload built on the device: ((row_ptr, col_idx, val),
    b, x*) with b = A x*, bit for bit the host generator's (workloads.config)."""
    import torch
    from . import workloads as W
    r = W.recipe(name)
    kb = None if r["sigma"] is None else W.block_values(r["N"], r["sigma"], r["seed"], r["block"])
    rp, ci, v = generate_stencil(r["N"], r["points"], kb, r["block"], stream)
    xs = random_vector(rp.numel() - 1, r["xseed"], stream)
    b = csr_times(rp, ci, v, xs, stream)
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return (rp, ci, v), b, xs


class DeviceCSR:
    """A device CSR (int32 / float64 tensors) accepted by Hierarchy."""

    def __init__(self, rp, ci, v):
        self.n, self.row_ptr, self.col_idx, self.val = rp.numel() - 1, rp, ci, v


# -- module-level calls (the Python form of amg_setup / amg_pcg_solve) ------
def setup(A, stream=None, **params) -> Hierarchy:
    """amg_setup: build the hierarchy of ``A`` (a ``torch.sparse_csr_tensor``
    of float64, on CUDA or host, or any object with ``n``, ``row_ptr``,
    ``col_idx``, ``val``).  Keyword arguments override ``amg_params`` fields.
    Raises AmgError when the setup fails."""
    return Hierarchy(A, stream=stream, **params)


def solve(h: Hierarchy, b, x0=None, tol=1e-6, maxit=1000):
    """amg_pcg_solve: Alg. 1 preconditioned by the hierarchy's cycle.
    Returns ``(x, iters, hist)``: the device solution (float64), the number
    of iterations and the host array ||r_i|| / ||b|| for i = 0..iters.  A run that stops
    at ``maxit`` without reaching ``tol`` still returns its iterate (status
    AMG_NOT_CONVERGED, available from ``h.pcg_solve``)."""
    out = h.pcg_solve(b, x0=x0, tol=tol, maxit=maxit)
    return out["x"], out["iters"], out["hist"]
