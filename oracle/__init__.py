"""CPU oracle of the AMG-preconditioned flexible CG (arXiv:2303.02352).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this package; the CUDA library never does and
shares no code with it.  The arithmetic lives in ``orc.c`` (plain FP64 C);
this module compiles it with gcc on first use and marshals numpy arrays.  The
serial build is the checker; the OpenMP build of the same source (``omp=True``)
is only the timed CPU baseline.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_SO_OMP = os.path.join(_BUILD, "liborc_omp.so")
_LOCK = threading.Lock()
_LIBS = {}

FP64, FP32, FP32_BF16FINE = 0, 1, 2
COARSE_L1JACOBI, COARSE_DENSE_CHOL = 0, 1
PROLONG_UNIT, PROLONG_W_NORMALIZED = 0, 1
OK, NOT_CONVERGED, ERR_ARG, ERR_BREAKDOWN = 0, 1, -1, -3


def build(force: bool = False, omp: bool = False) -> str:
    """Compile orc.c into _build/liborc.so (serial, the checker) or, with omp,
    _build/liborc_omp.so (the same source with its OpenMP row loops on: the
    timed CPU baseline).  No FMA contraction in either."""
    src = os.path.join(_HERE, "orc.c")
    so = _SO_OMP if omp else _SO
    if not force and os.path.exists(so) and os.path.getmtime(so) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "orc.h"))):
        return so
    os.makedirs(_BUILD, exist_ok=True)
    tmp = so + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"]
                          + (["-fopenmp"] if omp else []) + ["-o", tmp, src, "-lm"])
    os.replace(tmp, so)
    return so


class _Params(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int) for name in (
        "aggr_steps", "max_levels", "coarse_size", "pre_sweeps", "post_sweeps",
        "coarse_sweeps", "coarse_solver", "precision", "true_res_every", "num_parts", "cycle", "relax_type", "prolong_scale")]


def _lib(omp: bool = False):
    with _LOCK:
        if omp not in _LIBS:
            lib = ctypes.CDLL(build(omp=omp))
            P = ctypes.c_void_p
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            lib.orc_params_default.argtypes = [ctypes.POINTER(_Params)]
            lib.orc_weights.argtypes = [ctypes.c_int, i32p, i32p, f64p, f64p]
            lib.orc_match_greedy.argtypes = [ctypes.c_int, i32p, i32p, f64p, i32p]
            lib.orc_aggregate.argtypes = [ctypes.c_int, i32p, i32p]
            lib.orc_galerkin.argtypes = [ctypes.c_int, i32p, i32p, f64p, i32p, ctypes.c_int, P, P, P]
            lib.orc_galerkin.restype = ctypes.c_int64
            lib.orc_setup.argtypes = [ctypes.c_int, i32p, i32p, f64p, ctypes.POINTER(_Params)]
            lib.orc_setup.restype = P
            lib.orc_free.argtypes = [P]
            lib.orc_num_levels.argtypes = [P]
            lib.orc_level_n.argtypes = [P, ctypes.c_int]
            lib.orc_level_nnz.argtypes = [P, ctypes.c_int]
            lib.orc_level_nnz.restype = ctypes.c_int64
            lib.orc_level_csr.argtypes = [P, ctypes.c_int, i32p, i32p, f64p]
            lib.orc_level_agg.argtypes = [P, ctypes.c_int, i32p]
            lib.orc_level_l1.argtypes = [P, ctypes.c_int, f64p]
            lib.orc_num_pairwise.argtypes = [P]
            lib.orc_pairwise_n.argtypes = [P, ctypes.c_int]
            lib.orc_set_omega.argtypes = [P, ctypes.c_int, P]
            lib.orc_vcycle.argtypes = [P, f64p, f64p]
            lib.orc_spmv.argtypes = [P, ctypes.c_int, f64p, f64p]
            lib.orc_fcg.argtypes = [P, f64p, f64p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int), f64p, ctypes.POINTER(ctypes.c_double)]
            lib.orc_vcycle_loss.argtypes = [P, f64p, ctypes.c_int]
            lib.orc_vcycle_loss.restype = ctypes.c_double
            lib.orc_vcycle_loss_grad.argtypes = [P, f64p, ctypes.c_int, P]
            lib.orc_vcycle_loss_grad.restype = ctypes.c_double
            lib.orc_round_bf16.argtypes = [ctypes.c_float]
            lib.orc_round_bf16.restype = ctypes.c_float
            lib.orc_threads.argtypes = []
            _LIBS[omp] = lib
    return _LIBS[omp]


def threads(omp: bool = True) -> int:
    """Threads the row loops of the given build use (1 for the serial checker)."""
    return _lib(omp).orc_threads()


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def weights(rp, ci, v):
    """Matching weight of every stored entry (0 on the diagonal and on explicit zeros)."""
    rp, ci, v = _i32(rp), _i32(ci), _f64(v)
    out = np.zeros(len(ci), dtype=np.float64)
    if _lib().orc_weights(len(rp) - 1, rp, ci, v, out) != OK:
        raise ValueError("missing diagonal")
    return out


def match_greedy(rp, ci, wgt):
    rp, ci = _i32(rp), _i32(ci)
    mate = np.empty(len(rp) - 1, dtype=np.int32)
    _lib().orc_match_greedy(len(rp) - 1, rp, ci, _f64(wgt), mate)
    return mate


def aggregate(mate):
    mate = _i32(mate)
    agg = np.empty(len(mate), dtype=np.int32)
    nc = _lib().orc_aggregate(len(mate), mate, agg)
    return agg, nc


def galerkin(rp, ci, v, agg, nc):
    rp, ci, v, agg = _i32(rp), _i32(ci), _f64(v), _i32(agg)
    lib = _lib()
    nnz = lib.orc_galerkin(len(rp) - 1, rp, ci, v, agg, nc, None, None, None)
    rpc = np.zeros(nc + 1, dtype=np.int32)
    cic = np.zeros(nnz, dtype=np.int32)
    vc = np.zeros(nnz, dtype=np.float64)
    lib.orc_galerkin(len(rp) - 1, rp, ci, v, agg, nc, rpc.ctypes.data, cic.ctypes.data, vc.ctypes.data)
    return rpc, cic, vc


def round_bf16(x: float) -> float:
    return float(_lib().orc_round_bf16(float(x)))


@dataclass
class Params:
    aggr_steps: int = 3
    max_levels: int = 39
    coarse_size: int = 0
    pre_sweeps: int = 4
    post_sweeps: int = 4
    coarse_sweeps: int = 20
    coarse_solver: int = COARSE_L1JACOBI
    precision: int = FP64
    true_res_every: int = 50
    num_parts: int = 1
    cycle: int = 0
    relax_type: int = 4
    prolong_scale: int = PROLONG_UNIT  # PROLONG_W_NORMALIZED: ablation of the prolongator values

    def _c(self):
        p = _Params()
        for k in _Params._fields_:
            setattr(p, k[0], int(getattr(self, k[0])))
        return p


class Hierarchy:
    """Oracle AMG hierarchy (Alg. 3 with s-fold composition) plus the solve phase."""

    def __init__(self, A, params: Params | None = None, omp: bool = False, **kw):
        """omp: run on the OpenMP build (the timed CPU baseline) instead of the
        serial checker."""
        self.params = params or Params(**kw)
        rp, ci, v = _i32(A.row_ptr), _i32(A.col_idx), _f64(A.val)
        self._lib = _lib(omp)
        self._h = self._lib.orc_setup(A.n, rp, ci, v, ctypes.byref(self.params._c()))
        if not self._h:
            raise ValueError("oracle setup rejected the matrix")
        self.n = A.n

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._lib.orc_free(h)

    @property
    def num_levels(self) -> int:
        return self._lib.orc_num_levels(self._h)

    def level_n(self, k):
        return self._lib.orc_level_n(self._h, k)

    def level_nnz(self, k):
        return self._lib.orc_level_nnz(self._h, k)

    def level_csr(self, k):
        n, nnz = self.level_n(k), self.level_nnz(k)
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(nnz, np.int32)
        v = np.zeros(nnz, np.float64)
        self._lib.orc_level_csr(self._h, k, rp, ci, v)
        return rp, ci, v

    def level_agg(self, k):
        agg = np.zeros(self.level_n(k), np.int32)
        self._lib.orc_level_agg(self._h, k, agg)
        return agg

    def level_l1(self, k):
        out = np.zeros(self.level_n(k), np.float64)
        self._lib.orc_level_l1(self._h, k, out)
        return out

    @property
    def pairwise_sizes(self):
        return [self._lib.orc_pairwise_n(self._h, t) for t in range(self._lib.orc_num_pairwise(self._h))]

    def opc(self):
        return sum(self.level_nnz(k) for k in range(self.num_levels)) / self.level_nnz(0)

    def set_omega(self, k, omega):
        if omega is None:
            self._lib.orc_set_omega(self._h, k, None)
        else:
            om = _f64(omega)
            assert om.shape == (self.level_n(k),)
            self._lib.orc_set_omega(self._h, k, om.ctypes.data)

    def vcycle(self, r):
        r = _f64(r)
        z = np.zeros(self.n)
        self._lib.orc_vcycle(self._h, r, z)
        return z

    def spmv(self, k, x):
        x = _f64(x)
        y = np.zeros(self.level_n(k))
        self._lib.orc_spmv(self._h, k, x, y)
        return y

    def fcg(self, b, x0=None, tol=1e-6, maxit=1000, precflag=1):
        b = _f64(b)
        u = np.zeros(self.n) if x0 is None else _f64(x0).copy()
        it = ctypes.c_int(0)
        tr = ctypes.c_double(0.0)
        hist = np.zeros(maxit + 1)
        st = self._lib.orc_fcg(self._h, b, u, tol, maxit, precflag, ctypes.byref(it), hist, ctypes.byref(tr))
        return {"x": u, "iters": it.value, "hist": hist[: it.value + 1].copy(),
                "true_rel_res": tr.value, "status": st}

    def loss(self, r0, m):
        return self._lib.orc_vcycle_loss(self._h, _f64(r0), m)

    def loss_grad(self, r0, m):
        grads = [np.zeros(self.level_n(k)) for k in range(self.num_levels)]
        ptrs = (ctypes.c_void_p * len(grads))(*[g.ctypes.data for g in grads])
        L = self._lib.orc_vcycle_loss_grad(self._h, _f64(r0), m, ptrs)
        return L, grads
