"""The allocation-free residual check, called through the C ABI.

amg_residual_norm_noalloc serves callers that may not allocate device memory
themselves (their host owns all device memory through its own allocator, or
an allocation's implicit synchronisation is not acceptable).  It must agree
with the solver's own residual: the true relative residual that amg_pcg_solve
reports, and b - A x formed with amg_spmv.  Two calls in a row check that the
shared scratch array is reset between calls.  This file runs last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2303_02352_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def amg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_02352_gb300 import amg as amg_mod
    from paper_2303_02352_gb300 import build
    build.build()
    amg_mod.load()
    return amg_mod


def _csr(amg, A):
    rp = torch.as_tensor(A.row_ptr).cuda()
    ci = torch.as_tensor(A.col_idx).cuda()
    v = torch.as_tensor(A.val).cuda()
    keep = (rp, ci, v)
    return amg.amg_csr(A.n, A.nnz, rp.data_ptr(), ci.data_ptr(), v.data_ptr()), keep


@pytest.mark.parametrize("N", [24, 37])
def test_noalloc_residual_matches_solver_twice(amg, N):
    A = W.diffusion7(N, 1.5, 900 + N)
    b_np = W.rhs_from_solution(A, W.random_vector(A.n, N))
    g = amg.Hierarchy(A)
    res = g.pcg_solve(b_np)
    x = res["x"]
    b = torch.as_tensor(b_np).cuda()
    ref_r = (b - g.spmv(0, x)).cpu().numpy()
    csr, keep = _csr(amg, A)
    lib = amg.load()
    stream = torch.cuda.current_stream()
    for call in range(2):
        r = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
        norms = torch.zeros(2, dtype=torch.float64, device="cuda")
        st = lib.amg_residual_norm_noalloc(ctypes.byref(csr), b.data_ptr(), x.data_ptr(), r.data_ptr(),
                                           norms.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert st == amg.OK, lib.amg_last_error(None)
        torch.cuda.synchronize()
        nr, nb = norms.cpu().numpy()
        assert abs(nb - np.linalg.norm(b_np)) <= 1e-12 * np.linalg.norm(b_np)
        assert abs(nr / nb - res["true_rel_res"]) <= 1e-12 * res["true_rel_res"], call
        rr = r.cpu().numpy()
        assert np.linalg.norm(rr - ref_r) <= 1e-14 * np.linalg.norm(b_np), call
    # r is optional
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = lib.amg_residual_norm_noalloc(ctypes.byref(csr), b.data_ptr(), x.data_ptr(), None, norms.data_ptr(),
                                       ctypes.c_void_p(stream.cuda_stream))
    assert st == amg.OK
    torch.cuda.synchronize()
    assert abs(float(norms[0] / norms[1]) - res["true_rel_res"]) <= 1e-12 * res["true_rel_res"]


def test_noalloc_rejects_oversize_and_null(amg):
    lib = amg.load()
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    big = amg.amg_csr(2_097_153, 2_097_153, p, p, p)
    st = lib.amg_residual_norm_noalloc(ctypes.byref(big), p, p, None, p, None)
    assert st == amg.ERR_TOO_LARGE
    assert b"exceeds" in lib.amg_last_error(None)
    st = lib.amg_residual_norm_noalloc(ctypes.byref(big), None, p, None, p, None)
    assert st == amg.ERR_INVALID_ARG


def test_noalloc_at_the_size_that_fills_the_scratch_array(amg):
    """n = 2,097,152 rows (7-point Poisson 128^3): 8,192 blocks, every partial
    sum slot of the fixed array and the ticket counter right after them.  Two
    calls in a row against scipy's b - A x."""
    import scipy.sparse  # noqa: F401  (A.to_scipy)
    A = W.poisson7(128)
    assert A.n == 2_097_152
    b_np = W.rhs_from_solution(A, W.random_vector(A.n, 41))
    x_np = W.random_vector(A.n, 42)
    ref = b_np - A.to_scipy() @ x_np
    csr, keep = _csr(amg, A)
    lib = amg.load()
    b, x = torch.as_tensor(b_np).cuda(), torch.as_tensor(x_np).cuda()
    stream = torch.cuda.current_stream()
    for call in range(2):
        r = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
        norms = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.amg_residual_norm_noalloc(ctypes.byref(csr), b.data_ptr(), x.data_ptr(), r.data_ptr(),
                                           norms.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert st == amg.OK, lib.amg_last_error(None)
        torch.cuda.synchronize()
        rr = r.cpu().numpy()
        assert np.max(np.abs(rr - ref)) <= 1e-14 * np.max(np.abs(b_np)), call
        nr, nb = norms.cpu().numpy()
        assert abs(nr - np.linalg.norm(ref)) <= 1e-12 * np.linalg.norm(ref), call
        assert abs(nb - np.linalg.norm(b_np)) <= 1e-12 * np.linalg.norm(b_np), call
