"""The Python form of the boundary: ``amg.setup`` on a ``torch.sparse_csr_tensor``
and ``amg.solve`` returning ``(x, iters, hist)``, and ``learned.VCycleFn`` as a
``torch.autograd.Function``.  The sparse-tensor route must give the same
hierarchy and the same solve, bit for bit, as the plain CSR route, whatever the
index type and device of the tensor."""
import numpy as np
import pytest

from paper_2303_02352_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _sparse(A, device, index_dtype):
    return torch.sparse_csr_tensor(torch.tensor(A.row_ptr, dtype=index_dtype),
                                   torch.tensor(A.col_idx, dtype=index_dtype),
                                   torch.tensor(A.val, dtype=torch.float64),
                                   size=(A.n, A.n)).to(device)


@pytest.mark.parametrize("device,index_dtype", [("cuda", torch.int32), ("cuda", torch.int64),
                                                ("cpu", torch.int64)])
def test_setup_from_sparse_csr_tensor_matches_csr_route(device, index_dtype):
    _need_gpu()
    from paper_2303_02352_gb300 import amg
    A = W.diffusion27(20, 2.0, 3)
    b = W.rhs_from_solution(A, W.random_vector(A.n, 4))
    h0 = amg.setup(A)
    h1 = amg.setup(_sparse(A, device, index_dtype))
    try:
        i0, i1 = h0.info(), h1.info()
        assert i0["n"] == i1["n"] and i0["nnz"] == i1["nnz"]
        for k in range(i0["num_levels"] - 1):
            assert np.array_equal(h0.aggregates(k), h1.aggregates(k))
        x0, it0, hist0 = amg.solve(h0, b)
        x1, it1, hist1 = amg.solve(h1, torch.tensor(b, device="cuda"))
        assert it0 == it1 and it0 > 0
        assert np.array_equal(hist0, hist1)
        assert torch.equal(x0, x1)
        assert hist0.shape == (it0 + 1,) and abs(hist0[0] - 1.0) < 1e-14 and hist0[-1] < 1e-6
        # x0 argument: starting from the solution converges at once
        x2, it2, hist2 = amg.solve(h1, b, x0=x1, tol=1e-3)
        assert it2 <= 1 and torch.allclose(x2, x1, rtol=0, atol=1e-6 * float(x1.abs().max()))
    finally:
        h0.close()
        h1.close()


def test_solve_reports_not_converged_with_its_iterate():
    _need_gpu()
    from paper_2303_02352_gb300 import amg
    A = W.poisson7(24)
    b = W.rhs_from_solution(A, W.random_vector(A.n, 5))
    h = amg.setup(A)
    try:
        x, it, hist = amg.solve(h, b, maxit=3)
        assert it == 3 and hist.shape == (4,) and hist[-1] > 1e-6
        full = h.pcg_solve(b, maxit=3)
        assert full["status"] == amg.NOT_CONVERGED and torch.equal(full["x"], x)
    finally:
        h.close()


def test_vcycle_fn_is_an_autograd_function():
    _need_gpu()
    from paper_2303_02352_gb300 import amg, learned
    assert issubclass(learned.VCycleFn, torch.autograd.Function)
    A = W.poisson7(16)
    h = amg.setup(A)
    try:
        r = torch.tensor(W.random_vector(A.n, 6), device="cuda")
        oms = [torch.full((nk,), 0.9, dtype=torch.float64, device="cuda", requires_grad=True)
               for nk in h.level_sizes()]
        z = learned.VCycleFn.apply(h, r, *oms)
        for k in range(h.num_levels):
            h.set_omega(k, torch.full((h.level_sizes()[k],), 0.9, dtype=torch.float64, device="cuda"))
        assert torch.equal(z, h.vcycle(r))
        z.sum().backward()
        assert all(om.grad is not None and om.grad.shape == om.shape for om in oms)
    finally:
        h.close()
