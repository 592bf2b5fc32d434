"""Failure detection without a GPU fault.

Every failure here is made on the host (an injected allocation failure, a
matching-loop step cap set far below its proof-level bound, an indefinite
matrix) or by a device wait on a barrier phase that nothing completes.  After
each one the CUDA context must still be usable.
"""
import os
import time

import numpy as np
import pytest

import oracle as O
from paper_2303_02352_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_02352_gb300 import build
    build.build()
    from paper_2303_02352_gb300 import amg
    return amg.load()


def still_usable():
    from paper_2303_02352_gb300 import amg
    A = W.poisson7(10)
    r = amg.Hierarchy(A).pcg_solve(W.rhs_from_solution(A, W.random_vector(A.n, 1)))
    assert r["status"] == 0 and r["true_rel_res"] < 1e-6


def test_bounded_wait_gives_up_and_reports():
    from paper_2303_02352_gb300 import amg
    lib = amg.load()
    t0 = time.time()
    st = lib.amg_check_bounded_wait(20000, None)  # 20 ms limit
    dt = time.time() - t0
    assert st == amg.ERR_TIMEOUT
    assert dt < 5.0
    still_usable()


def test_matching_step_cap_reports_timeout(monkeypatch):
    from paper_2303_02352_gb300 import amg
    monkeypatch.setenv("AMG_SUITOR_CAP", "1")
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy(W.poisson7(12))
    assert e.value.status == amg.ERR_TIMEOUT
    monkeypatch.delenv("AMG_SUITOR_CAP")
    still_usable()


@pytest.mark.parametrize("k", [0, 3, 17, 40, 70])
def test_allocation_failure_is_reported_and_cleaned_up(monkeypatch, k):
    from paper_2303_02352_gb300 import amg
    A = W.poisson7(12)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("AMG_FAIL_ALLOC_AFTER", str(k))
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy(A)
    assert e.value.status == amg.ERR_OOM
    monkeypatch.delenv("AMG_FAIL_ALLOC_AFTER")
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) < (64 << 20)  # nothing of the failed handle is left behind
    still_usable()


def test_breakdown_on_an_indefinite_matrix_matches_oracle():
    n = 50
    i = np.arange(n)
    cols = np.stack([i - 1, i, i + 1], axis=1)
    vals = np.tile([-2.0, 1.0, -2.0], (n, 1))
    mask = (cols >= 0) & (cols < n)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum(mask.sum(1))
    A = W.CSR(n, rp, cols[mask].astype(np.int32), vals[mask])
    b = np.ones(n)  # b^T A b = n - 4 (n - 1) < 0
    from paper_2303_02352_gb300 import amg
    g = amg.Hierarchy(A)
    rg = g.cg_solve(b)
    ro = O.Hierarchy(A).fcg(b, precflag=0)
    assert rg["status"] == amg.ERR_BREAKDOWN == ro["status"]
    assert rg["iters"] == ro["iters"] == 0
    assert float(rg["x"].abs().max()) == 0.0  # the last good iterate is u_0
    still_usable()
