"""The general sparse product (amg_spgemm) and the w-normalised prolongators
built with it, through the C ABI.

amg_spgemm against scipy on random rectangular matrices: the structural
pattern exactly (every product that exists is kept, also where values cancel),
the values to 1e-13 of the sum of the magnitudes of their products, bitwise
reproducible, ragged rows (empty rows, rows longer than a warp), empty
products, invalid inputs.

prolong_scale = 1 (Sec. 3.1: P_{i,I} = w_i / |w on I|, w_next = P^T w) against
the oracle's ablation, which keeps the unit matrices A^k and the equivalent
smoother diagonal: aggregates bit-exact; the GPU's level matrices, formed by
the general product, equal W_k^-1 A^k W_k^-1 (w from the aggregates) to 1e-12;
their l1 norms scaled by w_I^2 equal the oracle's diagonal; one V-cycle to
1e-12 (level 0 is the same matrix in both forms); FCG iterations within 1 and
the iterate at equal count to 1e-9; W-cycle, Jacobi and decoupled aggregation
the same way; the FP32 hierarchy to the FP32 bar against the FP64 oracle.
"""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

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


def G(A, **kw):
    from paper_2303_02352_gb300 import amg
    return amg.Hierarchy(A, **kw)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def maxerr(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


def random_csr(m, n, rng, density, long_rows=0, empty_frac=0.1):
    """Random m x n CSR (sorted columns, mixed-sign values), with some empty rows
    and `long_rows` rows of 40-120 entries."""
    rows = []
    for i in range(m):
        if rng.random() < empty_frac:
            k = 0
        elif i < long_rows:
            k = int(rng.integers(40, min(n, 120) + 1))
        else:
            k = int(rng.binomial(n, density))
        cols = np.sort(rng.choice(n, size=min(k, n), replace=False)) if k else np.zeros(0, np.int64)
        rows.append(cols)
    rp = np.zeros(m + 1, np.int32)
    rp[1:] = np.cumsum([len(c) for c in rows])
    ci = np.concatenate(rows).astype(np.int32) if rp[-1] else np.zeros(0, np.int32)
    v = rng.standard_normal(len(ci)) * rng.choice([1.0, 1e-3, 1e3], size=len(ci))
    return sp.csr_matrix((v, ci, rp), shape=(m, n))


def dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def gpu_spgemm(A, B):
    from paper_2303_02352_gb300 import amg
    args = [dev(A.indptr, torch.int32), dev(A.indices, torch.int32), dev(A.data, torch.float64),
            dev(B.indptr, torch.int32), dev(B.indices, torch.int32), dev(B.data, torch.float64)]
    crp, cci, cv = amg.spgemm(*args, ncols=B.shape[1])
    return crp.cpu().numpy(), cci.cpu().numpy(), cv.cpu().numpy()


CASES = [  # (m, k, n, density A, density B, long rows of A)
    (1, 1, 1, 1.0, 1.0, 0),
    (37, 50, 29, 0.1, 0.1, 0),
    (500, 300, 400, 0.02, 0.03, 5),
    (2000, 2000, 1000, 0.004, 0.005, 20),
    (300, 200, 5, 0.05, 0.5, 10),  # few output columns: many products per entry
]


@pytest.mark.parametrize("case", CASES)
def test_spgemm_matches_scipy(case):
    m, k, n, da, db, lr = case
    rng = np.random.default_rng(m + k + n)
    A = random_csr(m, k, rng, da, long_rows=lr)
    B = random_csr(k, n, rng, db)
    crp, cci, cv = gpu_spgemm(A, B)
    # structural pattern: products of |A| and |B| (no cancellation)
    S = (abs(A) @ abs(B)).tocsr()
    S.sort_indices()
    assert np.array_equal(crp, S.indptr) and np.array_equal(cci, S.indices)
    ref = (A @ B).toarray()
    got = np.zeros((m, n))
    rows = np.repeat(np.arange(m), np.diff(crp))
    got[rows, cci] = cv
    mag = S.toarray()
    assert np.all(np.abs(got - ref) <= 1e-13 * mag)
    # bitwise reproducible
    crp2, cci2, cv2 = gpu_spgemm(A, B)
    assert np.array_equal(cv.view(np.uint64), cv2.view(np.uint64)) and np.array_equal(cci, cci2)


def test_spgemm_keeps_cancelling_products():
    # row 0 of A times B: (1)(1) + (1)(-1) = 0 in column 0, kept as a stored zero
    A = sp.csr_matrix(np.array([[1.0, 1.0]]))
    B = sp.csr_matrix(np.array([[1.0, 2.0], [-1.0, 0.0]]))
    B.eliminate_zeros()
    crp, cci, cv = gpu_spgemm(A, B)
    assert list(crp) == [0, 2] and list(cci) == [0, 1] and list(cv) == [0.0, 2.0]


def test_spgemm_empty_inputs():
    A = sp.csr_matrix((3, 4))
    B = random_csr(4, 5, np.random.default_rng(1), 0.5)
    crp, cci, cv = gpu_spgemm(A, B)
    assert list(crp) == [0, 0, 0, 0] and len(cci) == 0
    crp, cci, cv = gpu_spgemm(sp.csr_matrix((0, 4)), B)
    assert list(crp) == [0] and len(cci) == 0


def test_spgemm_rejects_bad_inputs():
    from paper_2303_02352_gb300 import amg
    A = sp.csr_matrix(np.ones((2, 2)))
    # a row of B with descending columns
    Bd = sp.csr_matrix((np.array([1.0, 2.0]), np.array([1, 0], np.int32), np.array([0, 2, 2], np.int32)),
                       shape=(2, 2))
    with pytest.raises(amg.AmgError, match="ascending"):
        gpu_spgemm(A, Bd)
    # a column of B beyond the stated number of columns
    Bo = sp.csr_matrix((np.array([1.0]), np.array([1], np.int32), np.array([0, 1, 1], np.int32)), shape=(2, 2))
    args = [dev(A.indptr, torch.int32), dev(A.indices, torch.int32), dev(A.data, torch.float64),
            dev(Bo.indptr, torch.int32), dev(Bo.indices, torch.int32), dev(Bo.data, torch.float64)]
    with pytest.raises(amg.AmgError, match="range"):
        amg.spgemm(*args, ncols=1)
    lib = amg.load()
    n = ctypes.c_int64(0)
    assert lib.amg_spgemm(-1, 1, 1, None, None, None, None, None, None, None, None, None, ctypes.byref(n),
                          None) == amg.ERR_INVALID_ARG


# ---------------------------------------------------------------------------
# w-normalised prolongators against the oracle's ablation


PROBLEMS = {
    "poisson13": lambda: W.poisson7(13),
    "diff7_20": lambda: W.diffusion7(20, 2.0, 1001),
    "diff27_12": lambda: W.diffusion27(12, 2.0, 3),
    "rand5k_mixed": lambda: W.random_spd(5000, 8, mixed_sign=True),
    "rand4k_zeros": lambda: W.random_spd(4000, 21, mixed_sign=True, zero_frac=0.3),
}


def smooth_vectors(o):
    """w^0 = 1, w^{k+1}_I = sqrt(sum over the members of I of (w^k_i)^2), from the aggregates."""
    ws = [np.ones(o.level_n(0))]
    for k in range(o.num_levels - 1):
        agg = o.level_agg(k)
        ws.append(np.sqrt(np.bincount(agg, weights=ws[-1] ** 2, minlength=o.level_n(k + 1))))
    return ws


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_w_normalised_hierarchy_matches_oracle(name):
    A = PROBLEMS[name]()
    g = G(A, prolong_scale=1)
    o = O.Hierarchy(A, prolong_scale=O.PROLONG_W_NORMALIZED)
    info = g.info()
    assert info["num_levels"] == o.num_levels and info["setup_spgemm_ms"] > 0
    for k in range(o.num_levels - 1):
        assert np.array_equal(g.aggregates(k), o.level_agg(k))
    ws = smooth_vectors(o)
    for k in range(o.num_levels):
        grp, gci, gv = g.level_csr(k)
        orp, oci, ov = o.level_csr(k)  # unit matrices (the oracle keeps those)
        assert np.array_equal(grp, orp) and np.array_equal(gci, oci)
        rows = np.repeat(np.arange(len(orp) - 1), np.diff(orp))
        w = ws[k]
        ref = ov / (w[rows] * w[oci])
        assert np.max(np.abs(gv - ref)) <= 1e-12 * np.max(np.abs(ref)), k
        if k == 0:
            assert np.array_equal(gv, ov)
        # the smoother diagonal in unit coordinates: w_I^2 sum_J |a_IJ| / (w_I w_J)
        mref = np.bincount(rows, weights=np.abs(ov) * w[rows] / w[oci], minlength=len(w))
        assert np.max(np.abs(g.l1(k) * w ** 2 - mref) / mref) < 1e-12, k
    r = W.random_vector(A.n, 5)
    zg, zo = g.vcycle(r).cpu().numpy(), o.vcycle(r)
    assert rel(zg, zo) < 1e-12 and maxerr(zg, zo) < 1e-12
    b = W.rhs_from_solution(A, W.random_vector(A.n, 6))
    rg, ro = g.pcg_solve(b), o.fcg(b)
    assert rg["status"] == 0 and ro["status"] == 0 and rg["true_rel_res"] < 1e-6
    assert abs(rg["iters"] - ro["iters"]) <= 1
    m = min(rg["iters"], ro["iters"])
    xg = g.pcg_solve(b, tol=0.0, maxit=m)["x"].cpu().numpy()
    xo = o.fcg(b, tol=0.0, maxit=m)["x"]
    assert rel(xg, xo) < 1e-9 and maxerr(xg, xo) < 1e-9


@pytest.mark.parametrize("kw", [dict(cycle=2), dict(relax_type=0), dict(num_parts=3)])
def test_w_normalised_variants_match_oracle(kw):
    A = W.diffusion7(16, 2.5, 77)
    g = G(A, prolong_scale=1, **kw)
    o = O.Hierarchy(A, prolong_scale=O.PROLONG_W_NORMALIZED, **kw)
    for k in range(o.num_levels - 1):
        assert np.array_equal(g.aggregates(k), o.level_agg(k))
    r = W.random_vector(A.n, 3)
    zg, zo = g.vcycle(r).cpu().numpy(), o.vcycle(r)
    assert rel(zg, zo) < 1e-12 and maxerr(zg, zo) < 1e-12
    b = W.rhs_from_solution(A, W.random_vector(A.n, 4))
    rg, ro = g.pcg_solve(b), o.fcg(b)
    assert abs(rg["iters"] - ro["iters"]) <= 1 and rg["true_rel_res"] < 1e-6


@pytest.mark.parametrize("prec", [1, 2])
def test_w_normalised_low_precision(prec):
    A = W.diffusion27(12, 2.0, 3)
    g = G(A, prolong_scale=1, precision=prec)
    o64 = O.Hierarchy(A, prolong_scale=O.PROLONG_W_NORMALIZED)
    r = W.random_vector(A.n, 9)
    assert rel(g.vcycle(r).cpu().numpy(), o64.vcycle(r)) < (1e-5 if prec == 1 else 2e-2)
    b = W.rhs_from_solution(A, W.random_vector(A.n, 1))
    rg, ro = g.pcg_solve(b), o64.fcg(b)
    assert rg["status"] == 0 and rg["true_rel_res"] < 1e-6 and abs(rg["iters"] - ro["iters"]) <= 2


def test_w_normalised_timing_entries_and_adjoint_rejected():
    from paper_2303_02352_gb300 import amg
    A = W.diffusion7(24, 2.0, 5)
    g = G(A, prolong_scale=1)
    assert g.info()["bottom_level"] == g.num_levels  # the fused bottom is for unit prolongators
    for kid in (amg.K_RESTRICT, amg.K_PROLONG, amg.K_RESTRICT_FIRST):
        assert g.time_kernel(kid, 0, reps=3) > 0
    with pytest.raises(amg.AmgError, match="unit prolongators"):
        g.vcycle_backward(W.random_vector(A.n, 1), W.random_vector(A.n, 2))
    with pytest.raises(amg.AmgError):
        G(A, prolong_scale=2)
