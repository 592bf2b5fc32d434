"""Unstructured matrices against the oracle, through the C ABI: random graphs
(no grid) with rows of 1 to about 220 entries, isolated rows (the diagonal
alone), many equal matching weights (values on a 1/64 grid), mixed-sign
off-diagonals, explicit zeros in the pattern (never matched; coarse entries
that cancel to zero are kept), and coarse levels whose rows hold hundreds of
entries (rows too
long for the pipelined tiles, so the fallback row kernels and the fused bottom
see them).  Same bars as the structured problems: hierarchy bit-exact, one
V-cycle to 1e-12, SpMV to 1e-13, FCG iterations within 1 and the iterate at the
same iteration count to 1e-9; low precision against the oracle's emulation."""
import numpy as np
import pytest

import oracle as O
from paper_2303_02352_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RAND = {
    "rand5k": lambda: W.random_spd(5000, 7),
    "rand5k_mixed": lambda: W.random_spd(5000, 8, mixed_sign=True),
    "rand20k": lambda: W.random_spd(20000, 9),
    "rand3k_light": lambda: W.random_spd(3001, 10, max_partners=12),
    "rand4k_zeros": lambda: W.random_spd(4000, 21, mixed_sign=True, zero_frac=0.3),  # explicit zeros
    "rand7": lambda: W.random_spd(7, 12, mixed_sign=True),
    "rand1": lambda: W.random_spd(1, 11),
}


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
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def maxerr(a, b):
    """Largest element-wise difference, relative to the largest entry of b."""
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("name", list(RAND))
def test_hierarchy_bit_exact(name):
    A = RAND[name]()
    g, o = G(A), O.Hierarchy(A)
    info = g.info()
    assert info["num_levels"] == o.num_levels
    assert info["num_pairwise"] == len(o.pairwise_sizes)
    for k in range(o.num_levels):
        assert info["n"][k] == o.level_n(k) and info["nnz"][k] == o.level_nnz(k)
        grp, gci, gv = g.level_csr(k)
        orp, oci, ov = o.level_csr(k)
        assert np.array_equal(grp, orp) and np.array_equal(gci, oci)
        assert np.array_equal(gv.view(np.uint64), ov.view(np.uint64))
        assert np.array_equal(g.l1(k).view(np.uint64), o.level_l1(k).view(np.uint64))
        if k < o.num_levels - 1:
            assert np.array_equal(g.aggregates(k), o.level_agg(k))


@pytest.mark.parametrize("name", list(RAND))
def test_vcycle_spmv_and_fcg(name):
    A = RAND[name]()
    g, o = G(A), O.Hierarchy(A)
    for seed in (1, 2):
        r = W.random_vector(A.n, seed)
        zg, zo = g.vcycle(r).cpu().numpy(), o.vcycle(r)
        assert rel(zg, zo) < 1e-12 and maxerr(zg, zo) < 1e-12
    x = W.random_vector(A.n, 7)
    for k in range(o.num_levels):
        xk = x[: o.level_n(k)]
        assert rel(g.spmv(k, xk).cpu().numpy(), o.spmv(k, xk)) < 1e-13
    b = W.rhs_from_solution(A, W.random_vector(A.n, 3))
    rg, ro = g.pcg_solve(b), o.fcg(b)
    assert rg["status"] == 0 and ro["status"] == 0
    assert abs(rg["iters"] - ro["iters"]) <= 1 and rg["true_rel_res"] < 1e-6
    m = min(rg["iters"], ro["iters"])
    xg = g.pcg_solve(b, tol=0.0, maxit=m)["x"].cpu().numpy()
    xo = o.fcg(b, tol=0.0, maxit=m)["x"]
    assert rel(xg, xo) < 1e-9 and maxerr(xg, xo) < 1e-9


# every kernel-form switch of the setup; each run is compared with the oracle
FORMS = [
    {"AMG_PIPE": "0"},                        # non-pipelined tiled kernels everywhere
    {"AMG_BOTTOM": "1"},                      # fused bottom whatever the owner spread
    {"AMG_BOTTOM": "0"},                      # bottom levels as separate launches
    {"AMG_FUSE": "0"},                        # restriction / prolongation as separate kernels
    {"AMG_BIG": "4"}, {"AMG_BIG": "2"}, {"AMG_BIG": "5"},    # the long-row forms (off by default)
    {"AMG_MIN_TPR": "4"}, {"AMG_MIN_TPR": "32"},
    {"AMG_SMALL_ROWS": "100000000"},          # pipelined forms off on every level
]


@pytest.mark.parametrize("env", FORMS, ids=lambda e: ",".join(f"{k}={v}" for k, v in e.items()))
@pytest.mark.parametrize("name", ["rand5k_mixed", "rand20k", "rand3k_light"])
def test_kernel_forms(name, env, monkeypatch):
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    A = RAND[name]()
    g, o = G(A), O.Hierarchy(A)
    if name == "rand3k_light" and env == {"AMG_BOTTOM": "1"}:
        # both coarse levels (602 and 370 rows) in the cluster: restriction,
        # prolongation and the gathers of a random graph through shared memory
        assert g.info()["bottom_level"] == 1
    r = W.random_vector(A.n, 5)
    assert rel(g.vcycle(r).cpu().numpy(), o.vcycle(r)) < 1e-12
    b = W.rhs_from_solution(A, W.random_vector(A.n, 6))
    rg, ro = g.pcg_solve(b), o.fcg(b)
    assert abs(rg["iters"] - ro["iters"]) <= 1 and rg["true_rel_res"] < 1e-6


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name", ["rand5k", "rand5k_mixed"])
def test_low_precision(name, prec):
    A = RAND[name]()
    g, olo, o64 = G(A, precision=prec), O.Hierarchy(A, precision=prec), O.Hierarchy(A)
    r = W.random_vector(A.n, 9)
    zg = g.vcycle(r).cpu().numpy()
    zlo = olo.vcycle(r)
    # bars: a few times the gaps measured on the GPU (see test_gpu_parity.LOWP_*)
    assert rel(zg, zlo) < 1e-6 and maxerr(zg, zlo) < 1e-6
    assert rel(zg, o64.vcycle(r)) < (1e-6 if prec == 1 else 1e-2)
    b = W.rhs_from_solution(A, W.random_vector(A.n, 1))
    rg, rlo = g.pcg_solve(b), olo.fcg(b)
    assert rg["status"] == 0 and rg["true_rel_res"] < 1e-6
    assert abs(rg["iters"] - rlo["iters"]) <= 2


@pytest.mark.parametrize("kw", [dict(cycle=2), dict(relax_type=0), dict(num_parts=3), dict(aggr_steps=1),
                                dict(aggr_steps=2, coarse_size=50)])
def test_variants(kw):
    A = RAND["rand5k_mixed"]()
    g, o = G(A, **kw), O.Hierarchy(A, **kw)
    assert g.num_levels == o.num_levels
    for k in range(o.num_levels - 1):
        assert np.array_equal(g.aggregates(k), o.level_agg(k))
    r = W.random_vector(A.n, 4)
    assert rel(g.vcycle(r).cpu().numpy(), o.vcycle(r)) < 1e-12
    b = W.rhs_from_solution(A, W.random_vector(A.n, 2))
    rg, ro = g.pcg_solve(b), o.fcg(b)
    assert abs(rg["iters"] - ro["iters"]) <= 1 and rg["true_rel_res"] < 1e-6
