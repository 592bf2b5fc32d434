"""Pattern-coded columns: the row kernels of a level whose rows fall into at most
255 tuples of column offsets read a one-byte tuple id per row instead of the
column indices.  Same entries in the same order and the same arithmetic as the
CSR form, so every row pass of the same kernel form, and so the V-cycle, is
bitwise that of the CSR form (AMG_PAT=0); pattern-coded float levels with
short tiles also take the two-group form, which sums a row in another order.  The pattern forms' smaller stages let more blocks share a
multiprocessor, so the persistent outer kernel runs another number of blocks
and its dot products add their block partial sums in another (fixed) order:
the solves agree to rounding, at the oracle's bars.
"""
import numpy as np
import pytest

import oracle as O
from paper_2303_02352_gb300 import workloads as W
from pattern_fixtures import block_diagonal, paired_rows

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
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


STENCILS = {
    "poisson40": lambda: W.poisson7(40),                 # 64,000 rows, 27 tuples
    "diff27_40": lambda: W.diffusion27(40, 2.0, 3),      # 27 tuples, 64-row tiles with 4 threads per row
    "diff7_48": lambda: W.diffusion7(48, 2.0, 1001),
}


def expected_form(name, prec):
    """Column form of level 0's V-cycle kernels: FP64 levels whose rows take
    several threads (27-point) keep CSR columns, the others use form 1."""
    return 0 if (name == "diff27_40" and prec == 0) else 1


@pytest.mark.parametrize("name", sorted(STENCILS))
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_pattern_form_is_bitwise_the_csr_form(name, prec, monkeypatch):
    A = STENCILS[name]()
    g = G(A, precision=prec)
    info = g.info()
    # a 7- or 27-point stencil on an N^3 grid: 3 cases per axis (low face, interior, high face)
    form = expected_form(name, prec)
    assert info["column_form"][0] == form and info["column_patterns"][0] == (27 if form else 0)
    assert info["outer_patterns"] == (0 if name == "diff27_40" else 27)
    monkeypatch.setenv("AMG_PAT", "0")
    c = G(A, precision=prec)
    ic = c.info()
    assert all(p == 0 for p in ic["column_patterns"]) and ic["outer_patterns"] == 0
    assert info["n"] == ic["n"] and info["nnz"] == ic["nnz"]
    # the pattern form moves one id byte per row instead of four index bytes per entry
    if form:
        assert info["vcycle_bytes"] < ic["vcycle_bytes"]
    r = W.random_vector(A.n, 8)
    zg, zc = g.vcycle(r).cpu().numpy(), c.vcycle(r).cpu().numpy()
    if info["consumer_groups"] == ic["consumer_groups"]:
        assert np.array_equal(zg, zc)
    else:
        # pattern-coded float levels with short tiles take the two-group form
        # (half the threads per row): another order of each row's float sum
        assert name == "diff27_40" and prec > 0 and info["consumer_groups"][0] == 2
        assert rel(zg, zc) < 1e-6
    b = W.rhs_from_solution(A, W.random_vector(A.n, 9))
    rg, rc = g.pcg_solve(b), c.pcg_solve(b)
    assert rg["status"] == 0 and rg["true_rel_res"] < 1e-6 and abs(rg["iters"] - rc["iters"]) <= 1
    m = min(rg["iters"], rc["iters"])
    xg = g.pcg_solve(b, tol=0.0, maxit=m)["x"].cpu().numpy()
    xc = c.pcg_solve(b, tol=0.0, maxit=m)["x"].cpu().numpy()
    # the bars of the oracle comparisons: 1e-10 for FP64, and for float
    # hierarchies that round in another order 1e-9 (test_gpu_parity.py)
    assert rel(xg, xc) < (1e-10 if prec == 0 else 1e-9)
    if prec == 0:
        o = O.Hierarchy(A)
        assert rel(zg, o.vcycle(r)) < 1e-12


@pytest.mark.parametrize("name", sorted(STENCILS))
@pytest.mark.parametrize("prec", [0, 2])
def test_rows_from_tuple_lengths_equal_rows_from_row_pointers(name, prec, monkeypatch):
    """Form 2 (AMG_PAT=2; one thread per row: a warp's rows located from one
    row pointer per 32 rows and the tuple lengths) against the default form 1
    (row pointers): the same stages and grid, so V-cycle and solve are bitwise
    equal.  27-point levels run 2-4 threads per row and keep their form."""
    A = STENCILS[name]()
    g = G(A, precision=prec)
    info = g.info()
    assert info["column_form"][0] == expected_form(name, prec)
    monkeypatch.setenv("AMG_PAT", "2")
    c = G(A, precision=prec)
    ic = c.info()
    two = name != "diff27_40"
    assert ic["column_form"][0] == (2 if two else expected_form(name, prec))
    assert ic["column_patterns"] == info["column_patterns"]
    if two:  # one row pointer per 32 rows instead of one per row
        assert ic["vcycle_bytes"] < info["vcycle_bytes"]
    r = W.random_vector(A.n, 3)
    assert np.array_equal(g.vcycle(r).cpu().numpy(), c.vcycle(r).cpu().numpy())
    b = W.rhs_from_solution(A, W.random_vector(A.n, 2))
    rg, rc = g.pcg_solve(b), c.pcg_solve(b)
    assert rg["iters"] == rc["iters"] and np.array_equal(rg["x"].cpu().numpy(), rc["x"].cpu().numpy())


@pytest.mark.parametrize("name", sorted(STENCILS))
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_staged_row_data_equals_loaded_row_data(name, prec, monkeypatch):
    """The small-stage pattern kernels bring the tile's row pointers and row
    vectors in by bulk copy; with AMG_STAGE=0 the consumers load them (the
    path taken when a source is not 16-byte aligned).  Same stages, grid and
    arithmetic: V-cycle and solve bitwise equal."""
    A = STENCILS[name]()
    g = G(A, precision=prec)
    monkeypatch.setenv("AMG_STAGE", "0")
    c = G(A, precision=prec)
    assert g.info()["column_form"] == c.info()["column_form"]
    r = W.random_vector(A.n, 12)
    assert np.array_equal(g.vcycle(r).cpu().numpy(), c.vcycle(r).cpu().numpy())
    b = W.rhs_from_solution(A, W.random_vector(A.n, 13))
    rg, rc = g.pcg_solve(b), c.pcg_solve(b)
    assert rg["status"] == 0 and rg["iters"] == rc["iters"]
    assert np.array_equal(rg["x"].cpu().numpy(), rc["x"].cpu().numpy())


@pytest.mark.parametrize("prec", [0, 1])
def test_per_row_damping_on_pattern_coded_levels(prec, monkeypatch):
    """Per-row damping (the learned smoother's D = omega / l1) on pattern-coded
    levels with staged row data: against the oracle with the same omegas (FP64,
    1e-12) and bitwise against CSR columns with the same omegas."""
    A = STENCILS["diff7_48"]()
    g = G(A, precision=prec)
    assert g.info()["column_form"][0] == 1
    monkeypatch.setenv("AMG_PAT", "0")
    c = G(A, precision=prec)
    rng = np.random.default_rng(7)
    oms = [0.6 + 0.8 * rng.random(n) for n in g.info()["n"]]
    for k, om in enumerate(oms):
        g.set_omega(k, om)
        c.set_omega(k, om)
    r = W.random_vector(A.n, 21)
    zg = g.vcycle(r).cpu().numpy()
    assert np.array_equal(zg, c.vcycle(r).cpu().numpy())
    if prec == 0:
        o = O.Hierarchy(A)
        for k, om in enumerate(oms):
            o.set_omega(k, om)
        assert rel(zg, o.vcycle(r)) < 1e-12


VARIANTS = {"w_cycle": dict(cycle=2), "jacobi": dict(relax_type=0), "decoupled3": dict(num_parts=3),
            "w_normalised": dict(prolong_scale=1)}


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_method_variants_on_pattern_coded_levels(variant, monkeypatch):
    """The method variants on a pattern-coded hierarchy (59,319 rows, an odd
    grid: aggregates of unequal sizes, so the w-normalised prolongator and the
    3 row blocks change the operator): V-cycle within 1e-12 of the oracle's
    same variant and bitwise equal to CSR columns."""
    kw = VARIANTS[variant]
    A = W.poisson7(39)
    g = G(A, **kw)
    assert g.info()["column_form"][0] == 1
    okw = dict(kw)
    if "prolong_scale" in okw:
        okw["prolong_scale"] = O.PROLONG_W_NORMALIZED
    o = O.Hierarchy(A, **okw)
    r = W.random_vector(A.n, 31)
    zg = g.vcycle(r).cpu().numpy()
    assert rel(zg, o.vcycle(r)) < 1e-12
    monkeypatch.setenv("AMG_PAT", "0")
    assert np.array_equal(zg, G(A, **kw).vcycle(r).cpu().numpy())


def test_checkpoint_of_a_pattern_coded_hierarchy(tmp_path):
    """A saved hierarchy rebuilds the same pattern-coded columns when loaded:
    the same tuple counts and a bitwise equal V-cycle."""
    from paper_2303_02352_gb300 import amg
    A = W.poisson7(40)
    g = G(A)
    path = str(tmp_path / "poisson40.amgh")
    g.save(path)
    h = amg.Hierarchy.load(path)
    assert h.info()["column_patterns"] == g.info()["column_patterns"]
    assert h.info()["column_patterns"][0] == 27
    r = W.random_vector(A.n, 32)
    assert np.array_equal(g.vcycle(r).cpu().numpy(), h.vcycle(r).cpu().numpy())
    h.close()


@pytest.mark.parametrize("dmax, singleton, expect", [(127, True, 255), (128, False, 0)])
def test_tuple_count_boundary(dmax, singleton, expect, monkeypatch):
    """255 distinct offset tuples take the pattern form (ids 0 .. 254), 256
    leave the level on CSR columns; the V-cycle is the oracle's either way."""
    A = paired_rows(dmax, singleton, 3)
    assert A.n >= 32768
    g = G(A)
    info = g.info()
    assert info["column_patterns"][0] == expect
    o = O.Hierarchy(A)
    r = W.random_vector(A.n, 5)
    zg = g.vcycle(r).cpu().numpy()
    assert rel(zg, o.vcycle(r)) < 1e-12
    monkeypatch.setenv("AMG_PAT", "0")
    assert np.array_equal(zg, G(A).vcycle(r).cpu().numpy())


def test_table_larger_than_the_cap_keeps_csr_columns():
    """231 tuples of up to 21 entries: 4,851 table entries, above the 1,024 the
    row kernels hold in shared memory, so the level keeps CSR columns."""
    A = block_diagonal(list(range(1, 22)), 160)
    assert A.n >= 32768
    g = G(A)
    assert g.info()["column_patterns"][0] == 0
    o = O.Hierarchy(A)
    r = W.random_vector(A.n, 4)
    assert rel(g.vcycle(r).cpu().numpy(), o.vcycle(r)) < 1e-12


def test_irregular_level_keeps_csr_columns():
    """A random sparse graph has more distinct tuples than ids: CSR columns."""
    A = W.random_spd(40000, 11, max_partners=12)
    g = G(A)
    assert g.info()["column_patterns"][0] == 0
    o = O.Hierarchy(A)
    r = W.random_vector(A.n, 6)
    assert rel(g.vcycle(r).cpu().numpy(), o.vcycle(r)) < 1e-12
