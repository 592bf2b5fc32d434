"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks one part of the method (Alg. 1, Alg. 2 / operator B^k, Alg. 3,
the l1-Jacobi smoother of Sec. 3.1) against brute force, closed forms, library
routines the oracle does not use, or values printed in the paper.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle as O
from paper_2303_02352_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# helpers written independently of the oracle


def random_graph_csr(nv, p, rng, uniform=False):
    """Symmetric weight pattern on nv vertices as CSR (diagonal stored, weight 0)."""
    W_ = np.zeros((nv, nv))
    for i in range(nv):
        for j in range(i + 1, nv):
            if rng.random() < p:
                w = 1.0 if uniform else float(rng.integers(1, 6)) / 4.0
                W_[i, j] = W_[j, i] = w
    rp, ci, wv = [0], [], []
    for i in range(nv):
        for j in range(nv):
            if j == i or W_[i, j] != 0:
                ci.append(j)
                wv.append(W_[i, j] if j != i else 0.0)
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32), np.array(wv), W_


def brute_force_mwm(W_):
    """Maximum total weight over all matchings (exhaustive)."""
    nv = W_.shape[0]
    edges = [(i, j) for i in range(nv) for j in range(i + 1, nv) if W_[i, j] > 0]
    best = 0.0

    def rec(k, used, tot):
        nonlocal best
        if k == len(edges):
            best = max(best, tot)
            return
        rec(k + 1, used, tot)
        i, j = edges[k]
        if not (used >> i) & 1 and not (used >> j) & 1:
            rec(k + 1, used | (1 << i) | (1 << j), tot + W_[i, j])

    rec(0, 0, 0.0)
    return best


def sequential_suitor(W_):
    """Sequential Suitor (Manne-Halappanavar) under the strict order
    (weight desc, smaller endpoint pair first), written without the oracle."""
    nv = W_.shape[0]
    suitor = [-1] * nv

    def better(u, v, w_new, cur):
        # is proposer u better for v than the current suitor cur?
        if cur < 0:
            return True
        if W_[u, v] != W_[cur, v]:
            return W_[u, v] > W_[cur, v]
        return u < cur  # among edges sharing v the smaller other endpoint wins

    for u0 in range(nv):
        cur = u0
        while cur >= 0:
            best, bw = -1, 0.0
            for v in range(nv):
                w = W_[cur, v]
                if v == cur or w <= 0:
                    continue
                if better(cur, v, w, suitor[v]):
                    if best < 0 or w > bw or (w == bw and v < best):
                        best, bw = v, w
            if best < 0:
                cur = -1
            else:
                prev = suitor[best]
                suitor[best] = cur
                cur = prev
    mate = [-1] * nv
    for v in range(nv):
        u = suitor[v]
        if u >= 0 and suitor[u] == v:
            mate[v] = u
    return mate


def dense(rp, ci, v, n):
    return sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()


def prolongator(agg, nc):
    n = len(agg)
    return sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, nc))


# ----------------------------------------------------------------------------
# matching (Alg. 3 "apply MWM"; Sec. 4.1 suitor, half approximation)


@pytest.mark.parametrize("seed", range(40))
def test_greedy_matching_half_approx_maximal_equals_suitor(seed):
    rng = np.random.default_rng(seed)
    nv = int(rng.integers(2, 13))
    rp, ci, wv, W_ = random_graph_csr(nv, 0.45, rng, uniform=(seed % 4 == 0))
    mate = O.match_greedy(rp, ci, wv)
    # a valid matching
    for i, m in enumerate(mate):
        if m >= 0:
            assert mate[m] == i and W_[i, m] > 0
    # maximal: no positive edge with both ends free
    for i in range(nv):
        for j in range(i + 1, nv):
            if W_[i, j] > 0:
                assert mate[i] >= 0 or mate[j] >= 0
    tot = sum(W_[i, m] for i, m in enumerate(mate) if m > i)
    assert tot >= 0.5 * brute_force_mwm(W_) - 1e-12
    assert list(mate) == sequential_suitor(W_)


def test_weights_1d_laplacian_closed_form():
    A = W.laplace1d(10)
    w = O.weights(A.row_ptr, A.col_idx, A.val)
    off = A.col_idx != np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    assert np.all(w[off] == 1.5)  # 1 - 2(-1)/(2+2)
    assert np.all(w[~off] == 0.0)
    mate = O.match_greedy(A.row_ptr, A.col_idx, w)
    assert list(mate) == [1, 0, 3, 2, 5, 4, 7, 6, 9, 8]


def test_poisson_pairwise_steps_give_2x2x2_cubes():
    """7-point Poisson: weight 7/6 -> x pairs; then 1.1 (x) < 1.2 (y, z) -> y pairs;
    then 1.125 < 1.25 (z) -> z pairs, so three steps make 2x2x2 cubes."""
    N = 8
    A = W.poisson7(N)
    rp, ci, v = A.row_ptr, A.col_idx, A.val
    agg_total = np.arange(A.n)
    expect_w = [{7.0 / 6.0}, {1.1, 1.2}, {1.125, 1.25}]
    for step in range(3):
        w = O.weights(rp, ci, v)
        off = ci != np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        assert set(np.round(w[off], 12)) == {round(x, 12) for x in expect_w[step]}
        mate = O.match_greedy(rp, ci, w)
        agg, nc = O.aggregate(mate)
        assert nc * 2 == len(rp) - 1
        rp, ci, v = O.galerkin(rp, ci, v, agg, nc)
        agg_total = agg[agg_total]
    i = np.arange(A.n)
    xs, ys, zs = i % N, (i // N) % N, i // (N * N)
    cube = (xs // 2) + (N // 2) * (ys // 2) + (N // 2) ** 2 * (zs // 2)
    assert np.array_equal(agg_total, cube)
    assert sorted(set(v.tolist())) == [-4.0, 24.0]


# ----------------------------------------------------------------------------
# Galerkin product (Alg. 3 "compute A^{k+1} = R^k A^k P^k")


def test_galerkin_1d_laplacian_halves():
    A = W.laplace1d(16)
    agg = np.arange(16) // 2
    rp, ci, v = O.galerkin(A.row_ptr, A.col_idx, A.val, agg, 8)
    Ac = dense(rp, ci, v, 8)
    ref = 2 * np.eye(8) - np.eye(8, k=1) - np.eye(8, k=-1)
    assert np.array_equal(Ac, ref)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_galerkin_matches_library_triple_product(seed):
    A = W.diffusion27(6, 2.0, seed)
    w = O.weights(A.row_ptr, A.col_idx, A.val)
    mate = O.match_greedy(A.row_ptr, A.col_idx, w)
    agg, nc = O.aggregate(mate)
    rp, ci, v = O.galerkin(A.row_ptr, A.col_idx, A.val, agg, nc)
    P = prolongator(agg, nc)
    ref = (P.T @ A.to_scipy() @ P).toarray()
    got = dense(rp, ci, v, nc)
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    assert np.array_equal(got, got.T)  # bitwise symmetric by construction
    # columns sorted within rows
    for I in range(nc):
        assert np.all(np.diff(ci[rp[I]:rp[I + 1]]) > 0)


def test_hierarchy_invariants_random_coefficient():
    A = W.diffusion7(16, 1.5, 7)
    h = O.Hierarchy(A, coarse_size=40)
    assert h.num_levels >= 3
    for k in range(h.num_levels - 1):
        n, nc = h.level_n(k), h.level_n(k + 1)
        agg = h.level_agg(k)
        assert agg.min() >= 0 and agg.max() == nc - 1
        P = prolongator(agg, nc)
        assert np.allclose(P @ np.ones(nc), 1.0)          # P 1 = 1
        sizes = np.asarray((P.T @ P).diagonal()).ravel()
        assert sizes.max() <= 8 and sizes.min() >= 1       # P^T P = diag(sizes), sizes <= 2^s
        rp, ci, v = h.level_csr(k)
        rpc, cic, vc = h.level_csr(k + 1)
        Ak = dense(rp, ci, v, n)
        Ac = dense(rpc, cic, vc, nc)
        assert np.array_equal(Ac, Ac.T)
        np.linalg.cholesky(Ac)                              # SPD
        ref = (P.T @ sp.csr_matrix(Ak) @ P).toarray()
        assert np.allclose(Ac, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        assert np.allclose(Ac.sum(axis=1), P.T @ (Ak @ np.ones(n)), rtol=1e-12, atol=1e-10)


def test_hierarchy_closed_form_sizes_poisson():
    h = O.Hierarchy(W.poisson7(32))
    assert [(h.level_n(k), h.level_nnz(k)) for k in range(h.num_levels)] == \
        [(32768, 223232), (4096, 27136), (1024, 6528)]
    h = O.Hierarchy(W.poisson7(64))
    assert [(h.level_n(k), h.level_nnz(k)) for k in range(h.num_levels)] == \
        [(262144, 1810432), (32768, 223232), (4096, 27136), (2048, 13312)]
    assert abs(h.opc() - (1810432 + 223232 + 27136 + 13312) / 1810432) < 1e-15


def test_paper_level_counts_130():
    gold = json.load(open(os.path.join(GOLD, "paper_structure.json")))
    h = O.Hierarchy(W.poisson7(130))
    assert h.num_levels == gold["levels"]["130"]
    assert abs(h.opc() - gold["opc_about"]) < gold["opc_tolerance"]


@pytest.mark.slow
def test_paper_level_counts_300():
    gold = json.load(open(os.path.join(GOLD, "paper_structure.json")))
    h = O.Hierarchy(W.poisson7(300))
    assert h.num_levels == gold["levels"]["300"]
    assert abs(h.opc() - gold["opc_about"]) < gold["opc_tolerance"]


def test_default_params_follow_listing1():
    gold = json.load(open(os.path.join(GOLD, "paper_settings.json")))
    p = O.Params()
    L = gold["listing1"]
    assert p.aggr_steps == L["aggrsweeps"] + 1 and 2 ** p.aggr_steps == gold["sec5"]["max_aggregate_size"]
    assert p.max_levels == L["max_levels"]
    assert (p.pre_sweeps, p.post_sweeps, p.coarse_sweeps) == (L["prerelax_sweeps"], L["postrelax_sweeps"],
                                                               L["relaxnumber_coarse"])
    h = O.Hierarchy(W.poisson7(24))
    assert h.level_n(h.num_levels - 1) <= gold["sec5"]["coarsest_size_per_nd"] * 24


# ----------------------------------------------------------------------------
# V-cycle (Alg. 2 read through the operator B^k of Sec. 3.1)


def dense_B(h, n):
    return np.stack([h.vcycle(e) for e in np.eye(n)], axis=1)


def error_propagation(h, k, pre, post, coarse, jacobi=False):
    """I - B_k A_k = S^post (I - P B_{k+1} P^T A_k) S^pre, S = I - D A, written densely
    (D = 1 / sum_j |a_ij|, or 1 / a_ii for Jacobi)."""
    rp, ci, v = h.level_csr(k)
    n = h.level_n(k)
    A = dense(rp, ci, v, n)
    D = np.diag(1.0 / (np.diag(A) if jacobi else np.abs(A).sum(axis=1)))
    S = np.eye(n) - D @ A
    if k == h.num_levels - 1:
        return np.linalg.matrix_power(S, coarse) if coarse >= 0 else np.zeros((n, n))
    agg = h.level_agg(k)
    nc = h.level_n(k + 1)
    P = prolongator(agg, nc).toarray()
    rpc, cic, vc = h.level_csr(k + 1)
    Ac = dense(rpc, cic, vc, nc)
    Ec = error_propagation(h, k + 1, pre, post, coarse, jacobi)
    Bc = (np.eye(nc) - Ec) @ np.linalg.inv(Ac)
    return np.linalg.matrix_power(S, post) @ (np.eye(n) - P @ Bc @ P.T @ A) @ np.linalg.matrix_power(S, pre)


@pytest.mark.parametrize("gen", ["poisson", "diffusion"])
def test_vcycle_equals_error_propagation_formula(gen):
    A = W.poisson7(5) if gen == "poisson" else W.diffusion7(5, 2.0, 11)
    h = O.Hierarchy(A, coarse_size=8, aggr_steps=2)
    assert h.num_levels >= 2
    B = dense_B(h, A.n)
    Ad = A.to_scipy().toarray()
    E = error_propagation(h, 0, 4, 4, 20)
    assert np.allclose(np.eye(A.n) - B @ Ad, E, atol=1e-12)
    assert np.allclose(B, B.T, atol=1e-13)
    np.linalg.cholesky(B)


@pytest.mark.parametrize("gen", ["poisson", "diffusion"])
def test_jacobi_relaxation_vcycle_equals_error_propagation_formula(gen):
    """Listing 1 relax_type 0: D = 1 / a_ii on every level (the l1 norms stay
    the row sums of |a_ij|)."""
    A = W.poisson7(5) if gen == "poisson" else W.diffusion7(5, 2.0, 11)
    h = O.Hierarchy(A, coarse_size=8, aggr_steps=2, relax_type=0)
    B = dense_B(h, A.n)
    Ad = A.to_scipy().toarray()
    E = error_propagation(h, 0, 4, 4, 20, jacobi=True)
    assert np.allclose(np.eye(A.n) - B @ Ad, E, atol=1e-12)
    assert np.allclose(B, B.T, atol=1e-13)
    # the two relaxations differ (on a 7-point Poisson row M_ii is 6 vs 12)
    h4 = O.Hierarchy(A, coarse_size=8, aggr_steps=2)
    assert not np.allclose(B, dense_B(h4, A.n))
    assert np.allclose(h.level_l1(0), h4.level_l1(0))
    # the oracle accepts only the two relaxations it implements
    with pytest.raises(ValueError):
        O.Hierarchy(A, relax_type=1)


def test_vcycle_exact_coarse_spectrum_in_unit_interval():
    A = W.diffusion7(5, 1.0, 3)
    h = O.Hierarchy(A, coarse_size=10, coarse_solver=O.COARSE_DENSE_CHOL)
    B = dense_B(h, A.n)
    Ad = A.to_scipy().toarray()
    ev = sla.eigvals(B @ Ad).real
    assert ev.min() > 0 and ev.max() <= 1 + 1e-12


def test_single_level_exact_coarse_solve_converges_in_one_iteration():
    A = W.laplace1d(50)
    h = O.Hierarchy(A, coarse_size=100, coarse_solver=O.COARSE_DENSE_CHOL)
    assert h.num_levels == 1
    b = np.sin(np.arange(50))
    res = h.fcg(b, tol=1e-12)
    assert res["iters"] == 1 and res["true_rel_res"] < 1e-13
    ref = sla.solve_banded((1, 1), np.vstack([np.r_[0, -np.ones(49)], 2 * np.ones(50), np.r_[-np.ones(49), 0]]), b)
    assert np.allclose(res["x"], ref, rtol=1e-12, atol=1e-12)


def test_l1_norms_are_absolute_row_sums():
    A = W.diffusion27(5, 2.0, 9)
    h = O.Hierarchy(A, coarse_size=10)
    for k in range(h.num_levels):
        rp, ci, v = h.level_csr(k)
        ref = np.asarray(abs(sp.csr_matrix((v, ci, rp))).sum(axis=1)).ravel()
        assert np.allclose(h.level_l1(k), ref, rtol=1e-14)


# ----------------------------------------------------------------------------
# Alg. 1 (flexible PCG)


def textbook_pcg(A, B, b, tol, maxit):
    """Standard preconditioned CG with a fixed SPD preconditioner matrix B."""
    x = np.zeros_like(b)
    r = b.copy()
    z = B @ r
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    it = 0
    while np.linalg.norm(r) / nb >= tol and it < maxit:
        Ap = A @ p
        a = rz / (p @ Ap)
        x += a * p
        r -= a * Ap
        it += 1
        z = B @ r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it


def test_fcg_equals_textbook_pcg_for_fixed_preconditioner():
    A = W.diffusion7(6, 1.0, 5)
    h = O.Hierarchy(A, coarse_size=20)
    B = dense_B(h, A.n)
    b = W.random_vector(A.n, 3)
    Ad = A.to_scipy().toarray()
    res = h.fcg(b, tol=1e-10)
    x_ref, it_ref = textbook_pcg(Ad, B, b, 1e-10, 1000)
    assert abs(res["iters"] - it_ref) <= 1
    xs = np.linalg.solve(Ad, b)
    assert np.linalg.norm(res["x"] - xs) / np.linalg.norm(xs) < 1e-8
    assert np.linalg.norm(x_ref - xs) / np.linalg.norm(xs) < 1e-8


def test_unpreconditioned_cg_1d_reaches_thomas_solution():
    n = 64
    A = W.laplace1d(n)
    h = O.Hierarchy(A)
    b = W.random_vector(n, 8)
    res = h.fcg(b, tol=1e-12, precflag=0)
    assert res["status"] == O.OK and res["iters"] <= n
    ab = np.vstack([np.r_[0, -np.ones(n - 1)], 2 * np.ones(n), np.r_[-np.ones(n - 1), 0]])
    ref = sla.solve_banded((1, 1), ab, b)
    assert np.allclose(res["x"], ref, rtol=1e-9, atol=1e-9)


def test_fcg_known_solution_and_history():
    A = W.poisson7(16)
    xs = W.random_vector(A.n, 1)
    b = W.rhs_from_solution(A, xs)
    h = O.Hierarchy(A)
    res = h.fcg(b)
    assert res["status"] == O.OK
    assert res["hist"][-1] < 1e-6 <= res["hist"][-2]
    assert res["true_rel_res"] < 1e-6
    Ad = A.to_scipy()
    r = b - Ad @ res["x"]
    assert abs(np.linalg.norm(r) / np.linalg.norm(b) - res["true_rel_res"]) < 1e-12
    assert np.linalg.norm(res["x"] - xs) / np.linalg.norm(xs) < 1e-4


def test_fcg_zero_rhs_and_maxit():
    A = W.poisson7(8)
    h = O.Hierarchy(A)
    res = h.fcg(np.zeros(A.n))
    assert res["iters"] == 0 and np.all(res["x"] == 0)
    res = h.fcg(W.random_vector(A.n, 2), tol=1e-14, maxit=2)
    assert res["status"] == O.NOT_CONVERGED and res["iters"] == 2


# ----------------------------------------------------------------------------
# periodic true-residual replacement of the low-precision hierarchy (r <- b - A u
# every k iterations; the recurrences of Alg. 1 are otherwise unchanged)

def _true_residuals(h, A, b, iters):
    """|b - A u_it| / |b| by scipy for the iterates u_it of h.fcg(tol=0, maxit=it)."""
    S, nb = A.to_scipy(), np.linalg.norm(b)
    return {it: np.linalg.norm(b - S @ h.fcg(b, tol=0.0, maxit=it)["x"]) / nb for it in iters}


@pytest.mark.parametrize("prec,k", [(O.FP32, 2), (O.FP32, 3), (O.FP32_BF16FINE, 3), (O.FP32_BF16FINE, 4)])
def test_periodic_true_residual_replacement_iterations_and_values(prec, k):
    """Run far past convergence (tol = 0): the recursive residual of Alg. 1 keeps
    falling geometrically while b - A u stagnates at round-off.  A replacement
    therefore shows as a rise of the history back to the true residual, exactly
    at the multiples of k; between replacements the history falls again."""
    A = W.poisson7(14)
    b = W.rhs_from_solution(A, W.random_vector(A.n, 3))
    M = 45
    h = O.Hierarchy(A, precision=prec, true_res_every=k)
    hist = h.fcg(b, tol=0.0, maxit=M)["hist"]
    plain = O.Hierarchy(A, precision=prec, true_res_every=0).fcg(b, tol=0.0, maxit=M)["hist"]
    # the same recurrences up to the first replacement
    assert np.array_equal(hist[:k], plain[:k])
    stag = int(np.argmax(plain < 1e-20))  # the recursive residual has left the true one far behind
    assert 10 <= stag < M - 2 * k
    tr = _true_residuals(h, A, b, range(1, M + 1))
    noise = np.median([tr[it] for it in range(stag, M + 1)])
    assert noise < 1e-14
    for it in range(stag, M + 1):
        if it % k == 0:
            # replaced: the history holds |b - A u_it| (two summation orders of a
            # round-off-level quantity agree to a small factor), above its predecessor
            assert 0.25 < hist[it] / tr[it] < 4.0, (it, hist[it], tr[it])
            assert hist[it] > hist[it - 1], it
        else:
            # recursive steps after the last replacement: below it
            assert hist[it] < hist[it - (it % k)], it
    # without replacement the recursive residual ends far below the true one
    assert plain[M] < 1e-3 * noise
    # before stagnation each replaced entry is the true residual of u_it itself
    # (a residual of u_{it-1} would be a convergence factor off)
    for it in range(k, stag - 4, k):
        assert abs(hist[it] - tr[it]) <= 1e-8 * tr[it], (it, hist[it], tr[it])
        assert abs(hist[it] - hist[it - 1]) > 0.5 * hist[it]


def test_true_residual_replacement_only_in_low_precision_and_solves_converge():
    A = W.diffusion7(12, 2.0, 5)
    b = W.rhs_from_solution(A, W.random_vector(A.n, 3))
    ref64 = O.Hierarchy(A).fcg(b, tol=0.0, maxit=30)["hist"]
    for k in (1, 2, 3):
        # FP64 hierarchy: the recursive residual is never replaced
        r64 = O.Hierarchy(A, true_res_every=k).fcg(b, tol=0.0, maxit=30)
        assert np.array_equal(r64["hist"], ref64)
    for prec in (O.FP32, O.FP32_BF16FINE):
        base = O.Hierarchy(A, precision=prec, true_res_every=0).fcg(b)
        for k in (1, 2, 3):
            res = O.Hierarchy(A, precision=prec, true_res_every=k).fcg(b)
            assert res["status"] == O.OK and res["true_rel_res"] < 1e-6
            assert abs(res["iters"] - base["iters"]) <= 1
            nb = np.linalg.norm(b)
            assert abs(res["true_rel_res"] - np.linalg.norm(b - A.to_scipy() @ res["x"]) / nb) < 1e-12


# ----------------------------------------------------------------------------
# mixed precision emulation and bf16 rounding


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.standard_normal(2000).astype(np.float32),
                         np.array([1.00390625, 1.01171875, -3.0e38, 1e-40, 0.0, -0.0], np.float32)])
    ref = torch.tensor(xs).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([O.round_bf16(float(x)) for x in xs], np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("prec", [O.FP32, O.FP32_BF16FINE])
def test_mixed_precision_oracle_converges(prec):
    A = W.diffusion27(12, 2.0, 3)
    b = W.rhs_from_solution(A, W.random_vector(A.n, 3))
    h64 = O.Hierarchy(A)
    hlo = O.Hierarchy(A, precision=prec)
    r64, rlo = h64.fcg(b), hlo.fcg(b)
    assert rlo["status"] == O.OK and rlo["true_rel_res"] < 1e-6
    assert abs(rlo["iters"] - r64["iters"]) <= 3
    # one V-cycle: the low-precision hierarchy is a perturbation of the FP64 one
    r = W.random_vector(A.n, 4)
    z64, zlo = h64.vcycle(r), hlo.vcycle(r)
    tol = 1e-5 if prec == O.FP32 else 2e-2
    assert np.linalg.norm(zlo - z64) / np.linalg.norm(z64) < tol


# ----------------------------------------------------------------------------
# learned damping: loss gradient against central finite differences


def test_loss_gradient_matches_finite_differences():
    A = W.diffusion7(5, 1.5, 21)
    h = O.Hierarchy(A, coarse_size=10, aggr_steps=2)
    rng = np.random.default_rng(1)
    om = [0.7 + 0.6 * rng.random(h.level_n(k)) for k in range(h.num_levels)]
    for k in range(h.num_levels):
        h.set_omega(k, om[k])
    r0 = W.random_vector(A.n, 9)
    m = 2
    L, g = h.loss_grad(r0, m)
    assert abs(L - h.loss(r0, m)) < 1e-14
    eps = 1e-6
    for k in range(h.num_levels):
        for i in rng.choice(h.level_n(k), size=min(6, h.level_n(k)), replace=False):
            op, omn = om[k].copy(), om[k].copy()
            op[i] += eps
            omn[i] -= eps
            h.set_omega(k, op)
            Lp = h.loss(r0, m)
            h.set_omega(k, omn)
            Lm = h.loss(r0, m)
            h.set_omega(k, om[k])
            fd = (Lp - Lm) / (2 * eps)
            assert abs(fd - g[k][i]) <= 1e-5 * max(abs(fd), 1e-3), (k, i, fd, g[k][i])


@pytest.mark.parametrize("m", [1, 3])
def test_loss_equals_dense_stationary_iteration(m):
    """The training loss is (1/m) ln(|(I - A B)^m r0| / |r0|): m steps of the
    stationary iteration r <- r - A B r, with B the V-cycle written as a dense
    matrix from its columns (damping per row on every level)."""
    A = W.diffusion7(5, 1.5, 21)
    h = O.Hierarchy(A, coarse_size=10, aggr_steps=2)
    rng = np.random.default_rng(3)
    for k in range(h.num_levels):
        h.set_omega(k, 0.6 + 0.8 * rng.random(h.level_n(k)))
    B = dense_B(h, A.n)
    E = np.eye(A.n) - A.to_scipy().toarray() @ B
    r0 = W.random_vector(A.n, 9)
    ref = np.log(np.linalg.norm(np.linalg.matrix_power(E, m) @ r0) / np.linalg.norm(r0)) / m
    assert ref < 0.0
    assert abs(h.loss(r0, m) - ref) < 1e-12


def test_unit_omega_reproduces_plain_smoother_bitwise():
    A = W.poisson7(8)
    h = O.Hierarchy(A)
    r = W.random_vector(A.n, 5)
    z0 = h.vcycle(r)
    for k in range(h.num_levels):
        h.set_omega(k, np.ones(h.level_n(k)))
    assert np.array_equal(z0, h.vcycle(r))


# ----------------------------------------------------------------------------
# reference of the damping network (oracle/mlp.py)


def test_mlp_reference_backward_matches_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(mlp.NPARAM) * 0.3
    feats = rng.standard_normal((7, 4))
    dom = rng.standard_normal(7)
    g = mlp.backward(theta, feats, dom)
    eps = 1e-6
    for p in rng.choice(mlp.NPARAM, size=40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += eps
        tm[p] -= eps
        fd = (dom @ mlp.forward(tp, feats) - dom @ mlp.forward(tm, feats)) / (2 * eps)
        assert abs(fd - g[p]) <= 1e-6 * max(1.0, abs(fd)), p


def test_mlp_reference_zero_last_layer_gives_unit_damping():
    from oracle import mlp
    rng = np.random.default_rng(4)
    theta = rng.standard_normal(mlp.NPARAM)
    theta[1216:] = 0.0
    assert np.all(mlp.forward(theta, rng.standard_normal((20, 4))) == 1.0)


def test_features_reference_on_poisson():
    from oracle import mlp
    A = W.poisson7(6)
    h = O.Hierarchy(A)
    f = mlp.features(A.row_ptr, A.col_idx, A.val, h.level_l1(0), 0)
    # interior row of the 7-point stencil: l1 = 12, diagonal 6, 7 stored entries
    i = 2 + 6 * 2 + 36 * 2
    assert np.allclose(f[i], [0.5, 0.0, 7 / 27, 0.0])
    # corner row: 4 entries, l1 = 9 ; neighbours have l1 = 10
    assert np.allclose(f[0], [6 / 9, np.log(9) - np.mean(np.log([9, 10, 10, 10])), 4 / 27, 0.0])


# ----------------------------------------------------------------------------
# decoupled aggregation (Sec. 4.1) and the W-cycle (Listing 1 cycle_type 2)


def test_decoupled_matching_1d_closed_form():
    A = W.laplace1d(10)
    h = O.Hierarchy(A, num_parts=2, coarse_size=8, aggr_steps=1)
    # blocks [0,5) and [5,10): (0,1),(2,3), 4 alone | (5,6),(7,8), 9 alone
    agg = h.level_agg(0)
    assert list(agg) == [0, 0, 1, 1, 2, 3, 3, 4, 4, 5]


@pytest.mark.parametrize("np_", [1, 3, 8])
def test_decoupled_aggregates_stay_inside_blocks(np_):
    A = W.diffusion7(14, 1.5, 17)
    h = O.Hierarchy(A, num_parts=np_)
    href = O.Hierarchy(A)
    if np_ == 1:
        for k in range(h.num_levels - 1):
            assert np.array_equal(h.level_agg(k), href.level_agg(k))
    # composed map of level 0: every aggregate lies in one block of level 0
    agg = h.level_agg(0)
    bnd = [(q * A.n) // np_ for q in range(np_ + 1)]
    part = np.searchsorted(bnd, np.arange(A.n), side="right") - 1
    for J in range(h.level_n(1)):
        assert len(set(part[agg == J])) == 1
    b = W.rhs_from_solution(A, W.random_vector(A.n, 2))
    assert h.fcg(b)["status"] == O.OK


def test_wcycle_equals_error_propagation_formula():
    A = W.diffusion7(5, 1.0, 13)
    h = O.Hierarchy(A, coarse_size=8, aggr_steps=2, cycle=2)
    assert h.num_levels >= 3
    B = dense_B(h, A.n)

    def ew(k):
        rp, ci, v = h.level_csr(k)
        n = h.level_n(k)
        Ak = dense(rp, ci, v, n)
        S = np.eye(n) - np.diag(1.0 / np.abs(Ak).sum(axis=1)) @ Ak
        if k == h.num_levels - 1:
            return np.linalg.matrix_power(S, 20)
        P = prolongator(h.level_agg(k), h.level_n(k + 1)).toarray()
        rpc, cic, vc = h.level_csr(k + 1)
        Ac = dense(rpc, cic, vc, h.level_n(k + 1))
        Ec = ew(k + 1)
        Bc = (np.eye(len(Ac)) - Ec @ Ec) @ np.linalg.inv(Ac)  # two coarse visits
        return np.linalg.matrix_power(S, 4) @ (np.eye(n) - P @ Bc @ P.T @ Ak) @ np.linalg.matrix_power(S, 4)

    Ad = A.to_scipy().toarray()
    assert np.allclose(np.eye(A.n) - B @ Ad, ew(0), atol=1e-12)
    assert np.allclose(B, B.T, atol=1e-13)


# ----------------------------------------------------------------------------
# prolongator values (Sec. 3.1: entries from the smooth vector, w^{k+1} = R w^k):
# the w-normalised ablation against the literal dense construction


def _normalised_hierarchy(A, h):
    """Literal w-normalised hierarchy: P_{i,I} = w_i / |w on I|, w^{k+1} = P^T w^k,
    A^{k+1} = P^T A^k P, from the level-0 matrix and the oracle's aggregates."""
    Ak = A.to_scipy().toarray()
    w = np.ones(A.n)
    mats, Ps, ws = [Ak], [], [w]
    for k in range(h.num_levels - 1):
        agg = h.level_agg(k)
        nc = h.level_n(k + 1)
        norms = np.sqrt(np.bincount(agg, weights=w * w, minlength=nc))
        P = np.zeros((len(agg), nc))
        P[np.arange(len(agg)), agg] = w / norms[agg]
        assert np.allclose(P.T @ P, np.eye(nc), atol=1e-14)
        w = P.T @ w
        Ak = P.T @ Ak @ P
        mats.append(Ak)
        Ps.append(P)
        ws.append(w)
    return mats, Ps, ws


def test_w_normalised_prolongator_vcycle_equals_literal_construction():
    A = W.diffusion7(5, 2.0, 11)  # aggregates of unequal sizes
    hn = O.Hierarchy(A, coarse_size=8, aggr_steps=2, prolong_scale=O.PROLONG_W_NORMALIZED)
    hu = O.Hierarchy(A, coarse_size=8, aggr_steps=2)
    assert hn.num_levels == hu.num_levels >= 3
    for k in range(hn.num_levels - 1):
        assert np.array_equal(hn.level_agg(k), hu.level_agg(k))
    mats, Ps, _ = _normalised_hierarchy(A, hn)

    def err(k):  # I - B_k A_k on the normalised matrices, l1 of their own rows
        Ak = mats[k]
        S = np.eye(len(Ak)) - np.diag(1.0 / np.abs(Ak).sum(axis=1)) @ Ak
        if k == len(mats) - 1:
            return np.linalg.matrix_power(S, 20)
        P = Ps[k]
        Bc = (np.eye(len(mats[k + 1])) - err(k + 1)) @ np.linalg.inv(mats[k + 1])
        S4 = np.linalg.matrix_power(S, 4)
        return S4 @ (np.eye(len(Ak)) - P @ Bc @ P.T @ Ak) @ S4

    Ad = A.to_scipy().toarray()
    Bn = dense_B(hn, A.n)
    assert np.allclose(np.eye(A.n) - Bn @ Ad, err(0), atol=1e-12)
    assert np.allclose(Bn, Bn.T, atol=1e-13)
    # with unequal aggregate sizes the two prolongator forms give different cycles
    assert np.abs(Bn - dense_B(hu, A.n)).max() > 1e-6
    # the learned part's gradient is defined for unit prolongators only
    assert np.isnan(hn.loss_grad(W.random_vector(A.n, 1), 1)[0])


def test_w_normalised_matching_weights_equal_unit_ones():
    """The weight of Sec. 3.1 / reading 1 on (A_norm^k, w^k) equals the weight on
    (A^k, 1) at every pairwise step (aggr_steps = 1: every step is a level), so
    the normalisation leaves the matching unchanged."""
    A = W.diffusion27(6, 2.0, 5)
    h = O.Hierarchy(A, coarse_size=4, aggr_steps=1)
    assert h.num_levels >= 4
    mats, _, ws = _normalised_hierarchy(A, h)
    for k in range(h.num_levels - 1):
        rp, ci, v = h.level_csr(k)
        unit = O.weights(rp, ci, v)
        An, w = mats[k], ws[k]
        rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        off = rows != ci
        a = An[rows, ci]
        d = np.diag(An)
        wn = 1.0 - 2.0 * a * w[rows] * w[ci] / (d[rows] * w[rows] ** 2 + d[ci] * w[ci] ** 2)
        assert np.allclose(wn[off], unit[off], rtol=0, atol=1e-12)


def test_w_normalised_equals_unit_on_equal_aggregate_sizes():
    """All aggregates of a level of one size: w is constant per level, w_I / w_J = 1
    exactly, and the two forms run the same arithmetic bit for bit."""
    A = W.poisson7(8)
    hn = O.Hierarchy(A, coarse_size=8, prolong_scale=O.PROLONG_W_NORMALIZED)
    hu = O.Hierarchy(A, coarse_size=8)
    assert hn.num_levels == 3
    b = W.rhs_from_solution(A, W.random_vector(A.n, 3))
    rn, ru = hn.fcg(b), hu.fcg(b)
    assert rn["iters"] == ru["iters"]
    assert np.array_equal(rn["x"], ru["x"]) and np.array_equal(rn["hist"], ru["hist"])
    with pytest.raises(ValueError):
        O.Hierarchy(A, prolong_scale=2)


def test_unstructured_workload_shape():
    """The random-graph workload of the unstructured GPU cases has what they
    rely on: rows of one entry (isolated) to a few hundred, a bitwise symmetric
    pattern and values, strict diagonal dominance, and a coarse level whose
    rows are longer than any pipelined tile of 8 rows holds."""
    A = W.random_spd(5000, 7)
    rl = np.diff(A.row_ptr)
    assert rl.min() == 1 and rl.max() >= 150
    S = A.to_scipy()
    assert (S != S.T).nnz == 0
    d = S.diagonal()
    assert np.all(d > np.abs(S).sum(axis=1).A1 - d)
    o = O.Hierarchy(A)
    assert o.num_levels >= 2
    assert np.diff(o.level_csr(1)[0]).max() > 256
    b = W.rhs_from_solution(A, W.random_vector(A.n, 3))
    assert o.fcg(b)["status"] == O.OK


def test_explicit_zeros_are_not_edges():
    """Reading 1: a stored entry with the value 0.0 is no edge of the matching
    graph (weight 0, never matched), and the Galerkin product keeps the
    structural zeros and the cancellations it produces."""
    A = W.random_spd(600, 21, mixed_sign=True, zero_frac=0.3)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    zero = (A.val == 0.0) & (rows != A.col_idx)
    assert zero.sum() > 100
    wgt = O.weights(A.row_ptr, A.col_idx, A.val)
    assert np.all(wgt[zero] == 0.0) and np.all(wgt[~zero & (rows != A.col_idx)] > 0.0)
    mate = O.match_greedy(A.row_ptr, A.col_idx, wgt)
    S = A.to_scipy()
    for i in np.flatnonzero(mate >= 0):
        assert S[i, mate[i]] != 0.0
    # pattern of A_c = P^T |pattern| P, values = P^T A P with the zeros kept
    agg, nc = O.aggregate(mate)
    rpc, cic, vc = O.galerkin(A.row_ptr, A.col_idx, A.val, agg, nc)
    P = sp.csr_matrix((np.ones(A.n), (np.arange(A.n), agg)), shape=(A.n, nc))
    pat = (P.T @ sp.csr_matrix((np.ones(A.nnz), A.col_idx, A.row_ptr), shape=(A.n, A.n)) @ P).tocsr()
    pat.sort_indices()
    assert np.array_equal(rpc, pat.indptr) and np.array_equal(cic, pat.indices)
    assert np.allclose(dense(rpc, cic, vc, nc), (P.T @ S @ P).toarray(), rtol=0, atol=1e-13)


def _laplace1d_l1_four(n):
    """tridiag(-1, 2, -1) with 3 in the two corner diagonal entries: every l1
    row norm is 4 on every level of its hierarchy (pairwise Galerkin keeps
    the form), so D = 1/4 and small-integer inputs keep every intermediate
    of a short V-cycle exact in float32."""
    A = W.laplace1d(n)
    v = A.val.copy()
    for i in (0, n - 1):
        for p in range(A.row_ptr[i], A.row_ptr[i + 1]):
            if A.col_idx[p] == i:
                v[p] = 3.0
    return W.CSR(n, A.row_ptr, A.col_idx, v)


@pytest.mark.parametrize("kw,levels", [
    (dict(coarse_size=4, aggr_steps=1, pre_sweeps=1, post_sweeps=2, coarse_sweeps=2), 4),
    (dict(coarse_size=4, aggr_steps=2, pre_sweeps=2, post_sweeps=2, coarse_sweeps=2), 3),
    (dict(coarse_size=4, aggr_steps=2, pre_sweeps=1, post_sweeps=1, coarse_sweeps=1, cycle=2), 3),
])
def test_low_precision_vcycle_equals_fp64_in_exact_arithmetic(kw, levels):
    """The float V-cycle of the mixed-precision emulation is separate code from
    the FP64 one; where no operation rounds (values, D = 1/4 and the
    intermediates of small-integer inputs are all exact in float32 and bf16),
    both must give the same bits, so a dropped term, a wrong index or a
    missing sweep in the float path shows up; with a generic input they differ
    by float32 rounding only."""
    A = _laplace1d_l1_four(16)
    hd = O.Hierarchy(A, **kw)
    assert hd.num_levels == levels
    assert all(np.all(hd.level_l1(k) == 4.0) for k in range(levels))
    r = np.floor(W.random_vector(A.n, 5) * 4)
    zd = hd.vcycle(r)
    rg = W.random_vector(A.n, 6)
    zg = hd.vcycle(rg)
    for prec in (O.FP32, O.FP32_BF16FINE):
        hf = O.Hierarchy(A, precision=prec, **kw)
        assert np.array_equal(hf.vcycle(r), zd)
        zf = hf.vcycle(rg)
        assert not np.array_equal(zf, zg) and np.linalg.norm(zf - zg) < 1e-6 * np.linalg.norm(zg)


# ----------------------------------------------------------------------------
# the OpenMP build of the oracle (timed CPU baseline only) computes the same solve


def test_openmp_build_matches_serial_checker():
    A = W.diffusion27(14, 2.0, 7)
    b = W.rhs_from_solution(A, W.random_vector(A.n, 2))
    ser, par = O.Hierarchy(A), O.Hierarchy(A, omp=True)
    assert O.threads(omp=False) == 1 and O.threads(omp=True) >= 1
    for k in range(ser.num_levels - 1):
        assert np.array_equal(ser.level_agg(k), par.level_agg(k))
    r = W.random_vector(A.n, 3)
    zs, zp = ser.vcycle(r), par.vcycle(r)
    assert np.array_equal(zs, zp)  # row loops only: every row sums in the same order
    rs, rp_ = ser.fcg(b), par.fcg(b)
    assert rp_["status"] == O.OK and abs(rs["iters"] - rp_["iters"]) <= 1
    m = min(rs["iters"], rp_["iters"])
    xs = ser.fcg(b, tol=0.0, maxit=m)["x"]
    xp = par.fcg(b, tol=0.0, maxit=m)["x"]
    assert np.linalg.norm(xs - xp) / np.linalg.norm(xs) < 1e-10  # the dot products sum in another order


def test_stored_oracle_reference_matches_the_oracle():
    """tests/golden/oracle_reference.json (written by make_oracle_reference.py,
    which calls only the oracle) still describes the oracle: the 32^3 entry is
    recomputed here; the GPU tests compare against the stored entries."""
    gold = json.load(open(os.path.join(GOLD, "oracle_reference.json")))
    ref = gold["poisson32:fp64"]
    A, b, _ = W.config("poisson32")
    h = O.Hierarchy(A)
    assert h.num_levels == ref["levels"]
    assert [h.level_n(k) for k in range(h.num_levels)] == ref["n"]
    assert [h.level_nnz(k) for k in range(h.num_levels)] == ref["nnz"]
    res = h.fcg(b)
    assert res["iters"] == ref["iters"] and res["status"] == ref["status"]
    assert abs(res["true_rel_res"] - ref["true_rel_res"]) <= 1e-12 * ref["true_rel_res"]
