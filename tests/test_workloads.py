"""The seeded input generators against definitions they do not share code with:
the published SplitMix64 sequence, the Kronecker-sum form of the 7-point
Dirichlet Laplacian, closed-form nonzero counts, and the special cases in which
the variable-coefficient problems reduce to the constant ones."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2303_02352_gb300 import workloads as W


def test_splitmix64_published_sequence():
    # the first outputs of SplitMix64 started at state 0 (Steele, Lea and
    # Flood's generator as published with its reference implementation)
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [int(v) for v in W.splitmix64(0, np.arange(4))] == want
    # counter form: output i of the stream started at seed s is output 0 of s + i * gamma
    gamma = 0x9E3779B97F4A7C15
    s = 12345
    for i in range(5):
        direct = int(W.splitmix64(s, np.array([i]))[0])
        assert direct == int(W.splitmix64((s + i * gamma) % 2 ** 64, np.array([0]))[0])
    u = W.uniform01(7, np.arange(100000))
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def _kron_laplacian(N):
    T = sp.diags([-np.ones(N - 1), 2 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1])
    I = sp.identity(N)
    K = (sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I)).tocsr()
    K.sum_duplicates()
    K.eliminate_zeros()
    return K


@pytest.mark.parametrize("N", [3, 5, 12])
def test_poisson7_is_the_kronecker_sum(N):
    A = W.poisson7(N)
    assert A.n == N ** 3 and A.nnz == 7 * N ** 3 - 6 * N ** 2
    K = _kron_laplacian(N)
    K.sort_indices()
    assert np.array_equal(A.row_ptr, K.indptr) and np.array_equal(A.col_idx, K.indices)
    assert np.array_equal(A.val, K.data)
    for i in range(0, A.n, max(1, A.n // 50)):  # columns strictly ascending
        assert np.all(np.diff(A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]) > 0)


def test_constant_coefficient_special_cases():
    N = 9
    # sigma = 0: k = 1 everywhere, harmonic means are exactly 1
    assert np.array_equal(W.diffusion7(N, 0.0, 3).val, W.poisson7(N).val)
    A = W.diffusion27(N, 0.0, 3)
    assert A.nnz == (3 * N - 2) ** 3
    S = A.to_scipy()
    off = S - sp.diags(S.diagonal())
    assert set(np.round(-off.data, 12)) == {1.0, 0.5, round(1 / 3, 12)}
    # every row's diagonal counts all 26 links (Dirichlet links included)
    assert np.allclose(S.diagonal(), 6 + 12 / 2 + 8 / 3, rtol=0, atol=1e-13)


@pytest.mark.parametrize("points", [7, 27])
def test_variable_coefficient_problems_are_symmetric_m_matrices(points):
    N = 10
    A = (W.diffusion7 if points == 7 else W.diffusion27)(N, 2.0, 5)
    S = A.to_scipy()
    assert (S != S.T).nnz == 0  # bitwise symmetric
    d = S.diagonal()
    off = S - sp.diags(d)
    assert np.all(off.data <= 0) and np.all(d > 0)
    rows = np.asarray(S.sum(axis=1)).ravel()
    assert np.all(rows >= -1e-12 * d)  # weakly diagonally dominant, strictly on the boundary
    # interior rows sum to zero (no Dirichlet link), boundary rows do not
    x, y, z = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    inner = (x > 0) & (x < N - 1) & (y > 0) & (y < N - 1) & (z > 0) & (z < N - 1)
    interior = inner.transpose(2, 1, 0).ravel()
    assert np.all(np.abs(rows[interior]) <= 1e-12 * d[interior])
    assert np.all(rows[~interior] > 1e-12 * d[~interior])


def test_block_field_is_blockwise_and_float32_exact():
    k = W.block_field(16, 2.0, 3, block=8)
    assert np.array_equal(k.astype(np.float32).astype(np.float64), k)
    g = k.reshape(16, 16, 16)  # z, y, x
    for bz in (0, 8):
        for by in (0, 8):
            for bx in (0, 8):
                blk = g[bz:bz + 8, by:by + 8, bx:bx + 8]
                assert np.all(blk == blk.flat[0])
    assert len(np.unique(k)) == 8


def test_rhs_and_vectors():
    A = W.poisson7(6)
    x = W.random_vector(A.n, 4)
    assert np.all(np.abs(x) <= 1.0)
    assert np.allclose(W.rhs_from_solution(A, x), A.to_scipy() @ x, rtol=0, atol=1e-14)
    b = W.config("poisson32")[1]
    assert np.allclose(b, W.poisson7(32).to_scipy() @ W.exact_solution("poisson32", 32 ** 3), rtol=0, atol=1e-13)
