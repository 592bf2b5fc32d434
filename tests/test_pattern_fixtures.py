"""CPU pins of the tuple counts the pattern-coded column tests rely on: the
number of distinct column-offset tuples (j - i over a row's entries, CSR
order) of the fixtures and of the stencil workloads, counted row by row."""
import numpy as np
import pytest

from paper_2303_02352_gb300 import workloads as W
from pattern_fixtures import block_diagonal, paired_rows


def tuples(A):
    rp, ci = A.row_ptr, A.col_idx
    return {tuple(int(c) - i for c in ci[rp[i]:rp[i + 1]]) for i in range(A.n)}


@pytest.mark.parametrize("make", [lambda: W.poisson7(12), lambda: W.diffusion7(12, 2.0, 5),
                                  lambda: W.diffusion27(10, 2.0, 3)])
def test_stencils_have_27_tuples(make):
    """Low face, interior and high face on each axis: 3^3 tuples for a 7- or
    27-point stencil on an N^3 grid (Dirichlet unknowns eliminated)."""
    assert len(tuples(make())) == 27


@pytest.mark.parametrize("dmax, singleton, expect", [(127, True, 255), (128, False, 256)])
def test_paired_rows_tuple_count(dmax, singleton, expect):
    A = paired_rows(dmax, singleton, 1)
    assert len(tuples(A)) == expect
    assert max(np.diff(A.row_ptr)) == 2
    S = A.to_scipy()
    assert (S != S.T).nnz == 0


def test_block_diagonal_tuple_count():
    A = block_diagonal(list(range(1, 22)), 1)
    assert len(tuples(A)) == 231 and max(np.diff(A.row_ptr)) == 21
