"""Saving a hierarchy to a file and loading it back (amg_save / amg_load),
through the C ABI.

A loaded handle must compute bit for bit what the saved one did: same level
sizes and kernel forms, the same V-cycle and the same solve, for the FP64,
FP32 and BF16-finest forms, with the learned damping applied, with the
w-normalised prolongator and with decoupled aggregation.  Loading with another
precision equals a fresh setup in that precision.  Files that are missing,
foreign, truncated or corrupt, and parameters that would change the
hierarchy, are rejected with an error.
"""
import os

import numpy as np
import pytest

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


def same_bits(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))


def check_same(g, h, A, b):
    ig, ih = g.info(), h.info()
    for key in ("num_levels", "n", "nnz", "tile_rows", "stage_scale", "bottom_level", "vcycle_launches",
                "precision"):
        assert ig[key] == ih[key], key
    for k in range(ig["num_levels"]):
        for x, y in zip(g.level_csr(k), h.level_csr(k)):
            assert np.array_equal(x, y)
        if k < ig["num_levels"] - 1:
            assert np.array_equal(g.aggregates(k), h.aggregates(k))
    r = W.random_vector(A.n, 17)
    assert same_bits(g.vcycle(r).cpu().numpy(), h.vcycle(r).cpu().numpy())
    rg, rh = g.pcg_solve(b), h.pcg_solve(b)
    assert rg["iters"] == rh["iters"] and same_bits(rg["x"].cpu().numpy(), rh["x"].cpu().numpy())
    assert np.array_equal(rg["hist"], rh["hist"])


@pytest.mark.parametrize("kw", [dict(), dict(precision=1), dict(precision=2), dict(prolong_scale=1),
                                dict(num_parts=4), dict(relax_type=0, cycle=2)])
def test_save_load_round_trip_bitwise(tmp_path, kw):
    from paper_2303_02352_gb300 import amg
    A = W.diffusion7(22, 2.0, 303)
    b = W.rhs_from_solution(A, W.random_vector(A.n, 4))
    g = G(A, **kw)
    path = str(tmp_path / "h.amg")
    g.save(path)
    assert os.path.getsize(path) > 12 * A.nnz
    h = amg.Hierarchy.load(path)
    assert h.params == g.params
    check_same(g, h, A, b)


def test_save_load_keeps_the_learned_damping(tmp_path):
    from paper_2303_02352_gb300 import amg, learned
    A = W.diffusion7(20, 2.0, 404)
    b = W.rhs_from_solution(A, W.random_vector(A.n, 5))
    theta = learned.init_theta(3)
    theta[1216:] = 0.3 * np.random.default_rng(8).standard_normal(33)  # a non-trivial last layer
    net = learned.Network(theta)
    g = G(A)
    g.apply_mlp(net.w)
    path = str(tmp_path / "learned.amg")
    g.save(path)
    h = amg.Hierarchy.load(path)
    check_same(g, h, A, b)
    # the damping is really there: a plain hierarchy differs
    r = W.random_vector(A.n, 17)
    assert not same_bits(G(A).vcycle(r).cpu().numpy(), h.vcycle(r).cpu().numpy())


def test_load_with_another_precision_equals_fresh_setup(tmp_path):
    from paper_2303_02352_gb300 import amg
    A = W.diffusion27(14, 2.0, 5)
    b = W.rhs_from_solution(A, W.random_vector(A.n, 6))
    path = str(tmp_path / "h64.amg")
    G(A).save(path)
    for prec in (1, 2):
        check_same(G(A, precision=prec), amg.Hierarchy.load(path, precision=prec, pre_sweeps=4), A, b)


def test_load_rejects_bad_files_and_parameters(tmp_path):
    from paper_2303_02352_gb300 import amg
    A = W.poisson7(12)
    path = str(tmp_path / "ok.amg")
    G(A).save(path)
    raw = open(path, "rb").read()
    with pytest.raises(amg.AmgError, match="cannot open|not a readable"):
        amg.Hierarchy.load(str(tmp_path / "missing.amg"))
    foreign = tmp_path / "foreign.amg"
    foreign.write_bytes(b"NOTAHIER" + raw[8:])
    with pytest.raises(amg.AmgError):
        amg.Hierarchy.load(str(foreign))
    trunc = tmp_path / "trunc.amg"
    trunc.write_bytes(raw[: len(raw) // 2])
    with pytest.raises(amg.AmgError, match="ends|truncated"):
        amg.Hierarchy.load(str(trunc))
    # a column index of level 0 out of range (the first column entry, after the
    # header, the level count, n, nnz and the row pointers)
    q = 14
    off = 8 + 4 + 4 + 4 * q + 4 + 4 + 4 + 8 + 4 * (A.n + 1)
    bad = bytearray(raw)
    bad[off:off + 4] = np.int32(10 ** 6).tobytes()
    corrupt = tmp_path / "corrupt.amg"
    corrupt.write_bytes(bytes(bad))
    with pytest.raises(amg.AmgError, match="column"):
        amg.Hierarchy.load(str(corrupt))
    with pytest.raises(amg.AmgError, match="must equal"):
        amg.Hierarchy.load(path, aggr_steps=2)
    # the file itself still loads
    h = amg.Hierarchy.load(path)
    assert h.pcg_solve(W.rhs_from_solution(A, W.random_vector(A.n, 1)))["status"] == 0
