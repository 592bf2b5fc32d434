"""The device problem generators (amg_generate_stencil, amg_random_vector,
amg_csr_times) against the host generator, through the C ABI: the stencil
matrices bit for bit (7 and 27 points, constant and block-wise coefficients,
blocks that do not divide N, the smallest grid), x* and b = A x* bit for bit,
a hierarchy built from the device matrix equal to one built from the host
matrix, and invalid arguments rejected."""
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


def same(dev, host, dtype):
    d = dev.cpu().numpy()
    h = np.asarray(host, dtype=dtype)
    return d.shape == h.shape and np.array_equal(d.view(np.uint8), h.view(np.uint8))


@pytest.mark.parametrize("N,points,sigma,block", [(3, 7, None, 8), (17, 7, None, 8), (12, 7, 2.0, 8), (13, 7, 1.5, 5),
                                                  (3, 27, 1.0, 8), (11, 27, 2.0, 4), (20, 27, 2.5, 8)])
def test_stencil_matches_host_generator(N, points, sigma, block):
    from paper_2303_02352_gb300 import amg
    if sigma is None:
        host = W.poisson7(N)
        kb = None
    else:
        host = (W.diffusion7 if points == 7 else W.diffusion27)(N, sigma, 77, block)
        kb = W.block_values(N, sigma, 77, block)
    rp, ci, v = amg.generate_stencil(N, points, kb, block)
    assert same(rp, host.row_ptr, np.int32) and same(ci, host.col_idx, np.int32)
    assert same(v, host.val, np.float64)


@pytest.mark.parametrize("name", ["poisson32", "poisson160", "diffusion7_48", "diffusion27_128"])
def test_named_workload_on_device(name):
    from paper_2303_02352_gb300 import amg
    (rp, ci, v), b, xs = amg.generate(name)
    A, b_host, _ = W.config(name)
    assert same(rp, A.row_ptr, np.int32) and same(ci, A.col_idx, np.int32) and same(v, A.val, np.float64)
    assert same(xs, W.exact_solution(name, A.n), np.float64)
    assert same(b, b_host, np.float64)


def test_hierarchy_from_device_matrix_equals_host_one():
    from paper_2303_02352_gb300 import amg
    (rp, ci, v), b, _ = amg.generate("diffusion7_24")
    A, b_host, _ = W.config("diffusion7_24")
    gd, gh = amg.Hierarchy(amg.DeviceCSR(rp, ci, v)), amg.Hierarchy(A)
    assert gd.info()["n"] == gh.info()["n"]
    for k in range(gd.num_levels - 1):
        assert np.array_equal(gd.aggregates(k), gh.aggregates(k))
    xd, xh = gd.pcg_solve(b)["x"].cpu().numpy(), gh.pcg_solve(b_host)["x"].cpu().numpy()
    assert np.array_equal(xd.view(np.uint64), xh.view(np.uint64))


def test_generators_reject_bad_arguments():
    from paper_2303_02352_gb300 import amg
    for N, pts in ((2, 7), (10, 9), (431, 27)):
        with pytest.raises(amg.AmgError):
            amg.generate_stencil(N, pts, None if pts == 7 else np.ones(1000, np.float32))
    with pytest.raises(amg.AmgError, match="coefficient"):
        amg.generate_stencil(10, 27, None)
    lib = amg.load()
    assert lib.amg_random_vector(-1, 1, None, None) == amg.ERR_INVALID_ARG
    assert amg.random_vector(0, 3).numel() == 0
