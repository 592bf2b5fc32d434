"""The bounds-checked build (AMG_CHECKED): every gather index of the
solve-phase kernels is checked on the device.  Run on small problems through
every kernel form, it must report no violation and give the normal build's
results bit for bit (the checks only read indices)."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from paper_2303_02352_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, problem, hierarchy parameters, environment of the setup)
CASES = [
    ("poisson13", "W.poisson7(13)", {}, {}),
    ("diff27_12", "W.diffusion27(12, 2.0, 3)", {}, {}),
    ("diff27_12_fp32", "W.diffusion27(12, 2.0, 3)", {"precision": 1}, {}),
    ("poisson32_bottom", "W.poisson7(32)", {}, {"AMG_BOTTOM": "1"}),
    ("poisson32_pair", "W.poisson7(32)", {}, {"AMG_PAIR": "2", "AMG_PAIR_SLACK": "1"}),
    ("poisson32_tiled", "W.poisson7(32)", {}, {"AMG_PIPE": "0"}),
    ("diff7_20_wcycle", "W.diffusion7(20, 2.0, 1001)", {"cycle": 2}, {}),
    ("diff7_20_bf16", "W.diffusion7(20, 2.0, 1001)", {"precision": 2}, {}),
    ("rand5k_mixed", "W.random_spd(5000, 8, mixed_sign=True)", {}, {}),
    ("rand5k_mixed_bottom", "W.random_spd(5000, 8, mixed_sign=True)", {}, {"AMG_BOTTOM": "1"}),
    ("rand20k_tiled", "W.random_spd(20000, 9)", {}, {"AMG_PIPE": "0"}),
    ("rand20k_fp32", "W.random_spd(20000, 9)", {"precision": 1}, {}),
]

RUNNER = r"""
import os, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
from paper_2303_02352_gb300 import amg, workloads as W
amg.load()
out = sys.argv[2]
for name, prob, kw, env in CASES:
    for k in ("AMG_BOTTOM", "AMG_PAIR", "AMG_PAIR_SLACK", "AMG_PIPE"):
        os.environ.pop(k, None)
    os.environ.update(env)
    A = eval(prob)
    g = amg.Hierarchy(A, **kw)
    r = W.random_vector(A.n, 3)
    z = g.vcycle(r).cpu().numpy()
    b = W.rhs_from_solution(A, W.random_vector(A.n, 4))
    res = g.pcg_solve(b)
    np.save(os.path.join(out, name + "_z.npy"), z)
    np.save(os.path.join(out, name + "_x.npy"), res["x"].cpu().numpy())
    g.close()
print("done")
"""


def _run(lib_path, outdir):
    code = "CASES = %r\n" % (CASES,) + RUNNER
    env = dict(os.environ)
    if lib_path:
        env["AMG_LIB"] = lib_path
    else:
        env.pop("AMG_LIB", None)
    r = subprocess.run([sys.executable, "-c", code, ROOT, outdir], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "done" in r.stdout


def test_checked_build_reports_nothing_and_matches_normal_build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_02352_gb300 import build
    normal = build.build()
    checked = build.build(checked=True)
    assert normal != checked and os.path.exists(checked)
    with tempfile.TemporaryDirectory() as d0, tempfile.TemporaryDirectory() as d1:
        _run(normal, d0)
        _run(checked, d1)  # an out-of-range index would raise AMG_ERR_CUDA in the child
        for name, *_ in CASES:
            for part in ("z", "x"):
                a = np.load(os.path.join(d0, f"{name}_{part}.npy"))
                c = np.load(os.path.join(d1, f"{name}_{part}.npy"))
                assert np.array_equal(a, c), (name, part)
