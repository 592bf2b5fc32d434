"""bench.py on CPU: the clock-sample summary, the replica plumbing (two gloo
ranks, barrier and the maximum over ranks of the per-rank step time, what the
benchmark reports for N > 1) and the reference arm (the oracle on the host
cores: its JSON line, and ranks other than 0 leaving without output)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, w, local = bench.dist_env()
    d = bench.Dist(w, "gloo")
    d.barrier()
    mx = d.max(10.0 + 5.0 * r)
    d.barrier()
    d.close()
    q.put((r, w, local, mx))


def test_two_gloo_ranks_report_the_maximum():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 0, 15.0), (1, 2, 1, 15.0)]


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench
    assert bench.dist_env() == (0, 1, 0)
    d = bench.Dist(1, "gloo")
    assert d.max(3.5) == 3.5
    d.barrier()
    d.close()


def _bench(args, env_extra=None):
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(root, "bench.py"), *args], env=env, cwd=root,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_line_on_cpu():
    """`bench.py --impl reference` (the oracle timed on the host cores) prints
    one JSON line with the contract's keys; it needs no GPU."""
    import json
    r = _bench(["--impl", "reference", "--workload", "poisson32", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "ms" and d["value"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is False
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["iters"] > 0 and "32^3" in d["config"]["workload"]


def test_reference_arm_other_ranks_exit_quietly():
    r = _bench(["--impl", "reference", "--workload", "poisson32", "--steps", "1", "--warmup", "0"],
               {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_clock_samples_summary():
    """The clock record of the bench line: median SM clock under load, the
    highest max clock and power, and every throttle reason seen active, for
    the bench's own GPU only."""
    import bench
    lines = [
        "0, 2070, 2070, 700.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1, 1200, 2070, 300.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "0, 2010, 2070, 810.9, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 650.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    c = bench.parse_clocks(lines, 0)
    assert c["samples"] == 3 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["power_w_max"] == 810.9 and c["reasons"] == ["sw_power_cap"]
    assert bench.parse_clocks(lines, 1)["reasons"] == ["hw_slowdown"]
    assert bench.parse_clocks(lines, 5) is None
