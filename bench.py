#!/usr/bin/env python
"""AMG-PCG solve-phase benchmark (arXiv:2303.02352 method on one GB300).

Metric: time of one AMG-preconditioned flexible CG solve to a 1e-6 relative
residual (setup excluded), plus the HBM roofline of the dominant kernel and of
the whole V-cycle.  One step = one complete solve of the workload from u_0 = 0:
every FCG iteration (V-cycle, SpMV + dots, axpys, stop test) through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload poisson320] [--precision fp64|fp32|bf16fine]

The default workload is the largest single-GPU configuration, 7-point Poisson
320^3 (32.8M rows, 228.8M nonzeros).

Several GPUs run independent replicas (the path has no exchange step on one
node's worth of work): each rank solves its own copy, the step time is the
maximum over ranks.  --impl reference times the CPU oracle on the same workload
(its OpenMP build, on every core of the host).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AMG-PCG solve ms to 1e-6 rel. residual; V-cycle HBM GB/s vs 8 TB/s peak"
UNIT = "ms"
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16fine": 2}
DTYPE = {"fp64": "f64", "fp32": "f32 hierarchy, f64 outer", "bf16fine": "bf16 level-0 values, f32 hierarchy, f64 outer"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="poisson320")
    ap.add_argument("--precision", choices=list(PRECISIONS), default="fp64")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--learned", action="store_true", help="time the solve with the trained damping network")
    ap.add_argument("--no-extra", action="store_true", help="skip the comparison solves of the other forms")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas)

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Dist:
    def __init__(self, world, backend):
        self.world = world
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if torch.cuda.is_available() and self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks during the timed region

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            lines = open(self.path).read().splitlines()
            os.unlink(self.path)
        except Exception:
            return None
        return parse_clocks(lines, self.idx)


def parse_clocks(lines, idx: int) -> dict | None:
    """Summary of nvidia-smi samples (Clocks.FIELDS, csv, no header) of GPU idx."""
    rows = []
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) >= 9 and f[0] == str(idx):
            rows.append(f)
    if not rows:
        return None

    def num(x):
        try:
            return float(x)
        except ValueError:
            return float("nan")

    sm = [num(r[1]) for r in rows]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower().startswith("active")})
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(num(r[2]) for r in rows),
            "power_w_max": max(num(r[3]) for r in rows), "samples": len(rows), "reasons": reasons,
            "window": "every 100 ms over the timed steps and 0.5 s of the same solves before and after"}


def gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


# ---------------------------------------------------------------------------
# roofline denominators and ncu traffic

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the sources that define the dominant kernel (the pipelined row kernel and the
# device helpers it uses); its launch shape on level 0 is checked separately
KERNEL_SOURCES = ("rows.cuh", "amg_internal.cuh")


# nominal dense FP64 rate of one GB300 (2 multiply-adds per clock per
# multiprocessor, 152 multiprocessors, 2.07 GHz)
FP64_TFLOPS = 1.25


def _code_only(text: str) -> str:
    """The source without comments and with runs of whitespace collapsed, so
    that a comment edit does not void a record of the compiled kernel."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_digest() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2303_02352_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(_code_only(open(os.path.join(d, f)).read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, precision: str, tile_rows: int, stage_scale: int, column_patterns: int):
    """DRAM bytes per launch of the dominant kernel from the committed ncu record,
    or None when that record was taken on other kernel sources or another
    launch shape (tile height, stage size, column form) of the level-0 kernel."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(f"{workload}:{precision}")
    if not d or d.get("kernel_digest") != kernel_digest():
        return None
    if d.get("tile_rows") != tile_rows or d.get("stage_scale") != stage_scale:
        return None
    if d.get("column_patterns", 0) != column_patterns:
        return None
    return d.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm)

def oracle_solve_ms(A, b, precision: str, maxit=1000):
    """One complete solve of the oracle's OpenMP build (every host core in the
    affinity mask); returns (solve ms, setup ms, iterations, x, threads)."""
    import oracle as O
    t0 = time.perf_counter()
    h = O.Hierarchy(A, omp=True, precision={"fp64": O.FP64, "fp32": O.FP32, "bf16fine": O.FP32_BF16FINE}[precision])
    t1 = time.perf_counter()
    res = h.fcg(b, maxit=maxit)
    t2 = time.perf_counter()
    return (t2 - t1) * 1e3, (t1 - t0) * 1e3, res["iters"], res["x"], O.threads(omp=True)


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_2303_02352_gb300 import workloads as W
    A, b, desc = W.config(args.workload)
    import oracle as O
    prec = {"fp64": O.FP64, "fp32": O.FP32, "bf16fine": O.FP32_BF16FINE}[args.precision]
    h = O.Hierarchy(A, precision=prec, omp=True)
    cores = O.threads(omp=True)
    # the first warm-up step is a complete solve: it fixes the iteration count
    t0 = time.perf_counter()
    full = h.fcg(b, tol=args.tol)
    t_full = time.perf_counter() - t0
    iters = max(1, full["iters"])
    per_step_budget = 200.0 / max(1, args.steps + args.warmup)
    sample_it = iters if t_full <= per_step_budget else max(1, int(per_step_budget / (t_full / iters)))
    for _ in range(max(0, args.warmup - 1)):
        h.fcg(b, tol=0.0, maxit=sample_it)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        h.fcg(b, tol=0.0 if sample_it < iters else args.tol, maxit=sample_it)
        times.append((time.perf_counter() - t0) * 1e3 * iters / sample_it)
    ms = sum(times) / len(times)
    kind = f"oracle (C, OpenMP build, {cores} threads)"
    sample = (f"{kind} on {desc}: each step one FCG solve to {args.tol:g}, setup excluded"
              if sample_it >= iters else
              f"{kind} on {desc}: each step {sample_it} of the {iters} FCG iterations, scaled to {iters}; "
              f"setup excluded")
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else DTYPE[args.precision],
            "data": "synthetic", "config": {"workload": desc, "precision": args.precision, "iters": full["iters"]},
            "cpu_baseline": {"value": ms, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm

def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    import numpy as np
    import torch

    from paper_2303_02352_gb300 import amg, build
    from paper_2303_02352_gb300 import workloads as W

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = Dist(world, "nccl")
    build.build()
    A, b_np, desc = W.config(args.workload)
    n = A.n

    # CPU baseline first (host only, rank 0, N = 1)
    cpu = None
    x_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ms_o, setup_o, it_o, x_oracle, cores = oracle_solve_ms(A, b_np, "fp64")
        cpu = {"value": ms_o, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"one complete oracle solve (C, fp64, OpenMP build: row loops of the SpMV, "
                         f"sweeps, residuals, dots and axpys over {cores} threads) of {desc} to "
                         f"{args.tol:g}: {it_o} iterations; oracle setup {setup_o:.0f} ms (serial) not included"}

    net = None
    if args.learned or not args.no_extra:
        from paper_2303_02352_gb300 import learned
        if os.path.exists(learned.DEFAULT_WEIGHTS):
            net = learned.Network.load()
        elif args.learned:
            raise SystemExit("--learned needs trained weights (python -m paper_2303_02352_gb300.train_omega)")
    g = amg.Hierarchy(A, precision=PRECISIONS[args.precision])
    if args.learned:
        g.apply_mlp(net.w)
    info = g.info()
    b = torch.as_tensor(b_np, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()

    def solve():
        x.zero_()
        return g.solve_into(b, x, args.tol, 1000)

    for _ in range(max(3, args.warmup)):
        res = solve()
    if res["status"] != 0 or res["true_rel_res"] >= args.tol:
        raise SystemExit(f"solve did not converge: {res}")
    iters = res["iters"]

    def load(seconds):
        # the same solves, untimed, so that the clock samples around the short
        # timed region are taken with the GPU under the same load
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end:
            solve()

    clocks = Clocks(gpu_index(local))
    clocks.start()
    load(0.5)
    dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(args.steps):
        res = solve()
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    dist.barrier()
    load(0.5)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = dist.max(ms)
    assert res["iters"] == iters

    # end to end through the host entry point: pinned host b and x, copies inside
    bh = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    xh = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    bh[:] = b_np
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        xh[:] = 0.0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rh = g.pcg_solve_host(bh, xh, tol=args.tol, maxit=1000)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e = dist.max(sum(e2e_ms) / len(e2e_ms))

    # roofline: dominant kernel = level-0 l1-Jacobi sweep, and the whole V-cycle
    peak, peak_kind = peaks()
    t_sweep = g.time_kernel(amg.K_SWEEP, 0, reps=50)
    by_sweep = g.kernel_bytes(amg.K_SWEEP, 0)
    fp64_flop = 2.0 * (info["nnz"][0] + info["n"][0]) if args.precision == "fp64" else 0.0
    ach = by_sweep / (t_sweep * 1e-3) / 1e9
    t_vc = g.time_vcycle(reps=20)
    vc_gbs = info["vcycle_bytes"] / (t_vc * 1e-3) / 1e9
    kernels = {}
    names = {amg.K_SWEEP: "sweep", amg.K_RESIDUAL: "residual", amg.K_RESTRICT_FIRST: "restrict_first_sweep",
             amg.K_SWEEP_PROLONG: "coarse_sweep_prolong", amg.K_SPMV_DOTS: "spmv_dots", amg.K_AXPY: "axpy"}
    for kid, nm in names.items():
        t = g.time_kernel(kid, 0, reps=30)
        by = g.kernel_bytes(kid, 0)
        kernels[nm] = {"ms": round(t, 5), "GB/s": round(by / (t * 1e-3) / 1e9, 1),
                       "frac": round(by / (t * 1e-3) / 1e9 / peak, 3)}

    launches_per_solve = g.info()["last_solve_launches"]  # the library counts the launches of its last solve

    xs = torch.as_tensor(W.exact_solution(args.workload, n), device="cuda")
    xo = torch.as_tensor(x_oracle, device="cuda") if x_oracle is not None else None

    def errors(xv):
        e = {}
        if xo is not None:
            e["rel_err_vs_fp64_oracle"] = float((xv - xo).norm() / xo.norm())
        if xs is not None:
            e["rel_err_vs_exact"] = float((xv - xs).norm() / xs.norm())
        return e

    head = {"ms": ms, "iters": iters, "true_rel_res": res["true_rel_res"], **errors(x)}
    forms = {("%s%s" % (args.precision, "+learned" if args.learned else "")): head}
    if not args.no_extra:
        for pname in ("fp64", "fp32", "bf16fine"):
            for use_net in (False, True):
                key = pname + ("+learned" if use_net else "")
                if key in forms or (use_net and net is None):
                    continue
                g2 = amg.Hierarchy(A, precision=PRECISIONS[pname])
                if use_net:
                    g2.apply_mlp(net.w)
                x2 = torch.zeros_like(b)
                for _ in range(2):
                    r2 = g2.solve_into(b, x2.zero_(), args.tol, 1000)
                torch.cuda.synchronize()
                q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                q0.record(stream)
                for _ in range(args.steps):
                    r2 = g2.solve_into(b, x2.zero_(), args.tol, 1000)
                q1.record(stream)
                torch.cuda.synchronize()
                forms[key] = {"ms": q0.elapsed_time(q1) / args.steps, "iters": r2["iters"],
                              "true_rel_res": r2["true_rel_res"], **errors(x2),
                              "vcycle_ms": g2.time_vcycle(reps=20), "vcycle_bytes": g2.info()["vcycle_bytes"]}
                g2.close()

    # the NEXT-row features on the same workload: plain CG (no preconditioner),
    # the W-cycle, decoupled aggregation over row blocks, the setup split
    extras = {}
    if not args.no_extra:
        def timed(hier, precond=True, maxit=1000):
            x2 = torch.zeros_like(b)
            hier.solve_into(b, x2.zero_(), args.tol, maxit, precond)
            torch.cuda.synchronize()
            q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            r2 = hier.solve_into(b, x2.zero_(), args.tol, maxit, precond)
            q1.record(stream)
            torch.cuda.synchronize()
            return {"ms": q0.elapsed_time(q1), "iters": r2["iters"], "true_rel_res": r2["true_rel_res"], **errors(x2)}

        extras["cg_no_preconditioner"] = timed(g, precond=False, maxit=5000)
        gw = amg.Hierarchy(A, precision=PRECISIONS[args.precision], cycle=2)
        extras["w_cycle"] = {**timed(gw), "cycle_ms": gw.time_vcycle(reps=10)}
        gw.close()
        for parts in (8, 64):
            gd = amg.Hierarchy(A, precision=PRECISIONS[args.precision], num_parts=parts)
            di = gd.info()
            extras["decoupled_%d_parts" % parts] = {**timed(gd), "levels": di["num_levels"], "n": di["n"],
                                                   "opc": round(di["opc"], 4)}
            gd.close()
        extras["setup_split_ms"] = {"total": info["setup_ms"], "matching": info["setup_match_ms"],
                                    "galerkin": info["setup_galerkin_ms"]}
        # the same hierarchy with CSR column indices in every row kernel (no
        # pattern-coded columns): same arithmetic, 4 bytes per entry more
        os.environ["AMG_PAT"] = "0"
        try:
            gc = amg.Hierarchy(A, precision=PRECISIONS[args.precision])
        finally:
            del os.environ["AMG_PAT"]
        ci = gc.info()
        t_sw = gc.time_kernel(amg.K_SWEEP, 0, reps=30)
        b_sw = gc.kernel_bytes(amg.K_SWEEP, 0)
        extras["csr_columns"] = {**timed(gc), "vcycle_ms": gc.time_vcycle(reps=10), "vcycle_bytes": ci["vcycle_bytes"],
                                 "sweep_ms": round(t_sw, 5), "sweep_bytes": b_sw,
                                 "sweep_frac": round(b_sw / (t_sw * 1e-3) / 1e9 / peak, 4)}
        gc.close()
        # w-normalised prolongator values (Sec. 3.1), level matrices by the general
        # sparse product: solve, and the setup split matching / pairwise Galerkin /
        # general product
        gn = amg.Hierarchy(A, precision=PRECISIONS[args.precision], prolong_scale=1)
        ni = gn.info()
        extras["w_normalised_prolongator"] = {**timed(gn), "setup_ms": {
            "total": ni["setup_ms"], "matching": ni["setup_match_ms"], "galerkin_pairwise": ni["setup_galerkin_ms"],
            "spgemm": ni["setup_spgemm_ms"]}}
        gn.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": desc, "precision": args.precision, "learned_damping": bool(args.learned),
                       "tol": args.tol,
                       "replicas": world, "l2": "inputs larger than L2 (level-0 matrix %.0f MB)" % (A.nnz * 12 / 1e6),
                       "levels": info["num_levels"], "n": info["n"], "nnz": info["nnz"],
                       "opc": round(info["opc"], 4), "iters": iters,
                       "kernel_forms": {"tile_rows": info["tile_rows"], "stage_scale": info["stage_scale"],
                                        "fused_bottom_from_level": info["bottom_level"],
                                        "column_patterns": info["column_patterns"],
                                        "outer_patterns": info["outer_patterns"]}},
            "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(ach / peak, 4),
                         "traffic": ncu_traffic(args.workload, args.precision, info["tile_rows"][0],
                                                info["stage_scale"][0], info["column_patterns"][0]),
                         "kernel": "l1-Jacobi sweep, level 0", "algorithmic_bytes_per_launch": by_sweep,
                         "launch_ms": round(t_sweep, 5), "peak_kind": peak_kind},
            # the same launch against the FP64 issue rate: one multiply-add per
            # entry and one per row (FP64 levels; 0 for float levels)
            "co_limit": {"bound": "fp64", "unit": "TFLOP/s", "peak": FP64_TFLOPS, "peak_kind": "nominal",
                         "flop_per_launch": fp64_flop,
                         "achieved": round(fp64_flop / (t_sweep * 1e-3) / 1e12, 4),
                         "frac": round(fp64_flop / (t_sweep * 1e-3) / 1e12 / FP64_TFLOPS, 4)},
            "vcycle": {"ms": round(t_vc, 4), "bytes": info["vcycle_bytes"], "GB/s": round(vc_gbs, 1),
                       "frac": round(vc_gbs / peak, 4), "launches": info["vcycle_launches"]},
            "kernels_level0": kernels,
            "iteration": {"ms": ms / max(1, iters), "bytes": info["iteration_bytes"],
                          "GB/s": round(info["iteration_bytes"] * iters / (ms * 1e-3) / 1e9, 1)},
            "setup_ms": info["setup_ms"],
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 8 * n},
            "gpu_launches": launches_per_solve * args.steps,
            "clocks": clk,
            "cpu_baseline": cpu,
            "forms": forms,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    g.close()
    dist.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
