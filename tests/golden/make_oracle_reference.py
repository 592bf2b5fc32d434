"""Writes oracle_reference.json: the CPU oracle's hierarchy and FCG results on the
benchmark workloads.  Calls only oracle/ and the seeded input generators.

Usage: python tests/golden/make_oracle_reference.py [config ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2303_02352_gb300 import workloads as W  # noqa: E402

PRECISIONS = {"fp64": O.FP64, "fp32": O.FP32, "bf16fine": O.FP32_BF16FINE}


def run(name, prec):
    A, b, desc = W.config(name)
    t0 = time.perf_counter()
    h = O.Hierarchy(A, precision=PRECISIONS[prec])
    t1 = time.perf_counter()
    res = h.fcg(b)
    t2 = time.perf_counter()
    return {"workload": desc, "precision": prec, "levels": h.num_levels,
            "n": [h.level_n(k) for k in range(h.num_levels)],
            "nnz": [h.level_nnz(k) for k in range(h.num_levels)], "opc": h.opc(),
            "iters": res["iters"], "true_rel_res": res["true_rel_res"], "status": res["status"],
            "oracle_setup_s": t1 - t0, "oracle_solve_s": t2 - t1}


def main(argv):
    out = os.path.join(HERE, "oracle_reference.json")
    data = json.load(open(out)) if os.path.exists(out) else {}
    data["_source"] = "written by tests/golden/make_oracle_reference.py (CPU oracle only); times are this machine's"
    jobs = [a.split(":") for a in argv] or [("poisson32", "fp64"), ("poisson160", "fp64"), ("poisson160", "fp32")]
    for name, prec in jobs:
        key = f"{name}:{prec}"
        data[key] = run(name, prec)
        print(key, data[key], flush=True)
        json.dump(data, open(out, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
