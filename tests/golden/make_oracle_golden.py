"""Writes tests/golden/oracle_iterations.json by running ONLY the CPU oracle.

Stored values: FGMRES iteration counts and true relative residuals of the
oracle (FP64, MGS, exact coarse solve) for the workloads the benchmark and
the GPU tests use at full size. Run:  python tests/golden/make_oracle_golden.py [NAME ...]
(no names: every workload; with names: only those, merged into the existing file).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import helm_inputs as hi  # noqa: E402
from oracle import solver  # noqa: E402


WORKLOADS = (hi.SMALL_P1, hi.GAUSS_P1, hi.RANDOM_P2, hi.RANDOM_P1_3D)


def main():
    path = os.path.join(HERE, "oracle_iterations.json")
    names = set(sys.argv[1:])
    out = {}
    if names and os.path.exists(path):
        with open(path) as f:
            out = json.load(f)
    for wl in WORKLOADS:
        if names and wl.name not in names:
            continue
        t0 = time.time()
        r = solver.build_problem(wl).solve()
        out[wl.name] = {"iters": r.iters, "relres_true": r.relres_true, "cycles": len(r.cycle_true),
                        "seconds": round(time.time() - t0, 1)}
        print(wl.name, out[wl.name], flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
