"""Writes tests/golden/oracle_iterations.json by running ONLY the CPU oracle.

Stored values: FGMRES iteration counts and true relative residuals of the
oracle (FP64, MGS, exact coarse solve) for the workloads the benchmark and
the GPU tests use at full size. Run:  python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import helm_inputs as hi  # noqa: E402
from oracle import solver  # noqa: E402


def main():
    out = {}
    for wl in (hi.SMALL_P1, hi.GAUSS_P1):
        t0 = time.time()
        r = solver.build_problem(wl).solve()
        out[wl.name] = {"iters": r.iters, "relres_true": r.relres_true, "cycles": len(r.cycle_true),
                        "seconds": round(time.time() - t0, 1)}
        print(wl.name, out[wl.name], flush=True)
    with open(os.path.join(HERE, "oracle_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
