#!/usr/bin/env python3
"""Writes tests/golden/c2_scale_study.json from the CPU oracle alone: the
choice of the scale factor omega_k (reading R5; Sec. 3.3) on the 128^3
benchmark system, AMP-PCG(FP16) with the linear criterion (ell = 5, C = 1),
latching and up to 3 FP64 verify-and-replace steps, tol 1e-10:
  - L2:  omega_k = 1/||r_k||, as printed in Alg. 3;
  - LINF_POW2: omega_k = 2^-ceil(log2 max|r_k|);
  - LINF_POW2_LAG: the previous iteration's power of two (reading R20).
For each: iterations, the u_r switch, the final true residual, and how many
scaled residual entries y_i (r_i != 0) fell below binary16's normal range
(subnormal or zero), summed over the iterations.  The three solves run in
parallel processes; about 17 minutes.  Nothing here calls the CUDA library.

    python tests/golden/make_scale_study.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "c2_scale_study.json")
MODES = {"L2": 1, "LINF_POW2": 2, "LINF_POW2_LAG": 3}


def run(name):
    import oracle
    import workloads as W
    a = W.diffusion3d(128, 2.0, seed=0)
    b = W.rhs_uniform(a.n, seed=1)
    pol = oracle.Policy(u0=oracle.FP16, criterion=oracle.LINEAR, ell=5, C=1.0, scale=MODES[name], latch=1,
                        verify_refresh=3)
    t0 = time.perf_counter()
    r = oracle.ampcg(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=20000, policy=pol)
    return name, {"iters": r.iters, "status": r.status, "switch_iter": list(r.switch_iter),
                  "refreshes": r.refreshes, "true_relres": r.true_relres,
                  "y16_below_normal": int(r.y16_small), "y16_nonzero": int(r.y16_total),
                  "y16_below_normal_frac": r.y16_small / max(r.y16_total, 1),
                  "scale_retries": r.scale_retries, "host_seconds": round(time.perf_counter() - t0, 1)}


def main():
    with mp.get_context("spawn").Pool(len(MODES)) as pool:
        res = dict(pool.map(run, list(MODES)))
    out = {"what": "oracle AMP-PCG(FP16) solves of the 128^3 diffusion benchmark system with three scale "
                   "factors; written by tests/golden/make_scale_study.py", **res}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
