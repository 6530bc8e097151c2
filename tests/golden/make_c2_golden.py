#!/usr/bin/env python3
"""Writes tests/golden/c2_diffusion128.json from the CPU oracle alone.

The benchmark system (128^3 7-point variable-coefficient diffusion, the
seeded recipe of workloads.diffusion3d(128, 2.0, seed=0), b = U[-1,1] seed 1,
x0 = 0) is solved by the oracle four times:
  - AMP-PCG(FP16) with the linear-convergence criterion (ell = 5, C = 1),
    latching and up to 3 FP64 verify-and-replace steps (Alg. 3 with readings
    R5, R9), tol 1e-10, once with LINF_POW2 scaling and once with the lagged
    power of two (reading R20);
  - PCG (Alg. 1) in FP64, tol 1e-10 (the baseline's iteration count);
  - PCG in FP64 to tol 1e-13: the reference solution x* (reading R11).
It stores iteration counts, switch points, the first 100 relative residuals,
the final true residuals, norms, the solutions at 1000 fixed indices and the
relative errors of the AMP solution against x*.  Nothing here calls the CUDA
library.  Takes about 35 minutes on one host core.

    python tests/golden/make_c2_golden.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "c2_diffusion128.json")
NSAMPLE = 1000


def main():
    a = W.diffusion3d(128, 2.0, seed=0)
    b = W.rhs_uniform(a.n, seed=1)
    idx = np.sort(np.random.default_rng(2024).choice(a.n, NSAMPLE, replace=False))
    amps = {}
    for key, scale in (("amp16_linear", oracle.SCALE_LINF_POW2), ("amp16_linear_lag", oracle.SCALE_LINF_POW2_LAG)):
        pol = oracle.Policy(u0=oracle.FP16, criterion=oracle.LINEAR, ell=5, C=1.0,
                            scale=scale, latch=1, verify_refresh=3)
        t0 = time.perf_counter()
        amps[key] = (oracle.ampcg(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=20000, policy=pol),
                     time.perf_counter() - t0)
    t0 = time.perf_counter()
    p64 = oracle.pcg64(a.rowptr, a.col, a.val, b, tol=1e-10, maxit=20000)
    t_p64 = time.perf_counter() - t0
    t0 = time.perf_counter()
    xs = oracle.pcg64(a.rowptr, a.col, a.val, b, tol=1e-13, maxit=40000)
    t_xs = time.perf_counter() - t0
    nxs = float(np.linalg.norm(xs.x))

    def rel(u, v):
        return float(np.linalg.norm(u - v) / np.linalg.norm(v))

    out = {
        "what": "oracle solves of the 128^3 diffusion benchmark system (workloads.diffusion3d(128, 2.0, "
                "seed=0), b = rhs_uniform(n, seed=1), x0 = 0); written by tests/golden/make_c2_golden.py",
        "n": int(a.n), "nnz": int(a.nnz),
        "sample_idx": idx.tolist(),
        **{key: {
            "policy": "AMP-PCG(FP16), linear criterion ell=5 C=1, " + ("lagged power-of-two scale (R20)"
                      if key.endswith("lag") else "LINF_POW2") + ", latch, verify_refresh=3, tol 1e-10",
            "status": amp.status, "iters": amp.iters, "switch_iter": list(amp.switch_iter),
            "refreshes": amp.refreshes, "true_relres": amp.true_relres, "scale_retries": amp.scale_retries,
            "updated_relres": amp.updated_relres, "relres_hist_100": amp.relres_hist[:100].tolist(),
            "x_norm": float(np.linalg.norm(amp.x)), "x_sample": amp.x[idx].tolist(),
            "err_vs_xstar": rel(amp.x, xs.x), "err_vs_xstar_sampled": rel(amp.x[idx], xs.x[idx]),
            "host_seconds": round(t_amp, 1)} for key, (amp, t_amp) in amps.items()},
        "pcg64": {"policy": "PCG (Alg. 1) FP64, Jacobi, tol 1e-10", "iters": p64.iters,
                  "true_relres": p64.true_relres, "x_norm": float(np.linalg.norm(p64.x)),
                  "x_sample": p64.x[idx].tolist(), "err_vs_xstar": rel(p64.x, xs.x),
                  "host_seconds": round(t_p64, 1)},
        "xstar": {"policy": "PCG (Alg. 1) FP64, Jacobi, tol 1e-13", "iters": xs.iters,
                  "true_relres": xs.true_relres, "x_norm": nxs, "x_sample": xs.x[idx].tolist(),
                  "host_seconds": round(t_xs, 1)},
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    for key in amps:
        print(json.dumps({k: v for k, v in out[key].items() if k not in ("x_sample", "relres_hist_100")}))
    print(json.dumps({k: v for k, v in out["pcg64"].items() if k != "x_sample"}))
    print(json.dumps({k: v for k, v in out["xstar"].items() if k != "x_sample"}))


if __name__ == "__main__":
    main()
