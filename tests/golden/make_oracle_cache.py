"""Write the oracle's solutions of a bench-size workload to tests/golden/oracle_<config>.npz.

This script calls only the CPU oracle (``oracle/``) and the seeded input generators
(``workloads/``); no value it stores comes from the CUDA path. At the bench sizes the
oracle needs tens of minutes per factorisation on a multi-core host (its Householder
QR is the unblocked textbook loop), so its results are cached here, keyed by the
SHA-256 of the generated inputs, and the GPU tests compare against them.

For each sketch seed it stores, from the implicit-form CSQRP-LSQR of Algorithm 1
(count sketch with s = 4n, Householder QR, LSQR on A R^-1 with per-step triangular
solves):
  * x_tol<seed>:   LSQR stopped by the Paige-Saunders rules at atol = btol = tol
                   (the benchmark's stopping rule), with its iteration count;
  * x_floor<seed>: LSQR run for a fixed number of iterations far past convergence,
                   at the floating-point floor of the iteration (the best estimate
                   of x_* = argmin ||Ax - b|| the oracle can give);
  * hist<seed>:    the ||r_k|| estimates of the tol run;
  * x_ref<seed>:   LSQR restarted once from x_tol<seed> (the correction from r = b - A x, same
                   stopping rule): per-step triangular solves limit the first solve's attainable
                   A-norm accuracy (its floor moves with the sketch by ~1e-9 on the 2D bench
                   workload); the restart removes that limit.
With --hhqr it also stores x_hh, the dense Householder least-squares solution (the
HHQR direct method of Section 4.1), an estimate of x_* by an independent route.

The spread between these estimates (two sketches, and the direct solve) is the
problem's own floating-point spread in the A-norm that Theorem 3.3 controls.

Usage: python tests/golden/make_oracle_cache.py --config cfg2 --seeds 1 2 [--hhqr] [--threads 8]
(A run resumes from the stored file: results already present for the same inputs are kept.)
"""
import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import config_problem, input_hash  # noqa: E402


def a_norm_rel(p, x, ref):
    return float(np.linalg.norm(oracle.spmv(p, x - ref)) / np.linalg.norm(oracle.spmv(p, ref)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="cfg2")
    ap.add_argument("--seeds", type=int, nargs="+", default=[1, 2])
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--floor-iters", type=int, default=250)
    ap.add_argument("--hhqr", action="store_true")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    out = args.out or os.path.join(HERE, "oracle_%s.npz" % args.config)
    nthr = oracle.set_threads(args.threads)
    p = config_problem(args.config)
    b = np.ascontiguousarray(p.b[0])
    s = oracle.sketch_size(p, 4.0)
    key = input_hash(p)
    print("%s: m=%d n=%d nnz=%d s=%d hash=%s threads=%d" % (args.config, p.m, p.n, p.nnz, s, key, nthr), flush=True)
    res = dict(config=args.config, input_hash=key, m=p.m, n=p.n, nnz=p.nnz, s=s, tol=args.tol,
               seeds=np.asarray(args.seeds), floor_iters=args.floor_iters)
    if os.path.exists(out):    # resume: keep what an earlier run stored for the same inputs
        old = dict(np.load(out, allow_pickle=False))
        if str(old.get("input_hash")) == key:
            for k, v in old.items():
                if k.startswith(("x_", "hist", "it_", "istop_", "rnorm_", "secs_")):
                    res[k] = v
    for seed in args.seeds:
        if all(("%s%d" % (k, seed)) in res for k in ("x_tol", "x_floor", "x_ref")):
            continue
        t0 = time.time()
        fac = oracle.factor(p, s, seed)
        t1 = time.time()
        R = fac["R"]
        fac = None
        if "x_floor%d" % seed not in res:
            x_tol, info, hist = oracle.lsqr(p, b, R, atol=args.tol, btol=args.tol, history=True)
            x_fl, info_fl = oracle.lsqr(p, b, R, fixed_iters=args.floor_iters)
            res["x_tol%d" % seed] = x_tol
            res["x_floor%d" % seed] = x_fl
            res["hist%d" % seed] = hist
            res["it_tol%d" % seed] = info["iterations"]
            res["istop_tol%d" % seed] = info["istop"]
            res["rnorm_floor%d" % seed] = float(np.linalg.norm(b - oracle.spmv(p, x_fl)))
        t2 = time.time()
        # one restart from the tol-stopped solution (the correction from r = b - A x), same rule
        x_ref, info_ref = oracle.lsqr(p, b, R, atol=args.tol, btol=args.tol, x0=res["x_tol%d" % seed])
        t3 = time.time()
        res["x_ref%d" % seed] = x_ref
        res["it_ref%d" % seed] = info_ref["iterations"]
        res["secs_factor%d" % seed] = t1 - t0
        res["secs_lsqr%d" % seed] = t3 - t1
        print("seed %d: factor %.0f s, lsqr %.0f s, %d + %d iterations, A-norm(tol vs floor) %.3e, (restart vs floor) "
              "%.3e" % (seed, t1 - t0, t3 - t1, int(res["it_tol%d" % seed]), info_ref["iterations"],
                        a_norm_rel(p, res["x_tol%d" % seed], res["x_floor%d" % seed]),
                        a_norm_rel(p, x_ref, res["x_floor%d" % seed])), flush=True)
        np.savez_compressed(out, **res)
    if args.hhqr and "x_hh" not in res:
        t0 = time.time()
        x_hh, _ = oracle.hhqr_solve(p.dense(), b)
        res["x_hh"] = x_hh
        res["secs_hhqr"] = time.time() - t0
        print("hhqr: %.0f s" % (time.time() - t0), flush=True)
        np.savez_compressed(out, **res)
    seeds = [sd for sd in args.seeds if "x_floor%d" % sd in res]
    ref = res["x_floor%d" % seeds[0]]
    for k in sorted(res):
        if k.startswith("x_"):
            print("%-10s A-norm vs x_floor%d: %.3e" % (k, seeds[0], a_norm_rel(p, res[k], ref)))


if __name__ == "__main__":
    main()
