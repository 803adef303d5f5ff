"""Benchmark: one full CSQRP-LSQR solve (count sketch + QR + LSQR) per step on
the 2D Poisson RFM workload (8 x 8 boxes, J = 200 tanh features each, 30 x 30
points per box plus boundary and C0/C1 interface rows: m = 65,280, n = 12,800,
14.4M nonzeros, s = 4n), binary64, synthetic seeded inputs.

Prints one JSON line. `value` is the device time per solve (seconds, lower is
better) over the whole job; `e2e` is the same solve through the public API with
host buffers (host->device copy of A and b, device->host copy of x inside the
timed region). Multi-GPU runs are independent replicas (one instance per rank).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solve time to rel. error 1e-10 (sketch+QR+LSQR); SpMV-pair HBM GB/s vs peak"
WORKLOADS = {
    "cfg2": "2D Poisson RFM, 8x8 boxes, J=200 tanh features, 30x30 points/box, m=65280 n=12800 nnz=14.4M, s=4n",
    "cfg1": "2D Poisson RFM, 2x2 boxes, J=100, 20x20 points/box, m=1920 n=400 nnz=208k, s=4n",
    "cfg3": "3D Poisson RFM, 4x4x4 boxes, J=400, 12^3 points/box, m=134784 n=25600 nnz=58.06M, s=4n",
    "cfg4a": "2D Poisson RFM cfg2 matrix with 64 right-hand sides sin(a pi x) sin(b pi y), block LSQR, s=4n",
    "cfg5": "random sparse 2e6 x 2e4, 10/row, columns scaled over 10 decades, s=4n",
    "rfm6x6": "2D Poisson RFM, 6x6 boxes, J=200, 30x30 points/box, m=36720 n=7200 nnz=8.06M, s=4n",
    "rfm6x6_64": "2D Poisson RFM rfm6x6 matrix with 64 right-hand sides sin(a pi x) sin(b pi y), block LSQR, s=4n",
    "cfg4b": "32 uneven 2D Poisson RFM instances (grids 2x2..6x6, J in {50,100,150}, 15..25 points/side), "
             "factored one by one, solved in one CUDA-graph launch",
}
WORKLOAD = WORKLOADS["cfg2"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="csls", choices=["csls", "reference"])
    ap.add_argument("--prec", default="f64emu", choices=["f64", "f32", "f64emu"])
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-FP64 solve timed beside")
    ap.add_argument("--cpu-library", action="store_true",
                    help="also time the method on NumPy/SciPy over all host cores (LAPACK QR, SciPy LSQR), in full")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle's CPU sample (cpu_baseline null), for secondary configurations")
    ap.add_argument("--config", default="cfg2")
    ap.add_argument("--assemble", action="store_true",
                    help="end-to-end leg: ship the RFM geometry and features, assemble the CSR on the GPU")
    ap.add_argument("--explicit", action="store_true",
                    help="the explicit form: B = A R^-1 formed densely, LSQR on B (Algorithm 1 steps 4-6)")
    ap.add_argument("--warm", action="store_true",
                    help="start LSQR from the sketch-and-solve point R^-1 Q^T S b (Remark 3.1)")
    ap.add_argument("--variant", default="qr", choices=["qr", "svd"],
                    help="preconditioner: QR of the sketch (Algorithm 1) or truncated SVD (Algorithm 2)")
    ap.add_argument("--backward", action="store_true",
                    help="each step also runs the adjoint backward of L = ||x - x_true||^2 (dL/db and dL/d values; "
                         "workloads with a known x_true)")
    ap.add_argument("--tol", type=float, default=1e-8,
                    help="LSQR stopping tolerance atol = btol (the tau of Section 4.1); with one restart the "
                         "A-norm accuracy is far below it (the first solve stops at its rounding floor anyway)")
    ap.add_argument("--refine", type=int, default=1,
                    help="LSQR restarts from the solution found (correction from r = b - A x); the first solve's "
                         "A-norm accuracy is limited by the per-step triangular solves, one restart removes that")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1890.0), "measured"
    return 6800.0, 1900.0, "fallback"


def read_ceiling_gbs(csls):
    """Streaming-read bandwidth of this GPU, the ceiling of a read-dominated kernel such as SpMV
    (the copy figure counts reads + writes): the library's probe kernel reads 2 GiB once per launch
    (integer checksum, so no FP64 pipe limit), swept over CTAs per SM and loads in flight per
    thread; the best configuration's median of 5 launches."""
    import torch
    nbytes = 2 << 30
    a = torch.ones(nbytes // 8, dtype=torch.float64, device="cuda")
    best, cfg = 0.0, None
    sweep = {}
    for ctas in (1, 2, 4):
        for unroll in (1, 2, 4, 8):
            csls.csls_read_probe(a, ctas, unroll)
            ts = []
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                csls.csls_read_probe(a, ctas, unroll)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            gbs = nbytes / (statistics.median(ts) * 1e-3) / 1e9
            sweep["%dx%d" % (ctas, unroll)] = round(gbs, 1)
            if gbs > best:
                sms = torch.cuda.get_device_properties(0).multi_processor_count
                best, cfg = gbs, {"ctas_per_sm": ctas, "loads_in_flight_per_thread": unroll,
                                  "bytes_in_flight": sms * ctas * 512 * unroll * 16}
    del a
    return best, cfg, sweep


def bf16_sustained():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f).get("bf16_tflops_sustained", 1700.0)
    return 1700.0


class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, world, device="cuda"):
    """The slowest rank's figure (whole-job time is set by the last rank to finish)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_problem(config, rank):
    """The workload of one replica: independent instances of the same recipe (a different seed per
    rank for the 2D bench workload), so N ranks solve N independent problems with no exchange."""
    from workloads import config_problem, poisson2d
    if config == "cfg2":
        return poisson2d(8, 8, 200, 30, 30, R=2.0, seed=2 + 1000 * rank)
    return config_problem(config)


# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per average launch of each factor family
# on the 2D bench workload: the per-unit bytes of one capture on the 6x6-box profiling workload (launch 41,
# outer block 40: L = 26,240 rows, n' = 4,576 trailing columns) times the units of an average bench launch
# (2.869e6 panel elements; 3.006e8 trailing-product elements). Traffic grows in proportion to these units:
# the products stream C once (vtc) or twice (update), the panel reads its block once.
TRAFFIC = {"k_obpanel": 12.28 * 2.869e6, "k_emu_vtc_tc": 8.199 * 3.006e8, "k_emu_update_tc": 15.875 * 3.006e8}
_TSRC = ("profiles/%s_rfm6x6.md (ncu --set full, launch 41 of the 6x6-box workload): %.3f B per %s, scaled to an "
         "average launch of the 2D bench workload")
TRAFFIC_SOURCE = {"k_obpanel": _TSRC % ("obpanel", 12.28, "panel element (L x 64)"),
                  "k_emu_vtc_tc": _TSRC % ("emu_vtc_tc", 8.199, "trailing element (L x n'; algorithmic 8)"),
                  "k_emu_update_tc": _TSRC % ("emu_update_tc", 15.875, "trailing element (L x n'; algorithmic 16)")}


def oracle_cache(p, config):
    """The oracle's cached solutions of this workload (tests/golden/oracle_<config>.npz), if they were
    computed for exactly these inputs (same SHA-256 of the CSR arrays and right-hand side)."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_%s.npz" % config)
    if not os.path.exists(path):
        return None
    from workloads import input_hash
    d = dict(np.load(path, allow_pickle=False))
    return d if str(d.get("input_hash")) == input_hash(p) else None


def csr_matvec_np(p, x):
    """A x from the CSR arrays (NumPy, for the accuracy figures)."""
    rows = np.repeat(np.arange(p.m), np.diff(p.row_ptr))
    return np.bincount(rows, weights=p.val * x[p.col], minlength=p.m)


def qr_flops(s, n):
    return 2.0 * s * n * n - 2.0 / 3.0 * n ** 3


def spmv_pair_bytes(m, n, nnz):
    # A x and A^T u: values (8 B) + column indices (4 B) per nonzero, row pointers (8 B),
    # the gathered vector and the written vector, for both passes.
    return 2 * (12 * nnz) + 8 * (m + 1) + 8 * (n + 1) + 8 * (m + n) * 2


# ----------------------------------------------------------------------------- reference arm (CPU oracle)

def oracle_sample_seconds(p, s, iters_full):
    """Time the oracle on a bounded sample of the workload and scale it to one
    full solve: the full sketch, Householder QR of the first k columns of the
    sketch (extrapolated by flop count; the QR's column loop runs on all host
    cores) and 2 LSQR iterations (scaled by the iteration count of the solve)."""
    import oracle
    threads = oracle.set_threads(len(os.sched_getaffinity(0)))
    t0 = time.perf_counter()
    h, d = oracle.hash_rows(p.m, s, 1)
    SA = oracle.sketch(p, s, h, d)
    t_sketch = time.perf_counter() - t0
    k = 320
    sub = np.asfortranarray(SA[:, :k])
    t0 = time.perf_counter()
    oracle.householder_qr(sub)
    t_qr_k = time.perf_counter() - t0
    flops_k = sum(4.0 * (s - j) * (k - j) for j in range(k))
    t_qr = t_qr_k * qr_flops(s, p.n) / flops_k
    R = np.eye(p.n) + np.triu(np.full((p.n, p.n), 1e-3), 1)
    t0 = time.perf_counter()
    oracle.lsqr(p, p.b[0], R, "qr", fixed_iters=2)
    t_it = (time.perf_counter() - t0) / 2.0
    total = t_sketch + t_qr + t_it * iters_full
    sample = ("oracle (C; the Householder column loop on %d threads) on %s: full sketch %.2fs + Householder QR "
              "of the first %d of %d sketch columns %.2fs scaled by flops to %.1fs + 2 LSQR iterations %.2fs/it x "
              "%d iterations" % (threads, WORKLOAD, t_sketch, k, p.n, t_qr_k, t_qr, t_it, iters_full))
    return total, sample, t_sketch + t_qr_k + 2 * t_it, threads


def library_cpu_solve(p, s, tol, refine):
    """The method on NumPy/SciPy over all host cores, as the paper's 2D experiments ran it (Python), timed in
    full: the count sketch as a sparse product S A (buckets and signs from NumPy's generator: Definition 2.3
    asks only for uniform buckets and balanced signs), LAPACK's Householder QR of the dense sketch
    (numpy.linalg.qr, dgeqrf), SciPy's LSQR on A R^-1 applied by triangular solves, and the same restarts
    as the GPU solve. Returns (seconds, x, iterations, phases)."""
    import scipy.linalg as sl
    import scipy.sparse as sp
    from scipy.sparse.linalg import LinearOperator, lsqr
    b = np.ascontiguousarray(p.b[0])
    t0 = time.perf_counter()
    A = sp.csr_matrix((p.val, p.col, p.row_ptr), shape=(p.m, p.n))
    rng = np.random.default_rng(1)
    h = rng.integers(0, s, p.m)
    d = rng.choice(np.array([-1.0, 1.0]), p.m)
    S = sp.csr_matrix((d, (h, np.arange(p.m))), shape=(s, p.m))
    SA = (S @ A).toarray()
    t1 = time.perf_counter()
    R = np.linalg.qr(SA, mode="r")
    del SA
    t2 = time.perf_counter()
    AT = A.T.tocsr()
    op = LinearOperator((p.m, p.n), matvec=lambda v: A @ sl.solve_triangular(R, v),
                        rmatvec=lambda u: sl.solve_triangular(R, AT @ u, trans="T"))
    out = lsqr(op, b, atol=tol, btol=tol, iter_lim=p.n)
    x = sl.solve_triangular(R, out[0])
    its = int(out[2])
    for _ in range(refine):
        out = lsqr(op, b - A @ x, atol=tol, btol=tol, iter_lim=p.n)
        x = x + sl.solve_triangular(R, out[0])
        its += int(out[2])
    t3 = time.perf_counter()
    return t3 - t0, x, its, {"sketch": t1 - t0, "qr": t2 - t1, "lsqr": t3 - t2}


def l2_policy(in_bytes):
    """Timing rule for the L2: inputs larger than the L2 need no flush between timed steps; smaller ones
    get one, a write of twice the L2's size before each timed step, outside that step's CUDA events.
    Returns (flush buffer or None, the note for the line's config)."""
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    l2 = int(getattr(props, "L2_cache_size", 0) or 129 * 2 ** 20)
    if in_bytes > l2:
        return None, "inputs larger than L2 (%.0f MB of inputs, %.0f MB of L2), no flush" % (in_bytes / 1e6, l2 / 1e6)
    buf = torch.empty(2 * l2 // 4, dtype=torch.int32, device="cuda")
    return buf, ("L2 flushed between timed steps: %.1f MB of inputs fit in the %.0f MB L2, so a %.0f MB write "
                 "precedes each step, outside its CUDA events" % (in_bytes / 1e6, l2 / 1e6, 2 * l2 / 1e6))


def run_reference(args):
    global WORKLOAD
    WORKLOAD = WORKLOADS.get(args.config, args.config)
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    from workloads import config_problem
    p = config_problem(args.config)
    s = 4 * p.n
    # the oracle's own iteration count at this workload (cached oracle run), else the GPU's last count
    cache = oracle_cache(p, args.config)
    iters = int(cache["it_tol1"]) if cache is not None and "it_tol1" in cache else 83
    vals = []
    sample = ""
    threads = 1
    for _ in range(args.warmup + args.steps):
        v, sample, _, threads = oracle_sample_seconds(p, s, iters)
        vals.append(v)
    v = statistics.median(vals[args.warmup:]) if args.steps > 0 else vals[-1]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": 1, "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def run_batch(args):
    """Config 4b: 32 uneven instances; a step factors every instance and solves the batch
    in one CUDA-graph launch (SpMV threads-per-row from the autotuner's cache)."""
    import torch
    from paper_2409_15818_gb300 import build, csls
    from workloads import batched_instances
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    build.build()
    probs = batched_instances(32)
    As = [csls.Csr.from_numpy(p.row_ptr, p.col, p.val, p.m, p.n) for p in probs]
    bs = [torch.tensor(p.b[0], device="cuda") for p in probs]
    opts = dict(seed=1, prec=args.prec, tol=1e-12)
    cache = os.path.join(ROOT, "paper_2409_15818_gb300", "_build", "spmv_autotune.json")

    fallbacks = []

    def step():
        Fs = [csls.csls_factor(A, **opts) for A in As]
        for F, A in zip(Fs, As):
            csls.csls_autotune(F, A, cache=cache)
        xs, reps, st = csls.csls_batch_solve(Fs, As, bs, raise_on_error=False, **opts)
        # binary32 factors rejected by the cond guard are refactored in emulated FP64 and the
        # rejected instances solved again as a second batch
        redo = [k for k, r in enumerate(reps) if r["status"] == 6]
        fallbacks.append(len(redo))
        if redo:
            F2 = [csls.csls_factor(As[k], **dict(opts, prec="f64emu")) for k in redo]
            for F, k in zip(F2, redo):
                csls.csls_autotune(F, As[k], cache=cache)
            x2, r2, st = csls.csls_batch_solve(F2, [As[k] for k in redo], [bs[k] for k in redo],
                                              raise_on_error=False, **dict(opts, prec="f64emu"))
            for j, k in enumerate(redo):
                xs[k], reps[k], Fs[k] = x2[j], r2[j], F2[j]
            st = next((r["status"] for r in reps if r["status"]), 0)
        return Fs, xs, reps, st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream()
    in_bytes = sum(A.row_ptr.numel() * 8 + A.col.numel() * 4 + A.val.numel() * 8 for A in As) + \
        sum(b.numel() * 8 for b in bs)
    flush, l2_note = l2_policy(in_bytes)
    launches, solve_ms, factor_ms, step_ms = 0, [], [], []
    for _ in range(args.steps):
        if flush is not None:
            flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Fs, xs, reps, st = step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        launches += sum(F.report["launches"] for F in Fs) + 6 * (1 + (fallbacks[-1] > 0))
        solve_ms.append(reps[0]["ms_solve"])
        factor_ms.append(sum(F.report["ms_factor"] + F.report["ms_sketch"] for F in Fs))
    clk = clocks.stop()
    ms = sum(step_ms) / max(args.steps, 1)
    iters = [r["iterations"] for r in reps]
    line = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": {"workload": WORKLOADS["cfg4b"], "instances": len(probs),
                       "n_range": [min(p.n for p in probs), max(p.n for p in probs)],
                       "m_range": [min(p.m for p in probs), max(p.m for p in probs)], "l2": l2_note},
            "status": csls.STATUS_NAMES.get(st, st), "iterations_range": [min(iters), max(iters)],
            "guard_fallbacks": fallbacks[-1] if fallbacks else 0,
            "phase_ms": {"factor_all": statistics.median(factor_ms), "batch_solve_graph": statistics.median(solve_ms)},
            "gpu_launches": int(launches), "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.config == "cfg4b":
        run_batch(args)
        return
    import torch
    import torch.distributed as dist
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2409_15818_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
        build.build()
    from paper_2409_15818_gb300 import csls
    from workloads import config_problem, poisson2d

    p = replica_problem(args.config, rank)   # one instance per replica
    m, n, nnz = p.m, p.n, p.nnz
    s = min(4 * n, m)
    global WORKLOAD
    WORKLOAD = WORKLOADS.get(args.config, args.config)
    if args.config.startswith("c1_"):
        WORKLOAD = ("rank-deficient sparse stand-in with the shape, rank and density of Table C.1's %s: m=%d n=%d "
                    "rank=%d nnz=%d, b = A x_true" % (args.config[3:], m, n, p.info["rank"], nnz))
    A = csls.Csr.from_numpy(p.row_ptr, p.col, p.val, m, n)
    b = torch.tensor(p.b[0] if p.nrhs == 1 else p.b, device="cuda")   # cfg4a: 64 right-hand sides
    opts = dict(seed=1, prec=args.prec, tol=args.tol, variant=args.variant, refine=args.refine)
    stream = torch.cuda.current_stream()
    if args.backward:
        assert getattr(p, "x_true", None) is not None and p.nrhs == 1 and not (args.explicit or args.warm), \
            "--backward needs a single right-hand side with a known x_true (the column-scaled workloads)"
        xt = torch.tensor(p.x_true, device="cuda")
        bopts = dict(opts, tol=1e-12)

    def step(time_kernels=0):
        # time_kernels: the factor brackets each launch of its QR kernel families with CUDA
        # events on its stream (the per-kernel roofline below)
        if args.explicit:
            F = csls.csls_factor(A, time_kernels=time_kernels, **opts)
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            Bt = csls.csls_form_b(F, A)
            f1.record(stream)
            x, rep = csls.csls_solve_explicit(F, Bt, b, raise_on_error=False, **opts)
            torch.cuda.synchronize()
            rep["ms_form_b"] = f0.elapsed_time(f1)
            del Bt
            return F, x, rep
        if args.warm:
            F, x0 = csls.csls_factor_warm(A, b, time_kernels=time_kernels, **opts)
            x, rep = csls.csls_solve(F, A, b, x=x0, warm_start=1, raise_on_error=False, **opts)
            return F, x, rep
        F = csls.csls_factor(A, time_kernels=time_kernels, **opts)
        x, rep = csls.csls_solve(F, A, b, raise_on_error=False, **opts)
        if args.backward:
            # adjoint of L = ||x - x_true||^2: CG on B^T B to 1e-12 (its own stopping rule)
            gb, gv, brep = csls.csls_solve_backward(F, A, b, x, 2.0 * (x - xt), **bopts)
            rep["ms_backward"] = brep["ms_solve"]
            rep["backward_iterations"] = brep["iterations"]
            rep["backward_status"] = brep["status"]
        return F, x, rep

    for _ in range(args.warmup):
        F, x, rep = step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    qr_ms, solve_ms, sketch_ms, iters, bwd_ms, step_ms = [], [], [], [], [], []
    kern_ms, kern_n, kern_flop = [0.0] * 3, [0] * 3, [0.0] * 3
    in_bytes = A.row_ptr.numel() * 8 + A.col.numel() * 4 + A.val.numel() * 8 + b.numel() * 8
    flush, l2_note = l2_policy(in_bytes)
    e0.record(stream)
    for _ in range(args.steps):
        if flush is not None:
            # inputs that fit in L2: flush it before the step and time the step alone
            torch.cuda.synchronize()
            flush.fill_(1)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            F, x, rep = step(time_kernels=1)
            a1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(a0.elapsed_time(a1))
        else:
            F, x, rep = step(time_kernels=1)
        for f in range(3):
            kern_ms[f] += F.report["kern_ms"][f]
            kern_n[f] += F.report["kern_launches"][f]
            kern_flop[f] += F.report["kern_flop"][f]
        launches += F.report["launches"] + rep["launches"]
        qr_ms.append(F.report["ms_factor"])
        sketch_ms.append(F.report["ms_sketch"])
        solve_ms.append(rep["ms_solve"])
        iters.append(rep["iterations"])
        if args.backward:
            bwd_ms.append(rep["ms_backward"])
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks((sum(step_ms) if flush is not None else e0.elapsed_time(e1)) / max(args.steps, 1), world)
    status = rep["status"]

    # the plain binary64 form (trailing updates on the FP64 MMA pipe), timed once beside the chosen form
    plain = None
    if args.prec != "f64" and not args.no_compare:
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        popts = dict(opts, prec="f64")
        p0.record(stream)
        Fp = csls.csls_factor(A, **popts)
        xp, repp = csls.csls_solve(Fp, A, b, raise_on_error=False, **popts)
        p1.record(stream)
        torch.cuda.synchronize()
        Ap = torch.sparse_csr_tensor(A.row_ptr, A.col.to(torch.int64), A.val, (m, n))
        dx = xp - x
        dx2, xp2 = dx.reshape(-1, n).t(), xp.reshape(-1, n).t()
        rel_a = float(torch.linalg.matrix_norm(Ap @ dx2) / torch.linalg.matrix_norm(Ap @ xp2))
        plain = {"dtype": "f64", "s_per_solve": p0.elapsed_time(p1) / 1e3, "iterations": int(repp["iterations"]),
                 "status": csls.STATUS_NAMES.get(repp["status"], repp["status"]),
                 "factor_ms": Fp.report["ms_factor"], "solve_ms": repp["ms_solve"],
                 "rel_diff_A_norm_vs_chosen": rel_a}
        del Fp, xp

    # SpMV pair (A z, A^T u) timed alone, for the HBM roofline of the Krylov step: 20 pairs captured
    # in a CUDA graph (as the solver issues them: back to back, no host work in between), replayed
    z = torch.randn(n, dtype=torch.float64, device="cuda")
    u = torch.randn(m, dtype=torch.float64, device="cuda")
    yz = torch.empty(m, dtype=torch.float64, device="cuda")
    yu = torch.empty(n, dtype=torch.float64, device="cuda")

    def pair():
        csls.csls_spmv(F, A, z, y=yz)
        csls.csls_spmv(F, A, u, trans=True, y=yu)

    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        pair()
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(20):
            pair()
    graph.replay()
    torch.cuda.synchronize()
    reps = 5
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(reps):
        graph.replay()
    s1.record(stream)
    torch.cuda.synchronize()
    pair_ms = s0.elapsed_time(s1) / (reps * 20)
    del graph
    hbm, bf16, src = peaks()
    bf16_sus = bf16_sustained()
    read_gbs, read_cfg, read_sweep = read_ceiling_gbs(csls)
    pair_gbs = spmv_pair_bytes(m, n, nnz) / (pair_ms * 1e-3) / 1e9

    # triangular-solve pair (z = R^-1 v, then R^-T z), each call timed with events on the stream
    # (includes the call's small status memsets), and the whole LSQR iteration from the solve time
    trsv = None
    if args.variant == "qr":
        v = torch.randn(n, dtype=torch.float64, device="cuda")
        csls.csls_precond_apply(F, v)
        tms = []
        for _ in range(5):
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            zz = csls.csls_precond_apply(F, v)
            csls.csls_precond_apply(F, zz, trans=True)
            t1.record(stream)
            torch.cuda.synchronize()
            tms.append(t0.elapsed_time(t1))
        trsv_ms = statistics.median(tms)
        trsv_bytes = 8 * n * (n + 1)   # the upper triangle of R read twice
        trsv = {"bound": "hbm", "ms": trsv_ms, "bytes": trsv_bytes, "achieved": trsv_bytes / (trsv_ms * 1e-3) / 1e9,
                "peak": hbm, "unit": "GB/s", "frac": trsv_bytes / (trsv_ms * 1e-3) / 1e9 / hbm,
                "fp64_floor_ms": n * n / (152 * 2 * 2.07e9) * 1e3,
                "fp64_floor_source": "n^2 FP64 FMAs at 2 per clock per SM (152 SMs, 2.07 GHz)"}
    it_bytes = spmv_pair_bytes(m, n, nnz) + 8 * n * (n + 1) + 48 * m + 64 * n
    it_ms = statistics.median(solve_ms) / max(1, int(statistics.median(iters)))
    iteration = {"ms": it_ms, "bytes": it_bytes, "achieved": it_bytes / (it_ms * 1e-3) / 1e9, "peak": hbm,
                 "unit": "GB/s", "frac": it_bytes / (it_ms * 1e-3) / 1e9 / hbm,
                 "bytes_source": "SpMV pair 2 (12 nnz) + 8 (m + 1) + 8 (n + 1) + 16 (m + n), TRSV pair 8 n (n + 1), "
                                 "vectors 48 m + 64 n"}
    # A-norm error against the oracle's cached solutions of these exact inputs (Theorem 3.3's norm)
    accuracy = None
    cache = oracle_cache(p, args.config) if args.variant == "qr" and not args.explicit else None
    if cache is not None:
        Ap = torch.sparse_csr_tensor(A.row_ptr, A.col.to(torch.int64), A.val, (m, n))
        def anorm(xa, ref):
            xa = xa.reshape(-1) if torch.is_tensor(xa) else torch.tensor(xa, device="cuda")
            r = torch.tensor(ref, device="cuda")
            return float(torch.linalg.vector_norm(Ap @ (xa - r).unsqueeze(1)) /
                         torch.linalg.vector_norm(Ap @ r.unsqueeze(1)))
        accuracy = {"rel_err_A_vs_oracle_floor": anorm(x, cache["x_floor1"]),
                    "rel_err_A_vs_oracle_tol": anorm(x, cache["x_tol1"]),
                    "oracle_iterations": int(cache["it_tol1"]),
                    "reference": "oracle CSQRP-LSQR (same sketch seed): run 250 iterations to the floating-point floor "
                                 "of the first solve; tol = the same stopping rule; restarted = tol run plus one restart "
                                 "from its x (tests/golden/oracle_%s.npz)" % args.config}
        if "x_ref1" in cache:
            accuracy["rel_err_A_vs_oracle_restarted"] = anorm(x, cache["x_ref1"])
            accuracy["oracle_iterations_restart"] = int(cache["it_ref1"])
        if "x_ref2" in cache:   # two sketches, each restarted: the solution both agree on
            accuracy["rel_err_A_vs_oracle_restarted_seed2"] = anorm(x, cache["x_ref2"])
            accuracy["oracle_restarted_spread_A"] = anorm(cache["x_ref2"], cache["x_ref1"])
        if "x_floor2" in cache:   # the problem's own spread: two sketches, each at the oracle's floor
            accuracy["oracle_spread_A"] = anorm(cache["x_floor2"], cache["x_floor1"])
        if "x_hh" in cache:       # the dense Householder direct solve against the implicit form's floor
            accuracy["oracle_hhqr_vs_floor_A"] = anorm(cache["x_hh"], cache["x_floor1"])

    # end to end through the public API with host buffers
    h_row = torch.tensor(p.row_ptr).pin_memory()
    h_col = torch.tensor(p.col).pin_memory()
    h_val = torch.tensor(p.val).pin_memory()
    h_b = (torch.tensor(p.b[0]) if p.nrhs == 1 else torch.tensor(p.b)).pin_memory()
    h_x = torch.empty(tuple(b.shape[:-1]) + (n,), dtype=torch.float64).pin_memory()
    h2d = h_row.numel() * 8 + h_col.numel() * 4 + h_val.numel() * 8 + h_b.numel() * 8
    if args.assemble:
        # the RFM geometry (row descriptors) and feature parameters instead of the CSR
        from workloads import rfm_row_descriptors
        h_rows = torch.from_numpy(rfm_row_descriptors(p).view(np.uint8).copy()).pin_memory()
        h_k = torch.tensor(p.k).pin_memory()
        h_c = torch.tensor(p.c).pin_memory()
        r_half = 0.5 / np.asarray(p.grid, dtype=np.float64)
        h2d = h_rows.numel() + h_k.numel() * 8 + h_c.numel() * 8 + h_b.numel() * 8
        # one untimed assembly, so that its kernels are loaded like those of the factor and solve,
        # which the timed steps above have already run
        csls.csls_rfm_assemble(p.dim, r_half, p.J, h_k.cuda(), h_c.cuda(), h_rows.cuda())
    d2h = h_x.numel() * 8
    if args.backward:   # the gradients come back too
        h_gb = torch.empty(m, dtype=torch.float64).pin_memory()
        h_gv = torch.empty(nnz, dtype=torch.float64).pin_memory()
        d2h += (m + nnz) * 8
    torch.cuda.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 2))
    q0.record(stream)
    for _ in range(e2e_steps):
        if args.assemble:
            A2 = csls.csls_rfm_assemble(p.dim, r_half, p.J, h_k.cuda(non_blocking=True), h_c.cuda(non_blocking=True),
                                        h_rows.cuda(non_blocking=True))
        else:
            A2 = csls.Csr(h_row.cuda(non_blocking=True), h_col.cuda(non_blocking=True),
                          h_val.cuda(non_blocking=True), m, n)
        b2 = h_b.cuda(non_blocking=True)
        if args.explicit:
            F2 = csls.csls_factor(A2, **opts)
            B2 = csls.csls_form_b(F2, A2)
            x2, _ = csls.csls_solve_explicit(F2, B2, b2, raise_on_error=False, **opts)
            del B2
        elif args.warm:
            F2, x0 = csls.csls_factor_warm(A2, b2, **opts)
            x2, _ = csls.csls_solve(F2, A2, b2, x=x0, warm_start=1, raise_on_error=False, **opts)
        else:
            F2 = csls.csls_factor(A2, **opts)
            x2, _ = csls.csls_solve(F2, A2, b2, raise_on_error=False, **opts)
            if args.backward:
                gb2, gv2, _ = csls.csls_solve_backward(F2, A2, b2, x2, 2.0 * (x2 - xt), **bopts)
                h_gb.copy_(gb2, non_blocking=True)
                h_gv.copy_(gv2, non_blocking=True)
        h_x.copy_(x2, non_blocking=True)
    q1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(q0.elapsed_time(q1) / e2e_steps, world)

    # roofline of the dominant kernel: of the factor's three kernel families (Householder panel,
    # W = V^T C, C -= V W), the one with the most device time over the timed steps, its CUDA-event
    # time summed over its launches (algorithmic flops per launch / average launch time)
    qr_gflops = qr_flops(s, n) / (statistics.median(qr_ms) * 1e-3) / 1e9
    fam_names = {"f64emu": ["k_obpanel (FP64 Householder outer-block panel, T and V digits)",
                            "k_emu_vtc_tc (W = V^T C, exact bf16 digit products on tcgen05)",
                            "k_emu_update_tc (C -= V W, exact bf16 digit products on tcgen05)"],
                 "f64": ["k_panel (FP64 Householder panel)", "k_vtc_f64 (W = V^T C, DMMA)",
                         "k_update_f64 (C -= V W, DMMA)"],
                 "f32": ["k_panel (FP32 Householder panel)", "k_vtc_f32 (W = V^T C, FP32 FMA)",
                         "k_update_f32 (C -= V W, FP32 FMA)"]}[args.prec]
    fp64_alu_peak = 152 * 2 * 2 * 2.07e9 / 1e12   # TFLOP/s: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz
    fp64_peak = 1100.0   # GFLOP/s: DMMA m16n8k16 .f64 with full-mantissa operands (= cuBLAS DGEMM on this part)
    # per family: its bound, the work it is rated on and the peak of that unit
    if args.prec == "f64emu":
        # the products: 21 exact bf16 digit-pair products per binary64 product (6 digits, levels
        # p + q <= 5), against the measured dense bf16 rate; the panel: FP64 arithmetic on the ALU pipe
        spec = [("alu", 1.0, fp64_alu_peak, "FP64 FMA pipe: 152 SMs x 2 FMA/clock x 2 flop x 2.07 GHz"),
                ("tensor", 21.0, bf16_sus, src + " bf16 sustained (kernel timed inside a multi-second step)"),
                ("tensor", 21.0, bf16_sus, src + " bf16 sustained (kernel timed inside a multi-second step)")]
    elif args.prec == "f64":
        dm = "measured DMMA m16n8k16 f64 rate with full-mantissa operands (1.10 TFLOP/s, = cuBLAS DGEMM)"
        spec = [("alu", 1.0, fp64_alu_peak, "FP64 FMA pipe: 152 SMs x 2 FMA/clock x 2 flop x 2.07 GHz"),
                ("tensor", 1.0, fp64_peak / 1e3, dm), ("tensor", 1.0, fp64_peak / 1e3, dm)]
    else:
        alu32 = 152 * 128 * 2 * 2.07e9 / 1e12
        spec = [("alu", 1.0, alu32, "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz")] * 3
    fams = {}
    for f in range(3):
        bound, mult, pk, psrc = spec[f]
        name = fam_names[f].split(" ")[0]
        secs = kern_ms[f] * 1e-3
        ach = mult * kern_flop[f] / secs / 1e12 if secs > 0 and kern_flop[f] > 0 else None
        traffic = TRAFFIC.get(name) if (args.config == "cfg2" and args.prec == "f64emu") else None
        fams[name] = {"kernel": fam_names[f], "bound": bound, "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                      "frac": ach / pk if ach else None, "peak_source": psrc, "ms_total": kern_ms[f],
                      "launches": kern_n[f], "avg_launch_ms": kern_ms[f] / max(kern_n[f], 1),
                      "share_of_factor": kern_ms[f] / max(sum(qr_ms), 1e-9),
                      "fp64_equivalent_tflops": kern_flop[f] / secs / 1e12 if secs > 0 else None,
                      "traffic": traffic, "traffic_source": TRAFFIC_SOURCE.get(name) if traffic else None}
    top = max(range(3), key=lambda f: kern_ms[f])
    tname = fam_names[top].split(" ")[0]
    roofline = {k: fams[tname][k] for k in ("bound", "kernel", "achieved", "peak", "unit", "frac", "traffic",
                                              "traffic_source", "peak_source", "launches", "avg_launch_ms",
                                              "fp64_equivalent_tflops")}
    roofline["families"] = fams
    roofline["qr_fp64_equivalent_tflops"] = qr_gflops / 1e3
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        total, sample, spent, threads = oracle_sample_seconds(p, s, int(statistics.median(iters)))
        cpu = {"value": total, "unit": "s", "cores": threads, "kind": "oracle", "sample": sample}
    cpu_lib = None
    if rank == 0 and args.cpu_library and p.nrhs == 1 and args.variant == "qr":
        secs, xl, its_l, ph = library_cpu_solve(p, s, args.tol, args.refine)
        cpu_lib = {"value": secs, "unit": "s", "cores": len(os.sched_getaffinity(0)), "iterations": its_l,
                   "phase_s": ph, "kind": "library (NumPy/SciPy: sparse count sketch, LAPACK dgeqrf through "
                                           "numpy.linalg.qr, SciPy LSQR with triangular solves), timed in full"}
        if cache is not None and "x_ref1" in cache:
            ref = cache["x_ref1"]
            cpu_lib["rel_err_A_vs_oracle_restarted"] = float(
                np.linalg.norm(csr_matvec_np(p, xl - ref)) / np.linalg.norm(csr_matvec_np(p, ref)))
    if rank == 0:
        line = {
            "metric": METRIC, "value": ms / 1e3 / world, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"f64": "f64", "f32": "f32 factor / f64 LSQR",
                      "f64emu": "f64 LSQR; factor panels f64, trailing products emulated from bf16 digit products "
                                "(47-bit operands, relative error ~2^-38)"}[args.prec],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "m": m, "n": n, "nnz": nnz, "s": s, "tol": args.tol, "restarts": args.refine,
                       "variant": args.variant, "start": "R^-1 Q^T S b" if args.warm else "0",
                       "form": "explicit B = A R^-1" if args.explicit else "implicit (per-step triangular solves)",
                       "global_batch": world, "parallelism": "replicas" if world > 1 else "single",
                       "l2": l2_note, "dense_sketch_bytes": 8 * s * n},
            "status": csls.STATUS_NAMES.get(status, status), "iterations": int(statistics.median(iters)),
            "iterations_restart": int(rep.get("iterations_refine", 0)),
            "phase_ms": {"sketch": statistics.median(sketch_ms), "factor": statistics.median(qr_ms),
                         "solve": statistics.median(solve_ms),
                         **({"form_b": rep.get("ms_form_b")} if args.explicit else {}),
                         **({"backward": statistics.median(bwd_ms)} if args.backward else {})},
            "backward": {"loss": "||x - x_true||^2", "outputs": "dL/db (m) and dL/d values of A (nnz)",
                         "method": "lambda = R^-1 mu, (B^T B) mu = R^-T g by CG reusing the forward factor",
                         "cg_tol": 1e-12, "iterations": int(rep["backward_iterations"]),
                         "status": csls.STATUS_NAMES.get(rep["backward_status"], rep["backward_status"]),
                         "forward_plus_backward_s": (statistics.median(sketch_ms) + statistics.median(qr_ms) +
                                                     statistics.median(solve_ms) + statistics.median(bwd_ms)) / 1e3}
            if args.backward else None,
            "roofline": roofline,
            "cond_est": rep.get("cond_est"),
            "accuracy": accuracy,
            "trsv_pair": trsv,
            "iteration": iteration,
            "spmv_pair": {"bound": "hbm", "achieved": pair_gbs, "peak": hbm, "unit": "GB/s", "frac": pair_gbs / hbm,
                          "ms": pair_ms, "bytes": spmv_pair_bytes(m, n, nnz), "peak_source": src + " copy (read + write)",
                          "read_only_ceiling": read_gbs, "frac_of_read_ceiling": pair_gbs / read_gbs,
                          "read_ceiling_source": "csls_read_probe: 2 GiB read once, 16-byte evict-first loads, integer "
                                                 "checksum; best of a sweep over CTAs per SM x loads in flight "
                                                 "per thread (GB/s per configuration in read_ceiling_sweep)",
                          "read_ceiling_config": read_cfg, "read_ceiling_sweep": read_sweep},
            "cpu_baseline": cpu,
            "cpu_library": cpu_lib,
            "plain_f64_beside": plain,
            "e2e": {"value": e2e_ms / 1e3 / world, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "inputs": "RFM row descriptors + features, CSR assembled on the GPU" if args.assemble
                    else "CSR matrix + right-hand side"},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
