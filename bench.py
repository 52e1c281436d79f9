#!/usr/bin/env python
"""Benchmark: NNLS solves/s of the anti-lopsided method on one GB300.

One step = one whole solve of the lopsided single-RHS workload (A 20000×5000
FP32 with log-uniform column scales, x_true 70% zeros, 1% noise): Alg. 1's
prepare (scale factors, Aᵀb, split-BF16 tensor-core Gram → Q) plus Alg. 2 in
FP32 to FP64 relative KKT ≤ 1e-6, including the FP64 KKT evaluation from A.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own
replica (the single-RHS path has no exchange step: replicas only) and `value`
counts all ranks' solves over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NNLS solves/s at rel KKT ≤1e-6, chosen form vs plain FP64 on one GB300"
UNIT = "solves/s"
D, N, TOL, SEED = 20000, 5000, 1e-6, 1002
WORKLOAD_FMT = ("lopsided_single_{d}x{n}_f32: A U[0,1] x log-uniform column scales [1e-2,1e2], "
                "x_true 70% zeros Exp(1), b = A x_true + 1% Gaussian noise")
WORKLOAD = WORKLOAD_FMT.format(d=D, n=N)
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--d", type=int, default=D, help="rows of A (smaller values: profiling cases)")
    ap.add_argument("--n", type=int, default=N, help="columns of A")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return FALLBACK_PEAKS, "fallback"


# ----------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------- CPU oracle
def cpu_baseline_sample(A, b, m):
    """The FP64 oracle, as it stands, on a bounded sample of the workload: the
    NNLS sub-problem on the first m columns of A (same d, same b) to rel KKT
    1e-6.  Gram and the dense Alg. 2 products of the oracle scale as n², so the
    full-size time is estimated as t_sample·(n/m)²."""
    import numpy as np
    from oracle import nnls as O
    A64 = np.asarray(A[:, :m], dtype=np.float64, order="F")
    b64 = np.asarray(b, dtype=np.float64)
    t0 = time.perf_counter()
    x, res, _ = O.antilop(A64, b64, tol=TOL)
    t = time.perf_counter() - t0
    scale = (A.shape[1] / m) ** 2
    return t, scale, res.iters


def blas_threads():
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(v):
            try:
                return int(os.environ[v])
            except ValueError:
                pass
    return os.cpu_count()


# ------------------------------------------------------------------- reference
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1502_01645_gb300 import workloads as W
    p = W.lopsided_single(d=D, n=N, seed=SEED)
    m = N // 2
    times = []
    for i in range(args.warmup + args.steps):
        t, scale, iters = cpu_baseline_sample(p.A, p.B[0], m)
        if i >= args.warmup:
            times.append(t * scale)
    per = sum(times) / len(times)
    value = 1.0 / per
    cores = blas_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "d": D, "n": N, "tol": TOL, "seed": SEED},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"oracle antilop on A[:, :{m}] (d={D}), time x (n/m)^2 = "
                                   f"{(N / m) ** 2:.0f}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------ ours
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1502_01645_gb300 import aln, build_lib, workloads as W
    build_lib.build()
    aln.load()

    p = W.lopsided_single(d=D, n=N, seed=SEED + rank)
    A_np, b_np = p.A, p.B[0]
    At = torch.from_numpy(np.ascontiguousarray(A_np.T)).cuda().t()  # (d, n) column-major
    bt = torch.from_numpy(np.ascontiguousarray(b_np[None, :])).cuda()
    Xt = torch.zeros((1, N), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    solver = aln.Solver("split_bf16", stream=stream.cuda_stream)

    def step():
        solver.prepare(At, bt)
        _, info = solver.solve(tol=TOL, X=Xt)
        st = solver.stats()
        return info[0], st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    launches0 = solver.stats().kernel_launches
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos, gram_ms, prep_ms, solve_ms, kkt_ms, iters = [], [], [], [], [], []
    iter_ms, qrows = [], []
    for _ in range(args.steps):
        info, st = step()
        infos.append(info)
        gram_ms.append(st.gram_ms)
        prep_ms.append(st.prepare_ms)
        solve_ms.append(st.solve_ms)
        kkt_ms.append(st.kkt_ms)
        iter_ms.append(st.iterate_ms)
        qrows.append(st.passive_rows + st.clipped_rows)
        iters.append(info.iters)
    ev1.record(stream)
    barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = solver.stats().kernel_launches - launches0
    clocks = sampler.stop()
    worst = max(i.rel_kkt for i in infos)
    if worst > TOL:
        raise SystemExit(f"invalid run: rel KKT {worst:.3e} above {TOL}")

    t = torch.tensor([elapsed], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tmax = float(t.item())
    value = world * args.steps / tmax

    # ---- end to end through the C ABI with host buffers (pinned) ----
    e2e = None
    if not args.no_e2e:
        A_h = torch.from_numpy(np.ascontiguousarray(A_np.T)).pin_memory().t()
        b_h = torch.from_numpy(np.ascontiguousarray(b_np[None, :])).pin_memory()
        X_h = torch.zeros((1, N), dtype=torch.float64).pin_memory()
        k_e2e = max(3, min(args.steps, 5))
        hsolver = aln.Solver("split_bf16", stream=stream.cuda_stream)
        hsolver.prepare(A_h, b_h)
        hsolver.solve(tol=TOL, X=X_h)
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            hsolver.prepare(A_h, b_h)
            _, hinfo = hsolver.solve(tol=TOL, X=X_h)
        barrier()
        te = time.perf_counter() - t0
        hsolver.close()
        te_t = torch.tensor([te], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(te_t, op=dist.ReduceOp.MAX)
        e2e = {"value": world * k_e2e / float(te_t.item()), "unit": UNIT,
               "h2d_bytes_per_step": int(A_np.nbytes + b_np.nbytes),
               "d2h_bytes_per_step": int(N * 8), "steps": k_e2e,
               "rel_kkt": hinfo[0].rel_kkt}

    # ---- plain FP64 method on the same workload (the metric's comparison) ----
    plain = None
    if not args.no_plain:
        psolver = aln.Solver("fp64", stream=stream.cuda_stream)
        psolver.prepare(At, bt)
        psolver.solve(tol=TOL, X=Xt)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kp = 2
        e0.record(stream)
        for _ in range(kp):
            psolver.prepare(At, bt)
            _, pinfo = psolver.solve(tol=TOL, X=Xt)
        e1.record(stream)
        barrier()
        tp = e0.elapsed_time(e1) / 1e3
        pst = psolver.stats()
        psolver.close()
        plain = {"value": kp / tp, "unit": UNIT, "steps": kp, "ms_per_step": tp / kp * 1e3,
                 "gram_ms": pst.gram_ms, "iters": pinfo[0].iters, "rel_kkt": pinfo[0].rel_kkt}

    solver.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    pk, pk_kind = peaks()
    gram = sum(gram_ms) / len(gram_ms)
    flops = 3.0 * D * N * (N + 1)              # three split products over n(n+1)/2 entries
    achieved = flops / (gram / 1e3) / 1e12
    peak = float(pk["bf16_tflops_sustained"])
    roof_gram = {"bound": "tensor", "kernel": "k_gram_tc (split-BF16 Gram)",
                 "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                 "frac": achieved / peak, "traffic": None,
                 "peak_kind": f"{pk_kind} bf16 sustained",
                 "algorithmic_per_launch": flops, "avg_launch_ms": gram}
    it_ms = sum(iter_ms) / len(iter_ms)
    qbytes = 4.0 * N * (sum(qrows) / len(qrows))   # FP32 rows of Q read (§4.2: n·S(n) per product)
    hbm = float(pk["hbm_gbs"])
    ach_it = qbytes / (it_ms / 1e3) / 1e9 if it_ms > 0 else 0.0
    roof_iter = {"bound": "hbm", "kernel": "k_alg2_persist (Alg. 2 loop)",
                 "achieved": ach_it, "peak": hbm, "unit": "GB/s", "frac": ach_it / hbm,
                 "traffic": None, "peak_kind": f"{pk_kind} hbm copy",
                 "algorithmic_per_launch": qbytes, "avg_launch_ms": it_ms,
                 "note": "Q (FP32, 100 MB) can stay in the 129 MB L2, so frac may exceed 1"}
    roofline, roof2 = (roof_iter, roof_gram) if it_ms >= gram else (roof_gram, roof_iter)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        m = N // 2
        ts, scale, _ = cpu_baseline_sample(A_np, b_np, m)
        cpu = {"value": 1.0 / (ts * scale), "unit": UNIT, "cores": blas_threads(),
               "kind": "oracle",
               "sample": f"oracle antilop on A[:, :{m}] (d={D}) in {ts:.2f} s, "
                         f"x (n/m)^2 = {scale:.0f} for the full size"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmax / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "d": D, "n": N, "tol": TOL, "seed": SEED,
                   "form": "split-BF16 tcgen05 Gram, FP32 Alg. 2, FP64 scale/KKT/refinement",
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (A 400 MB fp32, split copies 400 MB)",
                   "prepare_ms": sum(prep_ms) / len(prep_ms),
                   "gram_ms": gram, "solve_ms": sum(solve_ms) / len(solve_ms),
                   "iterate_ms": it_ms, "kkt_ms": sum(kkt_ms) / len(kkt_ms),
                   "iters": iters, "rel_kkt_max": worst},
        "roofline": roofline,
        "roofline_secondary": roof2,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "plain_fp64": plain,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    global D, N, WORKLOAD
    args = parse()
    D, N = args.d, args.n
    WORKLOAD = WORKLOAD_FMT.format(d=D, n=N)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
