"""Benchmark of the GCP solver on one GB300 (or N independent replicas).

Workload (default): one dense symmetric H, M=8192, N=2048, H = Q diag(eps) Q^T
with Q from the Householder QR of a seeded N(0,1) matrix, occupied levels
uniform in [-1, -0.005] and virtual in [0.005, 1] (gap 0.01); mixed precision
(split-FP16 tensor-core products, FP64 refinement) to ||D^2 - D||_F <= 1e-6,
from the paper's HPCP+ initial guess (Eq. hpcpguess; --guess canonical for
Eq. dmguess alone).  The plain FP64 GPU path it is compared with starts from
the same guess.

One step = one full solve (guess -> converged D -> energy).  `value` is the
effective GCP rate, 4 M^3 flops per applied step (two dense products) over
the solve time, in TFLOP/s.  Inputs (H is 512 MiB in FP64) exceed the 129 MB
L2, so no flush is needed between steps.  Multi-GPU: independent replicas
(each rank solves its own H), weak scaling, no collective on the data path.

--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded sample (a few purification steps of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M_DEFAULT, N_DEFAULT, GAP_DEFAULT = 8192, 2048, 0.01
TOL = 1e-6


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gcp", choices=["gcp", "reference"])
    p.add_argument("--M", type=int, default=M_DEFAULT)
    p.add_argument("--N", type=int, default=N_DEFAULT)
    p.add_argument("--gap", type=float, default=GAP_DEFAULT)
    p.add_argument("--prec", default="mixed_fp16")
    p.add_argument("--guess", default="hpcp+", choices=["canonical", "hpcp+", "hole"],
                   help="initial guess (default: the paper's HPCP+ guess, Eq. hpcpguess)")
    p.add_argument("--method", default="hpcp", choices=["hpcp", "pmcp"])
    p.add_argument("--skip-fp64", action="store_true", help="skip the plain FP64 GPU comparison")
    p.add_argument("--skip-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--skip-loop", action="store_true",
                   help="batched workload: skip the loop of single solves it is compared with")
    p.add_argument("--cpu-iters", type=int, default=2)
    p.add_argument("--no-graph", action="store_true",
                   help="host-driven loop (same kernels, one launch each; for launch lists)")
    p.add_argument("--workload", default="dense",
                   choices=["dense", "tb", "batched", "adjoint", "pbar"],
                   help="dense: the headline (one dense H); tb: tight-binding 20^3 insulator; "
                        "batched: 512 uneven instances; adjoint: dL/dH through 40 steps")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_input(M, N, gap, seed, qr_backend="torch"):
    from paper_1512_07236_gb300 import inputs
    return inputs.rotated_spectrum(M, N, (-1.0, -gap / 2), (gap / 2, 1.0), seed=seed,
                                   qr_backend=qr_backend)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def max_over_ranks(value, world, device="cpu"):
    """The slowest rank's time: replicas are timed each on its own GPU and the
    whole job lasts as long as the slowest one (a MAX all-reduce)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(flops_per_solve, steps, world, ms_total):
    """Every replica solves its own H each step (weak scaling): the job's
    rate is all ranks' work over the slowest rank's time."""
    return world * flops_per_solve * steps / (ms_total * 1e-3) / 1e12


def lookup_traffic(kernel, M):
    """DRAM bytes per launch of `kernel` at this M from the committed ncu
    summary table, or None when there is none or the kernel's source file
    changed since the capture (its SHA-256 is recorded beside the figure)."""
    import hashlib
    table = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if kernel is None or not os.path.exists(table):
        return None
    for line in open(table):
        f = line.split()
        if len(f) != 5 or line.startswith("#"):
            continue
        name, m, src, sha, nbytes = f
        if name != kernel or int(m) != M:
            continue
        path = os.path.join(ROOT, "paper_1512_07236_gb300", "csrc", src)
        if not os.path.exists(path):
            return None
        if hashlib.sha256(open(path, "rb").read()).hexdigest() != sha:
            return None
        return float(nbytes)
    return None


def oracle_sample(H, N, iters):
    """The FP64 oracle as it stands, `iters` purification steps of the
    workload; returns (seconds, applied steps)."""
    from oracle import gcp_oracle as o
    t0 = time.perf_counter()
    r = o.solve(H, N, fixed_iters=iters, record=False)
    return time.perf_counter() - t0, r["iters"]


def dtype_label(prec, M=None, tol=TOL):
    """The arithmetic a precision option runs: split products (two 16-bit
    halves, three products) then FP64 refinement for the mixed modes."""
    if prec == "mixed_auto":  # the library's rule (include/gcp.h)
        prec = "fp64" if (M is not None and M < 512) or tol < 1e-10 else "mixed_fp16"
    return {"fp64": "f64", "fp16x3": "fp16x3", "bf16x3": "bf16x3",
            "mixed_fp16": "fp16x3+f64", "mixed_bf16": "bf16x3+f64"}.get(prec, prec)


# The headline metric, shared by both arms.
METRIC = "GCP effective TFLOP/s (dense-equivalent 4 M^3 per step) to ||D^2-D||_F<=1e-6"


def workload_name(M, N, gap):
    return f"dense rotated spectrum M={M} N={N} gap={gap}, tol {TOL}"


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    M, N = args.M, args.N
    H, eps, Q = make_input(M, N, args.gap, seed=2, qr_backend="numpy")
    flops_step = 4.0 * M ** 3
    for _ in range(args.warmup):
        oracle_sample(H, N, 1)
    times = []
    for _ in range(args.steps):
        t, n = oracle_sample(H, N, args.cpu_iters)
        times.append(t / max(n, 1))
    per_step = statistics.mean(times)
    value = flops_step / per_step / 1e12
    line = {
        "impl": "reference", "metric": METRIC,
        "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(M, N, args.gap),
                   "M": M, "N": N, "gap": args.gap, "prec": "fp64 (CPU oracle)",
                   "sample": f"{args.cpu_iters} purification steps per timed step"},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cpu_cores(),
                         "kind": "oracle",
                         "sample": f"{args.cpu_iters} FP64 steps of M={M} (numpy, host BLAS)"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _cuda_ms(fn, reps, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps, out


def run_workload(args, rank):
    """The other workloads of the method, one JSON line each (rank 0)."""
    import numpy as np
    import torch

    from paper_1512_07236_gb300 import gcp, inputs

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    solver = gcp.Solver()
    W, K = max(args.warmup, 1), max(args.steps, 1)
    line = {"n_gpus": 1, "steps": K, "warmup": W, "scaling": "weak", "vs_baseline": None,
            "data": "synthetic"}
    if args.workload == "tb":
        Hf = inputs.tight_binding_cubic(L=20, seed=3)
        M, N = Hf.shape[0], Hf.shape[0] // 2
        Ht = torch.from_numpy(Hf).cuda()
        D = torch.empty((M, M), dtype=torch.float64, device="cuda")
        opts = dict(prec=args.prec, tol=TOL, guess=args.guess, method=args.method)
        for _ in range(W):
            solver.solve(Ht, N, out=D, **opts)
        with ClockSampler(0) as clk:
            ms, (_, info) = _cuda_ms(lambda: solver.solve(Ht, N, out=D, **opts), K, stream)
        H64 = Ht.double()
        lam = torch.linalg.eigvalsh(H64)
        E_ref = float(lam[:N].sum())
        R = float(torch.linalg.norm(D @ D - D))
        fp64_ms = None
        if not args.skip_fp64:
            fp64_ms, (_, i64) = _cuda_ms(lambda: solver.solve(Ht, N, prec="fp64", tol=TOL,
                                                              guess=args.guess), 1,
                                         stream)
        line.update({
            "metric": "time to ||D^2-D||_F<=1e-6, tight-binding insulator", "value": ms * 1e-3,
            "unit": "s", "higher_is_better": False, "ms_per_step": ms,
            "dtype": dtype_label(args.prec, M),
            "config": {"workload": "simple-cubic 20^3 tight-binding, t=-1, onsite +-0.5, "
                                   "disorder 0.1, FP32 storage, N=4000", "M": M, "N": N,
                       "prec": args.prec, "guess": args.guess, "iters": info["iters"]},
            "energy_err_per_site": abs(info["energy"] - E_ref) / M,
            "idem_fro": R, "trace_err": abs(float(torch.trace(D)) - N),
            "fp64_gpu_path_ms": fp64_ms,
            "speedup_vs_fp64_gpu": fp64_ms / ms if fp64_ms else None,
            "clocks": clk.summary()})
    elif args.workload == "batched":
        items = inputs.batched_rotated(512, qr_backend="torch")
        Hs = [torch.from_numpy(H).cuda() for H, _, _, _ in items]
        Ns = [N for _, N, _, _ in items]
        opts = dict(prec=args.prec, tol=TOL, guess=args.guess, method=args.method,
                    use_graph=not args.no_graph)
        for _ in range(W):
            solver.solve_batched(Hs, Ns, **opts)
        with ClockSampler(0) as clk:
            ms, (Ds, infos) = _cuda_ms(lambda: solver.solve_batched(Hs, Ns, **opts), K, stream)
        # work order of the tensor-core tiles, timed at the first solve
        order_choice, order_ms = solver.batched_order()
        loop_ms = None
        if not args.skip_loop:
            single = gcp.Solver()
            for H, N in zip(Hs[:4], Ns[:4]):
                single.solve(H, N, **opts)
            loop_ms, _ = _cuda_ms(lambda: [single.solve(H, N, **opts) for H, N in zip(Hs, Ns)],
                                  1, stream)
        # the same batch split by size class, each class timed on its own
        # (small instances are bound by per-tile latency, not by the MMAs)
        buckets = {}
        for lo, hi in ((64, 256), (257, 512), (513, 768), (769, 1024)):
            idx = [k for k, H in enumerate(Hs) if lo <= H.shape[0] <= hi]
            if not idx:
                continue
            Hb, Nb = [Hs[k] for k in idx], [Ns[k] for k in idx]
            solver.solve_batched(Hb, Nb, **opts)
            bms, _ = _cuda_ms(lambda: solver.solve_batched(Hb, Nb, **opts), 1, stream)
            buckets[f"M {lo}-{hi}"] = {"instances": len(idx), "solves_per_s": len(idx) / (bms * 1e-3),
                                       "ms": bms}
        errs = []
        for (H, N, eps, Q), Dk in zip(items[:32], Ds[:32]):
            Qo = torch.from_numpy(Q[:, :N]).cuda()
            errs.append(float(torch.linalg.norm(Dk - Qo @ Qo.T)) / np.sqrt(N))
        flops = sum(4.0 * H.shape[0] ** 3 * i["iters"] for H, i in zip(Hs, infos))
        line.update({
            "metric": "batched solves/s to ||D^2-D||_F<=1e-6", "value": 512 / (ms * 1e-3),
            "unit": "solves/s", "higher_is_better": True, "ms_per_step": ms,
            "dtype": dtype_label(args.prec),
            "config": {"workload": "512 rotated spectra, M in {64,96,...,1024}, N=M/4, "
                                   "gap U[0.02,0.2]", "prec": args.prec, "guess": args.guess,
                       "sum_M2": int(sum(H.shape[0] ** 2 for H in Hs))},
            "loop_of_single_solves_per_s": 512 / (loop_ms * 1e-3) if loop_ms else None,
            "speedup_vs_loop": loop_ms / ms if loop_ms else None,
            "effective_tflops": flops / (ms * 1e-3) / 1e12,
            "by_size": buckets,
            "work_order": {"choice": ["instance-major", "cost-sorted", "cost-sorted snake",
                                      "instance-major, largest first"][order_choice],
                           "gemm1_ms": {"instance-major": order_ms[0], "cost-sorted": order_ms[1],
                                        "cost-sorted snake": order_ms[2],
                                        "instance-major, largest first": order_ms[3]}},
            "status_ok": sum(1 for i in infos if i["status"] == 0),
            "max_subspace_err_first32": max(errs), "clocks": clk.summary()})
    elif args.workload == "pbar":
        # Fig. 3: mean iteration counts on the paper's diagonal M = 100 test
        # matrices, 32 per point, stop at Tr(D Dbar) <= 1e-6, one batched FP64
        # solve per point (HPCP / PMCP steps, canonical / HPCP+ guess)
        Mq, per = 100, 32
        thetas, gaps = (0.05, 0.1, 0.2, 0.3, 0.4, 0.5), (1.0, 1e-2, 1e-4)
        variants = (("hpcp", "canonical"), ("pmcp", "canonical"), ("hpcp", "hpcp+"))
        batches = []
        for th in thetas:
            for g in gaps:
                Nq = int(round(th * Mq))
                Hs = [torch.from_numpy(inputs.diagonal_spectrum(Mq, Nq, g, seed=1000 + k)[0]).cuda()
                      for k in range(per)]
                batches.append((th, g, Nq, Hs))
        table = []

        def run_all():
            out = []
            for th, g, Nq, Hs in batches:
                row = {"theta": th, "gap": g}
                for meth, gs in variants:
                    _, infos = solver.solve_batched(Hs, [Nq] * per, prec="fp64", stop="trace",
                                                    tol=1e-6, method=meth, guess=gs)
                    row[f"{meth}/{gs}"] = float(np.mean([i["iters"] for i in infos]))
                out.append(row)
            return out

        for _ in range(W):
            run_all()
        with ClockSampler(0) as clk:
            ms, table = _cuda_ms(run_all, K, stream)
        nsolve = len(batches) * per * len(variants)
        line.update({
            "metric": "p-bar study: batched FP64 solves/s (Fig. 3 matrices)",
            "value": nsolve / (ms * 1e-3), "unit": "solves/s", "higher_is_better": True,
            "ms_per_step": ms, "dtype": "f64",
            "config": {"workload": "diagonal M=100, eigenvalues in [-2.5, eps_N] u [eps_N+1, 2.5], "
                                   "32 per point, stop Tr(D Dbar) <= 1e-6",
                       "thetas": list(thetas), "gaps": list(gaps)},
            "pbar": table, "clocks": clk.summary()})
    else:  # adjoint
        M, N, Kst = 2048, 512, 40
        H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -0.025), (0.025, 1.0), seed=5,
                                            qr_backend="torch")
        V = inputs.symmetric_gaussian(M, 0.1, seed=6)
        Ht, Vt = torch.from_numpy(H).cuda(), torch.from_numpy(V).cuda()
        # the FP32 recursion (split-FP16 tensor-core products) and its adjoint
        H32, V32 = Ht.float(), Vt.float()
        g32 = torch.empty_like(H32)
        run = lambda: solver.backward(H32, N, Kst, G_D=V32, g_E=1.0, ckpt_every=8, out=g32,
                                      prec="fp32")
        for _ in range(W):
            run()
        with ClockSampler(0) as clk:
            ms, _ = _cuda_ms(run, K, stream)
        fwd_ms, _ = _cuda_ms(lambda: solver.solve(H32, N, prec="fp32", fixed_iters=Kst), 1,
                             stream)
        # the FP64 recursion and adjoint, once
        g64 = torch.empty_like(Ht)
        ms64, _ = _cuda_ms(lambda: solver.backward(Ht, N, Kst, G_D=Vt, g_E=1.0, ckpt_every=8,
                                                   out=g64), 1, stream)
        gH32 = g32.double().cpu().numpy()
        gH64 = g64.cpu().numpy()

        def loss(Hx):
            D, info = solver.solve(torch.from_numpy(Hx).cuda(), N, prec="fp64",
                                   fixed_iters=Kst)
            return float((D * Vt).sum()) + info["energy"]

        rng = np.random.default_rng(8)
        rel32, rel64 = [], []
        for _ in range(4):
            Ed = rng.standard_normal((M, M))
            Ed = Ed + Ed.T
            Ed /= np.linalg.norm(Ed)
            fd = (loss(H + 1e-4 * Ed) - loss(H - 1e-4 * Ed)) / 2e-4
            rel32.append(abs(float(np.sum(gH32 * Ed)) - fd) / max(abs(fd), 1e-30))
            rel64.append(abs(float(np.sum(gH64 * Ed)) - fd) / max(abs(fd), 1e-30))
        line.update({
            "metric": "dL/dH through 40 GCP steps (forward + adjoint)", "value": ms * 1e-3,
            "unit": "s", "higher_is_better": False, "ms_per_step": ms, "dtype": "f32",
            "config": {"workload": "M=2048 N=512 gap 0.05, L = Tr(DH) + Tr(DV), V ~ N(0,0.01)",
                       "fixed_iters": Kst, "ckpt_every": 8,
                       "prec": "fp32 (split-FP16 tensor-core products)"},
            "forward_only_ms": fwd_ms, "fd_rel_err_max": max(rel32),
            "fp64": {"s": ms64 * 1e-3, "fd_rel_err_max": max(rel64)},
            "max_abs_fp32_minus_fp64": float(np.abs(gH32 - gH64).max()),
            "clocks": clk.summary()})
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload != "dense":
        run_workload(args, rank)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1512_07236_gb300 import gcp

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    M, N = args.M, args.N
    H, eps, Q = make_input(M, N, args.gap, seed=2 + rank)
    Ht = torch.from_numpy(H).to(dev)
    D = torch.empty((M, M), dtype=torch.float64, device=dev)
    solver = gcp.Solver()
    stream = torch.cuda.current_stream()
    opts = dict(prec=args.prec, tol=TOL, max_iter=100, use_graph=not args.no_graph,
                guess=args.guess, method=args.method)

    def solve_once():
        return solver.solve(Ht, N, out=D, **opts)

    # warm-up (graph capture on the first call)
    for _ in range(args.warmup):
        _, info = solve_once()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        infos = []
        for _ in range(args.steps):
            _, info = solve_once()
            infos.append(info)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms_total = ev0.elapsed_time(ev1)
    ms_total = max_over_ranks(ms_total, world, dev)
    ms_step = ms_total / args.steps
    iters = infos[-1]["iters"]
    flops_step = 4.0 * M ** 3 * iters
    value = whole_job_tflops(flops_step, args.steps, world, ms_total)

    # --- accuracy of the returned D against the exact projector (FP64) ----
    acc = {}
    if rank == 0:
        Qo = torch.from_numpy(Q[:, :N]).to(dev)
        Dref = Qo @ Qo.T
        diff = D - Dref
        acc = {
            "fro_err_over_sqrtN": float(torch.linalg.norm(diff) / np.sqrt(N)),
            "max_abs_err": float(diff.abs().max()),
            "energy_rel_err": abs(infos[-1]["energy"] - float(eps[:N].sum())) / abs(float(eps[:N].sum())),
            "trace_err": abs(float(torch.trace(D)) - N),
            "idem_fro": infos[-1]["idem_fro"],
        }
        del Dref, diff, Qo

    # --- the products, each timed alone with CUDA events ------------------
    # Per launch, algorithmic work = one dense-equivalent product, 2 M^3.
    # Executed tensor work counts the computed 128 x 256 upper tiles: 3
    # products for a split GEMM, the digit-slice pairs for the exact D^2 (up
    # to M = 16384: the 43 pairs of weights 0..8 of eight base-64 slices plus
    # the (5, 5) square; beyond: 53 pairs of nine base-32 slices plus the
    # square), 3 for the refinement's (D^2 - D) D.
    split_prec = "bf16x3" if "bf16" in args.prec else "fp16x3"
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    fp16_note = "of measured" if "bf16_tflops" in peaks else "of fallback"
    Mp = ((M + 255) // 256) * 256
    ntiles = sum(min(2 * j + 2, Mp // 128) for j in range(Mp // 256))
    tile_flops = 2.0 * ntiles * 128 * 256 * Mp
    alg = 2.0 * M ** 3
    lp, l64 = infos[-1]["iters_lowp"], infos[-1]["iters_fp64"]
    kern = {}
    try:
        solver.solve(Ht, N, out=D, **opts)
        if "mixed" in args.prec or args.prec in ("fp16x3", "bf16x3"):
            t1, t2 = solver.time_kernels(M, N, prec=split_prec, reps=5)
            kern["tc_gemm_kernel"] = {
                "what": "split GEMM1 + GEMM2 of one step", "ms": [t1, t2],
                # every evaluation runs GEMM1 (lp steps + the final test), GEMM2 per step
                "launches_per_solve": 2 * lp + 1, "ms_per_solve": t1 * (lp + 1) + t2 * lp,
                "achieved_tflops": 2 * alg / ((t1 + t2) * 1e-3) / 1e12,
                "executed_tflops": 2 * 3 * tile_flops / ((t1 + t2) * 1e-3) / 1e12}
        if "mixed" in args.prec and l64 > 0:
            o1, o2, o3, npair = solver.time_kernels(M, N, prec=args.prec, reps=3, tol=TOL)
            # each refinement step: slice GEMM, refinement product, stop-test
            # product (the last step's stop test accepts D1 without a further
            # slice GEMM)
            kern["oz_gemm_kernel"] = {
                "what": f"digit-slice D^2 of one refinement step ({npair} digit-pair products)",
                "ms": o1, "launches_per_solve": l64, "ms_per_solve": o1 * l64,
                "achieved_tflops": alg / (o1 * 1e-3) / 1e12,
                "executed_tflops": npair * tile_flops / (o1 * 1e-3) / 1e12}
            kern["tc_gemm_kernel<3>"] = {
                "what": "refinement product (D^2 - D) D", "ms": o2, "launches_per_solve": l64,
                "ms_per_solve": o2 * l64, "executed_tflops": 3 * tile_flops / (o2 * 1e-3) / 1e12}
            kern["tc_gemm_kernel<4>"] = {
                "what": "stop-test product W = D1^2 - D^2 (K = 3M)", "ms": o3,
                "launches_per_solve": l64, "ms_per_solve": o3 * l64,
                "executed_tflops": 9 * tile_flops / (o3 * 1e-3) / 1e12}
    except Exception as e:  # noqa: BLE001
        kern["error"] = str(e)
    roof = {"bound": "tensor", "achieved": None, "peak": bf16_peak, "unit": "TFLOP/s",
            "frac": None, "traffic": None}
    timed = {k: v for k, v in kern.items() if isinstance(v, dict)}
    if timed:
        top = max(timed, key=lambda k: timed[k]["ms_per_solve"])
        kt = timed[top]
        ach = kt.get("achieved_tflops", kt["executed_tflops"])
        roof.update({"achieved": ach, "frac": ach / bf16_peak, "kernel": top,
                     "executed_tflops": kt["executed_tflops"],
                     "executed_frac": kt["executed_tflops"] / bf16_peak,
                     "share_of_solve": kt["ms_per_solve"] / ms_step,
                     "peak_note": f"bf16 dense burst {fp16_note} (fp16 has the same nominal "
                                  "rate); achieved = 2 M^3 per launch / mean launch time"})
    roof["traffic"] = lookup_traffic(top if timed else None, M)

    # --- end to end through the C ABI with host buffers --------------------
    # (after the timed region and the short kernel timings, before the long
    # FP64 comparison below, so that it runs in the timed region's clock state)
    # Every step copies its H in from pinned host memory and its D out to
    # pinned host memory inside the timed region.  The copies run on a second
    # stream, overlapped with the neighbouring solves: while step k solves,
    # step k+1's H goes in and step k-1's D comes out.  Consecutive steps
    # alternate between two pairs of device buffers, each with its own solver
    # handle (a handle's recorded graph is bound to its buffers).
    Hh = torch.from_numpy(H).pin_memory()
    Dh = torch.empty((M, M), dtype=torch.float64).pin_memory()
    copy = torch.cuda.Stream()
    Hd, Dd = [Ht, torch.empty_like(Ht)], [D, torch.empty_like(D)]
    handles = [solver, gcp.Solver()]
    Hd[1].copy_(Ht)
    handles[1].solve(Hd[1], N, out=Dd[1], **opts)  # records its graph, untimed
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy.wait_stream(stream)
    with torch.cuda.stream(copy):
        Hd[0].copy_(Hh, non_blocking=True)
    copy.synchronize()
    for k in range(args.steps):
        b = k % 2
        with torch.cuda.stream(copy):
            if k + 1 < args.steps:
                Hd[1 - b].copy_(Hh, non_blocking=True)
            if k > 0:
                Dh.copy_(Dd[1 - b], non_blocking=True)
        _, info = handles[b].solve(Hd[b], N, out=Dd[b], **opts)  # synchronous at exit
        copy.synchronize()
    Dh.copy_(Dd[(args.steps - 1) % 2], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    del handles, Hd, Dd
    e2e_value = whole_job_tflops(flops_step, args.steps, world, max_over_ranks(ms_e2e, world, dev))

    # --- plain FP64 GPU path: time to the same tolerance -------------------
    fp64 = None
    if not args.skip_fp64 and rank == 0:
        D64 = torch.empty_like(D)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, i64 = solver.solve(Ht, N, out=D64, prec="fp64", tol=TOL, max_iter=100,
                              guess=args.guess, method=args.method)
        b.record(stream)
        torch.cuda.synchronize()
        fp64 = {"ms": a.elapsed_time(b), "iters": i64["iters"], "status": i64["status"],
                "idem_fro": i64["idem_fro"]}
        del D64

    # --- CPU oracle baseline on a bounded sample ---------------------------
    cpu = None
    if rank == 0 and not args.skip_cpu:
        t, n = oracle_sample(H, N, args.cpu_iters)
        cpu = {"value": 4.0 * M ** 3 * n / t / 1e12, "unit": "TFLOP/s", "cores": cpu_cores(),
               "kind": "oracle",
               "sample": f"{n} FP64 purification steps of M={M} (numpy + host BLAS), "
                         f"{t:.1f} s"}

    # kernel launches per solve: guess 4; each WHILE body holds two steps and
    # runs (evaluations + 1) // 2 times, evaluations = applied steps + 1
    # (slice refinement: = applied steps, the stop test of the last step
    # ends the phase); split step 3 launches (GEMM1, control, GEMM2), FP64
    # step 3, slice refinement step 8 (slice, slice GEMM, finalize, control,
    # product, stop-test halves, stop-test product, stop-test control);
    # phase change 2; copy-out 1; energy 2
    split_phase = "mixed" in args.prec or args.prec in ("fp16x3", "bf16x3")
    f64_phase = "mixed" in args.prec or args.prec == "fp64"
    slices = "mixed" in args.prec and "oz_gemm_kernel" in kern
    ref_step = 8 if slices else 3
    per_solve = 4 + 1 + 2
    if split_phase:
        per_solve += 6 * ((lp + 2) // 2)
    if f64_phase:
        evals = l64 if slices else l64 + 1
        per_solve += 2 * ref_step * ((evals + 1) // 2) + (2 if "mixed" in args.prec else 0)
    launches = args.steps * per_solve

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype_label(args.prec, M),
            "data": "synthetic",
            "config": {"workload": workload_name(M, N, args.gap),
                       "M": M, "N": N, "gap": args.gap, "prec": args.prec,
                       "guess": args.guess, "method": args.method,
                       "iters": iters, "iters_lowp": lp, "iters_fp64": l64,
                       "l2": "inputs larger than L2 (H 512 MiB FP64)",
                       "parallelism": f"replicas x{world}"},
            "time_to_tol_s": ms_step * 1e-3,
            "fp64_gpu_path": fp64,
            "speedup_vs_fp64_gpu": (fp64["ms"] / ms_step) if fp64 else None,
            "accuracy": acc,
            "roofline": roof,
            "kernels": kern,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "TFLOP/s",
                    "h2d_bytes_per_step": M * M * 8, "d2h_bytes_per_step": M * M * 8,
                    "copies": "pinned host buffers; step k+1's H in and step k-1's D out on a "
                              "second stream during step k's solve"},
            "clocks": clk.summary(),
            "gpu_launches": launches,
            "status": infos[-1]["status"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
