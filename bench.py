#!/usr/bin/env python3
"""Benchmark: emulated-FP64 LU (partial pivoting) TFLOP/s on one GB300.

One step = one LU factorization with partial pivoting of a fresh n x n copy of
the synthetic input (emul_dgetrf: FP64 panel, emulated U12 solve and trailing
updates with s INT8 slices) plus the solve (emul_dgetrs).  The TFLOP/s
numerator is the HPL count 2/3 n^3 + 3/2 n^2.  The backward error
||Ax-b|| / (||A|| ||x|| n eps) of the last solve must stay <= 16.

--workload lu_nopiv times the Level-3-only LU without pivoting of Section 8
(emul_dgetrf_nopiv, block size --nb up to 4096) on a diagonally dominant
matrix, with the same solve, checks and JSON keys.  --range R > 0 draws the LU
input from the log-scaled generator u 10^e, e ~ U(-R, R).  --workload chol
times the blocked Cholesky (emul_dpotrf + emul_dpotrs) of an SPD matrix
Q diag(lam) Q^T with condition number --cond (numerator n^3/3 + 2 n^2).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (the
project's plain reference of the same method) on a bounded sample.
Multi-GPU (torchrun): replicas only; every rank factors its own matrix.
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

METRIC = "emulated-FP64 LU TFLOP/s vs native-FP64 LU on one GB300 at backward error ≤16"
METRIC_NOPIV = "emulated-FP64 LU without pivoting TFLOP/s on one GB300 at backward error ≤16"
METRIC_CHOL = "emulated-FP64 Cholesky TFLOP/s vs native-FP64 Cholesky on one GB300 at backward error ≤16"


# dram__bytes_read.sum + dram__bytes_write.sum (623.6 + 488.2 MB) of one launch of the
# product kernel (CTA pairs) on 8192^2 x 256 at s = 7 (full ncu capture), over the algorithmic
# bytes of the same launch (C 8192^2 x 16 B + slices 2 x 7 x 8192 x 256 x 2 B)
TRAFFIC_RATIO = (623.625216e6 + 488.196608e6) / (8192.0 * 8192.0 * 16.0 + 2 * 7 * 8192 * 256 * 2.0)


def lu_flops(n):
    return 2.0 / 3.0 * n ** 3 + 1.5 * n ** 2


def chol_flops(n):
    return n ** 3 / 3.0 + 2.0 * n ** 2


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.proc = None
        self.uuid = uuid

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x):
    """Largest value over the ranks (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world, flops_per_step, steps, ms_max):
    """Whole-job TFLOP/s of `world` replicas, each doing flops_per_step per step."""
    return world * flops_per_step * steps / (ms_max / 1e3) / 1e12


def cpu_oracle_lu(n, nb, s, seed, nopiv=False, update="emulated"):
    """Time the oracle's LU + solve of one n x n matrix (bounded sample):
    update = "emulated" (the method, s slices) or "fp64" (FP64 trailing updates)."""
    from oracle import lu as olu, residual
    from paper_2509_23565_gb300 import inputs
    A = inputs.diag_dominant(n, seed=seed) if nopiv else inputs.uniform(n, n, seed=seed)
    b = inputs.vector(n, seed=seed + 1)
    t0 = time.perf_counter()
    if nopiv:
        LU, _ = olu.getrf_nopiv(A, nb=nb, update=update, s=s)
        piv = np.arange(1, n + 1)
    else:
        LU, piv, _ = olu.getrf(A, nb=nb, update=update, s=s)
    x = olu.getrs(LU, piv, b)
    dt = time.perf_counter() - t0
    return dt, residual.backward_error(A, x, b)


def cpu_oracle_chol(n, nb, cond, seed):
    """Time the oracle's FP64 blocked Cholesky + solve of one SPD n x n matrix."""
    from oracle import lu as olu, residual
    from paper_2509_23565_gb300 import inputs
    A = inputs.spd(n, cond, seed=seed)
    b = inputs.vector(n, seed=seed + 1)
    t0 = time.perf_counter()
    L, _ = olu.potrf(A, nb=nb, update="fp64")
    x = olu.potrs(L, b)
    dt = time.perf_counter() - t0
    return dt, residual.backward_error(A, x, b)


def cpu_baseline(args, kind, s):
    """The oracle as it stands on the host cores, on bounded samples of the
    workload: its FP64 blocked factorization + solve (numpy BLAS threads for the
    trailing updates, the panel loop single-threaded) and, for LU, its emulated
    LU + solve with s slices (exact recombination in Python integers)."""
    cores = os.cpu_count()
    if kind == "chol":
        n = 2 * args.cpu_n
        dt, be = cpu_oracle_chol(n, 256, args.cond, 1234)
        return {"value": chol_flops(n) / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                "sample": f"oracle FP64 blocked Cholesky + solve of one SPD n={n} matrix (cond {args.cond:g}, "
                          f"nb=256; numpy BLAS threads, panel loop single-threaded)",
                "seconds": dt, "backward_error": be}
    nopiv = kind == "lu_nopiv"
    n = args.cpu_n
    dt, be = cpu_oracle_lu(n, 256, s, 1234, nopiv, update="fp64")
    edt, ebe = cpu_oracle_lu(args.cpu_emul_n, 64, s, 1235, nopiv, update="emulated")
    what = "no-pivot LU" if nopiv else "LU with partial pivoting"
    return {"value": lu_flops(n) / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle FP64 blocked {what} + solve of one n={n} uniform(-1,1) matrix (nb=256; numpy BLAS "
                      f"threads for the trailing updates, panel loop single-threaded)",
            "seconds": dt, "backward_error": be,
            "emulated_sample": {"value": lu_flops(args.cpu_emul_n) / edt / 1e12, "unit": "TFLOP/s",
                                "sample": f"oracle emulated {what} + solve of one n={args.cpu_emul_n} matrix "
                                          f"(nb=64, s={s}; exact recombination single-threaded)",
                                "seconds": edt, "backward_error": ebe}}


def run_reference(args, world, rank):
    if rank != 0:
        return
    n = args.cpu_emul_n
    for _ in range(args.warmup):
        cpu_oracle_lu(n, 64, args.slices, 1000)
    times, berr = [], None
    for k in range(args.steps):
        dt, berr = cpu_oracle_lu(n, 64, args.slices, 1000 + k)
        times.append(dt)
    tot = sum(times)
    value = lu_flops(n) * args.steps / tot / 1e12
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"LU partial pivoting, oracle sample n={n} nb=64 s={args.slices} uniform(-1,1)",
                   "n": n, "nb": 64, "slices": args.slices},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"oracle emulated LU + solve of one n={n} matrix per step (numpy BLAS threads, "
                                   f"exact recombination single-threaded)"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "backward_error": berr,
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    from paper_2509_23565_gb300 import inputs
    from paper_2509_23565_gb300.binding import ColMajor, Emul

    torch.cuda.set_device(local)
    n, nb, s = args.n, args.nb, args.slices
    kind = args.workload                  # lu, lu_nopiv, chol
    nopiv = kind == "lu_nopiv"
    chol = kind == "chol"
    flops = chol_flops if chol else lu_flops
    seed = 7000 + rank
    A_host = None
    if chol and n <= 8192:
        A0 = torch.from_numpy(inputs.spd(n, args.cond, seed=seed)).cuda()   # symmetric: store = matrix
    elif chol:
        A0 = inputs.spd_device(n, args.cond, seed=seed)
    elif args.range > 0:
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed)
        A0 = inputs.log_scaled_device(n, n, args.range, gen)         # store (n, n): column-major A
    else:
        # Fortran order; the no-pivot LU needs a matrix that elimination without pivoting keeps stable
        A_host = inputs.diag_dominant(n, seed=seed) if nopiv else inputs.uniform(n, n, seed=seed)
        A0 = torch.from_numpy(np.ascontiguousarray(A_host.T)).cuda()
    b_host = inputs.vector(n, seed=seed + 1)
    b0 = torch.from_numpy(b_host).cuda()
    work = ColMajor(torch.empty_like(A0), n, n)
    xb = ColMajor(torch.empty((1, n), dtype=torch.float64, device="cuda"), n, 1)
    lib = Emul()
    stream = torch.cuda.current_stream()
    if getattr(args, "nb_auto", False):
        # the library's block-size tuner (one timed factorization per candidate
        # of a synthetic matrix of this size), before any timed work
        nb = lib.autotune_nb("chol" if chol else "lu", n, s)

    def factor_solve():
        if chol:
            info = lib.dpotrf(work, nb=nb, slices=s)
            lib.dpotrs(work, xb)
            return info
        ipiv, info = (lib.dgetrf_nopiv if nopiv else lib.dgetrf)(work, nb=nb, slices=s)
        lib.dgetrs(work, ipiv, xb)
        return info

    def step():
        work.store.copy_(A0)
        xb.store[0].copy_(b0)
        return factor_solve()

    for _ in range(args.warmup):
        step()
    lib.sync_status()
    lib.profile_read()                      # reset counters
    lib.profile_enable(True)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        info = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = lib.profile_read()
    lib.profile_enable(False)
    lib.sync_status()
    ms_max = max_over_ranks(world, ms)
    # backward error of the last solve (device kernel, FP64)
    A_chk = ColMajor(A0, n, n)
    b_chk = ColMajor(b0.view(1, n), n, 1)
    berr = lib.backward_error(A_chk, xb, b_chk).cpu().numpy()
    info_v = int(info.item())

    value = aggregate_value(world, flops(n), args.steps, ms_max)
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
    achieved = prof["product_tensor_flops"] / (prof["product_ms"] / 1e3) / 1e12 if prof["product_ms"] > 0 else 0.0
    # DRAM traffic per launch: the full ncu capture of the product kernel on
    # 8192^2 x 256 measured 1.11 GB against 1.13 GB of algorithmic bytes; that
    # ratio scales this run's algorithmic bytes
    traffic = TRAFFIC_RATIO * prof["product_bytes"] / max(1, prof["product_launches"])
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
                "traffic_basis": "ncu DRAM bytes / algorithmic bytes = %.3f on the 8192^2 x 256 capture, "
                                 "times this run's algorithmic bytes per launch" % TRAFFIC_RATIO,
                "kernel": "gemm_kernel (slice-pair products)",
                "peak_kind": f"bf16 dense sustained, {peak_kind}",
                "launches": prof["product_launches"],
                "avg_launch_ms": prof["product_ms"] / max(1, prof["product_launches"]),
                "share_of_step": prof["product_ms"] / ms}

    if chol:
        workload = (f"Cholesky + solve, n={n} nb={nb} s={s}, SPD A = Q diag(lam) Q^T (Q from the QR of a Gaussian "
                    f"matrix, lam log-spaced 1..1/{args.cond:g}), b uniform(-1,1)")
    elif nopiv:
        workload = (f"LU without pivoting + solve, n={n} nb={nb} s={s}, A iid uniform(-1,1) with n on the diagonal, "
                    f"b uniform(-1,1)")
    elif args.range > 0:
        workload = (f"LU partial pivoting + solve, n={n} nb={nb} s={s}, A = u 10^e with u uniform(-1,1), "
                    f"e uniform(-{args.range:g},{args.range:g}); b uniform(-1,1)")
    else:
        workload = f"LU partial pivoting + solve, n={n} nb={nb} s={s}, A and b iid uniform(-1,1)"
    metric = METRIC_CHOL if chol else METRIC_NOPIV if nopiv else METRIC
    result = {
        "metric": metric, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload,
                   "n": n, "nb": nb, "slices": s, "parallelism": "replicas" if world > 1 else "single",
                   **({"nb_autotuned": [128, 256, 512]} if getattr(args, "nb_auto", False) else {}),
                   **({"cond": args.cond} if chol else {"range": args.range} if args.range > 0 else {}),
                   "l2": "inputs (8 n^2 bytes) larger than L2; each step restores A from a device copy"},
        "backward_error": float(berr[1]), "scaled_residual_eq8": float(berr[0]), "info": info_v,
        "roofline": roofline, "gpu_launches": int(prof["kernel_launches"]), "clocks": clk,
        "phases_ms_per_step": {k: round(v / args.steps, 2) for k, v in prof["phase_ms"].items()},
    }

    if rank == 0 and not args.no_e2e:
        # end to end through the C-ABI with host buffers: H2D of A and b, factor, solve, D2H of x
        if A_host is not None:
            A_pin = torch.from_numpy(np.ascontiguousarray(A_host.T)).pin_memory()
        else:
            A_pin = A0.cpu().pin_memory()
        b_pin = torch.from_numpy(b_host).pin_memory()
        x_pin = torch.empty(n, dtype=torch.float64).pin_memory()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.e2e_steps):
            work.store.copy_(A_pin, non_blocking=True)
            xb.store[0].copy_(b_pin, non_blocking=True)
            factor_solve()
            x_pin.copy_(xb.store[0], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = e0.elapsed_time(e1)
        result["e2e"] = {"value": flops(n) * args.e2e_steps / (e_ms / 1e3) / 1e12, "unit": "TFLOP/s",
                         "h2d_bytes_per_step": 8 * n * n + 8 * n, "d2h_bytes_per_step": 8 * n,
                         "steps": args.e2e_steps}
        del A_pin

    if rank == 0 and not args.no_native:
        # native FP64 factorization + solve (cuSOLVER through torch) on the same GPU and
        # input, with its backward error; one untimed full-size call first (handles,
        # workspace), then the timed one
        Am = A0.t()                        # column-major view of A

        def native():
            if chol:
                Lc = torch.linalg.cholesky(Am)
                return torch.cholesky_solve(b0.view(n, 1), Lc)
            LU, piv = torch.linalg.lu_factor(Am, pivot=not nopiv)
            return torch.linalg.lu_solve(LU, piv, b0.view(n, 1))

        native()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x = native()
        e1.record(stream)
        torch.cuda.synchronize()
        nms = e0.elapsed_time(e1)
        xn = ColMajor(x.t().contiguous(), n, 1)
        nb_err = lib.backward_error(A_chk, xn, b_chk).cpu().numpy()
        impl = ("torch.linalg.cholesky/cholesky_solve" if chol else
                "torch.linalg.lu_factor/lu_solve" + (" (pivot=False)" if nopiv else ""))
        result["native_fp64"] = {"value": flops(n) / (nms / 1e3) / 1e12, "unit": "TFLOP/s", "ms": nms,
                                 "backward_error": float(nb_err[1]), "impl": impl, "warmup": 1}
        result["speedup_vs_native"] = result["native_fp64"]["ms"] / result["ms_per_step"]
        del x
        torch.cuda.empty_cache()

    if rank == 0 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(args, kind, s)
    if rank == 0:
        print(json.dumps(result), flush=True)


def run_gemm(args):
    """Standalone emulated DGEMM C <- C - A B (the trailing-update form), m = n, k given."""
    import torch
    from paper_2509_23565_gb300.binding import ColMajor, Emul
    n, k, s = args.n, args.k, args.slices
    A = ColMajor(torch.rand(k, n, dtype=torch.float64, device="cuda") * 2 - 1, n, k)
    B = ColMajor(torch.rand(n, k, dtype=torch.float64, device="cuda") * 2 - 1, k, n)
    C = ColMajor(torch.rand(n, n, dtype=torch.float64, device="cuda"), n, n)
    lib = Emul()
    for _ in range(args.warmup):
        lib.dgemm(A, B, C, s, -1.0, 1.0)
    lib.sync_status()
    lib.profile_read()
    lib.profile_enable(True)
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        lib.dgemm(A, B, C, s, -1.0, 1.0)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = lib.profile_read()
    lib.sync_status()
    P = s * (s + 1) // 2
    peaks, kind = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    ach = prof["product_tensor_flops"] / (prof["product_ms"] / 1e3) / 1e12
    print(json.dumps({"metric": "emulated DGEMM TFLOP/s (C - A B)", "value": 2.0 * n * n * k / (ms / 1e3) / 1e12,
                      "unit": "TFLOP/s", "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
                      "config": {"workload": f"emulated DGEMM m=n={n} k={k} s={s}", "pairs": P},
                      "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                   "frac": ach / peak, "peak_kind": f"bf16 dense burst, {kind}"}}), flush=True)


def run_gemm_sweep(args):
    """Standalone emulated DGEMM sweep: m = n = k in {4096, 8192, 16384} x s in
    3..8 (C - A B form, one rounding per entry), TFLOP/s of the emulated FP64
    product and the product kernel's fraction of the measured BF16 burst peak;
    and, for inputs u 10^e with u ~ U(-1, 1), e ~ U(-r, r), r in {0, 4, 8, 16},
    the largest error on 32 sampled entries against the exact product (exact
    rational sums of the FP64 products), in units of k u (|A||B|)_ij."""
    import torch
    from fractions import Fraction
    from paper_2509_23565_gb300 import inputs
    from paper_2509_23565_gb300.binding import ColMajor, Emul
    lib = Emul()
    peaks, kind = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    u = 2.0 ** -53
    rows = []
    for n in (4096, 8192, 16384):
        for r in (0, 4, 8, 16):
            gen = torch.Generator(device="cuda")
            gen.manual_seed(n * 100 + r)
            A = ColMajor(inputs.log_scaled_device(n, n, r, gen), n, n)
            B = ColMajor(inputs.log_scaled_device(n, n, r, gen), n, n)
            C = ColMajor(torch.zeros((n, n), dtype=torch.float64, device="cuda"), n, n)
            rng = np.random.default_rng(n + r)
            samp = [(int(i), int(j)) for i, j in zip(rng.integers(0, n, 32), rng.integers(0, n, 32))]
            Ah = {i: A.store[:, i].cpu().numpy() for i, _ in samp}        # row i of A (column-major store)
            Bh = {j: B.store[j].cpu().numpy() for _, j in samp}           # column j of B
            for s in (3, 4, 5, 6, 7, 8):
                timed = r == 0 or (n == 4096)
                if not timed:
                    continue
                reps = 3 if n < 16384 else 2
                lib.dgemm(A, B, C, s, 1.0, 0.0)
                lib.profile_read()
                lib.profile_enable(True)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                for _ in range(reps):
                    lib.dgemm(A, B, C, s, 1.0, 0.0)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                prof = lib.profile_read()
                lib.profile_enable(False)
                lib.sync_status()
                ach = prof["product_tensor_flops"] / (prof["product_ms"] / 1e3) / 1e12
                Ch = C.store.cpu().numpy().T
                worst = 0.0
                for i, j in samp:
                    a, b = Ah[i], Bh[j]
                    exact = sum((Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b)), Fraction(0))
                    scale = float(np.abs(a) @ np.abs(b)) * n * u
                    if scale > 0:
                        worst = max(worst, abs(float(Fraction(float(Ch[i, j])) - exact)) / scale)
                rows.append({"n": n, "r": r, "s": s, "ms": ms, "tflops": 2.0 * n ** 3 / (ms / 1e3) / 1e12,
                             "frac_bf16_burst": ach / peak, "max_err_in_k_u_AB": worst})
            del A, B, C
            torch.cuda.empty_cache()
    print(json.dumps({"metric": "emulated DGEMM sweep (TFLOP/s, roofline fraction, error vs exact)",
                      "config": {"workload": "m=n=k in {4096, 8192, 16384}, s in 3..8, u 10^e inputs"},
                      "peak_kind": f"bf16 dense burst, {kind}", "rows": rows}), flush=True)


def run_table2(args):
    """The paper's scaling table of ParaWilk parameters (alpha = 1): for each n,
    the (d, b) it found to push the scaled residual (Eq. 8) above 16 with 6 and
    with 7 splits, and our residual for those parameters (one draw of the
    random fill, nb = 64), next to the printed value.  Reported, not asserted."""
    import torch
    from paper_2509_23565_gb300 import inputs
    from paper_2509_23565_gb300.binding import ColMajor, Emul
    lib = Emul()
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "table2_parawilk.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    out = []
    t0 = time.perf_counter()
    for n, d6, b6, r6, d7, b7, r7 in rows:
        n = int(n)
        bvec = inputs.vector(n, seed=n + 1)
        entry = {"n": n}
        for s, d, bb, want in ((6, d6, b6, r6), (7, d7, b7, r7)):
            A = inputs.parawilk_random(n, int(d), int(bb), 1.0, seed=n)
            A0 = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
            W = ColMajor(A0.clone(), n, n)
            x = ColMajor(torch.from_numpy(bvec.copy()).cuda().view(1, n), n, 1)
            ipiv, info = lib.dgetrf(W, nb=64, slices=s)
            lib.dgetrs(W, ipiv, x)
            be = lib.backward_error(ColMajor(A0, n, n), x, ColMajor(torch.from_numpy(bvec).cuda().view(1, n), n, 1))
            entry[f"s{s}"] = {"d": int(d), "b": int(bb), "scaled_residual": float(be.cpu().numpy()[0]),
                              "paper": want}
        out.append(entry)
    print(json.dumps({"metric": "scaled residual (Eq. 8) at the paper's ParaWilk parameters, 6 and 7 splits",
                      "config": {"workload": "ParaWilk_n(d, b, 1) with random fill, n = 256..2048, nb = 64"},
                      "seconds": time.perf_counter() - t0, "rows": out}), flush=True)


def run_fig1(args):
    """Fig. 1's sweep: LU + solve on HPL-style data A, b ~ U(-1/2, 1/2) for
    growing n with 6 and 7 splits and native FP64, scaled residual of Eq. 8
    (the paper reports that 6 splits fail the bar of 16 and 7 pass)."""
    import torch
    from paper_2509_23565_gb300 import inputs
    from paper_2509_23565_gb300.binding import ColMajor, Emul
    lib = Emul()
    rows = []
    for n in (256, 512, 1024, 2048, 4096, 8192, 16384):
        gen = torch.Generator(device="cuda")
        gen.manual_seed(n + 7919)          # another stream than A's
        A0 = inputs.uniform_device(n, n, seed=n, lo=-0.5, hi=0.5)
        b0 = torch.rand(n, generator=gen, device="cuda", dtype=torch.float64) - 0.5
        row = {"n": n}
        for s in (6, 7):
            W = ColMajor(A0.clone(), n, n)
            x = ColMajor(b0.clone().view(1, n), n, 1)
            ipiv, info = lib.dgetrf(W, nb=256 if n >= 4096 else 128, slices=s)
            lib.dgetrs(W, ipiv, x)
            be = lib.backward_error(ColMajor(A0, n, n), x, ColMajor(b0.view(1, n), n, 1)).cpu().numpy()
            row[f"s{s}"] = float(be[0])
        LU, piv = torch.linalg.lu_factor(A0.t())
        xn = torch.linalg.lu_solve(LU, piv, b0.view(n, 1))
        be = lib.backward_error(ColMajor(A0, n, n), ColMajor(xn.t().contiguous(), n, 1),
                                ColMajor(b0.view(1, n), n, 1)).cpu().numpy()
        row["fp64"] = float(be[0])
        del LU, piv, xn, A0
        rows.append(row)
    print(json.dumps({"metric": "scaled residual (Eq. 8) of the LU solve on U(-1/2,1/2), 6 and 7 splits",
                      "config": {"workload": "HPL-style A, b ~ U(-1/2, 1/2), n = 256..16384"}, "rows": rows}),
          flush=True)


def run_selector(args):
    """Ablation of the learned slice selector (mixed dynamic ranges): LU + solve with
    slices chosen per step by the trained network (plus the a-posteriori probe)
    against fixed s = 8, on a uniform and on a mixed-range matrix."""
    import torch
    from paper_2509_23565_gb300 import inputs
    from paper_2509_23565_gb300.binding import ColMajor, Emul
    lib = Emul()
    lib.selector_load(os.path.join(ROOT, "paper_2509_23565_gb300", "selector_weights.bin"))
    n, nb = args.n, args.nb
    out = {"metric": "learned slice selector vs fixed s=7 and s=8: LU TFLOP/s at backward error <= 16",
           "config": {"workload": f"LU partial pivoting + solve n={n} nb={nb}", "n": n, "nb": nb}, "cases": {}}
    for name, A in (("uniform", inputs.uniform(n, n, seed=8100)),
                    ("mixed_r_0_8_16", inputs.mixed_range(n, nb, (0, 8, 16), seed=8101))):
        b = inputs.vector(n, seed=8102)
        A0 = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
        b0 = torch.from_numpy(b).cuda()
        W = ColMajor(torch.empty_like(A0), n, n)
        x = ColMajor(torch.empty((1, n), dtype=torch.float64, device="cuda"), n, 1)
        row = {}
        for label, s in (("fixed_s7", 7), ("fixed_s8", 8), ("learned", 0)):
            times, st = [], None
            for rep in range(args.warmup + args.steps):
                W.store.copy_(A0)
                x.store[0].copy_(b0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ipiv, info, st = lib.dgetrf(W, nb=nb, slices=s, stats=True)
                lib.dgetrs(W, ipiv, x)
                torch.cuda.synchronize()
                if rep >= args.warmup:
                    times.append(time.perf_counter() - t0)
            be = lib.backward_error(ColMajor(A0, n, n), x, ColMajor(b0.view(1, n), n, 1)).cpu().numpy()
            t = statistics.median(times)
            row[label] = {"seconds": t, "tflops": lu_flops(n) / t / 1e12, "backward_error": float(be[1]),
                          "slices_mean": st.slices_mean, "slices_min": st.slices_min, "slices_max": st.slices_max,
                          "checks_failed": st.checks_failed}
        row["speedup_vs_s8"] = row["fixed_s8"]["seconds"] / row["learned"]["seconds"]
        row["speedup_vs_s7"] = row["fixed_s7"]["seconds"] / row["learned"]["seconds"]
        out["cases"][name] = row
    print(json.dumps(out), flush=True)


def run_batched(args):
    """Many uneven LU solves (n log-uniform in [64, 1024],
    uniform(-1,1) entries, half of them scaled with r = 8) in one persistent,
    graph-recorded launch: reduced-slice factorization + FP64 refinement."""
    import torch
    from paper_2509_23565_gb300 import inputs
    from paper_2509_23565_gb300.binding import ColMajor, Emul
    count = args.batch_count
    sizes = inputs.batch_sizes(count, 64, 1024, seed=9000)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(9001)
    As, bs, b0 = [], [], []
    for i, n in enumerate(sizes):
        r = 8 if i % 2 else 0
        As.append(ColMajor(inputs.log_scaled_device(int(n), int(n), r, gen), int(n), int(n)))
        v = torch.rand(int(n), generator=gen, device="cuda", dtype=torch.float64) * 2 - 1
        b0.append(v)
        bs.append(ColMajor(v.clone().view(1, int(n)), int(n), 1))
    lib = Emul()
    cache_dir = os.path.join(ROOT, "paper_2509_23565_gb300", "_build")   # build products, not tracked
    tune_path = os.path.join(cache_dir, "batched_autotune.json") if os.path.isdir(cache_dir) else None
    t0 = time.perf_counter()
    lib.autotune(tune_path)
    t_tune = time.perf_counter() - t0
    flops = sum(lu_flops(int(n)) for n in sizes)
    times = []
    for rep in range(args.warmup + args.steps):
        for b, v in zip(bs, b0):
            b.store[0].copy_(v)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        info, berr, iters = lib.dgesv_batched_ir(As, bs, max_iter=30)
        e1.record()
        torch.cuda.synchronize()
        if rep >= args.warmup:
            times.append(e0.elapsed_time(e1))
    lib.sync_status()
    ms = statistics.median(times)
    be = berr.cpu().numpy()
    it = iters.cpu().numpy()
    # native FP64 comparator: cuSOLVER batched LU + solve through torch, the
    # systems grouped by size rounded up to a multiple of 64 and padded with an
    # identity block (same solutions); rate counted on the unpadded flops
    groups = {}
    for i, n in enumerate(sizes):
        groups.setdefault((int(n) + 63) // 64 * 64, []).append(i)
    batches = []
    for npad, idx in sorted(groups.items()):
        Ab = torch.zeros((len(idx), npad, npad), dtype=torch.float64, device="cuda")
        bb = torch.zeros((len(idx), npad, 1), dtype=torch.float64, device="cuda")
        for t, i in enumerate(idx):
            n = int(sizes[i])
            Ab[t, :n, :n] = As[i].store[:, :n].t()
            if n < npad:
                Ab[t, n:, n:] = torch.eye(npad - n, dtype=torch.float64, device="cuda")
            bb[t, :n, 0] = b0[i]
        batches.append((Ab, bb))

    def native():
        for Ab, bb in batches:
            LU, piv = torch.linalg.lu_factor(Ab)
            torch.linalg.lu_solve(LU, piv, bb)

    native()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    native()
    e1.record()
    torch.cuda.synchronize()
    nms = e0.elapsed_time(e1)
    print(json.dumps({"metric": "batched uneven LU solves TFLOP/s (reduced-slice LU + FP64 refinement)",
                      "value": flops / (ms / 1e3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
                      "steps": args.steps, "warmup": args.warmup,
                      "config": {"workload": f"{count} systems, n log-uniform [64, 1024], r in {{0, 8}}",
                                 "total_lu_flops": flops},
                      "max_backward_error": float(be.max()), "mean_iterations": float(it.mean()),
                      "max_iterations": int(it.max()), "nonzero_info": int((info.cpu().numpy() != 0).sum()),
                      "native_fp64": {"value": flops / (nms / 1e3) / 1e12, "unit": "TFLOP/s", "ms": nms,
                                      "impl": "torch.linalg.lu_factor/lu_solve, batched per size rounded up to 64"},
                      "autotune_seconds": t_tune}), flush=True)


def main():
    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="lu",
                   choices=["lu", "lu_nopiv", "chol", "gemm", "gemm_sweep", "selector", "batched", "table2", "fig1"])
    p.add_argument("--range", type=float, default=0.0,
                   help="LU input u 10^e, e ~ U(-range, range) (0: uniform(-1,1))")
    p.add_argument("--cond", type=float, default=1e12, help="condition number of the Cholesky input")
    p.add_argument("--batch-count", type=int, default=4096)
    p.add_argument("--k", type=int, default=256)
    p.add_argument("--n", type=int, default=32768)
    p.add_argument("--nb", type=int, default=0,
                   help="block size (0: lu and chol tune it over {128, 256, 512} before the timed region; "
                        "1024 for lu_nopiv, 256 for the other workloads)")
    p.add_argument("--slices", type=int, default=7)
    p.add_argument("--cpu-n", type=int, default=4096,
                   help="size of the oracle's FP64 factorization sample (Cholesky: twice this)")
    p.add_argument("--cpu-emul-n", type=int, default=512,
                   help="size of the oracle's emulated LU sample (and of each --impl reference step)")
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--no-native", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    args = p.parse_args()
    args.nb_auto = args.nb == 0 and args.workload in ("lu", "chol")
    if args.nb == 0:
        args.nb = 1024 if args.workload == "lu_nopiv" else 256
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, world, rank)
        return
    if args.workload == "gemm":
        run_gemm(args)
        return
    if args.workload == "selector":
        run_selector(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "table2":
        run_table2(args)
        return
    if args.workload == "fig1":
        run_fig1(args)
        return
    if args.workload == "gemm_sweep":
        run_gemm_sweep(args)
        return
    world, rank, local = dist_setup()
    run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
