#!/usr/bin/env python3
"""Benchmark: batched FISTA at L1 = L2 = 256 through the C ABI.

Workload (one "step"): a batch of B independent snapshots, each drawn like the
single-snapshot 256 x 256 workload (32 x 32 half-wavelength array with N = 256
random elements, 8 off-grid sources with CN(0,1) amplitudes, 10 dB SNR, lam =
0.05 ||A^H y||_inf computed on the device), solved with T = 1000 FISTA
iterations: FP64 setup (Lambda, mu, b, lam), the fused FP32 iterations, and the
FP64 KKT / objective check, all in the library's kernels.

value = B * T * steps / time (instance-iterations per second, all ranks).
Under torchrun each rank solves its own B snapshots (weak scaling, no
collective on the data path).

``--impl reference`` times the FP64 dense oracle (the paper's "regular"
implementation) on the host cores on a bounded sample of the same workload.
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

METRIC = "batched FISTA iters/s at L1=L2=256; time to 1e-4 rel. error vs plain path"
UNIT = "instance-iterations/s"
WORKLOAD = dict(M1=32, M2=32, N=256, L1=256, L2=256, K=8, snr_db=10.0, lam_frac=0.05)
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128


def workload_name(B, T):
    return (f"batched FISTA: {B} snapshots/GPU, 32x32 half-wavelength array, N=256 random elements, "
            f"256x256 grid, 8 off-grid CN(0,1) sources, 10 dB, lam=0.05*||A^H y||_inf, {T} iterations")


def flops_per_inst_iter(L1, L2):
    """Algorithmic FP32 flops of one iteration on one L1 x L2 grid: a forward and an
    inverse 2D FFT at 5 L log2 L each, plus 18 L pointwise (real multiplier 2,
    + mu b 2, soft threshold 8, momentum 6)."""
    import math

    L = L1 * L2
    return 10.0 * L * math.log2(L) + 18.0 * L


def make_batch(B, first):
    import synth

    out = []
    for i in range(first, first + B):
        s = synth.make_snapshot(20000 + i, WORKLOAD["M1"], WORKLOAD["M2"], WORKLOAD["N"], WORKLOAD["L1"],
                                WORKLOAD["L2"], WORKLOAD["K"], WORKLOAD["snr_db"])
        out.append(s)
    return out


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples (one nvidia-smi row per 200 ms); BCCB_CLOCKS_DIR keeps them somewhere chosen
        out_dir = os.environ.get("BCCB_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons}


def gpu_index_for_smi(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


# ------------------------------------------------------------------------------------------
# CPU baseline: the FP64 dense oracle on a bounded sample
# ------------------------------------------------------------------------------------------


def cpu_oracle_sample(n_inst, iters, first=0):
    import oracle

    snaps = make_batch(n_inst, first)
    t0 = time.perf_counter()
    for s in snaps:
        A = oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2)
        lam = WORKLOAD["lam_frac"] * oracle.lambda_max(A, s.y)
        oracle.fista(A, s.y, lam, iters)
    dt = time.perf_counter() - t0
    return n_inst * iters / dt, dt


def cpu_fft_sample(n_inst, iters, first=0):
    """The paper's fast method (Section III-B) on the host cores, as timing context beside the
    dense oracle: FISTA on a batch of snapshots whose Gram products are IFFT2(Omega . FFT2(z))
    (eq:Rc) in FP64 with scipy.fft on every core; Omega is the FFT2 of the Gram's first column
    (eq:lambda), and A, b, lam come from the oracle (setup, not timed).  Returns instance-
    iterations per second of the iterations, the seconds they took and the last iterates
    (n_inst, L2, L1)."""
    import numpy as np
    import scipy.fft

    import oracle

    snaps = make_batch(n_inst, first)
    L1, L2 = WORKLOAD["L1"], WORKLOAD["L2"]
    omega = np.empty((n_inst, L2, L1))
    b = np.empty((n_inst, L2, L1), np.complex128)
    mu = np.empty((n_inst, 1, 1))
    kappa = np.empty((n_inst, 1, 1))
    for i, s in enumerate(snaps):
        A = oracle.dictionary(s.mask, s.M1, s.M2, L1, L2)
        omega[i] = scipy.fft.fft2(oracle.gram_first_column(A).reshape(L2, L1)).real
        b[i] = oracle.adjoint_measurements(A, s.y).reshape(L2, L1)
        mu[i] = 1.0 / omega[i].max()
        kappa[i] = mu[i] * WORKLOAD["lam_frac"] * np.abs(b[i]).max()
    beta = oracle.fista_momentum(iters)
    workers = os.cpu_count()
    c_prev = np.zeros_like(b)
    z = c_prev.copy()
    t0 = time.perf_counter()
    for t in range(iters):
        g = scipy.fft.ifft2(omega * scipy.fft.fft2(z, workers=workers), workers=workers)
        u = z - mu * g + mu * b
        mag = np.abs(u)
        c = u * (np.maximum(mag - kappa, 0.0) / np.where(mag > 0.0, mag, 1.0))
        z = c + beta[t] * (c - c_prev)
        c_prev = c
    dt = time.perf_counter() - t0
    return n_inst * iters / dt, dt, c_prev


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    n_inst, iters = 1, 300  # the dictionary's construction is amortised as in the GPU line's CPU baseline
    for _ in range(args.warmup):
        cpu_oracle_sample(n_inst, iters)
    t0 = time.perf_counter()
    for k in range(args.steps):
        cpu_oracle_sample(n_inst, iters, first=k)
    dt = time.perf_counter() - t0
    value = args.steps * n_inst * iters / dt
    sample = f"{n_inst} snapshot x {iters} FISTA iterations per step, dense FP64 oracle (setup included)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.batch, args.iters), "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------


# DRAM traffic of the fused kernel per instance, from one ncu capture of a small case of the
# variant named here (152 instances x 200 iterations of the 256x256 workload: dram__bytes_read.sum
# 177.97 MB + dram__bytes_write.sum 219.73 MB); the bytes do not grow with the iteration count past
# the dense first iterations, so they scale by instances
FUSED_TRAFFIC_VARIANT = (8192, 1)  # (tile, sparse_state)
FUSED_DRAM_BYTES_PER_INSTANCE = (177.968128e6 + 219.734784e6) / 152


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2509_13592_gb300 as bccb

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2509_13592_gb300 import shard

    B, T = args.batch, args.iters
    mine = shard.contiguous_range(B, rank)  # weak scaling: every rank solves its own B snapshots
    snaps = make_batch(B, mine.start)
    insts = [dict(M1=s.M1, M2=s.M2, L1=s.L1, L2=s.L2, mask=s.mask, y=s.y, lam=WORKLOAD["lam_frac"],
                  lam_is_frac=True) for s in snaps]
    stream = torch.cuda.Stream()  # graph capture needs a non-default stream
    solver = bccb.BatchSolver(insts, "fista", stream=stream)
    y_dev = torch.from_numpy(solver.y_host).cuda()
    c_dev = torch.empty(solver.total_c, dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()
    # untimed preparation: pick the fused kernel's tile per shape class, then capture
    # the whole solve (setup, T iterations, check) with its phase events in one graph
    bccb.bccb_batch_tune(solver.handle, y_dev, 20, args.tune_cache)
    tile, sparse_state = bccb.bccb_batch_variant(solver.handle, 256, 256)
    bccb.bccb_set_timing(solver.handle, True)
    bccb.bccb_batch_capture(solver.handle, y_dev, T, None, c_dev, None, True)

    def step():
        bccb.bccb_batch_replay(solver.handle)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    iterate_ms, setup_ms, check_ms, launches = [], [], [], 0
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_index_for_smi(local_rank)) as clocks:
        barrier()
        start.record(stream)
        for _ in range(args.steps):
            step()
            t = bccb.bccb_last_timing(solver.handle)  # waits for this step's events
            iterate_ms.append(t["iterate_ms"])
            setup_ms.append(t["setup_ms"])
            check_ms.append(t["check_ms"])
            launches += t["launches"]
        end.record(stream)
        barrier()
    elapsed = shard.max_over_ranks(start.elapsed_time(end) / 1e3, device="cuda")
    value = world * B * T * args.steps / elapsed
    clock = clocks.summary()

    # per-instance check of the last step
    torch.cuda.synchronize()
    res = solver.results()
    kkt_max = float(np.max(res["kkt"]))

    # ---- end to end through the host-buffer entry point (pinned host memory)
    y_pin = torch.from_numpy(solver.y_host).pin_memory()
    c_pin = torch.empty(solver.total_c, dtype=torch.complex64).pin_memory()
    bccb.bccb_set_timing(solver.handle, False)
    bccb.bccb_batch_solve_host_ptr(solver.handle, y_pin.data_ptr(), T, c_pin.data_ptr(), True)  # warm
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        bccb.bccb_batch_solve_host_ptr(solver.handle, y_pin.data_ptr(), T, c_pin.data_ptr(), True)
    barrier()
    e2e_elapsed = shard.max_over_ranks(time.perf_counter() - t0, device="cuda")
    e2e_value = world * B * T * args.steps / e2e_elapsed

    # ---- time to 1e-4: iterations until each sampled instance's iterate is within 1e-4 (relative
    # l2) of the plain path's T-iteration result.  The plain path is the single-instance entry point
    # (bccb_create + bccb_solve), run with the batch's tile; its result must equal the batched
    # solve's bit for bit.  FISTA's iterates do not depend on T, so a solve with t iterations gives
    # iterate t: a scan in steps of 10, then every iteration of the last window, finds each
    # instance's first t within 1e-4 (errors computed on the device).
    ttt = None
    if rank == 0 and not args.no_ttt:
        n_s = min(64, B)
        sub = insts[:n_s]
        gpu_name = torch.cuda.get_device_name(local_rank).replace(" ", "_")
        with tempfile.NamedTemporaryFile("w", suffix=".txt", delete=False) as f:
            f.write(f"{gpu_name} 256 256 0 {tile} {sparse_state}\n")
            cache = f.name
        batched = c_dev.view(-1)[: n_s * 65536].reshape(n_s, 65536).clone()
        refs, single_ms = [], []
        for i, d in enumerate(sub):
            h = bccb.bccb_create(d["M1"], d["M2"], d["mask"], d["L1"], d["L2"], bccb.FISTA, 1.0, stream)
            y1 = torch.from_numpy(np.asarray(d["y"], np.complex64)).cuda()
            c1 = torch.empty(65536, dtype=torch.complex64, device="cuda")
            bccb.bccb_batch_tune(h, y1, 1, cache)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            bccb.bccb_solve(h, y1, d["lam"], True, T, None, c1, check=False)  # warm-up
            e0.record(stream)
            bccb.bccb_solve(h, y1, d["lam"], True, T, None, c1, check=False)
            e1.record(stream)
            torch.cuda.synchronize()
            single_ms.append(e0.elapsed_time(e1))
            refs.append(c1)
            bccb.bccb_destroy(h)
        ref = torch.stack(refs)
        identical = bool(torch.equal(ref, batched))
        ref_norm = torch.linalg.vector_norm(ref, dim=1).clamp_min(1e-30)
        sub_solver = bccb.BatchSolver(sub, "fista", stream=stream)
        ys = torch.from_numpy(sub_solver.y_host).cuda()
        bccb.bccb_batch_tune(sub_solver.handle, ys, 1, cache)
        cur = torch.empty(n_s * 65536, dtype=torch.complex64, device="cuda")

        def errs(t):
            sub_solver.solve(ys, t, cur, check=False)
            torch.cuda.synchronize()  # the solve runs on `stream`, the norms on torch's current stream
            return (torch.linalg.vector_norm(cur.view(n_s, 65536) - ref, dim=1) / ref_norm).cpu().numpy()

        t_star = np.full(n_s, -1)
        prev = 0
        for t in list(range(10, T, 10)) + [T]:
            e = errs(t)
            hit = (e <= 1e-4) & (t_star < 0)
            if hit.any():
                for tt in range(prev + 1, t + 1):  # the first iteration within 1e-4 in (prev, t]
                    ee = e if tt == t else errs(tt)
                    new = hit & (ee <= 1e-4) & (t_star < 0)
                    t_star[new] = tt
            prev = t
            if (t_star > 0).all():
                break
        sub_solver.close()
        os.unlink(cache)
        per_iter_ms = statistics.median(iterate_ms) / T
        t_max = int(t_star.max())
        # batched: the whole batch's setup and t_max iterations, per instance; plain: each snapshot alone
        batched_ms = (statistics.median(setup_ms) + t_max * per_iter_ms) / B
        single_at_t = [ms * ts / T for ms, ts in zip(single_ms, t_star)]
        ttt = {"plain_path": "single-instance entry point (bccb_create + bccb_solve), same tile as the batch",
               "plain_equals_batched_bitwise": identical, "sampled_instances": n_s, "reference_iters": T,
               "t_star": {"min": int(t_star.min()), "median": float(np.median(t_star)), "max": t_max,
                          "resolution_iters": 1},
               "time_ms_full_batch": t_max * per_iter_ms,
               "batched_ms_per_instance": batched_ms,
               "single_instance_ms_at_t_star": float(statistics.median(single_at_t)),
               "single_instance_ms_T": float(statistics.median(single_ms)),
               "batched_speedup_vs_single": float(statistics.median(single_at_t)) / batched_ms,
               "note": f"the FP64 KKT residual after T = {T} iterations is up to {kkt_max:.2f}: FISTA is far from the "
                       f"LASSO minimiser on this workload, so its iterates still move near T and t* is close to T"}

    if rank == 0:
        peaks = load_peaks()
        props = torch.cuda.get_device_properties(local_rank)
        sm_count = props.multi_processor_count
        sm_max = peaks.get("sm_max_mhz", 2070.0)
        peak_tflops = sm_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        flops_launch = flops_per_inst_iter(256, 256) * B * T
        it_ms = statistics.mean(iterate_ms)
        achieved = flops_launch / (it_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": None,
                "kernel": f"fused_solve_kernel<256,256,FISTA,tile={tile}"
                          f"{',sparse state' if sparse_state else ''}> (one launch per step)",
                "peak_note": f"FP32: {sm_count} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {sm_max:.0f} MHz",
                "frac_at_median_clock": (achieved / (sm_count * FP32_LANES_PER_SM * 2 * clock["sm_mhz"] * 1e6 / 1e12)
                                         if clock.get("sm_mhz") else None)}
        # the derived FP32 peak confirmed on this GPU by a multiply-add microbenchmark (after the timed
        # region; scalar FFMA and the paired f32x2 form the solver's butterflies use)
        fma_rate = {"ffma": bccb.bccb_fp32_fma_rate(False), "ffma2": bccb.bccb_fp32_fma_rate(True)}
        roof["peak_measured_fma_tflops"] = fma_rate
        roof["frac_of_measured_fma"] = achieved / max(fma_rate.values())
        if args.traffic_bytes is not None:
            roof["traffic"] = args.traffic_bytes
        elif FUSED_TRAFFIC_VARIANT == (tile, sparse_state) and T > 0:
            # DRAM bytes per launch scaled by instances from an ncu capture of this kernel variant
            roof["traffic"] = FUSED_DRAM_BYTES_PER_INSTANCE * B
            roof["traffic_note"] = "ncu small-case capture of the same variant, scaled by instances"
        cpu = None
        if not args.no_cpu:
            n_cpu, it_cpu = 2, 300
            v, dt = cpu_oracle_sample(n_cpu, it_cpu, first=10**6)
            cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"{n_cpu} snapshots x {it_cpu} FISTA iterations of the same workload, dense FP64 "
                             f"oracle with setup ({dt:.1f} s)"}
            n_fft, it_fft = 8, 200
            v_fft, dt_fft, _ = cpu_fft_sample(n_fft, it_fft, first=10**6)
            cpu["fft_method"] = {"value": v_fft, "unit": UNIT, "cores": os.cpu_count(),
                                 "kind": "the paper's FFT method on the host (FP64, scipy.fft on every core)",
                                 "sample": f"{n_fft} snapshots x {it_fft} FISTA iterations of the same workload, "
                                           f"iterations only ({dt_fft:.1f} s)"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(B, T), "batch_per_gpu": B, "L1": 256, "L2": 256, "iters": T,
                       "tile": tile, "sparse_state": bool(sparse_state),
                       "launch": "CUDA graph of the whole solve, replayed per step",
                       "l2_policy": f"inputs larger than L2: {solver.total_c * 8 * 7 / 2**30:.1f} GiB resident per GPU",
                       "parallelism": f"instances sharded over {world} GPU(s)"},
            "phases_ms": {"setup": statistics.mean(setup_ms), "iterate": it_ms, "check": statistics.mean(check_ms)},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(solver.y_host.nbytes),
                    "d2h_bytes_per_step": int(solver.total_c * 8)},
            "gpu_launches": launches,
            "clocks": clock,
            "kkt_max": kkt_max,
            "time_to_1e-4": ttt,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------------------------
# secondary workloads (one JSON line each; the default run is the batched 256x256 metric)
# ------------------------------------------------------------------------------------------


def _solve_timed(bccb, torch, insts, algo, iters, rho=1.0, prec="f32", reps=3, check=False, method="fft"):
    stream = torch.cuda.Stream()
    solver = bccb.BatchSolver(insts, algo, rho, stream=stream, prec=prec)
    if method != "fft":
        solver.set_method(method)
    cdt = torch.complex128 if prec == "f64" else torch.complex64
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=cdt, device="cuda")
    aux = torch.zeros_like(c) if algo == "admm" else None
    torch.cuda.synchronize()
    if prec == "f32":
        bccb.bccb_batch_tune(solver.handle, y, 10, None)
    bccb.bccb_set_timing(solver.handle, True)
    solver.solve(y, iters, c, aux_out=aux, check=check)  # warm-up
    times = []
    for _ in range(reps):
        solver.solve(y, iters, c, aux_out=aux, check=check)
        times.append(bccb.bccb_last_timing(solver.handle))
    res = solver.results() if check else None
    torch.cuda.synchronize()
    out = (c.cpu().numpy(), None if aux is None else aux.cpu().numpy())
    solver.close()
    tot = [t["setup_ms"] + t["iterate_ms"] + t["check_ms"] for t in times]
    return out, {"ms": statistics.median(tot), "iterate_ms": statistics.median(t["iterate_ms"] for t in times),
                 "setup_ms": statistics.median(t["setup_ms"] for t in times)}, res


def run_workload(args):
    import numpy as np
    import torch

    import oracle
    import paper_2509_13592_gb300 as bccb
    import synth

    torch.cuda.set_device(0)
    if args.workload == "ragged":
        B, T = args.batch, args.iters
        snaps = synth.workload_batch("ragged", B)
        insts = [dict(M1=s.M1, M2=s.M2, L1=s.L1, L2=s.L2, mask=s.mask, y=s.y, lam=0.1, lam_is_frac=True)
                 for s in snaps]
        _, t, _ = _solve_timed(bccb, torch, insts, "fista", T, check=True)
        elems = sum(s.L1 * s.L2 for s in snaps)
        # A/B: the same instances, each (L1, L2) class solved on its own (its own solver and launch,
        # one after another), against the one call above whose class launches run concurrently
        classes = {}
        for d in insts:
            classes.setdefault((d["L1"], d["L2"]), []).append(d)
        solo = {}
        for key, group in sorted(classes.items()):
            _, tk, _ = _solve_timed(bccb, torch, group, "fista", T, check=False)
            solo[f"{key[0]}x{key[1]}"] = {"instances": len(group), "iterate_ms": tk["iterate_ms"]}
        seq_ms = sum(v["iterate_ms"] for v in solo.values())
        line = {"workload": f"ragged FISTA batch: {B} snapshots, L1,L2 uniform on {{64,128,256}}, M_i = L_i/4, "
                            f"25% occupancy, K in 1..10, SNR 0..30 dB, {T} iterations",
                "value": B * T / (t["ms"] / 1e3), "unit": "instance-iterations/s", "phases_ms": t,
                "grid_elements": elems, "flop_rate_tflops": sum(flops_per_inst_iter(s.L1, s.L2) for s in snaps)
                * T / (t["iterate_ms"] / 1e3) / 1e12,
                "ab_classes": {"concurrent_iterate_ms": t["iterate_ms"], "one_class_at_a_time_iterate_ms": seq_ms,
                               "per_class": solo}}
    elif args.workload == "precision1024":
        # the precision study at full length: FP32 and FP64 GPU paths, ADMM x 2000 at the stated rho = 0.5
        # and at rho = N = 1024, each result's error against the stored FP64 oracle reference
        sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
        import make_admm1024 as golden

        s = synth.workload_snapshot("admm1024", 0)
        s.y = s.y.astype(np.complex64).astype(np.complex128)  # the measurements the reference was given
        inst = [dict(M1=s.M1, M2=s.M2, L1=s.L1, L2=s.L2, mask=s.mask, y=s.y, lam=0.05, lam_is_frac=True)]
        T = golden.ITERS
        studies = []
        for tag in ("0p5", "1024"):
            ref = golden.read(tag)
            row = {"rho": ref["rho"], "norm_z": ref["norm_z"], "norm_c": ref["norm_c"], "norm_v": ref["norm_v"],
                   "oracle_nonzeros_z": int(ref["z_idx"].size)}
            for prec in ("f32", "f64"):
                (z, c), t, r = _solve_timed(bccb, torch, inst, "admm", T, rho=ref["rho"], prec=prec, reps=1,
                                            check=True)
                row[prec] = {"ms": t, "rel_err_vs_oracle": golden.errors(z.astype(np.complex128),
                                                                          c.astype(np.complex128), ref),
                             "nonzeros_z": int(np.count_nonzero(z)), "kkt": float(r["kkt"][0]),
                             "objective": float(r["objective"][0])}
            studies.append(row)
        # the FP64 oracle on the host cores (Kronecker-factored products: the dense A would be 16 GiB),
        # timed at 20 and 60 iterations and extrapolated to the study's length
        K = oracle.KronDictionary(s.mask, s.M1, s.M2, s.L1, s.L2)
        lam_o = 0.05 * float(np.abs(K.adjoint(s.y)).max())
        t_cpu = {}
        for n_it in (5, 20, 60):  # the first call warms the BLAS threads and caches
            t0 = time.perf_counter()
            oracle.admm_kron(K, s.y, lam_o, 1024.0, n_it)
            t_cpu[n_it] = time.perf_counter() - t0
        per_it = (t_cpu[60] - t_cpu[20]) / 40
        cpu_oracle = {"kind": "oracle.admm_kron (FP64, products through the Kronecker factors of D)",
                      "cores": os.cpu_count(), "s_per_iteration": per_it,
                      "s_setup": max(t_cpu[20] - 20 * per_it, 0.0),
                      "extrapolated_s_for_study": max(t_cpu[20] - 20 * per_it, 0.0) + T * per_it,
                      "sample": "20 and 60 iterations timed after a warm-up call, extrapolated linearly to the study's length"}
        line = {"workload": f"1024x1024 grid, 64x64 array N=1024, 20 off-grid sources, 15 dB, lam=0.05||A^H y||_inf, "
                            f"ADMM {T} iterations, single snapshot; rho = 0.5 (stated) and rho = N",
                "reference": "FP64 oracle (tests/golden/admm1024_rho*.txt): z^(T) in full, c^(T) on 1024 sampled "
                             "entries and in norm",
                "studies": studies, "cpu_oracle": cpu_oracle}
    elif args.workload == "learned":
        # unrolled FISTA, 16 layers with learned per-layer step and threshold multipliers (fixed 32x32
        # array, N = 256, 256x256 grid), judged against 1000-iteration plain FISTA
        from paper_2509_13592_gb300 import learned as Lm

        cfg = Lm.TrainConfig()
        path = args.params or os.path.join(ROOT, "paper_2509_13592_gb300", "unrolled_fista16_256.json")
        if os.path.exists(path):
            with open(path) as f:
                p = json.load(f)
            scale = torch.tensor(p["scale"], dtype=torch.float32, device="cuda")
            thresh = torch.tensor(p["thresh"], dtype=torch.float32, device="cuda")
            trained = {"file": os.path.relpath(path, ROOT), "snapshots": p["train_snapshots"]}
        else:  # no stored multipliers: a short training run here
            cfg.steps = 100
            scale, thresh, hist = Lm.train(cfg, log=None)
            trained = {"file": None, "snapshots": cfg.steps * cfg.batch, "loss_last": hist[-1]}
        n_eval, T = 8192, cfg.target_iters
        mask = Lm.fixed_mask(cfg)
        y = Lm.snapshot_batch(cfg, mask, 10**7, n_eval)
        L = cfg.L1 * cfg.L2
        one = dict(M1=cfg.M1, M2=cfg.M2, L1=cfg.L1, L2=cfg.L2, mask=mask, y=np.zeros(cfg.N, np.complex64),
                   lam=cfg.lam_frac, lam_is_frac=True)
        stream = torch.cuda.Stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def timed(fn):
            torch.cuda.synchronize()
            ev0.record()
            out = fn()
            ev1.record()
            torch.cuda.synchronize()
            return out, ev0.elapsed_time(ev1)

        solver = bccb.BatchSolver([one] * n_eval, "fista")
        bccb.bccb_batch_tune(solver.handle, y, 5, None)
        ref = torch.empty(n_eval * L, dtype=torch.complex64, device="cuda")
        solver.solve(y, 10, ref, check=False)  # warm-up

        def plain(iters, yy=y, s=solver, n=n_eval, c0=None):
            o = torch.empty(n * L, dtype=torch.complex64, device="cuda")
            s.solve(yy, iters, o, c0=c0, check=False)
            torch.cuda.synchronize()
            return o

        ref, t_ref = timed(lambda: plain(T))
        net = Lm.UnrolledNet(cfg.M1, cfg.M2, mask, cfg.L1, cfg.L2, n_eval, cfg.lam_frac)
        with torch.no_grad():
            Lm.net_forward(net, y, scale, thresh)  # warm-up
            c_net, t_net = timed(lambda: Lm.net_forward(net, y, scale, thresh))
        e_net = Lm.relative_errors(c_net, ref, n_eval, L)
        sweep = {}
        for it in (16, 32, 48, 64, 128, 256):
            o, t = timed(lambda: plain(it))
            e = Lm.relative_errors(o, ref, n_eval, L)
            sweep[it] = {"ms": t, "rel_err_mean": e.mean().item()}
        net.close()
        # time to 1e-4 of the target on a 64-snapshot sample: plain FISTA from zero, and the network
        # followed by plain FISTA warm-started from its output (momentum restarted), the fallback path
        n_s = 64
        ys = y[: n_s * cfg.N].contiguous()
        refs = ref[: n_s * L].view(n_s, L)
        rn = torch.linalg.vector_norm(refs, dim=1)
        sub = bccb.BatchSolver([one] * n_s, "fista")

        def worst(o):
            return float((torch.linalg.vector_norm(o.view(n_s, L) - refs, dim=1) / rn).max())

        t_plain = next((t for t in range(10, T + 1, 10) if worst(plain(t, ys, sub, n_s)) <= 1e-4), None)
        if t_plain is not None:
            t_plain = next(t for t in range(t_plain - 9, t_plain + 1) if worst(plain(t, ys, sub, n_s)) <= 1e-4)
        c_sub = c_net[: n_s * L].contiguous()
        fb = {k: worst(plain(k, ys, sub, n_s, c0=c_sub)) for k in (1, 10, 100, 250, 500, 1000, 2000)}
        k_hit = next((k for k, w in fb.items() if w <= 1e-4), None)
        sub.close()
        per_it = t_ref / T / n_eval
        # plain single-instance FISTA (bccb_create + bccb_solve), T iterations, first 8 snapshots
        single = []
        for i in range(8):
            h = bccb.bccb_create(cfg.M1, cfg.M2, mask, cfg.L1, cfg.L2, bccb.FISTA, 1.0, stream)
            y1 = y[i * cfg.N:(i + 1) * cfg.N].contiguous()
            c1 = torch.empty(L, dtype=torch.complex64, device="cuda")
            bccb.bccb_solve(h, y1, cfg.lam_frac, True, T, None, c1, check=False)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bccb.bccb_solve(h, y1, cfg.lam_frac, True, T, None, c1, check=False)
            e1.record(stream)
            torch.cuda.synchronize()
            single.append(e0.elapsed_time(e1))
            bccb.bccb_destroy(h)
        solver.close()
        line = {"workload": f"unrolled FISTA: 16 layers with learned per-layer step and threshold multipliers, fixed "
                            f"32x32 array N=256, 256x256 grid, K in 1..8 off-grid, SNR 0..30 dB, lam=0.05||A^H y||_inf; "
                            f"inference on {n_eval} snapshots; judge: {T}-iteration plain FISTA",
                "trained": trained,
                "target_batched_ms": t_ref, "net_ms": t_net,
                "net_rel_err_mean": e_net.mean().item(), "net_rel_err_median": e_net.median().item(),
                "plain_batched": sweep,
                "time_to_1e-4_of_target": {
                    "sample": n_s, "plain_batched_iters": t_plain,
                    "plain_batched_ms_per_instance": None if t_plain is None else t_plain * per_it,
                    "plain_single_instance_ms": statistics.median(single) * (t_plain or T) / T,
                    "net_then_fallback_worst_rel_err_after_k_iters": fb, "net_then_fallback_iters": k_hit,
                    "net_then_fallback_ms_per_instance": None if k_hit is None else t_net / n_eval + k_hit * per_it}}
    elif args.workload == "peaks":
        # harmonic / angle extraction (Section II-A) on the solutions of the batched 256x256 workload
        B, T, K = args.batch, args.iters, 16
        snaps = make_batch(B, 0)
        insts = [dict(M1=s.M1, M2=s.M2, L1=s.L1, L2=s.L2, mask=s.mask, y=s.y, lam=WORKLOAD["lam_frac"],
                      lam_is_frac=True) for s in snaps]
        stream = torch.cuda.Stream()
        solver = bccb.BatchSolver(insts, "fista", stream=stream)
        y = torch.from_numpy(solver.y_host).cuda()
        c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
        solver.solve(y, T, c, check=False)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            out = solver.peaks(c, K, 0.05)  # warm-up
            ev0.record(stream)
            for _ in range(5):
                out = solver.peaks(c, K, 0.05)
            ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / 5
        cnt = out["count"].cpu().numpy()
        c_host = c[: 16 * 65536].cpu().numpy()
        t0 = time.perf_counter()
        for i in range(16):
            oracle.peaks.peaks(c_host[i * 65536:(i + 1) * 65536].reshape(256, 256), K, 0.05)
        cpu_s = (time.perf_counter() - t0) / 16
        solver.close()
        line = {"workload": f"peak extraction and harmonic-to-angle map, K={K}, rel_thresh=0.05, on the {T}-iteration "
                            f"FISTA solutions of {B} 256x256 snapshots", "value": B / (ms / 1e3),
                "unit": "instances/s", "ms_per_batch": ms, "peaks_per_instance_median": float(np.median(cnt)),
                "bytes_read_per_instance_pass": 65536 * 8,
                "cpu_oracle": {"ms_per_instance": cpu_s * 1e3, "cores": 1, "sample": "16 instances"}}
    elif args.workload == "torchfft":
        # Context only, outside the library: the same FISTA iteration written with torch.fft (cuFFT) on
        # the same FP32 setup (q, Bt, mu, lam taken from the library's solver), against the fused solver
        B, T = args.batch, args.iters
        snaps = [synth.make_snapshot(20000 + i, 32, 32, 256, 256, 256, 8, 10.0) for i in range(B)]
        insts = [dict(M1=q.M1, M2=q.M2, L1=q.L1, L2=q.L2, mask=q.mask, y=q.y, lam=0.05, lam_is_frac=True) for q in snaps]
        (c_fused, _), t_fused, res = _solve_timed(bccb, torch, insts, "fista", T, reps=3, check=True)
        solver = bccb.BatchSolver(insts, "fista")
        y = torch.from_numpy(solver.y_host).cuda()
        c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
        solver.solve(y, 1, c, check=False)
        q = torch.empty(solver.total_c, dtype=torch.float32, device="cuda")
        bt = torch.empty(solver.total_c, dtype=torch.complex64, device="cuda")
        solver.get(2, q)
        solver.get(3, bt)
        r1 = solver.results()
        solver.close()
        kappa = torch.tensor(np.asarray(r1["mu"]) * np.asarray(r1["lam"]), dtype=torch.float32, device="cuda").view(B, 1, 1)
        q, bt = q.view(B, 256, 256), bt.view(B, 256, 256)
        tk, beta = 1.0, []
        for _ in range(T):
            tn = (1.0 + (1.0 + 4.0 * tk * tk) ** 0.5) / 2.0
            beta.append((tk - 1.0) / tn)
            tk = tn

        def torch_fista():
            z = torch.zeros(B, 256, 256, dtype=torch.complex64, device="cuda")
            c_prev = torch.zeros_like(z)
            for t in range(T):
                g = torch.fft.ifft2(q * torch.fft.fft2(z) - bt, norm="forward")  # unnormalised inverse
                u = z - g
                mag = u.abs()
                cn = u * torch.clamp(1.0 - kappa / torch.clamp(mag, min=1e-30), min=0.0)
                z = cn + beta[t] * (cn - c_prev)
                c_prev = cn
            return c_prev

        torch_fista()  # warm-up (cuFFT plans)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(3):
            e0.record()
            c_t = torch_fista()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        t_torch = statistics.median(ts)
        ct = c_t.reshape(-1).cpu().numpy().astype(np.complex128)
        cf = c_fused.astype(np.complex128)
        line = {"workload": f"context only, not the library: FISTA x {T} on {B} snapshots of the 256x256 workload written "
                            f"with torch.fft (cuFFT), FP32, on the library's q, Bt, mu and lam",
                "value": B * T / (t_torch / 1e3), "unit": UNIT, "ms": t_torch,
                "fused_value": B * T / (t_fused["iterate_ms"] / 1e3), "fused_iterate_ms": t_fused["iterate_ms"],
                "fused_over_torch": t_torch / t_fused["iterate_ms"],
                "rel_diff_vs_fused": float(np.linalg.norm(ct - cf) / np.linalg.norm(cf))}
    elif args.workload == "toeplitz":
        # element spacing 0.4 wavelength (gamma != 1/2): Toeplitz Gram, 2L1 x 2L2 circulant embedding
        B, T, g = min(args.batch, 1024), args.iters, (0.4, 0.4)
        snaps = [synth.make_snapshot(60000 + i, 32, 32, 256, 128, 128, 8, 10.0, gamma=g) for i in range(B)]
        insts = [dict(M1=s.M1, M2=s.M2, L1=s.L1, L2=s.L2, mask=s.mask, y=s.y, lam=0.05, lam_is_frac=True)
                 for s in snaps]
        stream = torch.cuda.Stream()
        solver = bccb.BatchSolver(insts, "fista", stream=stream, gamma=g)
        y = torch.from_numpy(solver.y_host).cuda()
        c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
        torch.cuda.synchronize()
        bccb.bccb_set_timing(solver.handle, True)
        solver.solve(y, 1, c, check=False)  # first solve: includes the mask-only setup (spectrum, mu)
        first_setup = bccb.bccb_last_timing(solver.handle)["setup_ms"]
        bccb.bccb_batch_tune(solver.handle, y, 10, None)
        bccb.bccb_set_timing(solver.handle, True)
        solver.solve(y, T, c, check=True)  # warm-up
        times = []
        for _ in range(3):
            solver.solve(y, T, c, check=True)
            times.append(bccb.bccb_last_timing(solver.handle))
        res = solver.results()
        it_ms = statistics.median(t["iterate_ms"] for t in times)
        su_ms = statistics.median(t["setup_ms"] for t in times)
        # oracle on a bounded sample: the dense FP64 solve of two snapshots, 100 iterations
        t0 = time.perf_counter()
        for s in snaps[:2]:
            A = oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2, *g)
            oracle.fista(A, s.y, 0.05 * oracle.lambda_max(A, s.y), 100)
        cpu = 2 * 100 / (time.perf_counter() - t0)
        solver.close()
        line = {"workload": f"gamma = 0.4 array (Toeplitz Gram): {B} snapshots, 32x32 array, N=256, 128x128 grid "
                            f"(256x256 circulant embedding), 8 off-grid sources, 10 dB, lam=0.05||A^H y||_inf, "
                            f"FISTA {T} iterations", "value": B * T / (it_ms / 1e3), "unit": "instance-iterations/s",
                "phases_ms": {"setup": su_ms, "iterate": it_ms},
                "setup_first_solve_ms": first_setup,
                "setup_note": "the mask-only setup (embedding spectrum and mu) runs on a solver's first solve only",
                "kkt_max": float(np.max(res["kkt"])),
                "cpu_oracle": {"value": cpu, "unit": "instance-iterations/s", "cores": os.cpu_count(),
                               "sample": "2 snapshots x 100 FISTA iterations, dense FP64 oracle incl. setup"}}
    elif args.workload == "single64":
        s = synth.workload_snapshot("fista64", 0)
        inst = [dict(M1=s.M1, M2=s.M2, L1=s.L1, L2=s.L2, mask=s.mask, y=s.y, lam=0.1, lam_is_frac=True)]
        _, t, _ = _solve_timed(bccb, torch, inst, "fista", 500, reps=5, check=True)
        per_it_s = t["iterate_ms"] / 500 / 1e3
        achieved = flops_per_inst_iter(64, 64) / per_it_s / 1e12
        props = torch.cuda.get_device_properties(0)
        sm_max = load_peaks().get("sm_max_mhz", 2070.0)
        sm_peak = FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        line = {"workload": "single snapshot: 16x16 array, N=64, 64x64 grid, 3 on-grid sources, 20 dB, FISTA 500 "
                            "iterations, lam=0.1||A^H y||_inf", "latency_ms": t,
                "per_iteration_us": 1e6 * per_it_s,
                # one CTA on one SM: the fraction of that SM's FP32 peak and of the chip's
                "roofline": {"bound": "alu", "achieved": achieved, "unit": "TFLOP/s", "peak_one_sm": sm_peak,
                             "frac_one_sm": achieved / sm_peak,
                             "frac_chip": achieved / (sm_peak * props.multi_processor_count)}}
    elif args.workload == "table1":
        rows = []
        for algo in ("ista", "fista", "admm"):
            for L1 in (64, 128, 256, 512):
                for it in (50, 100, 200, 400):
                    errs, errs32, t_reg, t_gpu, t_dense, t_fast_it, eps_dense, dense_gbs = ([] for _ in range(8))
                    for trial in range(args.trials):
                        s = synth.paper_experiment_snapshot(trial, L1)
                        A = oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2)
                        lam = 0.1 * oracle.lambda_max(A, s.y)
                        t0 = time.perf_counter()
                        if algo == "ista":
                            ref = oracle.ista(A, s.y, lam, it)
                        elif algo == "fista":
                            ref = oracle.fista(A, s.y, lam, it)
                        else:
                            ref = oracle.admm(A, s.y, lam, float(s.N), it)[0]
                        t_reg.append(1e3 * (time.perf_counter() - t0))
                        inst = [dict(M1=s.M1, M2=s.M2, L1=s.L1, L2=s.L2, mask=s.mask, y=s.y, lam=lam)]
                        (c64, _), t64, _ = _solve_timed(bccb, torch, inst, algo, it, rho=float(s.N), prec="f64",
                                                        reps=1)
                        (c32, _), t32, _ = _solve_timed(bccb, torch, inst, algo, it, rho=float(s.N), reps=1)
                        (cd, _), td, _ = _solve_timed(bccb, torch, inst, algo, it, rho=float(s.N), reps=1,
                                                      method="dense")
                        nr = np.linalg.norm(ref)
                        errs.append(float(np.linalg.norm(c64 - ref) / nr) if nr else 0.0)
                        errs32.append(float(np.linalg.norm(c32 - ref) / nr) if nr else 0.0)
                        nd = np.linalg.norm(cd)
                        eps_dense.append(float(np.linalg.norm(cd - c32) / nd) if nd else 0.0)
                        t_gpu.append(t32["ms"])
                        t_fast_it.append(t32["iterate_ms"])
                        t_dense.append(td["iterate_ms"])
                        L = L1 * 32
                        dense_gbs.append(8.0 * L * L * it / (td["iterate_ms"] / 1e3) / 1e9)
                    rows.append({"algo": algo, "L1": L1, "n_iter": it, "eps_r_fp64_gpu": float(np.mean(errs)),
                                 "eps_r_fp32_gpu": float(np.mean(errs32)), "t_reg_cpu_ms": float(np.mean(t_reg)),
                                 "t_fast_gpu_ms": float(np.mean(t_gpu)),
                                 "t_reg_gpu_iter_ms": float(np.mean(t_dense)),
                                 "t_fast_gpu_iter_ms": float(np.mean(t_fast_it)),
                                 "t_reg_over_t_fast_gpu": float(np.mean(t_dense) / np.mean(t_fast_it)),
                                 "eps_r_reg_vs_fast_fp32_gpu": float(np.mean(eps_dense)),
                                 "dense_gram_gbs": float(np.mean(dense_gbs))})
        line = {"workload": f"paper experiment shape: M1=51, M2=16, N=40, L2=32, 15 dB, K in 1..10, "
                            f"{args.trials} trials; ADMM rho = N", "rows": rows, "cpu_cores": os.cpu_count()}
    else:
        raise SystemExit(f"unknown workload {args.workload}")
    line["impl"] = "ours"
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=4096, help="snapshots per GPU")
    ap.add_argument("--iters", type=int, default=1000)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-1e-4 measurement")
    ap.add_argument("--tune-cache", default=None, help="autotuner cache file (default: measure every run)")
    ap.add_argument("--workload", default="batched256",
                    choices=["batched256", "ragged", "precision1024", "single64", "table1", "peaks", "toeplitz",
                             "learned", "torchfft"],
                    help="batched256 is the benchmark metric; the others print their own line")
    ap.add_argument("--trials", type=int, default=3, help="trials per Table I cell (--workload table1)")
    ap.add_argument("--params", default=None, help="trained multipliers of the unrolled network (--workload learned)")
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="DRAM bytes per launch of the fused kernel from an ncu capture")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload != "batched256":
        return run_workload(args)
    return run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
