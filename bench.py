"""Benchmark of the Chebyshev-Hutchinson log-determinant on one GB300.

One step = one whole estimate: spectral interval (Gershgorin pass on the
device, or the workload's known interval), probe signs, n fused recurrence
steps, moment reduction, coefficients and final sum, read back to the host.

Default workload (config 2): sparse random SPD, d = 1e7, 5 picks per row
(about 1.1e8 stored entries), FP32 values, FP32 recurrence vectors, n = 100,
M = 32 probes, probe seed 0.  The metric is the algorithmic HBM bandwidth of
the estimate: n x B_gather / time, with per degree step
    B_gather = nnz (s_v + 4) + 8 (d + 1) + nnz_off * M * 4 + 3 d M 4
(each off-diagonal entry gathers one M-wide FP32 row of w_j; w_j, w_{j-1} are
read and w_{j+1} written once).  Inputs are larger than L2 (one recurrence
vector block is 1.28 GB), so no flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU FP64 oracle
on a bounded probe sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "logdet time & HBM GB/s (% of peak) at stated rel. error; adjoint/forward ratio"


def algorithmic_bytes_per_step(B, M, s_v):
    nnz = B.nnz
    rows = np.repeat(np.arange(B.d), np.diff(B.rowptr))
    nnz_off = int(np.count_nonzero(B.col != rows))
    b_gather = nnz * (s_v + 4) + 8 * (B.d + 1) + nnz_off * M * 4 + 3 * B.d * M * 4
    b_min = nnz * (s_v + 4) + 8 * (B.d + 1) + 3 * B.d * M * 4
    return b_gather, b_min, nnz_off


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            j = json.load(open(p))
            return float(j["hbm_gbs"]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running.
    The raw samples go to a CSV in $CLD_CLOCKS_DIR (default: the temp dir);
    the JSON line carries their summary."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0, name="clocks_bench.csv"):
        self.proc = None
        self.f = None
        self.failure = None
        import tempfile

        self.path = os.path.join(os.environ.get("CLD_CLOCKS_DIR") or tempfile.gettempdir(), name)
        self.gpu_index = gpu_index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
        except OSError as e:
            self.failure = "clock log not writable: %s" % e
            return self
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError as e:
            self.proc = None
            self.failure = "nvidia-smi unavailable: %s" % e
            self.f.close()
            self.f = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.f is not None:
            self.f.close()
            self.f = None

    def summary(self):
        if self.failure is not None or self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [self.failure or "nvidia-smi unavailable"]}
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            try:
                pw.append(float(parts[3]))
            except ValueError:
                pass
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "sm_min_mhz": float(min(sm)),
                "power_w": float(np.median(pw)) if pw else None, "samples": len(sm), "reasons": sorted(reasons)}


def build_workload(cfg_id, d_override=None):
    cfg = dict(workloads.CONFIGS[cfg_id])
    if d_override:
        if cfg["kind"] == "grid_gmrf":
            cfg["N"] = int(round(d_override ** 0.5))
        else:
            cfg["d"] = int(d_override)
    t0 = time.time()
    B = workloads.make(cfg)
    gen_s = time.time() - t0
    if cfg["kind"] == "grid_gmrf":
        interval = (cfg["kappa2"], cfg["kappa2"] + 8.0)
        desc = "grid_gmrf N=%d (d=%d) kappa2=%g" % (cfg["N"], B.d, cfg["kappa2"])
    else:
        interval = None
        desc = "sparse_random_spd d=%d picks=%d seed=%d" % (B.d, cfg["picks"], cfg["seed"])
    return cfg, B, interval, desc, gen_s


def cpu_sample(B, v64, a, b, n, M, budget_s=20.0):
    """Times the oracle on probe 0 with as many degree steps as fit a budget.
    Returns (seconds, steps, probes, moments of probe 0 or None, threads)."""
    import oracle

    V = oracle.rademacher(0, B.d, [0])
    t0 = time.time()
    oracle.moments(B.rowptr, B.col, v64, a, b, 2, V)
    t2 = time.time() - t0
    per_step = max(t2 / 2.0, 1e-6)
    steps = int(max(1, min(n, budget_s / per_step)))
    t0 = time.time()
    t = oracle.moments(B.rowptr, B.col, v64, a, b, steps, V)
    dt = time.time() - t0
    return dt, steps, 1, (t if steps == n else None), oracle.num_threads()


def run_reference(args, rank, world):
    import oracle

    oracle.build()
    if rank != 0:
        return
    cfg, B, interval, desc, _ = build_workload(args.config, args.d)
    stored, v64 = B.stored(args.dtype)
    s_v = {"f32": 4, "bf16": 2, "f64": 8}[args.dtype]
    a, b = interval if interval is not None else oracle.gershgorin(B.rowptr, B.col, v64)
    n, M = cfg["n"], cfg["M"]
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_sample(B, v64, a, b, n, M, budget_s=min(budget, 5.0))
    times, steps_done = [], 0
    for _ in range(args.steps):
        dt, steps, probes, _, threads = cpu_sample(B, v64, a, b, n, M, budget_s=budget)
        times.append(dt)
        steps_done = steps
    bg, bmin, nnz_off = algorithmic_bytes_per_step(B, 1, s_v)
    t = float(np.mean(times))
    value = steps_done * bg / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "n": n, "M": M, "nnz": B.nnz},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle",
                             "sample": "probe 0 of %d, %d of %d degree steps, full d=%d" % (M, steps_done, n, B.d)},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x: float, world: int, device: str = "cpu") -> float:
    """The slowest rank's time (all ranks take part; identity for one rank)."""
    if world <= 1:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def time_estimates(m, n, M, seed, interval, steps, warmup, torch, world):
    """Warm-up, then `steps` timed estimates (interval + estimate each) with CUDA
    events on the launching stream.  Returns (ms per step, kernel ms per general
    step launch, general launches, total launches, last result)."""

    def step():
        if interval is None:
            m.auto_interval(0)
        else:
            m.set_interval(*interval)
        return m.estimate(n, M, seed)

    for _ in range(warmup):
        step()
    m.set_profiling(True)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms, step_launches, total_launches, r = 0.0, 0, 0, None
    for i in range(steps):
        ev[i][0].record(stream)
        r = step()
        ev[i][1].record(stream)
        ms, sl, tl = m.last_timing()
        step_ms += ms
        step_launches += sl
        total_launches += tl + (2 if interval is None else 1)  # + interval kernels
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_ms = max_over_ranks(float(sum(ev[i][0].elapsed_time(ev[i][1]) for i in range(steps))), world, "cuda")
    m.set_profiling(False)
    return total_ms / steps, step_ms / max(1, step_launches), step_launches, total_launches, r


def run_only(args):
    """One leg alone (profiling captures on smaller cases): prints its JSON."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    leg = {"dense": dense_leg, "adjoint": adjoint_leg, "paper": paper_leg, "latency": latency_leg,
           "gmrf": gmrf_leg, "config1": config1_leg, "batch": batch_leg}[args.only]
    out = leg(args, torch, 1) if args.only == "adjoint" else leg(args, torch)
    key = {"config1": "gmrf_config1"}.get(args.only, args.only)
    if not args.no_cpu_baseline and key in ("latency", "gmrf_config1", "paper", "gmrf", "dense"):
        reference_errors({key: out})
    print(json.dumps({"only": args.only, **out}), flush=True)


def run_ours(args, rank, world):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1503_06394_gb300 import CsrLogdet, logdet_host
    from paper_1503_06394_gb300 import _binding as Bd

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    cfg, B, interval, desc, gen_s = build_workload(args.config, args.d)
    stored, v64 = B.stored(args.dtype)
    s_v = {"f32": 4, "bf16": 2, "f64": 8}[args.dtype]
    n, M = cfg["n"], cfg["M"]
    seed = cfg["probe_seed"] + rank  # independent replicas on independent probe streams
    m = CsrLogdet(B.rowptr, B.col, stored, dtype=args.dtype)
    if interval is None:
        m.auto_interval(0)
    else:
        m.set_interval(*interval)
    if args.variant is None:
        variant, _ = m.autotune(n, M)
    else:
        variant = args.variant
        m.set_kernel_variant(variant)
    m.reserve(n, M)
    bg, bmin, nnz_off = algorithmic_bytes_per_step(B, M, s_v)
    # the grid stencil's neighbour rows are L2 hits (its roofline is B_min);
    # uniformly random columns miss L2 (B_gather)
    model = "B_min" if args.config == 1 else "B_gather"
    bstep = bmin if args.config == 1 else bg
    peak, peak_src = read_peaks()
    with ClockSampler(local) as clk:
        ms_per_step, kernel_avg_ms, step_launches, total_launches, r_last = time_estimates(
            m, n, M, seed, interval, args.steps, args.warmup, torch, world)
    value = world * n * bstep / (ms_per_step / 1e3) / 1e9
    achieved = bstep / (kernel_avg_ms / 1e3) / 1e9
    panel, lpr, ctas, threads = m.launch_config(M)
    a_e, b_e = (interval if interval is not None else Bd.cld_auto_interval(m.h, 0))
    rr = m.estimate(n, M, cfg["probe_seed"], details=True)
    gp0_ours = float(rr["gamma_p"][0])
    m.close()
    del m
    torch.cuda.empty_cache()

    # end to end through the host-buffer entry point (pinned host arrays), right
    # after the device-timed region and under the same conditions
    rp = torch.from_numpy(B.rowptr).pin_memory()
    cl = torch.from_numpy(B.col).pin_memory()
    vv = torch.from_numpy(stored.view(np.int16) if args.dtype == "bf16" else stored).pin_memory()
    need = Bd.cld_host_workspace_size(B.d, B.nnz, {"f32": 0, "bf16": 1, "f64": 2}[args.dtype], n, M)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    logdet_host(rp, cl, vv, a_e, b_e, n, M, seed, dtype=args.dtype, workspace=ws)
    torch.cuda.synchronize()
    e2e_t = []
    with ClockSampler(local, "clocks_e2e.csv") as clk_e2e:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            logdet_host(rp, cl, vv, a_e, b_e, n, M, seed, dtype=args.dtype, workspace=ws)
            e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.mean(e2e_t))
    h2d = (B.d + 1) * 8 + B.nnz * 4 + B.nnz * s_v
    del ws
    torch.cuda.empty_cache()

    # BF16-stored values on the same GPU (FP32 recurrence vectors)
    bf16 = None
    if args.dtype == "f32" and not args.no_bf16:
        st16, v16 = B.stored("bf16")
        m16 = CsrLogdet(B.rowptr, B.col, st16, dtype="bf16")
        iv16 = interval
        if iv16 is None:
            iv16 = m16.auto_interval(0)
        v16, _ = m16.autotune(n, M)
        bg16, bmin16, _ = algorithmic_bytes_per_step(B, M, 2)
        bg16 = bmin16 if args.config == 1 else bg16
        ms16, k16, _, _, _ = time_estimates(m16, n, M, seed, interval, args.steps, max(1, args.warmup - 1), torch, world)
        m16.set_interval(*iv16)
        r16 = m16.estimate(n, M, cfg["probe_seed"], details=True)
        bf16 = {"value": world * n * bg16 / (ms16 / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": ms16, "variant": v16,
                "kernel_ms": k16, "logdet": r16["logdet"], "gamma_p0": float(r16["gamma_p"][0]),
                "vs_fp32_time": ms16 / ms_per_step}
        m16.close()
        del m16
        torch.cuda.empty_cache()

    adjoint = None
    if not args.no_adjoint and args.d is None:
        adjoint = adjoint_leg(args, torch, world)
    batched = None
    if not args.no_batch and args.d is None:
        batched = batch_leg(args, torch)
    dense = None
    if not args.no_dense and args.d is None:
        dense = dense_leg(args, torch)
    latency = None
    if not args.no_latency and args.d is None:
        latency = latency_leg(args, torch)
    config1 = None
    if not args.no_config1 and args.d is None:
        config1 = config1_leg(args, torch)
    paper = None
    if not args.no_paper and args.d is None:
        paper = paper_leg(args, torch)
    gmrf = None
    if not args.no_gmrf and args.d is None:
        gmrf = gmrf_leg(args, torch)

    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": desc, "n": n, "M": M, "nnz": B.nnz, "nnz_off": nnz_off,
                       "value_dtype": args.dtype, "vector_dtype": "f32",
                       "l2": "inputs larger than L2 (recurrence block %.2f GB)" % (B.d * panel * 4 / 1e9)
                       if B.d * panel * 4 > 2e8 else "L2-resident workload (no flush)",
                       "interval": "gershgorin on device each step" if interval is None else "closed form %s" % (interval,),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "launch": {"panel": panel, "lanes_per_row": lpr, "ctas": ctas, "threads": threads,
                                  "variant": variant}},
            "logdet": r_last["logdet"], "stderr": r_last["stderr"],
            "logdet_s": ms_per_step / 1e3, "pct_of_peak": 100.0 * value / world / peak,
            "bytes_model": model, "b_gather_per_step": bg, "b_min_per_step": bmin,
            "effective_gbs_bmin": world * n * bmin / (ms_per_step / 1e3) / 1e9,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": profiled_traffic(args, B, variant),
                         "kernel": "step_kernel (general recurrence step, j >= 2)",
                         "avg_launch_ms": kernel_avg_ms, "peak_source": peak_src},
            "gpu_launches": total_launches,
            "e2e": {"value": world * n * bstep / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": 32, "seconds_per_step": e2e_s,
                    "seconds_each": [round(t, 5) for t in e2e_t], "clocks": clk_e2e.summary()},
            "clocks": clk.summary(), "generation_s": gen_s}
    if bf16 is not None:
        line["bf16"] = bf16
    if adjoint is not None:
        line["adjoint"] = adjoint
    if batched is not None:
        line["batched"] = batched
    if dense is not None:
        line["dense"] = dense
    if latency is not None:
        line["latency"] = latency
    if config1 is not None:
        line["gmrf_config1"] = config1
    if paper is not None:
        line["paper"] = paper
    if gmrf is not None:
        line["gmrf"] = gmrf
    if not args.no_cpu_baseline:
        # the oracle on the original FP64 values, probe 0: the CPU baseline and
        # the reference for the relative errors of the FP32 and BF16 results
        import oracle

        # the oracle takes its own interval (closed form, or its Gershgorin pass)
        a_c, b_c = interval if interval is not None else oracle.gershgorin(B.rowptr, B.col, B.val)
        dt, steps, probes, t_cpu, threads = cpu_sample(B, B.val, a_c, b_c, n, M, budget_s=args.cpu_budget)
        bg1, _, _ = algorithmic_bytes_per_step(B, 1, s_v)
        line["cpu_baseline"] = {"value": steps * bg1 / dt / 1e9, "unit": "GB/s", "cores": threads,
                                "kind": "oracle",
                                "sample": "probe 0 of %d, %d of %d degree steps, full d=%d, FP64" % (M, steps, n, B.d)}
        if t_cpu is not None:
            gp0 = float(np.dot(oracle.cheb_coeffs(n, a_c, b_c), t_cpu[:, 0]))
            line["rel_err_probe0_vs_fp64_oracle"] = abs(gp0_ours - gp0) / abs(gp0)
            if bf16 is not None:
                bf16["rel_err_probe0_vs_fp64_oracle"] = abs(bf16["gamma_p0"] - gp0) / abs(gp0)
        reference_errors(line)
    print(json.dumps(line), flush=True)


def _forward_and_grad(K, n, M, a, b, steps, torch, checkpoint_too, variant=None):
    """CUDA-event times of cld_estimate and cld_grad on one matrix (autotuned
    unless ``variant`` pins the inner loop), and optionally of the
    checkpointed cld_grad."""
    from paper_1503_06394_gb300 import CsrLogdet

    v32, _ = K.stored("f32")
    m = CsrLogdet(K.rowptr, K.col, v32)
    m.set_interval(a, b)
    if variant is None:
        variant, _ = m.autotune(n, M)
    else:
        m.set_kernel_variant(variant)
    ws_all = m.reserve(n, M, 1)
    m.estimate(n, M, 0)
    m.grad(n, M, 0)
    stream = torch.cuda.current_stream()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    e[0].record(stream)
    for _ in range(steps):
        r = m.estimate(n, M, 0)
    e[1].record(stream)
    for _ in range(steps):
        g, G = m.grad(n, M, 0)
    e[2].record(stream)
    torch.cuda.synchronize()
    out = {"forward_ms": e[0].elapsed_time(e[1]) / steps, "grad_ms": e[1].elapsed_time(e[2]) / steps,
           "workspace_gb": ws_all / 1e9, "variant": variant, "logdet": r["logdet"], "grad_logdet": g}
    if checkpoint_too:
        # checkpointed reverse pass: pairs every K ~ sqrt(2n) steps, segments recomputed
        kc = max(2, int(round((2 * n) ** 0.5)))
        m.set_grad_checkpoint(kc)
        m.ws = None
        torch.cuda.empty_cache()
        ws_ck = m.reserve(n, M, 1)
        gc, Gc = m.grad(n, M, 0)
        torch.cuda.synchronize()
        e[2].record(stream)
        for _ in range(steps):
            gc, Gc = m.grad(n, M, 0)
        e[3].record(stream)
        torch.cuda.synchronize()
        grd_ck = e[2].elapsed_time(e[3]) / steps
        out["checkpointed"] = {"interval": kc, "grad_ms": grd_ck, "adjoint_forward_ratio": grd_ck / out["forward_ms"],
                               # (reverse pass + segment recomputation) / forward, the forward of cld_grad excluded
                               "reverse_over_forward": (grd_ck - out["forward_ms"]) / out["forward_ms"],
                               "workspace_gb": ws_ck / 1e9, "bit_identical_to_store_all": bool(gc == g and torch.equal(Gc, G))}
        del Gc
    m.close()
    del m, G
    torch.cuda.empty_cache()
    return out


def adjoint_leg(args, torch, world):
    """Config 3: Wendland kernel matrix (1e6 points, ell = 0.002, sigma2 = 0.1),
    n = 60, M = 32.  Times cld_estimate (forward) and cld_grad (forward storing
    every w_j + reverse pass + gradient map, and the checkpointed form) on the
    same matrix and probes, with the points numbered by cell of side ell
    (neighbours at nearby indices); the forward and gradient are also timed
    with the points numbered as drawn (the same matrix up to a permutation)."""
    cfg = dict(workloads.CONFIGS[3])
    if args.d:
        cfg["npts"] = int(args.d)
        cfg["ell"] = 0.002 * (1e6 / args.d) ** 0.5  # same expected neighbour count
    if args.n:
        cfg["n"] = int(args.n)
    n, M = cfg["n"], cfg["M"]
    steps = max(1, args.steps)
    res = {}
    for order in ("cell", "random"):
        K = workloads.make(dict(cfg, order=order))
        _, v64 = K.stored("f32")
        a = cfg["sigma2"]
        b = float(np.max(np.add.reduceat(np.abs(v64), K.rowptr[:-1])))
        res[order] = _forward_and_grad(K, n, M, a, b, steps, torch, order == "cell", args.variant)
        res[order]["interval"] = [a, b]
        nnz, d = K.nnz, K.d
        del K
    c = res["cell"]
    out = {"workload": "wendland npts=%d ell=%g sigma2=%g (nnz=%d, %.1f per row), n=%d, M=%d, points numbered by "
                       "cell of side ell" % (cfg["npts"], cfg["ell"], cfg["sigma2"], nnz, nnz / d, n, M),
           "interval": c["interval"], "forward_ms": c["forward_ms"], "grad_ms": c["grad_ms"],
           "forward_variant": c["variant"],
           "adjoint_forward_ratio": c["grad_ms"] / c["forward_ms"],
           "reverse_over_forward": (c["grad_ms"] - c["forward_ms"]) / c["forward_ms"],
           "storage": "all w_j kept in HBM (%.1f GB)" % (n * d * 32 * 4 / 1e9),
           "workspace_gb": c["workspace_gb"], "checkpointed": c["checkpointed"],
           "logdet": c["logdet"], "grad_logdet": c["grad_logdet"],
           "random_order": {"forward_ms": res["random"]["forward_ms"], "grad_ms": res["random"]["grad_ms"],
                            "forward_variant": res["random"]["variant"],
                            "adjoint_forward_ratio": res["random"]["grad_ms"] / res["random"]["forward_ms"],
                            "logdet": res["random"]["logdet"]}}
    return out


def batch_bytes(mats, M, s_v, general):
    """Algorithmic bytes of one degree step over all blocks: (B_gather, B_min).

    SPD blocks: one pass reads the CSR, w_j and w_{j-1} and writes w_{j+1}:
    B_min = csr + 3 d M 4; B_gather adds one M-wide row of w_j per stored
    off-diagonal entry.  General blocks (Algorithm 2): a first pass y = C w_j
    reads C's CSR and w_j and writes y; a second applies C^T to y with the
    recurrence, reading C^T's CSR, y, w_j and w_{j-1} and writing w_{j+1}:
    B_min = 2 csr + 6 d M 4 (y spans all blocks, far more than L2, so it
    goes to DRAM and back); B_gather adds the gathered rows of both passes."""
    bg = bm = 0
    for m in mats:
        rows = np.repeat(np.arange(m.d), np.diff(m.rowptr))
        off = int(np.count_nonzero(m.col != rows))
        csr = m.nnz * (s_v + 4) + 8 * (m.d + 1)
        if general:
            bm += 2 * csr + 6 * m.d * M * 4
            bg += 2 * csr + 2 * off * M * 4 + 6 * m.d * M * 4
        else:
            bm += csr + 3 * m.d * M * 4
            bg += csr + off * M * 4 + 3 * m.d * M * 4
    return bg, bm


def batch_leg(args, torch):
    """Config 4: 512 matrices, d log-uniform in [1e3, 2e5]; the SPD half and the
    general half (1/2 logdet C^T C) each in one batched estimate replayed as a
    CUDA graph, against a loop of single-matrix estimates on the same GPU.
    Each arm is timed as `reps` separately timed estimates (CUDA events);
    the median is reported with the spread.  The roofline of the batched step
    kernel is its mean launch time (profiled estimate) against B_min: every
    block's w_j is at most 12.8 MB, so gathers are L2 hits and the DRAM
    traffic a launch must move is the CSR plus the recurrence blocks."""
    from paper_1503_06394_gb300 import CsrBatchLogdet, CsrLogdet

    cfg = workloads.CONFIGS[4]
    n, M = cfg["n"], cfg["M"]
    spd, gen = workloads.batch_mixed(cfg["count"], cfg["dmin"], cfg["dmax"], cfg["seed"])
    peak, src = read_peaks()
    out = {"workload": "%d matrices, d log-uniform in [%g, %g] (sum d = %d), half SPD, half general; n=%d, M=%d" % (
        cfg["count"], cfg["dmin"], cfg["dmax"], sum(m.d for m in spd + gen), n, M),
           "bytes_model": "B_min per degree step: SPD csr + 3 d M 4, general 2 csr + 6 d M 4 (see batch_bytes)",
           "peak_gbs": peak, "peak_source": src}
    reps = max(7, args.steps)
    for dtype in ("f32", "bf16"):
        tot_ms, tot_bmin = 0.0, 0
        for kind, mats in (("spd", spd), ("general", gen)):
            br, S = workloads.block_diag(mats)
            st, _ = S.stored(dtype)
            bt = CsrBatchLogdet(br, S.rowptr, S.col, st, dtype=dtype, kind=kind)
            bt.auto_intervals()
            if args.variant is None:
                v, _ = bt.autotune(n, M)
            else:  # pinned (profiling captures): no autotuner launches
                v = args.variant
                bt.set_kernel_variant(v)
                if args.tile_rows:
                    bt.set_tile_rows(args.tile_rows)
            tile_rows = bt.tile_rows
            bt.reserve(n, M)
            # the step kernel alone: plain launches with profiling events
            bt.set_graph(False)
            bt.set_profiling(True)
            bt.estimate(n, M, 0)
            kms, klaunch, _ = bt.last_timing()
            bt.set_profiling(False)
            bt.set_graph(True)
            for _ in range(3):
                bt.estimate(n, M, 0)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            torch.cuda.synchronize()
            for e0, e1 in ev:
                e0.record()
                bt.estimate(n, M, 0)
                e1.record()
            torch.cuda.synchronize()
            each = sorted(e0.elapsed_time(e1) for e0, e1 in ev)
            ms = float(np.median(each))
            bt.close()
            del bt
            s_v = 2 if dtype == "bf16" else 4
            bg, bm = batch_bytes(mats, M, s_v, kind == "general")
            # mean time of one general degree step (both passes for general blocks)
            kernel_ms = kms / max(1, klaunch)
            key = "%s_%s" % (kind, dtype)
            out[key + "_ms"] = ms
            out[key + "_ms_min_max"] = [each[0], each[-1]]
            out[key + "_gbs_bmin"] = n * bm / (ms / 1e3) / 1e9
            out[key + "_gbs_gather"] = n * bg / (ms / 1e3) / 1e9
            out[key + "_step_kernel_ms"] = kernel_ms
            out[key + "_step_frac_bmin"] = bm / (kernel_ms / 1e3) / 1e9 / peak
            out[key + "_variant"] = v
            out[key + "_tile_rows"] = tile_rows
            tot_ms += ms
            tot_bmin += n * bm
        out["batched_%s_ms" % dtype] = tot_ms
        out["batched_%s_gbs_bmin" % dtype] = tot_bmin / (tot_ms / 1e3) / 1e9
        out["batched_%s_frac_bmin" % dtype] = tot_bmin / (tot_ms / 1e3) / 1e9 / peak
    # per-matrix loop (FP32): one handle per matrix, estimates one after another
    handles = []
    for kind, mats in (("spd", spd), ("general", gen)):
        for m in mats:
            v32, _ = m.stored("f32")
            h = CsrLogdet(m.rowptr, m.col, v32, kind=kind)
            h.auto_interval(0)
            h.reserve(n, M)
            handles.append(h)
    for h in handles[:4]:
        h.estimate(n, M, 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h in handles:
        h.estimate(n, M, 0)
    torch.cuda.synchronize()
    loop_ms = (time.perf_counter() - t0) * 1e3
    for h in handles:
        h.close()
    del handles
    torch.cuda.empty_cache()
    out["loop_f32_ms"] = loop_ms
    out["speedup_vs_loop"] = loop_ms / out["batched_f32_ms"]
    out["bf16_vs_f32_time"] = out["batched_bf16_ms"] / out["batched_f32_ms"]
    return out


def gmrf_leg(args, torch):
    """The paper's GMRF experiment (Sec. 5.2, Fig. 3): a sample x of the
    4-neighbour GMRF on a 5000 x 5000 grid (d = 2.5e7) with partial
    correlation rho = -0.22, drawn by a chequerboard Gibbs sampler
    (x_i | rest ~ N(rho * sum of neighbours, 1)); then the log-likelihood
    1/2 logdet J(rho) - 1/2 x^T J(rho) x over a grid of rho, logdet J(rho)
    estimated on the GPU (n = 60, M = 16).  The exact logdet from the
    separable spectrum 1 - rho (2 cos(pi i/(N+1)) + 2 cos(pi j/(N+1))) and
    the argmax it gives are added by the CPU-baseline block."""
    from paper_1503_06394_gb300 import CsrLogdet

    N = int(round((args.d or 25_000_000) ** 0.5))
    rho0, sweeps = -0.22, 200
    g = torch.Generator(device="cuda").manual_seed(1007)
    x = torch.zeros((N + 2, N + 2), dtype=torch.float64, device="cuda")  # zero halo
    ii, jj = torch.meshgrid(torch.arange(N, device="cuda"), torch.arange(N, device="cuda"), indexing="ij")
    colour = ((ii + jj) % 2).bool()
    torch.cuda.synchronize()
    t0 = time.time()
    for _ in range(sweeps):
        for c in (False, True):
            nb = x[:-2, 1:-1] + x[2:, 1:-1] + x[1:-1, :-2] + x[1:-1, 2:]
            z = torch.randn((N, N), dtype=torch.float64, device="cuda", generator=g)
            inner = x[1:-1, 1:-1]
            inner[colour == c] = (rho0 * nb + z)[colour == c]
    xs = x[1:-1, 1:-1].contiguous()
    sum_sq = float((xs * xs).sum())
    xax = float(2 * ((xs[:-1, :] * xs[1:, :]).sum() + (xs[:, :-1] * xs[:, 1:]).sum()))  # x^T A x
    gibbs_s = time.time() - t0
    del x, ii, jj, colour, xs
    rowptr, col, diag = workloads.grid_pattern_device(N, torch)
    vals = torch.ones(col.shape[0], dtype=torch.float32, device="cuda")
    m = CsrLogdet(rowptr, col, vals)
    n, M = 60, 16
    sweep = []
    torch.cuda.synchronize()
    t0 = time.time()
    for rho in np.round(np.arange(-0.245, 0.0001, 0.005), 4):
        m.val.copy_(torch.where(diag, 1.0, float(rho)).float())  # values of J(rho), same pattern
        m.set_interval(1 - 4 * abs(rho) - 1e-6, 1 + 4 * abs(rho) + 1e-6)
        r = m.estimate(n, M, 0)
        quad = sum_sq - rho * xax
        sweep.append({"rho": float(rho), "logdet": r["logdet"], "stderr": r["stderr"],
                      "loglik": 0.5 * r["logdet"] - 0.5 * quad, "quad": quad})
    sweep_s = time.time() - t0
    nnz = int(col.shape[0])
    m.close()
    del m, rowptr, col, diag, vals
    torch.cuda.empty_cache()
    best = max(sweep, key=lambda e: e["loglik"])
    return {"workload": "GMRF grid %d x %d (d=%d, nnz=%d), Gibbs sample at rho=%g (%d sweeps), n=%d, M=%d" % (
                N, N, N * N, nnz, rho0, sweeps, n, M),
            "N": N, "argmax_rho": best["rho"], "true_rho": rho0,
            "gibbs_s": gibbs_s, "sweep_s": sweep_s, "estimates": len(sweep), "sweep": sweep}


def paper_leg(args, torch):
    """The paper's timing experiment (Sec. 5.1, Fig. 1a): Algorithm 2 on its own
    sparse random generator (five U[-1,1] off-diagonals per row, mirrored,
    diagonal = absolute row sum + 1e-3) with m = 10, n = 15,
    sigma_min = 1e-3, sigma_max = ||C||_1, at d = 3e7 (about 3.3e8 stored
    entries, built on the device).  The paper reports 500 s on a 3.40 GHz
    Intel i7.  Accuracy point: the same setting at d = 1e4 (numpy generator);
    its error against numpy's log|det C| is added by the CPU-baseline block."""
    from paper_1503_06394_gb300 import CsrLogdet

    n, M = 15, 10
    out = {"paper_seconds": 500.0, "paper_hardware": "3.40 GHz Intel i7, 24 GB RAM (Sec. 5.1)", "n": n, "m": M}
    for d in (10_000, args.d or 30_000_000):
        t0 = time.time()
        if d <= 20000:
            C = workloads.paper_sparse_random(d, 1006)
            rowptr, col = C.rowptr, C.col
            v32, v64 = C.stored("f32")
            smax = float(np.max(np.add.reduceat(np.abs(v64), C.rowptr[:-1])))  # ||C||_1 = ||C||_inf
            nnz = C.nnz
        else:
            rowptr, col, v64 = workloads.paper_sparse_random_device(d, 1006, torch)
            v32 = v64.float()
            rows = torch.repeat_interleave(torch.arange(d, device="cuda"), torch.diff(rowptr))
            smax = float(torch.zeros(d, dtype=torch.float64, device="cuda").index_add_(0, rows, v32.double().abs()).max())
            nnz = int(col.shape[0])
            del v64, rows
        torch.cuda.synchronize()
        gen = time.time() - t0
        m = CsrLogdet(rowptr, col, v32, kind="general")
        m.set_interval(1e-6, smax ** 2)
        m.reserve(n, M)
        m.estimate(n, M, 0)
        torch.cuda.synchronize()
        reps = 3
        t0 = time.perf_counter()
        for _ in range(reps):
            r = m.estimate(n, M, 0)
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t0) / reps
        m.close()
        del m, rowptr, col, v32
        torch.cuda.empty_cache()
        out["d%d" % d] = {"nnz": nnz, "seconds": sec, "logdet": r["logdet"], "stderr": r["stderr"],
                          "speedup_vs_paper": (500.0 / sec) if d >= 30_000_000 else None, "generation_s": gen,
                          "generator": "numpy (workloads.paper_sparse_random)" if d <= 20000 else
                          "device (workloads.paper_sparse_random_device)"}
    return out


def config1_leg(args, torch):
    """Config 1: the GMRF precision 0.1 I + L on a 1000 x 1000 grid (d = 1e6,
    5-point Dirichlet Laplacian, nnz = 4,996,000), FP32, n = 50, M = 64, the
    closed-form interval [0.1, 8.1].  Whole-estimate time (CUDA events) and the
    general step kernel's mean launch time against B_min: the stencil's
    neighbour rows are L2 hits, so each step must move the CSR once and
    w_{j-1}, w_j, w_{j+1} once."""
    from paper_1503_06394_gb300 import CsrLogdet

    cfg = workloads.CONFIGS[1]
    B = workloads.make(cfg)
    v32, _ = B.stored("f32")
    n, M = cfg["n"], cfg["M"]
    interval = (cfg["kappa2"], cfg["kappa2"] + 8.0)
    m = CsrLogdet(B.rowptr, B.col, v32)
    m.set_interval(*interval)
    if args.variant is None:
        variant, _ = m.autotune(n, M)
    else:  # pinned (profiling captures): no autotuner launches
        variant = args.variant
        m.set_kernel_variant(variant)
    m.reserve(n, M)
    ms, kernel_ms, launches, _, r = time_estimates(m, n, M, cfg["probe_seed"], interval, max(3, args.steps),
                                                  max(3, args.warmup), torch, 1)
    m.close()
    del m
    torch.cuda.empty_cache()
    _, bmin, _ = algorithmic_bytes_per_step(B, M, 4)
    peak, src = read_peaks()
    return {"workload": "grid_gmrf N=%d (d=%d, nnz=%d) kappa2=%g, FP32, n=%d, M=%d, interval %s" % (
                cfg["N"], B.d, B.nnz, cfg["kappa2"], n, M, list(interval)),
            "ms_per_estimate": ms, "variant": variant, "step_kernel_ms": kernel_ms,
            "b_min_per_step": bmin, "step_gbs_bmin": bmin / (kernel_ms / 1e3) / 1e9,
            "step_frac_bmin": bmin / (kernel_ms / 1e3) / 1e9 / peak, "peak_gbs": peak, "peak_source": src,
            "estimate_gbs_bmin": n * bmin / (ms / 1e3) / 1e9, "logdet": r["logdet"], "stderr": r["stderr"]}


def latency_leg(args, torch):
    """Config 0 (d = 2048, n = 30, M = 30): a launch- and latency-bound size.
    Time per estimate with plain launches and with the whole estimate replayed
    as one CUDA graph, the interval from the device's own Gershgorin pass.  The
    errors against the oracle (same probes) and the exact Cholesky value are
    added by the CPU-baseline block (``reference_errors``)."""
    from paper_1503_06394_gb300 import CsrLogdet

    cfg = workloads.CONFIGS[0]
    B = workloads.make(cfg)
    v32, _ = B.stored("f32")
    n, M = cfg["n"], cfg["M"]
    m = CsrLogdet(B.rowptr, B.col, v32)
    m.reserve(n, M)
    a_gpu, b_gpu = m.auto_interval(0)  # the device's own Gershgorin pass
    out = {"workload": "sparse_random_spd d=%d picks=%d seed=%d, n=%d, M=%d" % (B.d, cfg["picks"], cfg["seed"], n, M)}
    reps = 50
    for mode in ("launches", "graph"):
        m.set_graph(mode == "graph")
        for _ in range(5):
            r = m.estimate(n, M, cfg["probe_seed"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            r = m.estimate(n, M, cfg["probe_seed"])
        out["%s_us" % mode] = (time.perf_counter() - t0) / reps * 1e6
    m.close()
    out.update({"interval": [a_gpu, b_gpu], "logdet": r["logdet"], "stderr": r["stderr"],
                "timing": "host wall clock per estimate call (includes the result read-back)"})
    return out


def reference_errors(line):
    """Part of the CPU-baseline leg: the oracle's and the closed forms' values
    for the small legs, and the GPU results' errors against them.  Runs after
    every GPU measurement; no value here feeds a GPU call."""
    import oracle

    lat = line.get("latency")
    if lat is not None:
        cfg = workloads.CONFIGS[0]
        B = workloads.make(cfg)
        _, v64 = B.stored("f32")
        a, b = oracle.gershgorin(B.rowptr, B.col, v64)  # the oracle's own interval
        ref = oracle.estimate(B.rowptr, B.col, v64, a, b, cfg["n"], cfg["M"], seed=cfg["probe_seed"])
        exact = oracle.logdet_cholesky(workloads.Csr(B.rowptr, B.col, v64).dense())
        lat.update({"interval_rel_diff_vs_oracle": max(abs(lat["interval"][0] - a) / a, abs(lat["interval"][1] - b) / b),
                    "oracle_logdet": ref["gamma"], "exact_cholesky": exact,
                    "rel_err_vs_oracle": abs(lat["logdet"] - ref["gamma"]) / abs(ref["gamma"]),
                    "rel_err_vs_exact": abs(lat["logdet"] - exact) / abs(exact)})
    pl = line.get("paper")
    if pl is not None and "d10000" in pl:
        C = workloads.paper_sparse_random(10_000, 1006)
        exact = float(np.linalg.slogdet(C.dense())[1])
        pl["d10000"].update({"exact": exact, "rel_err": abs(pl["d10000"]["logdet"] - exact) / abs(exact)})
    gm = line.get("gmrf")
    if gm is not None:
        N = gm["N"]
        c = np.cos(np.pi * np.arange(1, N + 1) / (N + 1))
        for e in gm["sweep"]:
            exact = float(np.sum(np.log(1.0 - e["rho"] * 2.0 * (c[:, None] + c[None, :]))))
            e["logdet_exact"] = exact
            e["loglik_exact"] = 0.5 * exact - 0.5 * e["quad"]
        gm["argmax_rho_exact_logdet"] = max(gm["sweep"], key=lambda e: e["loglik_exact"])["rho"]
        gm["max_rel_err_logdet"] = max(abs(e["logdet"] - e["logdet_exact"]) / abs(e["logdet_exact"])
                                       for e in gm["sweep"] if e["logdet_exact"] != 0)
        gm["max_err_in_stderrs"] = max(abs(e["logdet"] - e["logdet_exact"]) / e["stderr"] for e in gm["sweep"]
                                       if e["stderr"] > 0)
    dn = line.get("dense")
    if dn is not None:
        exact = oracle.kms_logdet(dn["d"], dn["rho"])
        dn.update({"exact_closed_form": exact, "rel_err_vs_exact": abs(dn["logdet"] - exact) / abs(exact),
                   "err_in_stderrs": abs(dn["logdet"] - exact) / dn["stderr"]})
    g1 = line.get("gmrf_config1")
    if g1 is not None:
        cfg = workloads.CONFIGS[1]
        exact = oracle.grid_laplacian_logdet(cfg["N"], cfg["kappa2"])
        g1.update({"exact_closed_form": exact, "rel_err_vs_exact": abs(g1["logdet"] - exact) / abs(exact),
                   "err_in_stderrs": abs(g1["logdet"] - exact) / g1["stderr"]})


def dense_leg(args, torch):
    """Dense kernel-matrix path (tensor cores): the Kac-Murdock-Szego matrix
    A_ik = 0.5^|i-k| at d = 32768 in BF16 (2.1 GB; 0.5^k is exact in BF16 down
    to the 1e-40 range, the rest rounds to 0), n = 30, M = 32, on its known
    spectral interval [1/3, 3].  Its exact logdet is (d - 1) log(0.75)
    (added by the CPU-baseline block).  The step streams B once: bytes per
    step = 2 d^2 + 12 d M (vectors); the MMA work is 3 x 2 d^2 M (three BF16
    parts of w_j)."""
    from paper_1503_06394_gb300 import DenseLogdet

    d, n, M, rho = args.d or 32768, args.n or 30, 32, 0.5
    Ab = torch.empty((d, d), dtype=torch.bfloat16, device="cuda")
    cols = torch.arange(d, device="cuda", dtype=torch.float32)
    for r0 in range(0, d, 2048):
        rows = torch.arange(r0, min(d, r0 + 2048), device="cuda", dtype=torch.float32)
        Ab[r0:r0 + rows.numel()] = torch.pow(rho, (rows[:, None] - cols[None, :]).abs()).to(torch.bfloat16)
    del cols
    m = DenseLogdet(Ab, d)
    # eigenvalues of rho^|i-k| lie in ((1 - rho)/(1 + rho), (1 + rho)/(1 - rho))
    a, b = (1 - rho) / (1 + rho), (1 + rho) / (1 - rho)
    m.set_interval(a, b)
    m.estimate(n, M, 0)
    steps = max(1, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        r = m.estimate(n, M, 0)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    m.close()
    del m, Ab
    torch.cuda.empty_cache()
    peak, src = read_peaks()
    step_bytes = 2 * d * d + 12 * d * M
    gbs = n * step_bytes / (ms / 1e3) / 1e9
    return {"workload": "dense Kac-Murdock-Szego matrix 0.5^|i-k|, BF16, d=%d, n=%d, M=%d" % (d, n, M),
            "d": d, "rho": rho, "interval": [a, b], "ms_per_estimate": ms, "gbs": gbs, "pct_of_peak": 100 * gbs / peak,
            "tensor_tflops": n * 3 * 2 * d * d * M / (ms / 1e3) / 1e12, "logdet": r["logdet"], "stderr": r["stderr"],
            "kernel": "dense_step_kernel (tcgen05.mma kind::f16, TMA, TMEM)"}


def step_sources_sha256(csrc):
    """sha256 of the step kernels' device code, value loads and grid sizing:
    their headers, and the argument block (struct StepArgs) of the shared
    internal header, whose other declarations do not reach these kernels."""
    import hashlib

    h = hashlib.sha256()
    for name in ("step_kernel.cuh", "step_wide.cuh", "step_staged.cuh", "step_window.cuh", "async_copy.cuh",
                 "step_launch.cuh"):
        h.update(open(os.path.join(csrc, name), "rb").read())
    internal = open(os.path.join(csrc, "cld_internal.cuh"), "rb").read()
    i = internal.index(b"struct StepArgs {")
    h.update(internal[i:internal.index(b"};", i) + 2])
    return h.hexdigest()


def profiled_traffic(args, B, variant):
    """DRAM bytes (read + write) per general-step launch of inner-loop variant
    ``variant`` from the committed ncu summary of this workload, if the step
    kernel's source is the one it was captured with."""
    path = os.path.join(ROOT, "profiles", "step_kernel_config2_traffic.md")
    csrc = os.path.join(ROOT, "paper_1503_06394_gb300", "csrc")
    if args.config != 2 or args.d or args.dtype != "f32" or not os.path.exists(path):
        return None
    text = open(path).read()
    want = step_sources_sha256(csrc)
    vals = dict(line.split(":", 1) for line in text.splitlines() if ":" in line and line[:1].isalpha())
    if vals.get("step_kernels_sha256", "").strip() != want:
        return None
    try:
        return float(vals["traffic_bytes_per_launch_v%d" % variant].strip())
    except (KeyError, ValueError):
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=[0, 1, 2])
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f64"])
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--d", type=int, default=None, help="override the dimension (small profiling cases)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16-storage measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward (config 3) measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched (config 4) measurement")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense tensor-core measurement")
    ap.add_argument("--no-latency", action="store_true", help="skip the config-0 latency measurement")
    ap.add_argument("--no-config1", action="store_true", help="skip the config-1 (grid GMRF) measurement")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper's Sec. 5.1 timing replay")
    ap.add_argument("--no-gmrf", action="store_true", help="skip the paper's Sec. 5.2 GMRF likelihood sweep")
    ap.add_argument("--only", choices=["dense", "adjoint", "paper", "latency", "gmrf", "config1", "batch"],
                    default=None,
                    help="run one leg alone (with --d / --n overrides) and print its JSON")
    ap.add_argument("--n", type=int, default=None, help="degree override for --only")
    ap.add_argument("--variant", type=int, default=None, choices=[0, 1, 2, 3, 4, 5, 6, 7],
                    help="pin the recurrence-step inner-loop variant instead of autotuning it")
    ap.add_argument("--tile-rows", type=int, default=None,
                    help="with --variant and --only batch: rows per work tile of the batched step")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch

        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.only:
        run_only(args)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
