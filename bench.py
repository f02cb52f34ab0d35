"""Benchmark of the CIL hot path on B300 (one JSON line on rank 0).

One step = one pass of the whole hot path over one batch of synthetic input
(the 64x64 FitzHugh-Nagumo workload: 2 sets x 64 realisations, 10^4 FP32
Euler steps, u-only patterns of d = 4096, 16 radii, 200 resamples):
  initial state -> integration (+ FP64 residual) -> pattern Gram + exact
  recheck -> radii / bins / counts -> bootstrap counts -> mean, covariance,
  Cholesky, log-determinant, cost and log-likelihood.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

value  = cell-updates per second of the whole step (a cell-update = one grid
         node, both species, one time step), device-timed with CUDA events,
         max over ranks, inputs resident in HBM.
e2e    = the same through the public API with host buffers: every step
         copies the initial fields host->device and the statistics back.
--impl reference runs the plain FP64 CPU oracle on a bounded sample of the
same workload (rank 0 only; other ranks exit).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

# FP32-pipe instructions of the implemented update per cell-update: two
# neighbour sums (3 + 3), then FHN u 6, v 3; GM u 9, v 5 (deviation form;
# the division's reciprocal runs on the MUFU pipe and is not counted);
# BZ u 8 (a + u0, U*U, *b, fma P, e0 + P, fma f, fma, fma), v 6 (-e0 - P,
# fma g, fma, fma, fma -4, ...); DIFF 2 + 2.
FP32_INST_PER_CELL = {W.FHN: 15, W.GM: 20, W.DIFF: 10, W.BZ: 22}

# DRAM bytes (read + write) of one stepper launch on this workload, from the
# ncu capture summarised in profiles/rd_resident_scalar_kernel_fhn64_c2.md,
# keyed by a hash of the stepper sources: reported only while the kernel is
# the one that was measured.
STEPPER_TRAFFIC = {"6f89ac52bd0c99eb": 4223232, "a1b8429f6f299483": 4223488, "7c8c62601c860730": 4223488}
STEPPER_SOURCES = ["paper_2203_14742_b300/csrc/stepper.cu", "paper_2203_14742_b300/csrc/tile.cuh",
                   "paper_2203_14742_b300/csrc/common.cuh"]


def stepper_traffic():
    import hashlib
    h = hashlib.sha256()
    for f in STEPPER_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return STEPPER_TRAFFIC.get(h.hexdigest()[:16])
L2_BYTES = 126 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-reference-path", action="store_true")
    ap.add_argument("--variant", type=int, default=-1,
                    help="fixed stepper tile variant (skips the autotuner; for profiling)")
    ap.add_argument("--graph", action="store_true",
                    help="also time the pass captured in a CUDA graph and replayed")
    ap.add_argument("--gram-large", action="store_true",
                    help="also time the tensor-core Gram on 2 x 1024 patterns of d = 32768")
    ap.add_argument("--adjoint", action="store_true",
                    help="also time the adjoint (smoothed-CIL gradient) on the FHN 64x64 adjoint workload "
                         "(32 realisations, 5000 steps)")
    ap.add_argument("--stream", action="store_true",
                    help="also time the streaming stepper (TMA tiles, temporal blocking) on FHN 512x512 x 128 "
                         "realisations, against the HBM roofline")
    ap.add_argument("--stream-only", action="store_true",
                    help="time only the streaming stepper (for profiling)")
    ap.add_argument("--mcil", action="store_true",
                    help="also time the multi-feature correlation integral (six distances) at the FHN 64x64 "
                         "and GM 128x128 set shapes")
    ap.add_argument("--mcil-only", action="store_true",
                    help="time only the multi-feature correlation integral (for profiling)")
    ap.add_argument("--rkc", action="store_true",
                    help="add the adaptive stabilised RK2 (App. B.2) against the Euler stepper on c2")
    ap.add_argument("--rkc-only", action="store_true",
                    help="run only the adaptive stabilised RK2 comparison and print it")
    ap.add_argument("--imex", action="store_true",
                    help="add the semi-implicit Euler stepper against the Euler stepper on c2")
    ap.add_argument("--imex-only", action="store_true",
                    help="run only the semi-implicit Euler comparison and print it")
    ap.add_argument("--gram-large-only", action="store_true",
                    help="time only the tensor-core Gram and correlation integral on 2 x 1024 patterns of "
                         "d = 32768 (for profiling); prints that object alone")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
                "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled through NVML (the
    driver library nvidia-smi reads, called through ctypes) every few
    milliseconds on a thread, so that even a timed region of a few tens of
    milliseconds has samples.  Call begin() and end() around the timed
    region; summary() keeps the samples taken between them."""

    # nvmlClocksEventReason* bits of the NVML API
    REASONS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
               ("sw_power_cap", 0x4))
    NVML_CLOCK_SM = 1

    def __init__(self, index, interval_s=0.005):
        self.index = index
        self.interval = interval_s
        self.samples = []
        self.t_begin = self.t_end = None
        self.thread = None
        self.stop = threading.Event()

    def __enter__(self):
        try:
            import ctypes as C
            nv = C.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return self
            h = C.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.index), C.byref(h)) != 0:
                return self
            mx = C.c_uint(0)
            nv.nvmlDeviceGetMaxClockInfo(h, C.c_int(self.NVML_CLOCK_SM), C.byref(mx))
            self.max_mhz = int(mx.value)
            get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons

            def loop():
                clk, rs = C.c_uint(0), C.c_ulonglong(0)
                while not self.stop.is_set():
                    if nv.nvmlDeviceGetClockInfo(h, C.c_int(self.NVML_CLOCK_SM), C.byref(clk)) == 0 and \
                            get_reasons(h, C.byref(rs)) == 0:
                        self.samples.append((time.perf_counter(), int(clk.value),
                                             [n for n, m in self.REASONS if rs.value & m]))
                    self.stop.wait(self.interval)

            self.thread = threading.Thread(target=loop, daemon=True)
            self.thread.start()
            time.sleep(0.05)
        except Exception:
            self.thread = None
        return self

    def begin(self):
        self.t_begin = time.perf_counter()

    def end(self):
        self.t_end = time.perf_counter()

    def __exit__(self, *a):
        if self.thread is not None:
            self.stop.set()
            self.thread.join(timeout=2)

    def summary(self):
        if self.thread is None or self.t_begin is None:
            return None
        t1 = self.t_end if self.t_end is not None else float("inf")
        inside = [s for s in self.samples if self.t_begin <= s[0] <= t1]
        if not inside:
            return None
        reasons = sorted(set(r for s in inside for r in s[2]))
        return {"sm_mhz": statistics.median(s[1] for s in inside), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(inside), "source": "NVML every 5 ms in the timed region"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
# ---------------------------------------------------------------------------
# multi-rank host logic (weak scaling: every rank runs its own independent
# batch; no collective on the data path, only the timing is reduced)
# ---------------------------------------------------------------------------
RANK_SEED_STRIDE = 7919


def rank_groups(cfg, rank):
    """The workload's groups for one rank: the same shapes, seeds offset by
    rank so that every rank integrates an independent batch."""
    out = []
    for gd in cfg["groups"]:
        gd = dict(gd)
        gd["seed"] = gd["seed"] + RANK_SEED_STRIDE * rank
        out.append(gd)
    return out


def max_over_ranks(x, device, world):
    """The largest value of x over all ranks (x itself when world == 1)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t)


def whole_job_rate(units_per_rank, world, ms):
    """Units processed by all ranks per second, over the slowest rank's time."""
    return units_per_rank * world / (ms * 1e-3)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2203_14742_b300 as p
    from paper_2203_14742_b300 import build as B

    B.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    cfg = W.config(args.config)
    gds = rank_groups(cfg, rank)
    groups = [p.Group.from_dict(gd) for gd in gds]
    n1, n2, M, b, T = cfg["n1"], cfg["n2"], cfg["M"], cfg["b"], cfg["T_res"]
    sets = [(n1, n2, gd["species_mask"]) for gd in gds]
    pipe = p.Pipeline(groups, sets, M, b, T, cfg["seed"] + rank, device=dev)
    sim = pipe.sim
    multi = len(groups) > 1
    if args.variant >= 0:
        for g in groups:
            assert p.lib().rd_set_variant(g.model, g.G, args.variant) == 0
        variant = args.variant
    elif not multi:
        chosen = sim.autotune(steps=300)      # tile shape per (model, G); untimed set-up
        variant = chosen[groups[0].model * 3 + {32: 0, 64: 1, 128: 2}[groups[0].G]]
    else:
        variant = "persistent"
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    cell_updates = sum(g.n_real * g.G * g.G * g.n_steps for g in groups)
    inst = sum(g.n_real * g.G * g.G * g.n_steps * FP32_INST_PER_CELL[g.model] for g in groups)
    pairs = n1 * n2 * len(groups)

    # ---- warm-up -------------------------------------------------------------
    for _ in range(args.warmup):
        pipe.run()
    torch.cuda.synchronize()
    assert sim.sync_status() == 0, "non-finite field during warm-up"

    # ---- device-timed whole steps (L2 flushed between steps) -----------------
    def evs():
        return [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    marks = [evs() for _ in range(args.steps)]
    launches0 = p.lib().rd_kernel_launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        clk.begin()
        for i in range(args.steps):
            flush.fill_(float(i))
            e = marks[i]
            e[0].record(stream)
            sim.reinit()
            e[1].record(stream)
            _check_int(p, sim, pipe)
            e[2].record(stream)
            for (X1, X2), out in zip(pipe.views, pipe.cil_out):
                p.cil(X1, X2, b=b, M=M, work=pipe.work, out=out)
            e[3].record(stream)
            p.synlik(pipe.bins, M, T, pipe.seed, y_obs=pipe.C, out=pipe.stats, work=pipe.syn_work)
            e[4].record(stream)
        torch.cuda.synchronize()
        clk.end()
    launches = p.lib().rd_kernel_launches() - launches0
    step_ms = sum(m[0].elapsed_time(m[4]) for m in marks)
    k_ms = [m[1].elapsed_time(m[2]) for m in marks]
    cil_ms = [m[2].elapsed_time(m[3]) for m in marks]
    syn_ms = [m[3].elapsed_time(m[4]) for m in marks]
    step_ms = max_over_ranks(step_ms, dev, world)
    assert sim.sync_status() == 0
    ms_per_step = step_ms / args.steps
    value = whole_job_rate(cell_updates, world, ms_per_step)
    nre = int(sum(int(o["n_rechecked"]) for o in pipe.cil_out))

    # ---- the same pass captured in a CUDA graph and replayed -----------------
    graph_ms = None
    if args.graph:
        pipe.capture()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pipe.replay()
        torch.cuda.synchronize()
        g0.record(stream)
        for _ in range(args.steps):
            pipe.replay()
        g1.record(stream)
        torch.cuda.synchronize()
        graph_ms = g0.elapsed_time(g1) / args.steps
        pipe.graph = None

    # ---- end to end through the public API with host buffers -----------------
    host = {"fields": torch.empty(sim.fields.shape, dtype=torch.float32, pin_memory=True)}
    sim.reinit()
    host["fields"].copy_(sim.fields)
    outs = {"mu": pipe.stats["mu"], "cov": pipe.stats["cov"], "chol": pipe.stats["chol"],
            "scalars": pipe.stats["scalars"], "status": pipe.stats["status"], "C": pipe.C,
            "residual": pipe.residual}
    for k, t in outs.items():
        host[k] = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)

    def e2e_step():
        sim.fields.copy_(host["fields"], non_blocking=True)
        pipe.run(reinit=False)
        for k, t in outs.items():
            host[k].copy_(t, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, dev, world)
    h2d = host["fields"].numel() * 4
    d2h = sum(host[k].numel() * host[k].element_size() for k in outs)

    # ---- plain single-realisation FP32 path on a slice (same GPU) ------------
    ref_rate = None
    if not args.no_reference_path and rank == 0:
        gsl = dict(gds[0])
        gsl["n_real"] = 2
        ssl = p.Simulation([p.Group.from_dict(gsl)], device=dev)
        nsl = 500
        ssl.integrate_reference(steps=50)
        torch.cuda.synchronize()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        ssl.integrate_reference(steps=nsl)
        r1.record(stream)
        torch.cuda.synchronize()
        ref_rate = 2 * gsl["G"] ** 2 * nsl / (r0.elapsed_time(r1) * 1e-3)

    # ---- roofline of the dominant kernel (the stepper) ----------------------
    pk, src = peaks()
    k_avg_ms = sum(k_ms) / len(k_ms)
    achieved = inst / (k_avg_ms * 1e-3) / 1e12                          # T FP32 instructions / s
    peak_alu = 148 * 128 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12   # FP32 lanes x clock
    cil_avg = sum(cil_ms) / len(cil_ms)
    if multi:
        kname = "rd_batch_kernel (persistent)"
    else:
        pk_, ty_, tx_ = p.variant_shape(groups[0].G, variant)
        kname = "%s<%s,%d,%dx%d> variant %s" % ("rd_resident_kernel" if pk_ else "rd_resident_scalar_kernel",
                                               {0: "FHN", 1: "GM", 2: "DIFF", 3: "BZ"}[groups[0].model],
                                               groups[0].G, ty_, tx_, variant)
    workload = {"c2": "c2: FHN 64x64, 2 sets x 64 realisations, 10^4 Euler steps, u-only d=4096, M=16, "
                      "b=1.3, 200 resamples",
                "c4": "c4: 64 parameter vectors x 128 realisations, FHN+GM at 64^2 (10^4 steps) and 128^2 "
                      "(2x10^4 steps) in one persistent launch, 2 x 64 sets per vector, M=16, 200 resamples",
                "c1": "c1: FHN 32x32, 2 x 16, 2000 steps, d=2048, M=8, 50 resamples",
                "c3": "c3: GM 128x128, 2 x 256, 2x10^4 steps, d=32768, M=16, 200 resamples",
                "c5": "c5: FHN 64x64, 32 realisations, 5000 steps",
                "c6": "c6: Brusselator 64x64, 2 sets x 64 realisations, 25600 Euler steps (T = 100), both "
                      "species d=8192, M=16, b=1.3, 200 resamples"}[args.config]
    out = {
        "metric": "RD cell-updates/s + CIL pair-dists/s at stated tol; % HBM/tensor roofline",
        "value": value,
        "unit": "cell-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 stepper, bf16x3 Gram + f64 recheck, f64 statistics",
        "data": "synthetic (seeded counter-based initial noise; the paper's data are simulated too)",
        "config": {"workload": workload, "groups": len(groups),
                   "realisations_per_gpu": sum(g.n_real for g in groups),
                   "grids": sorted(set(g.G for g in groups)), "pairs": pairs, "radii": M, "resamples": T,
                   "l2": "flushed between timed steps (256 MB write)"},
        "pair_dists_per_s": pairs / (cil_avg * 1e-3),
        "cil_pairs_rechecked_exactly": nre,
        "stepper_variant": variant,
        "stepper_ms": k_avg_ms,
        "cil_ms": cil_avg,
        "synlik_ms": sum(syn_ms) / len(syn_ms),
        "graph_replay_ms_per_step": graph_ms,
        "e2e": {"value": whole_job_rate(cell_updates, world, e2e_ms), "unit": "cell-updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_alu, "unit": "Tinst/s",
                     "frac": achieved / peak_alu,
                     "traffic": stepper_traffic() if variant == 0 and args.config == "c2" else None,
                     "kernel": kname,
                     "note": "FP32 pipe instructions of the update (FHN 15, GM 20, BZ 22 per cell-update) x "
                             "cell-updates / stepper time; peak = 148 SM x 128 FP32 lanes x max SM clock "
                             "(%s peaks file)" % src},
        "plain_fp32_path_cell_updates_per_s": ref_rate,
        "batched_vs_plain": (cell_updates / (k_avg_ms * 1e-3)) / ref_rate if ref_rate else None,
    }
    cs = clk.summary()
    if cs:
        out["clocks"] = cs
    if args.gram_large and rank == 0:
        out["gram_large"] = gram_large(p, torch, dev, stream, pk, src)
    if args.adjoint and rank == 0:
        out["adjoint"] = adjoint_c5(p, torch, dev, stream)
    if args.mcil and rank == 0:
        out["mcil"] = mcil_bench(p, torch, dev, stream)
        out["scil"] = scil_bench(p, torch, dev, stream)
    if args.stream and rank == 0:
        out["stream"] = stream_bench(p, torch, dev, stream, pk, src)
    if args.rkc and rank == 0:
        out["rkc"] = rkc_bench(p, torch, dev, stream, pk, src)
    if args.imex and rank == 0:
        out["imex"] = imex_bench(p, torch, dev, stream, pk, src)
    return out


def _check_int(p, sim, pipe):
    """rd_integrate_batch with the pipeline's residual buffer."""
    import ctypes
    st = p.lib().rd_integrate_batch(sim.handle, ctypes.c_void_p(sim.fields.data_ptr()), -1,
                                    ctypes.c_void_p(pipe.residual.data_ptr()),
                                    ctypes.c_void_p(__import__("torch").cuda.current_stream().cuda_stream))
    if st != 0:
        raise RuntimeError("rd_integrate_batch failed: %d" % st)


def gram_large(p, torch, dev, stream, pk, src):
    """Tensor-core Gram at the paper's SCIL scale (N_syn = 1000): 2 sets x
    1024 patterns of d = 32768 (GM 128x128 both species, synthetic cosine
    fields), plus the whole correlation integral on them."""
    n, G = 1024, 128
    X = torch.from_numpy(W.cosine_patterns(2 * n, G, 2, 77, amp=0.8, offset=2.0)).to(dev)
    X1, X2 = X[:n], X[n:]
    d = X.shape[1]
    c = p.cil(X1, X2, b=1.3, M=16)          # packs the workspace (and warms up)
    torch.cuda.synchronize()
    reps = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fl = p.gram_only(n, n, d, dev)
    e1.record(stream)
    torch.cuda.synchronize()
    t_gram = e0.elapsed_time(e1) / reps * 1e-3
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(reps):
        c = p.cil(X1, X2, b=1.3, M=16)
    c1.record(stream)
    torch.cuda.synchronize()
    t_cil = c0.elapsed_time(c1) / reps * 1e-3
    tf = fl / t_gram / 1e12                  # bf16 MMA work executed: 3 products per element pair
    alg = 2.0 * n * n * d / t_gram / 1e12    # algorithmic: one product per element pair
    return {"pairs": n * n, "d": d, "gram_ms": t_gram * 1e3,
            "gram_tflops_executed": tf, "gram_tflops_algorithmic": alg,
            "peak_bf16_tflops": pk["bf16_tflops"], "frac_of_peak": tf / pk["bf16_tflops"],
            "frac_of_peak_algorithmic": alg / pk["bf16_tflops"],
            "frac_of_sustained_peak": tf / pk.get("bf16_tflops_sustained", pk["bf16_tflops"]),
            "peak_note": "bf16 dense burst peak (%s peaks file); executed = hi.hi + hi.lo + lo.hi bf16 "
                         "products (3 x 2 n1 n2 d flops), algorithmic = 2 n1 n2 d" % src,
            "cil_ms": t_cil * 1e3, "pair_dists_per_s": n * n / t_cil,
            "rechecked": int(c["n_rechecked"])}


def stream_bench(p, torch, dev, stream, pk, src, depths=(1, 2, 4, 8)):
    """Streaming stepper on FHN 512x512, 128 realisations (268 MB of fields,
    above L2): 64 Euler steps per depth.  Algorithmic HBM bytes per launch =
    the fields read and written once (16 B per cell), so 16/S B per
    cell-update at depth S."""
    G, n, steps = 512, 128, 64
    g = p.Group(W.FHN, G, n, (2.8e-4, 0.05, 10.0, 0.95), 2.0 ** -16, steps, (-0.05, 0.05), 4242)
    sim = p.Simulation([g], device=dev)
    cells = n * G * G
    out = []
    for S in depths:
        sim.set_stream_depth(S)
        sim.reinit()
        sim.integrate(residual=False)
        torch.cuda.synchronize()
        reps = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            sim.integrate(residual=False)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps * 1e-3
        launches = (steps + S - 1) // S
        gbs = 16.0 * cells * launches / t / 1e9
        out.append({"depth": S, "ms": t * 1e3, "cell_updates_per_s": cells * steps / t,
                    "hbm_algorithmic_gbs": gbs, "hbm_frac": gbs / pk["hbm_gbs"],
                    "bytes_per_cell_update": 16.0 / S})
    assert sim.sync_status() == 0
    return {"workload": "FHN 512x512, 128 realisations, 64 Euler steps (dt 2^-16)", "peak_hbm_gbs": pk["hbm_gbs"],
            "peak_note": "%s peaks file; achieved = 16 B per cell per launch / time" % src, "depths": out}


# FP32 instructions per cell per RHS stage of the adaptive RK2 kernel (FHN):
# stage state Y_0 + D 2, 5-point sums 6, Laplacian centre terms 2,
# kinetics u 3 (a*a, a - b, fma), v 1, increment recurrence u 5 (g0 mul,
# kinetics fma, Laplacian fma, nu fma, mu fma), v 5.
RKC_FP32_INST_PER_CELL_STAGE = {W.FHN: 24}


def rkc_bench(p, torch, dev, stream, pk, src, tols=(1e-5, 1e-6, 1e-7)):
    """Adaptive stabilised second-order RK (App. B.2, Chebyshev
    coefficients) against the explicit Euler stepper on the FHN 64x64
    workload (2 x 64 realisations, integrated to T = 10^4 x 2^-10): time to
    T on the GPU, RHS evaluations, and the accuracy of both on a sample of
    two realisations against an accurate oracle reference (adaptive,
    tolerance 1e-9)."""
    import oracle
    cfg = W.config("c2")
    gd = cfg["groups"][0]
    G, n = gd["G"], gd["n_real"]
    T = gd["dt"] * gd["n_steps"]
    sim = p.Simulation([p.Group.from_dict(gd)], device=dev)
    w0 = sim.group_fields(0)[:2].cpu().numpy()
    ref, _, failed = oracle.rkc_adaptive(gd["model"], gd["params"], T, 1e-3, 1e-9, 1e-9, w0)
    assert failed == 0

    def rel(a):
        a = np.asarray(a, np.float64)
        num = np.abs(a - ref).reshape(2, 2, -1).max(-1)
        return float((num / np.abs(ref).reshape(2, 2, -1).max(-1)).max())

    def timed(fn, reps=3):
        ts = []
        for _ in range(reps + 1):
            sim.reinit()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        return min(ts[1:]), r

    t_eul, _ = timed(lambda: sim.integrate(residual=False))
    assert sim.sync_status() == 0
    err_eul = rel(sim.group_fields(0)[:2].cpu().numpy())
    peak_alu = 148 * 128 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    # fixed schedule (no step control): the pure per-stage cost, per tile
    # shape; the fastest shape is kept for the adaptive rows that follow
    s_fix, n_fix = 16, 128
    shapes = []
    for v in range(p.lib().rd_rkc_n_variants()):
        p.rkc_set_variant(G, v)
        tv, _ = timed(lambda: sim.integrate_rkc(0.1, s_fixed=s_fix, n_fixed=n_fix))
        shapes.append({"variant": v, "us_per_stage": tv * 1e6 / (1 + s_fix * n_fix)})
    best = min(range(len(shapes)), key=lambda i: shapes[i]["us_per_stage"])
    p.rkc_set_variant(G, best)
    t_fix, _ = timed(lambda: sim.integrate_rkc(0.1, s_fixed=s_fix, n_fixed=n_fix))
    assert sim.sync_status() == 0
    n_rhs = n * (1 + s_fix * n_fix)
    inst = n_rhs * G * G * RKC_FP32_INST_PER_CELL_STAGE[gd["model"]]
    fixed = {"s": s_fix, "steps": n_fix, "h": 0.1, "ms": t_fix * 1e3, "variant": best, "shapes": shapes,
             "us_per_stage": t_fix * 1e6 / (1 + s_fix * n_fix),
             "cell_stage_updates_per_s": n_rhs * G * G / t_fix, "alu_tinst_per_s": inst / t_fix / 1e12,
             "alu_frac": inst / t_fix / 1e12 / peak_alu}
    rows = []
    for tol in tols:
        t, (st, _) = timed(lambda: sim.integrate_rkc(1e-3, rtol=tol, atol=tol))
        assert sim.sync_status() == 0
        st = st.cpu().numpy()
        err = rel(sim.group_fields(0)[:2].cpu().numpy())
        n_rhs = int(st[:, 2].sum())
        inst = n_rhs * G * G * RKC_FP32_INST_PER_CELL_STAGE[gd["model"]]
        rows.append({"tol": tol, "ms": t * 1e3, "steps_mean": float(st[:, 0].mean()),
                     "rejected_mean": float(st[:, 1].mean()), "rhs_mean": float(st[:, 2].mean()),
                     "s_max_used": int(st[:, 3].max()), "rel_err_sample": err,
                     "cell_stage_updates_per_s": n_rhs * G * G / t,
                     "alu_tinst_per_s": inst / t / 1e12, "alu_frac": inst / t / 1e12 / peak_alu,
                     "speedup_vs_euler": t_eul / t, "as_accurate_as_euler": err <= err_eul})
    rdode = rdode_c7(p, torch, dev, stream)
    c3 = rkc_c3(p, torch, dev, stream)
    # the FP64 oracle's adaptive run of a sample of c2 realisations on the
    # host, at the middle tolerance
    n_s, tol_s = 4, 1e-6
    w0s = oracle.init_fields(gd["model"], G, n_s, gd["params"], gd["noise"][0], gd["noise"][1], gd["seed"])
    t0 = time.perf_counter()
    _, _, failed = oracle.rkc_adaptive(gd["model"], gd["params"], T, 1e-3, tol_s, tol_s, w0s)
    t_o = time.perf_counter() - t0
    assert failed == 0
    row_s = [r for r in rows if r["tol"] == tol_s][0]
    cpu = {"kind": "oracle", "sample": "%d realisations of c2 to T at tol %g" % (n_s, tol_s), "s": t_o,
           "cores": oracle.threads(), "realisations_per_s": n_s / t_o,
           "gpu_realisations_per_s": n / (row_s["ms"] * 1e-3)}
    return {"workload": "FHN 64x64, 2 x 64 realisations, 0 -> T = 10^4 x 2^-10 (the c2 horizon)",
            "rdode_c7": rdode,
            "gm128_c3": c3,
            "cpu_baseline": cpu,
            "fixed_schedule": fixed,
            "euler": {"ms": t_eul * 1e3, "steps": gd["n_steps"], "rel_err_sample": err_eul},
            "reference": "oracle adaptive, tolerance 1e-9, realisations 0 and 1",
            "peak_note": "alu peak = 148 SM x 128 FP32 lanes x max SM clock (%s peaks file); "
                         "%d FP32 instructions per cell per RHS stage" % (src, RKC_FP32_INST_PER_CELL_STAGE[gd["model"]]),
            "tolerances": rows}


def imex_bench(p, torch, dev, stream, pk, src, dts=(2 ** -6, 2 ** -5, 2 ** -4)):
    """Semi-implicit Euler (diffusion implicit through the cosine basis,
    reaction explicit) against the explicit Euler stepper on the FHN 64x64
    workload (2 x 64 realisations) to the same horizon T = 10^4 x 2^-10:
    time on the GPU, FP32 FMA rate of the products against the FP32 peak,
    and the accuracy of two realisations against an accurate oracle
    reference (adaptive RK2, tolerance 1e-9)."""
    import oracle
    cfg = W.config("c2")
    gd = cfg["groups"][0]
    G, n = gd["G"], gd["n_real"]
    T = gd["dt"] * gd["n_steps"]
    sim = p.Simulation([p.Group.from_dict(gd)], device=dev)
    w0 = sim.group_fields(0)[:2].cpu().numpy()
    ref, _, failed = oracle.rkc_adaptive(gd["model"], gd["params"], T, 1e-3, 1e-9, 1e-9, w0)
    assert failed == 0

    def rel(a):
        a = np.asarray(a, np.float64)
        num = np.abs(a - ref).reshape(2, 2, -1).max(-1)
        return float((num / np.abs(ref).reshape(2, 2, -1).max(-1)).max())

    def timed(s_, fn, reps=3):
        ts = []
        for _ in range(reps + 1):
            s_.reinit()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        return min(ts[1:]), r

    t_eul, _ = timed(sim, lambda: sim.integrate(residual=False))
    assert sim.sync_status() == 0
    err_eul = rel(sim.group_fields(0)[:2].cpu().numpy())
    fma_peak = 148 * 128 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12   # T FMA/s
    rows = []
    for dt in dts:
        steps = int(round(T / dt))
        gi = dict(gd, dt=dt, n_steps=steps)
        s2 = p.Simulation([p.Group.from_dict(gi)], device=dev)
        t, res = timed(s2, lambda: s2.integrate_imex(residual=True))
        assert s2.sync_status() == 0
        err = rel(s2.group_fields(0)[:2].cpu().numpy())
        # four G^3 products per species and step; the even/odd split (variant
        # 4) forms each from two half-length sums: half the FMAs
        fma = (4.0 if p.imex_get_variant(G) == 4 else 8.0) * G ** 3 * n * steps
        rows.append({"dt": dt, "steps": steps, "ms": t * 1e3, "us_per_step": t * 1e6 / steps,
                     "cell_updates_per_s": n * G * G * steps / t,
                     "product_tfma_per_s": fma / t / 1e12, "fma_frac": fma / t / 1e12 / fma_peak,
                     "rel_err_sample": err, "speedup_vs_euler": t_eul / t,
                     "residual_max": float(res[:, 0].max())})
    # the long run (Sec. 5.1: the RD models are integrated to t = 100, by
    # then at their steady state for the paper's parameters): Euler at its
    # dt against the semi-implicit step at 2^-4 from the same initial
    # states, on c2's FHN and on GM 64x64 with c3's parameters
    T100, dt_i = 100.0, 2 ** -4
    c3g = W.config("c3")["groups"][0]
    long_runs = []
    for name, gl in (("FHN 64x64 (c2)", dict(gd)),
                     ("GM 64x64 (c3's parameters)", dict(c3g, G=64, n_real=128, dt=2 ** -8))):
        nl = gl["n_real"]
        se = p.Simulation([p.Group.from_dict(dict(gl, n_steps=int(round(T100 / gl["dt"]))))], device=dev)
        t_e, res_e = timed(se, lambda: se.integrate(residual=True), reps=1)
        fe = se.group_fields(0).cpu().numpy().astype(np.float64)
        si = p.Simulation([p.Group.from_dict(dict(gl, dt=dt_i, n_steps=int(round(T100 / dt_i))))], device=dev)
        t_i, res_i = timed(si, lambda: si.integrate_imex(residual=True), reps=1)
        fi = si.group_fields(0).cpu().numpy().astype(np.float64)
        dif = (np.abs(fe - fi).reshape(nl, 2, -1).max(-1) / np.abs(fe).reshape(nl, 2, -1).max(-1)).max(-1)
        long_runs.append({"workload": name, "t_end": T100, "euler_dt": gl["dt"], "euler_ms": t_e * 1e3,
                          "imex_dt": dt_i, "imex_ms": t_i * 1e3, "speedup": t_e / t_i,
                          "euler_residual_max": float(res_e[:, 0].max()),
                          "imex_residual_max": float(res_i[:, 0].max()),
                          "same_pattern_1e-3": int((dif < 1e-3).sum()), "realisations": nl,
                          "rel_diff_median": float(np.median(dif))})
    return {"workload": "FHN 64x64, 2 x 64 realisations, 0 -> T = 10^4 x 2^-10 (the c2 horizon)",
            "t100": long_runs,
            "variant": p.imex_get_variant(G),
            "euler": {"ms": t_eul * 1e3, "steps": gd["n_steps"], "dt": gd["dt"], "rel_err_sample": err_eul},
            "reference": "oracle adaptive RK2, tolerance 1e-9, realisations 0 and 1",
            "peak_note": "FMA peak = 148 SM x 128 FP32 lanes x max SM clock (%s peaks file); the "
                         "products take 128 of the 148 SMs (one CTA per realisation)" % src,
            "rows": rows}


def rkc_c3(p, torch, dev, stream, tols=(1e-5, 1e-6)):
    """The GM 128x128 workload c3 (2 x 256 realisations, to T = 2*10^4 x
    2^-10): Euler against the adaptive stabilised RK2 (one 4-CTA cluster
    per realisation), accuracy of two realisations against an accurate
    oracle reference (adaptive, tolerance 1e-9)."""
    import oracle
    cfg = W.config("c3")
    gd = cfg["groups"][0]
    T = gd["dt"] * gd["n_steps"]
    sim = p.Simulation([p.Group.from_dict(gd)], device=dev)
    w0 = sim.group_fields(0)[:2].cpu().numpy()
    ref, _, failed = oracle.rkc_adaptive(gd["model"], gd["params"], T, 1e-3, 1e-9, 1e-9, w0)
    assert failed == 0

    def rel(a):
        a = np.asarray(a, np.float64)
        num = np.abs(a - ref).reshape(2, 2, -1).max(-1)
        return float((num / np.abs(ref).reshape(2, 2, -1).max(-1)).max())

    def timed(fn, reps=2):
        ts = []
        for _ in range(reps + 1):
            sim.reinit()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        return min(ts[1:]), r

    t_eul, _ = timed(lambda: sim.integrate(residual=False))
    assert sim.sync_status() == 0
    err_eul = rel(sim.group_fields(0)[:2].cpu().numpy())
    rows = []
    for tol in tols:
        t, (st, _) = timed(lambda: sim.integrate_rkc(1e-3, rtol=tol, atol=tol))
        assert sim.sync_status() == 0
        st = st.cpu().numpy()
        rows.append({"tol": tol, "ms": t * 1e3, "steps_mean": float(st[:, 0].mean()),
                     "rhs_mean": float(st[:, 2].mean()), "rel_err_sample": rel(sim.group_fields(0)[:2].cpu().numpy()),
                     "cell_stage_updates_per_s": float(st[:, 2].sum()) * gd["G"] ** 2 / t,
                     "speedup_vs_euler": t_eul / t})
    return {"workload": "GM 128x128, 2 x 256 realisations, 0 -> T = 2*10^4 x 2^-10 (c3)",
            "euler": {"ms": t_eul * 1e3, "steps": gd["n_steps"], "rel_err_sample": err_eul},
            "tolerances": rows}


def rdode_c7(p, torch, dev, stream):
    """The 1-D reaction-diffusion-ODE workload c7 (Sec. 4.3, Table 1: 64
    nodes, t in [0, 50], 2 x 100 realisations), adaptive stabilised RK2 at
    the configured tolerance, one warp per realisation; the oracle's FP64
    run of a sample of realisations on the host for comparison."""
    import oracle
    cfg = W.config("c7")
    gd = cfg["groups"][0]
    tol = cfg["rkc_tol"]
    sim = p.Simulation([p.Group.from_dict(gd)], device=dev)
    ts = []
    for _ in range(4):
        sim.reinit()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, _ = sim.integrate_rkc(1e-3, rtol=tol, atol=tol)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    assert sim.sync_status() == 0
    t = min(ts[1:])
    st = st.cpu().numpy()
    n, N = gd["n_real"], gd["G"]
    # the rest of a likelihood evaluation on these patterns (both species,
    # d = 2N): CIL with Table 1's linear radii law, M = 13, and the
    # synthetic-likelihood statistics of 200 resampled set pairs
    X = sim.group_fields(0).reshape(n, 2 * N)
    half = n // 2
    tl = []
    for _ in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c = p.cil_linear(X[:half], X[half:], M=cfg["M"])
        sl = p.synlik(c["bins"], cfg["M"], cfg["T_res"], cfg["seed"])
        e1.record(stream)
        torch.cuda.synchronize()
        tl.append(e0.elapsed_time(e1) * 1e-3)
    t_lik = min(tl[1:])
    sample = 8
    w0 = oracle.rdode_init(N, sample, gd["noise"][0], gd["noise"][1], gd["seed"], 10)
    T = gd["dt"] * gd["n_steps"]
    t0 = time.perf_counter()
    _, ost, failed = oracle.rkc_adaptive(W.RDODE, gd["params"], T, 1e-3, tol, tol, w0)
    t_orc = time.perf_counter() - t0
    return {"workload": "RD-ODE 64 nodes, 200 realisations, t in [0, 50], tol %g" % tol, "ms": t * 1e3,
            "cil_linear_synlik_ms": t_lik * 1e3, "counts": c["counts"].cpu().numpy().tolist(),
            "realisations_per_s": n / t, "steps_mean": float(st[:, 0].mean()), "rhs_mean": float(st[:, 2].mean()),
            "cell_stage_updates_per_s": float(st[:, 2].sum()) * 2 * N / t,
            "oracle_sample": {"realisations": sample, "s": t_orc, "realisations_per_s": sample / t_orc,
                              "threads": oracle.threads(), "steps_mean": float(ost[:, 0].mean())}}


def mcil_bench(p, torch, dev, stream):
    """Multi-feature correlation integral (L2, Linf, W12, W12', W1inf,
    W1inf'; Sec. 3.1) on synthetic cosine-mode fields of two set shapes:
    2 x 64 patterns of one 64x64 species and 2 x 256 of two 128x128
    species; raw and min-max scaled."""
    res = []
    for (n, G, nsp) in ((64, 64, 1), (256, 128, 2)):
        X = torch.from_numpy(W.cosine_patterns(2 * n, G, nsp, 91, amp=0.8, offset=1.0)).to(dev)
        for scale in (False, True):
            work = p.mcil_workspace(n, n, G, nsp, 63, scale, 16, dev)
            r = p.mcil(X[:n], X[n:], G, nsp, b=1.3, M=16, scale=scale, work=work)
            torch.cuda.synchronize()
            reps = 5
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                r = p.mcil(X[:n], X[n:], G, nsp, b=1.3, M=16, scale=scale, work=work)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / reps * 1e-3
            res.append({"pairs": n * n, "G": G, "species": nsp, "d": nsp * G * G, "scaled": scale,
                        "features": 6, "ms": t * 1e3, "pair_features_per_s": 6 * n * n / t,
                        "exact_pairs": int(r["n_exact"])})
    return res


def scil_bench(p, torch, dev, stream):
    """The synthetic-likelihood cost after the simulations, at the paper's
    SCIL scale (Alg. 6 with bootstrapping, Sec. 5.1: N_syn = 1000 patterns,
    N_set = 50 of them against the other 950, n_CIL = 1000 resampled set
    pairs, the six features): multi-feature CIL of GM-sized fields (2 species
    of 128x128, synthetic cosine modes), then bootstrap counts of the
    96-component vector and its statistics (tensor-core and SIMT counts)."""
    n_syn, n_set, G, nsp, M, T = 1000, 50, 128, 2, 16, 1000
    X = torch.from_numpy(W.cosine_patterns(n_syn, G, nsp, 93, amp=0.8, offset=2.0)).to(dev)
    X1, X2 = X[:n_set], X[n_set:]
    n2 = n_syn - n_set
    work = p.mcil_workspace(n_set, n2, G, nsp, 63, False, M, dev)
    swork = p.synlik_workspace(n_set, n2, M, T, 6, 1, dev)
    sout = p.synlik_outputs(1, 6 * M, T, dev)
    r = p.mcil(X1, X2, G, nsp, b=1.3, M=M, work=work)
    bins = r["bins"].unsqueeze(0).contiguous()
    yobs = r["C"].unsqueeze(0).contiguous()
    p.synlik(bins, M, T, 2203, y_obs=yobs, n_feat=6, work=swork, out=sout)
    torch.cuda.synchronize()

    def timed(fn, reps=5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_mcil = timed(lambda: p.mcil(X1, X2, G, nsp, b=1.3, M=M, work=work))
    t_syn = timed(lambda: p.synlik(bins, M, T, 2203, y_obs=yobs, n_feat=6, work=swork, out=sout))
    Y_tc = sout["Y"].clone()
    t_simt = timed(lambda: p.synlik(bins, M, T, 2203, y_obs=yobs, n_feat=6, out=sout, simt=True), reps=2)
    return {"n_syn": n_syn, "n_set": n_set, "d": nsp * G * G, "features": 6, "M": M, "n_cil": T,
            "mcil_ms": t_mcil, "bootstrap_stats_ms": t_syn, "bootstrap_stats_simt_ms": t_simt,
            "same_counts": bool(torch.equal(Y_tc, sout["Y"])), "status": int(sout["status"][0]),
            "cost_f": float(sout["scalars"][0, 1]), "total_ms": t_mcil + t_syn}


def adjoint_c5(p, torch, dev, stream):
    """Smoothed-CIL gradient (discrete adjoint with sqrt(N) checkpoints) on
    the FHN 64x64 adjoint workload: 32 realisations (2 x 16), 5000 steps,
    M = 16 radii from the unperturbed run, tau_k = 0.05 R_k, cotangent 1/M."""
    cfg = W.config("c5")
    gd = dict(cfg["groups"][0])
    sim = p.Simulation([p.Group.from_dict(gd, adjoint=True)], device=dev)
    f0 = sim.fields.clone()
    n, G, N = gd["n_real"], gd["G"], gd["n_steps"]
    sim.integrate()
    X = sim.fields.view(n, 2 * G * G)[:, :G * G] if gd["species_mask"] == 1 else sim.fields.view(n, 2 * G * G)
    half = n // 2
    c = p.cil(X[:half], X[half:], b=cfg["b"], M=cfg["M"])
    radii = c["radii"].clone()
    cot = torch.full((cfg["M"],), 1.0 / cfg["M"], dtype=torch.float64, device=dev)
    s1, s2 = list(range(half)), list(range(half, n))
    sim.adjoint(0, f0, gd["species_mask"], s1, s2, radii, cfg["tau_frac"], cot)   # warm-up
    torch.cuda.synchronize()
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        Cv, g = sim.adjoint(0, f0, gd["species_mask"], s1, s2, radii, cfg["tau_frac"], cot)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / reps * 1e-3
    C = math.ceil(math.sqrt(N))
    cells = n * G * G * N
    ckpt = (math.ceil(N / C) * n + C * n) * 2 * G * G * 4
    return {"workload": "FHN 64x64, 32 realisations, 5000 steps, M=16, tau=0.05 R_k",
            "ms": t * 1e3, "trajectory_cell_updates_per_s": cells / t,
            "executed_cell_updates_per_s": 3 * cells / t,
            "note": "one trajectory = n G^2 N cell-updates; the adjoint executes 3 passes of it (recording "
                    "forward, segment recompute, reverse)",
            "checkpoint_bytes": ckpt, "segment": C, "grad": [float(x) for x in g.cpu()]}


# ---------------------------------------------------------------------------
# oracle (CPU) arm / baseline
# ---------------------------------------------------------------------------
def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo), or None."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def oracle_sample(cfg, n_steps_sample):
    """Time the oracle on a bounded sample: all realisations for
    n_steps_sample Euler steps (scaled to the full step count), plus the full
    CIL and bootstrap statistics.  Returns (cell-updates/s, seconds, note)."""
    import oracle
    g = cfg["groups"][0]
    G, n = g["G"], g["n_real"]
    t0 = time.perf_counter()
    f0 = oracle.init_fields(g["model"], G, n, g["params"], g["noise"][0], g["noise"][1], g["seed"])
    f = oracle.step(g["model"], g["params"], g["dt"], n_steps_sample, f0.astype(np.float64))
    oracle.residual(g["model"], g["params"], f)
    t_step = time.perf_counter() - t0
    t1 = time.perf_counter()
    X = oracle.patterns(f.astype(np.float32), g["species_mask"])
    o = oracle.cil(X[:cfg["n1"]], X[cfg["n1"]:cfg["n1"] + cfg["n2"]], b=cfg["b"], M=cfg["M"])
    oracle.synlik(o["bins"], cfg["M"], cfg["T_res"], cfg["seed"], y_obs=o["counts"] / (cfg["n1"] * cfg["n2"]))
    t_cil = time.perf_counter() - t1
    full_cells = n * G * G * g["n_steps"]
    t_full = t_step * (g["n_steps"] / n_steps_sample) + t_cil
    if n_steps_sample >= g["n_steps"]:
        note = ("the whole workload: all %d realisations x %d Euler steps + CIL + bootstrap statistics"
                % (n, g["n_steps"]))
    else:
        note = ("all %d realisations x %d of %d Euler steps (stepping time scaled by %.0fx) + full CIL "
                "and bootstrap statistics" % (n, n_steps_sample, g["n_steps"], g["n_steps"] / n_steps_sample))
    return full_cells / t_full, t_step + t_cil, note


def run_reference(args):
    import oracle
    cfg = W.config(args.config)
    # each step is the whole workload (about 5 s on 16 cores) while the run
    # stays within a few minutes; beyond 20 steps a proportional sample
    n_full = cfg["groups"][0]["n_steps"]
    n_sample = n_full if args.steps + args.warmup <= 20 else max(1000, n_full * 20 // (args.steps + args.warmup))
    oracle_sample(cfg, 10)           # warm (builds the library)
    vals, secs = [], 0.0
    for _ in range(args.warmup):
        oracle_sample(cfg, n_sample)
    for _ in range(args.steps):
        v, s, note = oracle_sample(cfg, n_sample)
        vals.append(v)
        secs += s
    value = statistics.mean(vals)
    cores = oracle.threads()
    g = cfg["groups"][0]
    return {
        "impl": "reference",
        "metric": "RD cell-updates/s + CIL pair-dists/s at stated tol; % HBM/tensor roofline",
        "value": value, "unit": "cell-updates/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": g["n_real"] * g["G"] ** 2 * g["n_steps"] / value * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "c2: FHN 64x64, 2 sets x 64 realisations, 10^4 Euler steps, "
                               "u-only d=4096, M=16, b=1.3, 200 resamples"},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": note},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args)))
        return
    if args.stream_only:
        import torch
        import paper_2203_14742_b300 as p
        from paper_2203_14742_b300 import build as B
        B.build()
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        pk, src = peaks()
        print(json.dumps(stream_bench(p, torch, dev, torch.cuda.current_stream(dev), pk, src)))
        return
    if args.mcil_only:
        import torch
        import paper_2203_14742_b300 as p
        from paper_2203_14742_b300 import build as B
        B.build()
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        st_ = torch.cuda.current_stream(dev)
        print(json.dumps({"mcil": mcil_bench(p, torch, dev, st_), "scil": scil_bench(p, torch, dev, st_)}))
        return
    if args.rkc_only:
        import torch
        import paper_2203_14742_b300 as p
        from paper_2203_14742_b300 import build as B
        B.build()
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        pk, src = peaks()
        print(json.dumps(rkc_bench(p, torch, dev, torch.cuda.current_stream(dev), pk, src)))
        return
    if args.imex_only:
        import torch
        import paper_2203_14742_b300 as p
        from paper_2203_14742_b300 import build as B
        B.build()
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        pk, src = peaks()
        print(json.dumps(imex_bench(p, torch, dev, torch.cuda.current_stream(dev), pk, src)))
        return
    if args.gram_large_only:
        import torch
        import paper_2203_14742_b300 as p
        from paper_2203_14742_b300 import build as B
        B.build()
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        pk, src = peaks()
        print(json.dumps(gram_large(p, torch, dev, torch.cuda.current_stream(dev), pk, src)))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world, local_rank)
    if rank == 0 and not args.no_cpu_baseline:
        cfg = W.config(args.config)
        v, secs, note = oracle_sample(cfg, cfg["groups"][0]["n_steps"])
        import oracle
        cores = oracle.threads()
        # one thread, on a sixteenth of the steps (stepping time scaled)
        oracle.set_threads(1)
        v1, secs1, note1 = oracle_sample(cfg, max(1, cfg["groups"][0]["n_steps"] // 16))
        oracle.set_threads(cores)
        out["cpu_baseline"] = {"value": v, "unit": "cell-updates/s", "cores": cores,
                               "kind": "oracle", "sample": note + " (%.1f s of CPU work)" % secs,
                               "one_thread": {"value": v1, "sample": note1 + " (%.1f s)" % secs1},
                               "cpu_model": cpu_model()}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
