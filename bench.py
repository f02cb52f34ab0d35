"""Benchmark of the CIL hot path on B300 (one JSON line on rank 0).

One step = one pass of the whole hot path over one batch of synthetic input.
The default workload is the largest single-GPU configuration, the batched
sampler sweep: 64 parameter vectors x 128 realisations, FHN and GM on 64x64
(10^4 Euler steps) and 128x128 (2x10^4 steps) in one persistent launch,
then per parameter vector the correlation integral of 2 sets x 64 patterns
(16 radii) and the bootstrap statistics (200 resamples):
  initial state -> integration (+ FP64 residual) -> pattern Gram + exact
  recheck -> radii / bins / counts -> bootstrap counts -> mean, covariance,
  Cholesky, log-determinant, cost and log-likelihood.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config c4|c2|...]

value  = cell-updates per second of the whole step (a cell-update = one grid
         node, both species, one time step), device-timed with CUDA events,
         max over ranks, inputs resident in HBM.
e2e    = the same through the public API with host buffers: every step
         copies the initial fields host->device and the statistics back.
The default run adds keys for the FHN 64x64 workload (c2), the tensor-core
Gram at the paper's SCIL scale, the streaming stepper against HBM, the
adjoint (c5) and one whole synthetic-likelihood cost evaluation (Alg. 6,
workload c8).
--impl reference runs the plain FP64 CPU oracle on a bounded sample of the
same workload (every group, a stated slice of its steps; rank 0 only).
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

# resident stepper kernel of each tile kind (rd_variant_shape)
RESIDENT_KERNEL = {0: "rd_resident_scalar_kernel", 1: "rd_resident_kernel", 2: "rd_resident_rot_kernel",
                   3: "rd_resident_rot2_kernel"}

# DRAM bytes (read + write) of one launch of the dominant kernel, from an ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum), keyed by workload
# (with ":v<n>" for a resident tile variant other than 0) and a hash of the
# stepper sources: reported, labelled as that capture's,
# only while the kernel is the one that was measured.  The resident and
# persistent steppers read the initial fields and write the final ones once
# per launch whatever the step count, so a capture of a shortened run gives
# the full launch's traffic.
STEPPER_TRAFFIC = {
    "c2": {"6f89ac52bd0c99eb": 4223232, "a1b8429f6f299483": 4223488, "7c8c62601c860730": 4223488,
           "60c7c52369dee980": 4297216, "bf9071c73da591c1": 4297216, "730afce9ca60e453": 4314112,
           "3af7521f7d8ea050": 4278016, "4a973e1119f01943": 4244480},
    "c2:v3": {"730afce9ca60e453": 4223488, "3af7521f7d8ea050": 4301312, "4a973e1119f01943": 4239872},
    "c4": {"250da058b95b29c7": 1285591296, "02a4865c70d95aa1": 1284856064, "60c7c52369dee980": 1290298112,
           "bf9071c73da591c1": 1290150912, "730afce9ca60e453": 1291938816,
           "3af7521f7d8ea050": 1289928192, "4a973e1119f01943": 1290087168},
}
STEPPER_SOURCES = ["paper_2203_14742_b300/csrc/stepper.cu", "paper_2203_14742_b300/csrc/tile.cuh",
                   "paper_2203_14742_b300/csrc/common.cuh"]


def sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in STEPPER_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stepper_traffic(config):
    """(bytes, source label) of the committed capture for this workload and
    the current stepper sources, or (None, reason)."""
    hs = sources_hash()
    v = STEPPER_TRAFFIC.get(config, {}).get(hs)
    if v is None:
        return None, "no ncu capture of the current stepper sources (hash %s) on this workload" % hs
    return v, "ncu capture of the stepper sources with hash %s (dram__bytes_read.sum + dram__bytes_write.sum)" % hs


WORKLOADS = {
    "c1": "c1: FHN 32x32, 2 x 16, 2000 steps, d=2048, M=8, 50 resamples",
    "c2": "c2: FHN 64x64, 2 sets x 64 realisations, 10^4 Euler steps, u-only d=4096, M=16, b=1.3, "
          "200 resamples",
    "c3": "c3: GM 128x128, 2 x 256, 2x10^4 steps, d=32768, M=16, 200 resamples",
    "c4": "c4: 64 parameter vectors x 128 realisations, FHN+GM at 64^2 (10^4 steps) and 128^2 "
          "(2x10^4 steps) in one persistent launch, 2 x 64 sets per vector, M=16, b=1.3, 200 resamples",
    "c5": "c5: FHN 64x64, 32 realisations, 5000 steps",
    "c6": "c6: Brusselator 64x64, 2 sets x 64 realisations, 25600 Euler steps (T = 100), both "
          "species d=8192, M=16, b=1.3, 200 resamples",
}


def config_json(name, cfg):
    """The `config` object of the JSON line (both arms)."""
    groups = cfg["groups"]
    return {"workload": WORKLOADS[name], "groups": len(groups),
            "realisations_per_gpu": sum(g["n_real"] for g in groups),
            "grids": sorted(set(g["G"] for g in groups)), "pairs": cfg["n1"] * cfg["n2"] * len(groups),
            "radii": cfg["M"], "resamples": cfg["T_res"],
            "l2": "flushed between timed steps (256 MB write)"}


L2_BYTES = 126 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c4")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the c2, tensor-core Gram, streaming-stepper, adjoint and SCIL keys of the default run")
    ap.add_argument("--stepper-only", action="store_true",
                    help="initial state and integration only, steps overridden by --steps-override "
                         "(for profiling the stepper on a shortened run)")
    ap.add_argument("--steps-override", type=int, default=-1)
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
            pipe.run_cils()
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

    # ---- plain batched FP32 path (every realisation of a group per launch,
    # one step per launch, state through HBM) on every group, 50 steps -----
    plain_rate = None
    if not args.no_reference_path and rank == 0:
        spl = p.Simulation(groups, device=dev)
        tmp = torch.empty(max(2 * g.G * g.G * g.n_real for g in groups), dtype=torch.float32, device=dev)
        npl = 50
        spl.integrate_plain(steps=5, tmp=tmp)
        torch.cuda.synchronize()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        spl.integrate_plain(steps=npl, tmp=tmp)
        r1.record(stream)
        torch.cuda.synchronize()
        plain_rate = sum(g.n_real * g.G * g.G for g in groups) * npl / (r0.elapsed_time(r1) * 1e-3)
        del spl, tmp

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
        kname = "%s<%s,%d,%dx%d> variant %s" % (RESIDENT_KERNEL[pk_],
                                               {0: "FHN", 1: "GM", 2: "DIFF", 3: "BZ"}[groups[0].model],
                                               groups[0].G, ty_, tx_, variant)
    if multi or variant == 0:
        traffic, tsrc = stepper_traffic(args.config)
    else:
        traffic, tsrc = stepper_traffic("%s:v%d" % (args.config, variant))
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
        "config": config_json(args.config, cfg),
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
                     "traffic": traffic, "traffic_source": tsrc,
                     "kernel": kname,
                     "note": "FP32 pipe instructions of the update (FHN 15, GM 20, BZ 22 per cell-update) x "
                             "cell-updates / stepper time; peak = 148 SM x 128 FP32 lanes x max SM clock "
                             "(%s peaks file)" % src},
        "plain_fp32_path_cell_updates_per_s": ref_rate,
        "batched_vs_plain": (cell_updates / (k_avg_ms * 1e-3)) / ref_rate if ref_rate else None,
        "plain_batched_fp32_path_cell_updates_per_s": plain_rate,
        "batched_vs_plain_batched": (cell_updates / (k_avg_ms * 1e-3)) / plain_rate if plain_rate else None,
        "plain_note": "plain = one Euler step per launch, state through HBM, the same FP32 update; "
                      "single-realisation: one realisation per launch (2 realisations of the first group, "
                      "500 steps); batched: every realisation of a group per launch (every group, 50 steps)",
    }
    cs = clk.summary()
    if cs:
        out["clocks"] = cs
    extras = not args.no_extras and rank == 0
    if extras and args.config != "c2":
        out["c2"] = c2_bench(p, torch, dev, stream, pk, src)
    if (args.gram_large or extras) and rank == 0:
        out["gram_large"] = gram_large(p, torch, dev, stream, pk, src)
    if (args.adjoint or extras) and rank == 0:
        out["adjoint"] = adjoint_c5(p, torch, dev, stream)
    if args.mcil and rank == 0:
        out["mcil"] = mcil_bench(p, torch, dev, stream)
    if (args.mcil or extras) and rank == 0:
        out["scil"] = scil_bench(p, torch, dev, stream)
    if (args.stream or extras) and rank == 0:
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


def stepper_only(p, torch, dev, args):
    """Initial state and integration of the workload's groups only, every
    group advanced --steps-override steps (default: its own step count):
    one warm-up launch, then --steps timed launches (for profiling the
    stepper on a shortened run; the persistent launch's DRAM traffic does
    not depend on the step count)."""
    cfg = W.config(args.config)
    groups = [p.Group.from_dict(gd) for gd in cfg["groups"]]
    sim = p.Simulation(groups, device=dev)
    steps = int(args.steps_override)
    stream = torch.cuda.current_stream(dev)
    sim.integrate(steps=steps, residual=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sim.reinit()
    e0.record(stream)
    for _ in range(max(1, args.steps)):
        sim.integrate(steps=steps, residual=False)
    e1.record(stream)
    torch.cuda.synchronize()
    assert sim.sync_status() == 0
    cells = sum(g.n_real * g.G * g.G * (steps if steps >= 0 else g.n_steps) for g in groups)
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    return {"workload": WORKLOADS[args.config], "steps_override": steps, "ms_per_launch": ms,
            "cell_updates_per_s": cells / (ms * 1e-3)}


def c2_bench(p, torch, dev, stream, pk, src, reps=5):
    """The FHN 64x64 workload (c2: 2 sets x 64 realisations, 10^4 Euler
    steps, u-only patterns, 16 radii, 200 resamples) as a key of the default
    run: whole pass and stepper time (CUDA events, L2 flushed between
    passes), the autotuned tile variant and the stepper against the FP32
    issue peak."""
    cfg = W.config("c2")
    gd = cfg["groups"][0]
    g = p.Group.from_dict(gd)
    pipe = p.Pipeline([g], [(cfg["n1"], cfg["n2"], gd["species_mask"])], cfg["M"], cfg["b"], cfg["T_res"],
                      cfg["seed"], device=dev)
    sim = pipe.sim
    chosen = sim.autotune(steps=300)
    variant = chosen[g.model * 3 + 1]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(3):
        pipe.run()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(reps)]
    for i in range(reps):
        flush.fill_(float(i))
        e = ev[i]
        e[0].record(stream)
        sim.reinit()
        e[1].record(stream)
        _check_int(p, sim, pipe)
        e[2].record(stream)
        pipe.run_cils()
        p.synlik(pipe.bins, cfg["M"], cfg["T_res"], pipe.seed, y_obs=pipe.C, out=pipe.stats, work=pipe.syn_work)
        e[3].record(stream)
    torch.cuda.synchronize()
    assert sim.sync_status() == 0
    step_ms = sum(e[0].elapsed_time(e[3]) for e in ev) / reps
    k_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / reps
    cells = g.n_real * g.G * g.G * g.n_steps
    inst = cells * FP32_INST_PER_CELL[g.model]
    peak = 148 * 128 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    ach = inst / (k_ms * 1e-3) / 1e12
    pk_, ty_, tx_ = p.variant_shape(g.G, variant)
    traffic, tsrc = stepper_traffic("c2" if variant == 0 else "c2:v%d" % variant)
    # accuracy against the oracle: the fields of two realisations after the
    # full step count (FP64 oracle from the same FP32 initial state; per
    # realisation and species max |a - b| / max |b|), and the correlation
    # integral recomputed by the oracle on the GPU's own fields
    import oracle
    sim.reinit()
    w0 = sim.group_fields(0)[:2].cpu().numpy().astype(np.float64)
    _check_int(p, sim, pipe)
    for (X1, X2), o in zip(pipe.views, pipe.cil_out):
        p.cil(X1, X2, b=cfg["b"], M=cfg["M"], work=pipe.work, out=o)
    torch.cuda.synchronize()
    wg = sim.group_fields(0)[:2].cpu().numpy().astype(np.float64).reshape(2, 2, -1)
    wo = oracle.step(g.model, g.params[:4], g.dt, g.n_steps, w0).reshape(2, 2, -1)
    field_err = float((np.abs(wg - wo).max(-1) / np.abs(wo).max(-1)).max())
    X1, X2 = pipe.views[0]
    oc = oracle.cil(X1.cpu().numpy(), X2.cpu().numpy(), b=cfg["b"], M=cfg["M"])
    cil_exact = bool(np.array_equal(pipe.cil_out[0]["counts"].cpu().numpy(), oc["counts"]) and
                     float(pipe.cil_out[0]["radii"][0]) == oc["R0"] and
                     np.array_equal(pipe.cil_out[0]["radii"][1:].cpu().numpy(), oc["radii"]))
    return {"workload": WORKLOADS["c2"], "ms_per_step": step_ms, "cell_updates_per_s": cells / (step_ms * 1e-3),
            "accuracy": {"field_rel_err_2_realisations": field_err, "field_tolerance": 1e-5,
                         "cil_radii_counts_equal_oracle": cil_exact,
                         "note": "fields: FP32 GPU vs FP64 oracle after 10^4 steps from the same initial state; "
                                 "CIL: the oracle's exact counts on the GPU's fields"},
            "stepper_ms": k_ms, "stepper_variant": variant,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Tinst/s", "frac": ach / peak,
                         "traffic": traffic, "traffic_source": tsrc,
                         "kernel": "%s<FHN,64,%dx%d> variant %d" % (
                             RESIDENT_KERNEL[pk_], ty_, tx_, variant)},
            "cil_pairs_rechecked_exactly": int(sum(int(o["n_rechecked"]) for o in pipe.cil_out))}


def gram_large(p, torch, dev, stream, pk, src):
    """Tensor-core Gram at the paper's SCIL scale (N_syn = 1000): 2 sets x
    1024 patterns of d = 32768 (GM 128x128 both species, synthetic cosine
    fields), plus the whole correlation integral on them; the default form
    (three bf16 products, hi.hi + hi.lo + lo.hi) and, for comparison, one
    product (hi.hi, the cross terms in the bound), with the pairs each
    leaves to tiers 2 and 3."""
    n, G = 1024, 128
    X = torch.from_numpy(W.cosine_patterns(2 * n, G, 2, 77, amp=0.8, offset=2.0)).to(dev)
    X1, X2 = X[:n], X[n:]
    d = X.shape[1]
    reps = 5

    def measure():
        c = p.cil(X1, X2, b=1.3, M=16)          # packs the workspace (and warms up)
        torch.cuda.synchronize()
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
        return fl, t_gram, c0.elapsed_time(c1) / reps * 1e-3, p.cil_queue_lengths(n, n, d, dev)

    products = p.gram_products(n, n, d)
    fl, t_gram, t_cil, rech = measure()

    # the HBM-bound shapes (arithmetic intensity n1 n2 / (n1 + n2) below the
    # ridge): c2's 2 x 64 x 4096 and c3's 2 x 256 x 32768, against the HBM
    # roofline on the algorithmic bytes 2 (n1 + n2) d (bf16 patterns once;
    # the kernel reads hi and lo, twice that)
    hbm = []
    for (ns_, G_, nsp_) in ((64, 64, 1), (256, 128, 2)):
        Xs = torch.from_numpy(W.cosine_patterns(2 * ns_, G_, nsp_, 81, amp=0.8, offset=2.0)).to(dev)
        ds = Xs.shape[1]
        p.cil(Xs[:ns_], Xs[ns_:], b=1.3, M=16)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for _ in range(20):
            p.gram_only(ns_, ns_, ds, dev)
        h1.record(stream)
        torch.cuda.synchronize()
        th = h0.elapsed_time(h1) / 20 * 1e-3
        alg_b = 2.0 * 2 * ns_ * ds
        hbm.append({"shape": "2 x %d x %d" % (ns_, ds), "gram_us": th * 1e6,
                    "algorithmic_gbs": alg_b / th / 1e9, "hbm_frac": alg_b / th / 1e9 / pk["hbm_gbs"],
                    "executed_gbs": 2 * alg_b / th / 1e9})
    try:
        p.set_gram_products(1)
        fl1, t_gram1, t_cil1, rech1 = measure()
    finally:
        p.set_gram_products(0)
    tf = fl / t_gram / 1e12                  # bf16 MMA work executed
    alg = 2.0 * n * n * d / t_gram / 1e12    # algorithmic: one product per element pair
    return {"pairs": n * n, "d": d, "products": products, "gram_ms": t_gram * 1e3,
            "gram_tflops_executed": tf, "gram_tflops_algorithmic": alg,
            "peak_bf16_tflops": pk["bf16_tflops"], "frac_of_peak": tf / pk["bf16_tflops"],
            "frac_of_peak_algorithmic": alg / pk["bf16_tflops"],
            "frac_of_sustained_peak": tf / pk.get("bf16_tflops_sustained", pk["bf16_tflops"]),
            "peak_note": "bf16 dense burst peak (%s peaks file); executed = the bf16 products the form "
                         "runs (products x 2 n1 n2 d_padded flops), algorithmic = 2 n1 n2 d" % src,
            "cil_ms": t_cil * 1e3, "pair_dists_per_s": n * n / t_cil,
            "tier2_pairs": rech[0], "exact_pairs": rech[1],
            "hbm_bound_shapes": hbm,
            "one_product": {"gram_ms": t_gram1 * 1e3,
                            "frac_of_peak": fl1 / t_gram1 / 1e12 / pk["bf16_tflops"],
                            "frac_of_peak_algorithmic": 2.0 * n * n * d / t_gram1 / 1e12 / pk["bf16_tflops"],
                            "cil_ms": t_cil1 * 1e3, "tier2_pairs": rech1[0], "exact_pairs": rech1[1]}}


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
    # G = 128 (one 4-CTA cluster per realisation): the GM 128x128 workload
    # c3 (512 realisations) to its horizon, against its explicit Euler run
    # (dt 2^-10, accurate to about 1e-5 there)
    gc3 = W.config("c3")["groups"][0]
    T3 = gc3["dt"] * gc3["n_steps"]
    s3 = p.Simulation([p.Group.from_dict(gc3)], device=dev)
    t_e3, _ = timed(s3, lambda: s3.integrate(residual=False), reps=1)
    assert s3.sync_status() == 0
    fe3 = s3.group_fields(0).cpu().numpy().astype(np.float64)
    n3 = gc3["n_real"]
    g128 = []
    for dt in (2 ** -6, 2 ** -4):
        steps = int(round(T3 / dt))
        si = p.Simulation([p.Group.from_dict(dict(gc3, dt=dt, n_steps=steps))], device=dev)
        t, res = timed(si, lambda: si.integrate_imex(residual=True), reps=2)
        assert si.sync_status() == 0
        fi = si.group_fields(0).cpu().numpy().astype(np.float64)
        dif = (np.abs(fe3 - fi).reshape(n3, 2, -1).max(-1) / np.abs(fe3).reshape(n3, 2, -1).max(-1)).max(-1)
        fma = 4.0 * 128 ** 3 * n3 * steps
        g128.append({"dt": dt, "steps": steps, "ms": t * 1e3, "us_per_step": t * 1e6 / steps,
                     "product_tfma_per_s": fma / t / 1e12, "fma_frac": fma / t / 1e12 / fma_peak,
                     "speedup_vs_euler": t_e3 / t, "rel_diff_vs_euler_median": float(np.median(dif)),
                     "rel_diff_vs_euler_max": float(dif.max()), "residual_max": float(res[:, 0].max())})
    c3_128 = {"workload": "GM 128x128, 512 realisations (c3), 0 -> T = 2*10^4 x 2^-10",
              "kernel": "one 4-CTA cluster per realisation",
              "euler": {"ms": t_e3 * 1e3, "steps": gc3["n_steps"], "dt": gc3["dt"]}, "rows": g128}
    return {"workload": "FHN 64x64, 2 x 64 realisations, 0 -> T = 10^4 x 2^-10 (the c2 horizon)",
            "g128": c3_128,
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


def scil_bench(p, torch, dev, stream, reps=3):
    """One evaluation of the synthetic-likelihood cost f(theta) with
    bootstrapping (Alg. 6) as one call (scil_evaluate), in Table 1's SCIL
    setting (workload c8): FHN 64x64 to T = 100 (102400 Euler steps), N_syn
    = 1000 model runs at theta from fresh initial states, N_set = 50 against
    the other 950, the six features on both species, M = 13 radii per
    feature (power law fitted to the range), n_CIL = 1000 resamples, the
    data vector of 50 patterns simulated at theta_0.  Whole-call time
    (CUDA events), and the stage split from the same stages run as separate
    calls."""
    cfg = W.config("c8")
    g = p.Group.from_dict(cfg["groups"][0])
    gd = p.Group.from_dict(cfg["data_group"])
    sim = p.Simulation([g], device=dev)
    dsim = p.Simulation([gd], device=dev)
    dsim.integrate(residual=False)
    data = dsim.fields.view(gd.n_real, -1)
    n_set, M, T, feats = cfg["n_set"], cfg["M"], cfg["T_res"], cfg["features"]
    sc = p.Scil(sim, 0, data, n_set=n_set, n_species=2, features=feats, law=cfg["law"], M=M, T=T, seed=cfg["seed"])
    sc.run()
    torch.cuda.synchronize()

    def timed(fn, n=reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    t_total = timed(sc.run)
    out = sc.out
    assert sim.sync_status() == 0
    # the stages as separate calls on the same fields
    X = sim.fields.view(g.n_real, -1)
    S1, S2 = X[:n_set], X[n_set:]
    work = p.mcil_workspace(max(n_set, gd.n_real), g.n_real - n_set, g.G, 2, feats, False, M, dev)
    t_sim = timed(lambda: (sim.reinit(), sim.integrate(residual=False)))
    r = p.mcil(S1, S2, g.G, 2, M=M, features=feats, work=work, law=cfg["law"])
    t_mcil = timed(lambda: p.mcil(S1, S2, g.G, 2, M=M, features=feats, work=work, law=cfg["law"]))
    t_data = timed(lambda: p.mcil_given(data, S2, g.G, 2, r["radii"], features=feats, work=work))
    K = bin(feats).count("1")
    bins = r["bins"].unsqueeze(0).contiguous()
    swork = p.synlik_workspace(n_set, g.n_real - n_set, M, T, K, 1, dev)
    sout = p.synlik_outputs(1, K * M, T, dev)
    yv = out["y_data"].unsqueeze(0).contiguous()
    t_stats = timed(lambda: p.synlik(bins, M, T, cfg["seed"], y_obs=yv, n_feat=K, work=swork, out=sout))
    cells = g.n_real * g.G * g.G * g.n_steps
    return {"workload": "c8: Alg. 6 in Table 1's SCIL setting: FHN 64x64 to T = 100 (102400 Euler steps), "
                        "N_syn = 1000 runs at theta, N_set = 50, six features (both species), M = 13, fitted "
                        "power law, n_CIL = 1000 resamples, data = 50 patterns at theta_0",
            "f_theta_ms": t_total, "evaluations_per_s": 1e3 / t_total,
            "stages_ms": {"simulate": t_sim, "mcil_s1_s2": t_mcil, "data_vector": t_data,
                          "bootstrap_stats": t_stats},
            "simulate_cell_updates_per_s": cells / (t_sim * 1e-3),
            "status": int(out["status"][0]), "cost_f": float(out["scalars"][1]),
            "loglik": float(out["scalars"][2]), "m_active": int(out["scalars"][3]),
            "pairs_exact": [int(x) for x in out["n_exact"].cpu()]}


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


# sizing of the oracle samples only (not a measurement): the FP64 oracle
# steps about 2e9 cell-updates/s on the GPU machine's 16 host cores
ORACLE_RATE_GUESS = 2e9


def full_cells(cfg):
    return sum(g["n_real"] * g["G"] * g["G"] * g["n_steps"] for g in cfg["groups"])


def oracle_sample(cfg, frac):
    """Time the oracle on a bounded sample of the whole workload: every group,
    all its realisations for max(1, round(frac * n_steps)) of its Euler steps
    (stepping time scaled to the full step count), then the full correlation
    integral and bootstrap statistics of every group on the stepped fields.
    Returns (cell-updates/s, seconds spent, description)."""
    import oracle
    t_full = spent = 0.0
    slices = set()
    for g in cfg["groups"]:
        G, n, N = g["G"], g["n_real"], g["n_steps"]
        ns = N if frac >= 1.0 else max(1, int(round(N * frac)))
        slices.add((ns, N))
        t0 = time.perf_counter()
        f0 = oracle.init_fields(g["model"], G, n, g["params"], g["noise"][0], g["noise"][1], g["seed"])
        f = oracle.step(g["model"], g["params"], g["dt"], ns, f0.astype(np.float64))
        oracle.residual(g["model"], g["params"], f)
        t_step = time.perf_counter() - t0
        t1 = time.perf_counter()
        X = oracle.patterns(f.astype(np.float32), g["species_mask"])
        o = oracle.cil(X[:cfg["n1"]], X[cfg["n1"]:cfg["n1"] + cfg["n2"]], b=cfg["b"], M=cfg["M"])
        oracle.synlik(o["bins"], cfg["M"], cfg["T_res"], cfg["seed"], y_obs=o["counts"] / (cfg["n1"] * cfg["n2"]))
        t_cil = time.perf_counter() - t1
        t_full += t_step * (N / ns) + t_cil
        spent += t_step + t_cil
    ng = len(cfg["groups"])
    steps_txt = ", ".join("%d of %d" % sl for sl in sorted(slices))
    if frac >= 1.0:
        note = "the whole workload: every group (%d) x all realisations x all Euler steps + CIL + bootstrap " \
               "statistics" % ng
    else:
        note = ("every group (%d), all realisations x %s Euler steps (stepping time scaled to the full step "
                "count) + the full CIL and bootstrap statistics of every group" % (ng, steps_txt))
    return full_cells(cfg) / t_full, spent, note


def run_reference(args):
    import oracle
    cfg = W.config(args.config)
    # each step a bounded sample, sized so that warm-up and timed steps
    # together stay within about 150 s of CPU work
    per_step = 150.0 / (args.steps + args.warmup + 1)
    frac = min(1.0, per_step * ORACLE_RATE_GUESS / full_cells(cfg))
    oracle_sample(W.config("c1", steps_scale=0.01), 1.0)      # warm (builds the library)
    vals = []
    note = ""
    for _ in range(args.warmup):
        oracle_sample(cfg, frac)
    for _ in range(args.steps):
        v, _, note = oracle_sample(cfg, frac)
        vals.append(v)
    value = statistics.mean(vals)
    cores = oracle.threads()
    return {
        "impl": "reference",
        "metric": "RD cell-updates/s + CIL pair-dists/s at stated tol; % HBM/tensor roofline",
        "value": value, "unit": "cell-updates/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": full_cells(cfg) / value * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": config_json(args.config, cfg),
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": note, "cpu_model": cpu_model()},
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
    if args.stepper_only:
        import torch
        import paper_2203_14742_b300 as p
        from paper_2203_14742_b300 import build as B
        B.build()
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        print(json.dumps(stepper_only(p, torch, dev, args)))
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
        # about 15 s of CPU work on all cores, a sixteenth of that on one
        frac = min(1.0, 15.0 * ORACLE_RATE_GUESS / full_cells(cfg))
        v, secs, note = oracle_sample(cfg, frac)
        import oracle
        cores = oracle.threads()
        out["cpu_baseline"] = {"value": v, "unit": "cell-updates/s", "cores": cores,
                               "kind": "oracle", "sample": note + " (%.1f s of CPU work)" % secs,
                               "cpu_model": cpu_model()}
        if len(cfg["groups"]) == 1:   # one thread on a sixteenth of the sample (single-group workloads)
            oracle.set_threads(1)
            v1, secs1, note1 = oracle_sample(cfg, frac / 16)
            oracle.set_threads(cores)
            out["cpu_baseline"]["one_thread"] = {"value": v1, "sample": note1 + " (%.1f s)" % secs1}
        else:   # one thread, stepping only, every eighth group on a sixteenth of the step slice
            oracle.set_threads(1)
            cells = 0
            t0 = time.perf_counter()
            for g in cfg["groups"][::8]:
                ns = max(1, int(round(g["n_steps"] * frac / 16)))
                f0 = oracle.init_fields(g["model"], g["G"], g["n_real"], g["params"], g["noise"][0], g["noise"][1],
                                        g["seed"])
                oracle.step(g["model"], g["params"], g["dt"], ns, f0.astype(np.float64))
                cells += g["n_real"] * g["G"] * g["G"] * ns
            secs1 = time.perf_counter() - t0
            oracle.set_threads(cores)
            out["cpu_baseline"]["one_thread"] = {
                "value": cells / secs1, "unit": "cell-updates/s (stepping only)",
                "sample": "every eighth group, all realisations x 1/16 of the step slice (%.1f s)" % secs1}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
