#!/usr/bin/env python3
"""Throughput benchmark: Q+Tw values per second on one GB300.

Workload (the synthetic active-region configuration): a 256x256x128 FP32 cube,
the potential field of 24 buried monopoles (seeded), unit spacing, curl by
central differences; Q (Method I, RKF45, tol_perp = 10^-3.2) and Tw on the z=0
plane at 4x oversampling (1024x1024 seeds), both directions. A "step" is one
Q+Tw map (tracer + Q assembly launches). The headline ``value`` is the FP32
tracer (FP32 error norm, compensated FP32 length/Tw sums, FP64 tolerance,
footpoints and Q assembly); the FP32 tracer with FP64 accumulation at every
step and the plain FP64 tracer are timed beside it. ``e2e`` is the same map through the C ABI from host memory: copy of B,
curl+pack, map, copy of Q and Tw back.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fqsl|reference]
N>1 runs as torchrun ranks, one GPU each, each rank mapping its own cube
(weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NU = NV = 1024
TOL = 10 ** -3.2
CONVERGED_TOL = 1e-10  # the oracle's map at this tolerance stands in for the exact map
CUBE = (256, 256, 128)
SEED = 2208
WORKLOAD = "monopole24_256x256x128_f32_z0plane_1024x1024_methodI_rkf45"
METRIC = "Q+Tw values/sec on 1 GB300 (FP32 vs FP64) at stated rel-err vs oracle"
# Algorithmic work of one RKF45 trial step of the FP32 tracer, counted from the
# kernel source (trace.cuh): 6 right-hand-side evaluations, 4 of them with the
# twist integrand at 145 flops each (trilinear weights 18, 8-corner x
# 6-component accumulation 96, normalisation and twist integrand 31) and the 2
# whose 4th-order weight is zero (stages 1 and 5) with B alone at 89 flops
# (accumulation 48, normalisation 23), plus 222 flops of stage combination; and
# 4 x 8 corner records of 32 bytes plus 2 x 8 B halves of 16 bytes requested
# from L1.
FLOPS_PER_TRIAL = 4 * 145 + 2 * 89 + 222
GATHER_BYTES_PER_TRIAL = 4 * 8 * 32 + 2 * 8 * 16
# The FP64 tracer (trace.cuh, FP64 gather and rhs): per evaluation 118 flops
# of trilinear gather (6 weights, 16 corner-weight products, 8 x 6 x 2
# accumulation) and 30 of right-hand side (3 divisions by the spacing, |bt|^2,
# |B|^2, 2 square roots, 6 for F, 1 for dl/dtau, 8 for the twist integrand);
# 6 evaluations and 222 flops of stage combination per trial. A division or a
# square root counts as one flop. Bytes: 6 x 8 corners x the 48 bytes of B
# and curl B of a 64-byte record.
FLOPS_PER_TRIAL_F64 = 6 * (118 + 30) + 222
GATHER_BYTES_PER_TRIAL_F64 = 6 * 8 * 48
FP32_LANES_PER_SM = 128
NUM_SMS = 152
# DRAM bytes (read + write) of one k_trace_f32 launch on this workload, from
# an ncu capture of that kernel on this map, valid while the tracer sources
# hash to TRACE_F32_SRC_HASH.
TRACE_F32_DRAM_BYTES = 309.030656e6 + 59.771648e6
TRACE_F32_SRC_HASH = "ef0edbdcc5075cb6"


def _trace_src_hash():
    import hashlib

    h = hashlib.sha256()
    for name in ("trace.cuh", "trace_f32.cu"):
        with open(os.path.join(ROOT, "paper_2208_12569_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def _smi_gpu_id(dev_index: int) -> str:
    """The nvidia-smi id of a CUDA device: its UUID (CUDA and NVML number
    visible devices differently when CUDA_VISIBLE_DEVICES is set), else the
    index."""
    try:
        import torch

        u = str(torch.cuda.get_device_properties(dev_index).uuid)
        u = u[4:] if u.startswith("GPU-") else u
        if len(u) == 36 and all(c in "0123456789abcdef-" for c in u.lower()):
            return "GPU-" + u
    except Exception:
        pass
    return str(dev_index)


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region. start()
    returns once the sampler has written its first line, so sampling is under
    way when the region begins; stop() keeps the samples stamped between the
    two calls. If the region is shorter than the sampling interval and holds
    no sample, the last sample before it and the first after it stand in
    (``bracketing``)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 20

    def __init__(self, gpu_index: int, smi: str = "nvidia-smi"):
        self.ids = [_smi_gpu_id(gpu_index)]
        if self.ids[0] != str(gpu_index):
            self.ids.append(str(gpu_index))
        self.smi = smi
        self.proc = None
        self.lines = []
        self.t0 = None

    def _spawn(self, gid):
        self.lines = []
        self.proc = subprocess.Popen([self.smi, "-i", gid, "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                     stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        deadline = time.monotonic() + 5.0
        while not self.lines and time.monotonic() < deadline and self.proc.poll() is None:
            time.sleep(0.002)
        return bool(self.lines)

    def start(self):
        self.proc = None
        for gid in self.ids:
            try:
                if self._spawn(gid):
                    break
            except OSError:
                self.proc = None
                break
            self._kill()
        self.t0 = time.monotonic()

    def mark(self):
        """The timed region begins now (start() may run before the warm-up,
        so that the GPU does not idle between the warm-up and the region
        while the sampler starts)."""
        self.t0 = time.monotonic()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def _kill(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)

    @staticmethod
    def _parse(ln):
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 9:
            return None
        try:
            sm, mx = float(parts[1]), float(parts[2])
        except ValueError:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        return sm, mx, {nm for nm, v in zip(names, parts[5:9]) if v.lower().startswith("active")}

    def stop(self):
        t1 = time.monotonic()
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        # one more interval, so that a sample after the region exists
        time.sleep(2 * self.INTERVAL_MS / 1000.0)
        self._kill()
        stamped = [(t, r) for t, r in ((t, self._parse(ln)) for t, ln in self.lines) if r is not None]
        inside = [r for t, r in stamped if self.t0 <= t <= t1]
        bracketing = not inside
        if bracketing:
            before = [r for t, r in stamped if t < self.t0][-1:]
            after = [r for t, r in stamped if t > t1][:1]
            inside = before + after
        sm = [r[0] for r in inside]
        mx = [r[1] for r in inside]
        reasons = set().union(*[r[2] for r in inside]) if inside else set()
        out = {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": sorted(reasons), "samples": 0 if bracketing else len(sm),
               "interval_ms": self.INTERVAL_MS, "region_ms": round((t1 - self.t0) * 1000.0, 1)}
        if bracketing:
            out["bracketing"] = len(sm)
        return out


def roofline(trials, trace_ms, trace64_ms, ceil, work_src):
    """Roofline of the FP32 tracer: algorithmic gather bytes and flops of
    `trials` RKF45 trial steps over its event-timed duration, against the
    gather and FMA ceilings measured by the probes; bound = the larger
    fraction. The FP64 tracer's fraction of the FP64 FMA ceiling beside it."""
    gather = trials * GATHER_BYTES_PER_TRIAL / (trace_ms / 1000.0) / 1e12
    flops = trials * FLOPS_PER_TRIAL / (trace_ms / 1000.0) / 1e12
    flops64 = trials * FLOPS_PER_TRIAL_F64 / (trace64_ms / 1000.0) / 1e12
    gather64 = trials * GATHER_BYTES_PER_TRIAL_F64 / (trace64_ms / 1000.0) / 1e12
    traffic = TRACE_F32_DRAM_BYTES if _trace_src_hash() == TRACE_F32_SRC_HASH else None
    per = {"trial_steps": trials, "source": work_src, "gather_bytes_per_trial": GATHER_BYTES_PER_TRIAL,
           "flops_per_trial": FLOPS_PER_TRIAL}
    if ceil is None:
        peaks, kind = _measured_peaks()
        sm = float(peaks.get("sm_max_mhz", 2070.0))
        alu = NUM_SMS * FP32_LANES_PER_SM * 2 * sm * 1e6 / 1e12
        return {"bound": "alu", "achieved": flops, "peak": alu, "unit": "TFLOP/s", "frac": flops / alu,
                "traffic": traffic, "work": per,
                "peak_source": "nominal: 152 SMs x 128 FP32 lanes x 2 x %.0f MHz (%s sm_max_mhz); probes skipped"
                               % (sm, kind)}
    fg = gather / ceil["gather_walk_TBs"]
    fa = flops / ceil["fma_f32_TFLOPs"]
    g_bound = fg >= fa
    return {"bound": "gather" if g_bound else "alu", "achieved": gather if g_bound else flops,
            "peak": ceil["gather_walk_TBs"] if g_bound else ceil["fma_f32_TFLOPs"],
            "unit": "TB/s" if g_bound else "TFLOP/s", "frac": max(fg, fa), "traffic": traffic,
            "peak_source": ("measured on this GPU: trilinear gathers of 32-byte records by 8x4-lane tiles walking "
                            "the cube (fqsl_probe_gather)" if g_bound else
                            "measured on this GPU: FP32 FMA chains (fqsl_probe_fma)"),
            "gather": {"achieved_TBs": gather, "ceiling_TBs": ceil["gather_walk_TBs"], "frac": fg},
            "alu": {"achieved_TFLOPs": flops, "ceiling_TFLOPs": ceil["fma_f32_TFLOPs"], "frac": fa},
            "ceilings": ceil, "work": per,
            "fp64_tracer": {"ms": trace64_ms, "achieved_TFLOPs": flops64,
                            "frac_of_fma_f64": flops64 / ceil["fma_f64_TFLOPs"], "gather_TBs": gather64,
                            "flops_per_trial": FLOPS_PER_TRIAL_F64,
                            "note": "a division or square root counts as one flop; the FP64 pipe runs each as "
                                    "several instructions"}}


def measure_ceilings(dev, cube=CUBE, target_ms=6.0):
    """Roofline ceilings measured on this GPU by the probe kernels of
    libfqsl_probes.so (include/fqsl_probes.h): trilinear gathers of 32-byte
    records over a cube of the workload's size (requested bytes per second, for
    three access patterns) and FP32 / FP64 FMA chains (flops per second). Each
    figure is the best over a few grid sizes; each launch runs about target_ms."""
    import ctypes as C

    import torch

    import __graft_entry__

    lib = C.CDLL(__graft_entry__._builder().build_probes())
    lib.fqsl_probe_gather.restype = C.c_int
    lib.fqsl_probe_fma.restype = C.c_int
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    nx, ny, nz = cube
    rec = torch.rand(nx * ny * nz * 8, dtype=torch.float32, device=dev)  # 32-byte records, > L2
    sink = torch.empty(sms * 64 * 256, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    sptr = C.c_void_p(stream.cuda_stream)

    def best_ms(launch, reps=3):
        launch()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            launch()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    def sized(run, work0):
        # calibrate the per-thread work so that one launch takes about target_ms
        t = best_ms(lambda: run(work0), reps=1)
        work = max(work0, int(work0 * target_ms / max(t, 1e-3)))
        return work, best_ms(lambda: run(work))

    out = {"sms": sms, "cube": list(cube), "record_bytes": 32}
    names = {0: "walk", 1: "tile", 2: "random"}
    for pat, name in names.items():
        best = 0.0
        for bps in (4, 8, 16):
            def run(g, bps=bps, pat=pat):
                rc = lib.fqsl_probe_gather(C.c_void_p(rec.data_ptr()), nx, ny, nz, pat, int(g), sms, bps,
                                           C.c_void_p(sink.data_ptr()), sptr)
                if rc:
                    raise RuntimeError("fqsl_probe_gather: %d" % rc)
            g, ms = sized(run, 64)
            best = max(best, sms * bps * 128 * g * 256 / (ms / 1000.0) / 1e12)
        out["gather_%s_TBs" % name] = best
    for fp64, name, w0 in ((0, "fma_f32_TFLOPs", 4096), (1, "fma_f64_TFLOPs", 256)):
        best = 0.0
        for bps in (4, 8):
            def run(it, bps=bps, fp64=fp64):
                rc = lib.fqsl_probe_fma(fp64, int(it), sms, bps, C.c_void_p(sink.data_ptr()), sptr)
                if rc:
                    raise RuntimeError("fqsl_probe_fma: %d" % rc)
            it, ms = sized(run, w0)
            best = max(best, sms * bps * 256 * 8 * it * 2 / (ms / 1000.0) / 1e12)
        out[name] = best
    del rec, sink
    torch.cuda.empty_cache()
    return out


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def monopole24_inputs(rank: int = 0, cube=CUBE):
    """Rank r maps its own cube: the same shape, sources seeded with 2208 + r."""
    import synth

    B, grid, _ = synth.monopole24_cube(seed=SEED + rank, n=cube)
    u = (float(cube[0] - 1) / NU, 0.0, 0.0)
    v = (0.0, float(cube[1] - 1) / NV, 0.0)
    return B, grid, u, v


def job_rate(ms_local: float, units_per_rank: int, dist=None, device="cpu"):
    """Whole-job throughput of a weak-scaling step: every rank processed
    units_per_rank units; the job's step time is the slowest rank's. Returns
    (max step ms over ranks, units of all ranks per second)."""
    import torch

    ws = 1
    ms = float(ms_local)
    if dist is not None:
        ws = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_per_rank * ws / (ms / 1000.0)


def cpu_baseline(B, grid, u, v, target_s=12.0, seed=5):
    """The oracle as it stands, on a seeded random sample of the same lattice,
    all host cores; rate in Q+Tw values per second."""
    import oracle

    oracle.build()
    B64 = B.astype(np.float64)
    J = oracle.curl(B64, grid)
    rng = np.random.default_rng(seed)
    p = oracle.params(tol=TOL)
    calib = np.sort(rng.choice(NU * NV, 512, replace=False))
    t0 = time.perf_counter()
    oracle.plane(B64, grid, (0.0, 0.0, 0.0), u, v, NU, NV, p, sample=calib, J=J)
    rate0 = len(calib) / max(time.perf_counter() - t0, 1e-6)
    m = int(min(NU * NV, max(1024, rate0 * target_s)))
    sample = np.sort(rng.choice(NU * NV, m, replace=False))
    t0 = time.perf_counter()
    ref = oracle.plane(B64, grid, (0.0, 0.0, 0.0), u, v, NU, NV, p, sample=sample, J=J)
    dt = time.perf_counter() - t0
    return {"value": m / dt, "unit": "Q+Tw values/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": "%d seeded-random seeds of the 1024x1024 lattice (%.1f s)" % (m, dt)}, sample, ref


def err_stats(g, ref, sample):
    """Relative Q and Tw error of a GPU map against the oracle on the sample."""
    gq, rq = g["Q"][sample], ref["Q"]
    ok = np.isfinite(rq) & np.isfinite(gq) & (rq < 1e6)
    rel = np.abs(gq[ok] / rq[ok] - 1)
    gt, rt = g["Tw"][sample], ref["Tw"]
    okt = np.isfinite(rt) & np.isfinite(gt)
    twr = np.abs(gt[okt] - rt[okt]) / np.maximum(np.abs(rt[okt]), 1e-3)
    return {"q_rel_median": float(np.median(rel)), "q_rel_p99": float(np.percentile(rel, 99)),
            "tw_rel_median": float(np.median(twr)), "tw_rel_p99": float(np.percentile(twr, 99)),
            "faces_equal": float(np.mean((g["face1"][sample] == ref["face1"]) & (g["face2"][sample] == ref["face2"]))),
            "status_equal": float(np.mean(g["status"][sample] == ref["status"])), "n": int(len(sample))}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    B, grid, u, v = monopole24_inputs(0)
    import oracle

    oracle.build()
    B64 = B.astype(np.float64)
    J = oracle.curl(B64, grid)
    p = oracle.params(tol=TOL)
    rng = np.random.default_rng(17)
    per_step = 4096
    times = []
    for it in range(args.warmup + args.steps):
        sample = np.sort(rng.choice(NU * NV, per_step, replace=False))
        t0 = time.perf_counter()
        oracle.plane(B64, grid, (0.0, 0.0, 0.0), u, v, NU, NV, p, sample=sample, J=J)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1000.0 * float(np.mean(times))
    value = per_step / (ms / 1000.0)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Q+Tw values/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "Q+Tw values/s", "cores": oracle.max_threads(),
                             "kind": "oracle", "sample": "%d seeded-random seeds per step" % per_step},
            "e2e": {"value": value, "unit": "Q+Tw values/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


VOL_CUBE = (1024, 1024, 512)
VOL_SEEDS = (512, 512, 256)
VOL_PLANE = (4096, 4096)
VOL_WORKLOAD = "monopole64_1024x1024x512_f32_volume512x512x256_plane4096x4096_methodI"


def run_volume(args, emit=True, sample_frac=0.0025, fp64_layers=32, conv_seeds=1000):
    """Large volume: 1024x1024x512 FP32 monopole cube (64 sources); Q and Tw on
    the 512x512x256 cell-centred seed volume spanning the cube (every z-layer
    its own S0) and on a 4096x4096 z=0 map. FP32 over the whole volume; FP64
    on the fp64_layers layers in the middle of it (a slab of the same volume,
    to bound the run: the whole FP64 volume takes about 50 s) and on the whole
    4096^2 map.
    Errors against the oracle on a seeded sample of sample_frac of the volume
    (FP64 on the sample's seeds in the slab), and FP32 and FP64 against the
    converged oracle map (tol_perp = 1e-10) on conv_seeds of the slab's seeds."""
    import torch

    import __graft_entry__
    import oracle
    import synth

    __graft_entry__._builder().build()
    import paper_2208_12569_gb300 as fq

    dev = torch.device("cuda", 0)
    n = VOL_CUBE
    t0 = time.perf_counter()
    Bd, grid, _ = synth.large_monopole(n=n, device=dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    vol = VOL_SEEDS
    step = tuple((n[a] - 1.0) / vol[a] for a in range(3))
    plane = VOL_PLANE
    u = ((n[0] - 1.0) / plane[0], 0.0, 0.0)
    v = (0.0, (n[1] - 1.0) / plane[1], 0.0)
    nvol = vol[0] * vol[1] * vol[2]
    slab = (vol[0], vol[1], fp64_layers)
    nslab = slab[0] * slab[1] * slab[2]
    k0 = (vol[2] - fp64_layers) // 2  # the slab's first layer in the volume
    off = k0 * vol[0] * vol[1]  # volume index of the slab's seed 0
    slab_origin = (0.0, 0.0, k0 * step[2])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def timed(fn, k):
        ms, kern = [], []
        for _ in range(k):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.mean(ms))

    res, outs = {}, {}
    for prec in ("f32", "f64"):
        field = fq.Field(Bd, grid.origin, grid.spacing, pack=(prec,))
        field.set_timing(True)
        p = fq.params(precision=prec, tol=TOL)
        lat = vol if prec == "f32" else slab
        org_v = (0.0, 0.0, 0.0) if prec == "f32" else slab_origin
        nl = lat[0] * lat[1] * lat[2]
        out = fq.alloc_out(nl, device=dev)
        run_v = lambda: fq.qmap_volume(field, org_v, step, *lat, p, out=out)  # noqa: E731
        run_v()  # warm-up
        torch.cuda.synchronize()
        ms_v = timed(run_v, 1)
        field.check()
        kern = field.times()
        outs[prec] = {k: t.cpu().numpy() for k, t in out.items() if t is not None}
        steps_total = float(outs[prec]["steps"].astype(np.int64).sum())
        del out
        outp = fq.alloc_out(plane[0] * plane[1], device=dev)
        run_p = lambda: fq.qmap_plane(field, (0.0, 0.0, 0.0), u, v, *plane, p, out=outp)  # noqa: E731
        run_p()
        torch.cuda.synchronize()
        ms_p = timed(run_p, 3 if prec == "f32" else 1)
        del outp
        field.close()
        res[prec] = {"volume": {"value": nl / (ms_v / 1000.0), "unit": "Q+Tw values/s", "ms": ms_v,
                                "seeds": list(lat), "kernels_ms": kern, "mean_trials_per_line": steps_total / nl,
                                "trials_per_s": steps_total / (ms_v / 1000.0)},
                     "plane_4096": {"value": plane[0] * plane[1] / (ms_p / 1000.0), "unit": "Q+Tw values/s",
                                    "ms": ms_p}}
        torch.cuda.empty_cache()
    del flush
    line = {"metric": METRIC, "workload": "large_volume", "unit": "Q+Tw values/s",
            "config": {"workload": VOL_WORKLOAD, "cube": list(n), "seeds": list(vol), "plane": list(plane),
                       "tol_perp": TOL, "fp64_volume_layers": [k0, k0 + fp64_layers],
                       "l2": "flushed between steps (inputs far larger than L2)"},
            "value": res["f32"]["volume"]["value"], "f32": res["f32"], "f64": res["f64"],
            "speedup_fp32_over_fp64_volume_per_trial": res["f32"]["volume"]["trials_per_s"] /
                                                       res["f64"]["volume"]["trials_per_s"],
            "generation_s": gen_s, "gpu_launches": 10}
    if not getattr(args, "no_cpu_baseline", False):
        # the oracle on a seeded sample of the volume (the FP32 volume) and of
        # its slab (the FP64 volume, bitwise)
        m = max(1000, int(nvol * sample_frac))
        sample = np.sort(np.random.default_rng(19).choice(nvol, m, replace=False))
        B64 = Bd.cpu().numpy().astype(np.float64)
        del Bd
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        J = oracle.curl(B64, grid)
        curl_s = time.perf_counter() - t0
        org, a1, a2, a3 = (0.0, 0.0, 0.0), (step[0], 0, 0), (0, step[1], 0), (0, 0, step[2])
        t0 = time.perf_counter()
        ref = oracle.qmap(B64, grid, org, a1, a2, a3, vol, oracle.params(tol=TOL), sample=sample, J=J)
        ora_s = time.perf_counter() - t0
        in_slab = (sample >= off) & (sample < off + nslab)
        ss = sample[in_slab] - off
        e64 = err_stats(outs["f64"], {k: v[in_slab] for k, v in ref.items()}, ss)
        e64["bitwise"] = bool(all(np.array_equal(outs["f64"][k][ss], ref[k][in_slab], equal_nan=True)
                                  for k in ("Q", "Tw", "face1", "face2", "status")))
        line["error_vs_oracle"] = {"f32": err_stats(outs["f32"], ref, sample), "f64_slab": e64,
                                   "sample": "%d seeded-random seeds of the volume (%.2f%%); FP64 on the %d of them "
                                             "in its slab" % (m, 100.0 * m / nvol, int(in_slab.sum()))}
        cs = np.sort(np.random.default_rng(37).choice(nslab, conv_seeds, replace=False))
        t1 = time.perf_counter()
        conv = oracle.qmap(B64, grid, org, a1, a2, a3, vol, oracle.params(tol=CONVERGED_TOL), sample=cs + off,
                           J=J)
        conv_s = time.perf_counter() - t1
        acc = {"reference": "oracle at tol_perp = %g on %d seeded-random seeds of the slab (%.1f s)"
                            % (CONVERGED_TOL, conv_seeds, conv_s),
               "f32": err_stats(outs["f32"], conv, cs + off), "f64": err_stats(outs["f64"], conv, cs)}
        acc["f32_p99_over_f64_p99"] = acc["f32"]["q_rel_p99"] / max(acc["f64"]["q_rel_p99"], 1e-300)
        line["accuracy_vs_converged"] = acc
        line["cpu_baseline"] = {"value": m / ora_s, "unit": "Q+Tw values/s", "cores": oracle.max_threads(),
                                "kind": "oracle", "sample": "%d seeded-random seeds of the volume (%.1f s; curl "
                                                            "%.1f s)" % (m, ora_s, curl_s)}
    if emit:
        print(json.dumps(line), flush=True)
    return line


RECT_WORKLOAD = "monopole24_stretched256x256x128_f32_z0plane_1024x1024_methodI_rkf45"


def run_stretched(args, emit=True):
    """The 24-monopole map on a stretched grid (Sec. 2.2-2.3): the same 24 monopoles
    sampled on 256x256x128 nodes over the same box, horizontal cells growing
    1 % per cell from the middle to the edges and vertical cells 2 % per cell
    upward; 1024x1024 seeds on z=0. FP32 and FP64, next to the uniform map
    (the paper reports 45-80 % of the uniform speed for its binary search);
    error against the oracle on a seeded sample."""
    import torch

    import __graft_entry__
    import oracle
    import synth

    __graft_entry__._builder().build()
    import paper_2208_12569_gb300 as fq

    dev = torch.device("cuda", 0)
    B, grid, _ = synth.monopole24_stretched(seed=SEED, n=CUBE)
    Bd = torch.from_numpy(B).to(dev)
    u = ((CUBE[0] - 1.0) / NU, 0.0, 0.0)
    v = (0.0, (CUBE[1] - 1.0) / NV, 0.0)
    n = NU * NV
    out = fq.alloc_out(n, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(field, p, k):
        for _ in range(args.warmup):
            fq.qmap_plane(field, (0.0, 0.0, 0.0), u, v, NU, NV, p, out=out)
        torch.cuda.synchronize()
        field.check()
        ms, kern = [], []
        for _ in range(k):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fq.qmap_plane(field, (0.0, 0.0, 0.0), u, v, NU, NV, p, out=out)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            kern.append(field.times())
        return float(np.mean(ms)), float(np.mean([k[0] for k in kern])), \
            {k: t.cpu().numpy() for k, t in out.items() if t is not None}

    res = {}
    fr = fq.Field(Bd, coords=grid.coords, pack=("f32", "f64"))
    fr.set_timing(True)
    for prec, k in (("f32", args.steps), ("f32acc64", args.steps), ("f64", max(1, args.fp64_steps))):
        ms, tr, o = timed(fr, fq.params(precision=prec, tol=TOL), k)
        res[prec] = {"value": n / (ms / 1000.0), "unit": "Q+Tw values/s", "ms_per_step": ms, "trace_ms": tr,
                     "mean_trials_per_line": float(o["steps"].astype(np.int64).sum()) / n, "out": o}
    fr.close()
    # the uniform 256x256x128 map in the same run, for the ratio
    Bu, ugrid, uu, vu = monopole24_inputs(0)
    Bud = torch.from_numpy(Bu).to(dev)
    fu = fq.Field(Bud, ugrid.origin, ugrid.spacing, pack=("f32",))
    fu.set_timing(True)
    ms_u, tr_u, _ = timed(fu, fq.params(precision="f32", tol=TOL), args.steps)
    fu.close()
    line = {"metric": METRIC, "workload": "stretched", "unit": "Q+Tw values/s", "value": res["f32"]["value"],
            "ms_per_step": res["f32"]["ms_per_step"], "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": RECT_WORKLOAD, "cube": list(CUBE), "seeds": [NU, NV], "tol_perp": TOL,
                       "stretch": "x, y cells x1.01 per cell from the middle; z cells x1.02 per cell upward",
                       "cell_width_range": [float(min(np.diff(grid.axis(a)).min() for a in range(3))),
                                            float(max(np.diff(grid.axis(a)).max() for a in range(3)))],
                       "l2": "flushed between steps (256 MB write)", "inputs_resident": True},
            "f32_acc64": {k: res["f32acc64"][k] for k in ("value", "ms_per_step", "trace_ms")},
            "fp64": {k: res["f64"][k] for k in ("value", "ms_per_step", "trace_ms")},
            "kernels_ms": {"trace_f32": res["f32"]["trace_ms"]},
            "work": {"mean_trials_per_line": res["f32"]["mean_trials_per_line"]},
            "uniform_f32": {"value": n / (ms_u / 1000.0), "ms_per_step": ms_u, "trace_ms": tr_u,
                               "stretched_over_uniform": ms_u / res["f32"]["ms_per_step"]},
            "gpu_launches": 3 * args.steps}
    if emit and not args.no_cpu_baseline:
        sample = np.sort(np.random.default_rng(23).choice(n, 2000, replace=False))
        t0 = time.perf_counter()
        ref = oracle.plane(B.astype(np.float64), grid, (0.0, 0.0, 0.0), u, v, NU, NV, oracle.params(tol=TOL),
                           sample=sample)
        dt = time.perf_counter() - t0
        line["error_vs_oracle"] = {p: err_stats(res[p]["out"], ref, sample) for p in ("f32", "f32acc64", "f64")}
        line["cpu_baseline"] = {"value": len(sample) / dt, "unit": "Q+Tw values/s", "cores": oracle.max_threads(),
                                "kind": "oracle", "sample": "%d seeded-random seeds of the map" % len(sample)}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_batch(args, emit=True):
    """Batched uneven workload: 48 monopole cubes with sizes drawn from
    {64^3, 128^2x64, 256^2x128, 384^2x192}, 8-64 sources each, each with the
    z=0 plane or the mid-y vertical slice of 512x256 seeds (6.29 M lines).
    Times per-cube launches, one batch run, its CUDA-graph replay and the
    autotuned graph; checks a sample of seeds against the oracle."""
    import torch

    import __graft_entry__
    import oracle
    import synth

    __graft_entry__._builder().build()
    import paper_2208_12569_gb300 as fq
    from paper_2208_12569_gb300 import autotune

    dev = torch.device("cuda", 0)
    specs = synth.batch_specs(seed=SEED)
    t0 = time.perf_counter()
    cubes = [synth.monopole_cube(sp["grid"], sp["charges"], dtype=np.float32, device=dev) for sp in specs]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    fields = [fq.Field(B, sp["grid"].origin, sp["grid"].spacing, pack=("f32",)) for B, sp in zip(cubes, specs)]
    planes = [sp["plane"] for sp in specs]
    total = sum(pl["nu"] * pl["nv"] for pl in planes)
    p = fq.params(precision="f32", tol=TOL)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    outs = [fq.alloc_out(pl["nu"] * pl["nv"], device=dev) for pl in planes]

    def timed(fn, k):
        ts = []
        for _ in range(k):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    def per_cube(pp=p):
        for fld, pl, o in zip(fields, planes, outs):
            fq.qmap_plane(fld, pl["origin"], pl["u"], pl["v"], pl["nu"], pl["nv"], pp, out=o)

    for _ in range(args.warmup):
        per_cube()
    ms_single = timed(per_cube, args.steps)
    batch = fq.Batch(fields, planes, p, outs=outs)
    for _ in range(args.warmup):
        batch.run()
    ms_batch = timed(batch.run, args.steps)
    graph = batch.graph()
    ms_graph = timed(graph.replay, args.steps)
    # autotune the batch's scheduling knobs (results are identical for all)
    space = {"refill_lanes": (1, 32), "sync_dirs": (0, 1), "blocks_per_sm": (0, 2, 3)}

    def run_with(pp):
        b = fq.Batch(fields, planes, pp, outs=outs)
        b.run()
        torch.cuda.synchronize()
        b.close()

    best, table = autotune.tune(run_with, p, key="batch48_512x256", space=space, reps=3, path="")
    tuned = fq.Batch(fields, planes, best, outs=outs)
    tuned.run()
    tgraph = tuned.graph()
    ms_tuned = timed(tgraph.replay, args.steps)
    torch.cuda.synchronize()
    res = [{k: t.cpu().numpy() for k, t in o.items() if t is not None} for o in outs]
    # the same batch traced in FP64 (one launch set)
    fields64 = [fq.Field(B, sp["grid"].origin, sp["grid"].spacing, pack=("f64",)) for B, sp in zip(cubes, specs)]
    outs64 = [fq.alloc_out(pl["nu"] * pl["nv"], device=dev) for pl in planes]
    batch64 = fq.Batch(fields64, planes, fq.params(precision="f64", tol=TOL), outs=outs64)
    batch64.run()
    torch.cuda.synchronize()
    ms64 = timed(batch64.run, 1)
    res64 = [{k: t.cpu().numpy() for k, t in o.items() if t is not None} for o in outs64]
    batch64.close()
    for fl in fields64:
        fl.close()
    del outs64
    # oracle on a sample of seeds of the four smallest cubes and the largest
    by_size = sorted(range(len(specs)), key=lambda k: np.prod(specs[k]["grid"].n))
    order = by_size[:4] + by_size[-1:]
    errs = []
    ora_n, ora_s = 0, 0.0
    for k in order:
        sp, pl = specs[k], planes[k]
        sample = np.sort(np.random.default_rng(k).choice(pl["nu"] * pl["nv"], 300, replace=False))
        B64 = cubes[k].cpu().numpy().astype(np.float64)
        t1 = time.perf_counter()
        ref = oracle.plane(B64, sp["grid"], pl["origin"], pl["u"], pl["v"], pl["nu"], pl["nv"],
                           oracle.params(tol=TOL), sample=sample)
        ora_s += time.perf_counter() - t1
        ora_n += len(sample)
        e = {"entry": int(k), "cube": list(sp["grid"].n), "f32": err_stats(res[k], ref, sample),
             "f64": err_stats(res64[k], ref, sample)}
        e["f64"]["bitwise"] = bool(all(np.array_equal(res64[k][c][sample], ref[c], equal_nan=True)
                                       for c in ("Q", "Tw", "face1", "face2", "status")))
        if k == by_size[0]:
            # the smallest cube (lattice step 1/8 cell): FP32 and FP64 against
            # the converged oracle map on the same seeds
            conv = oracle.plane(B64, sp["grid"], pl["origin"], pl["u"], pl["v"], pl["nu"], pl["nv"],
                                oracle.params(tol=CONVERGED_TOL), sample=sample)
            e["accuracy_vs_converged"] = {"reference": "oracle at tol_perp = %g" % CONVERGED_TOL,
                                          "f32": err_stats(res[k], conv, sample),
                                          "f64": err_stats(res64[k], conv, sample)}
        errs.append(e)
    line = {"metric": METRIC, "workload": "batch", "unit": "Q+Tw values/s",
            "config": {"workload": "batch48_monopole_mixed_sizes_512x256_seeds_methodI", "entries": len(specs),
                       "lines": total, "tol_perp": TOL, "l2": "flushed between steps"},
            "value": total / (ms_tuned / 1000.0),
            "per_cube_launches": {"ms": ms_single, "value": total / (ms_single / 1000.0)},
            "batch_run": {"ms": ms_batch, "value": total / (ms_batch / 1000.0)},
            "batch_graph": {"ms": ms_graph, "value": total / (ms_graph / 1000.0)},
            "batch_graph_autotuned": {"ms": ms_tuned, "value": total / (ms_tuned / 1000.0),
                                      "best": {k: getattr(best, k) for k in space}, "table": table},
            "fp64_batch_run": {"ms": ms64, "value": total / (ms64 / 1000.0)},
            "error_vs_oracle_sample": errs,
            "cpu_baseline": {"value": ora_n / ora_s, "unit": "Q+Tw values/s", "cores": oracle.max_threads(),
                             "kind": "oracle", "sample": "300 seeds of each of the 4 smallest cubes and the largest"},
            "generation_s": gen_s, "gpu_launches": 4 * args.steps}
    if emit:
        print(json.dumps(line), flush=True)
    for b in (batch, tuned):
        b.close()
    for fl in fields:
        fl.close()
    return line


ADJ_CUBE = (128, 128, 64)
ADJ_SEEDS = 256
ADJ_WORKLOAD = "adjoint_monopole24_twisttube_128x128x64_f32_z0plane_256x256_logQ_Tw_loss_methodI"
ADJ_METRIC = "adjoint s/grad"
ADJ_SAMPLE = 64  # oracle seeds per check (plus their 4-neighbour lines)
# Work of one accepted step in the reverse sweep, counted from adjoint.cu:
#   A1 (recompute)  5 right-hand sides of 145 flops, 8 x 32-byte corner records each
#   A2 (Jacobian)   5 stage Jacobians: trilinear value and 3 derivatives of 6
#                   components (8 x 6 x 4 FMAs = 384 flops), 3x3 local Jacobian and
#                   Tw gradient (~110), tangent products (~100)
#   C (VJP)         5 stage VJPs: the same gather with derivatives (384), local
#                   adjoint (~60), scatter of 8 x 6 products (96), position adjoint (36)
# plus stage combinations (~300). Gathers: 15 x 8 records of 32 bytes; scatter:
# 5 x 8 corners x 24 bytes of atomics.
REV_FLOPS_PER_STEP = 5 * 145 + 5 * (384 + 110 + 100) + 5 * (384 + 60 + 96 + 36) + 300
REV_GATHER_BYTES_PER_STEP = 15 * 8 * 32
REV_SCATTER_BYTES_PER_STEP = 5 * 8 * 24


def _adj_plane():
    u = (float(ADJ_CUBE[0] - 1) / ADJ_SEEDS, 0.0, 0.0)
    v = (0.0, float(ADJ_CUBE[1] - 1) / ADJ_SEEDS, 0.0)
    return (0.0, 0.0, 0.0), u, v, ADJ_SEEDS, ADJ_SEEDS


def run_adjoint(args, emit=True):
    """Differentiation workload: d(loss)/dB of the log-Q/Tw misfit on the z=0
    map of a 128x128x64 monopole cube with a twist tube (256x256 seeds). A
    step = repack B with its curl, the taped FP32 map, the loss and its
    gradient, and the reverse sweep into dB (s per gradient). Prints the JSON
    line (emit) and returns it."""
    import torch

    import __graft_entry__
    import oracle
    import synth
    from oracle import adjoint as oadj

    __graft_entry__._builder().build()
    import paper_2208_12569_gb300 as fq

    dev = torch.device("cuda", 0)
    B, Bt, grid = synth.adjoint_cubes(seed=SEED, n=ADJ_CUBE)
    plane = _adj_plane()
    n = ADJ_SEEDS * ADJ_SEEDS
    Bd = torch.from_numpy(B).to(dev)
    # one field per traced precision, as a user would create it (repacking a
    # field repacks every precision it holds); a third with both for the
    # FP64-forward / float-reverse check
    field = fq.Field(Bd, grid.origin, grid.spacing, pack=("f32",))
    field64 = fq.Field(Bd, grid.origin, grid.spacing, pack=("f64",))
    fieldx = fq.Field(Bd, grid.origin, grid.spacing, pack=("f32", "f64"))
    ftgt = fq.Field(torch.from_numpy(Bt).to(dev), grid.origin, grid.spacing, pack=("f32",))
    tgt = fq.qmap_plane(ftgt, *plane, fq.params(precision="f32", tol=TOL))
    out = fq.alloc_out(n, device=dev)
    dB = torch.zeros_like(Bd)
    dB64 = torch.zeros(Bd.shape, dtype=torch.float64, device=dev)
    lbuf = dict(sums=torch.empty(2, dtype=torch.float64, device=dev),
                loss=torch.empty((), dtype=torch.float64, device=dev),
                dQ=torch.empty(n, dtype=torch.float64, device=dev), dTw=torch.empty(n, dtype=torch.float64, device=dev))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    p32 = fq.params(precision="f32", tol=TOL, tape=1)
    p64 = fq.params(precision="f64", tol=TOL, tape=1)

    def step(pp, Bsrc, g):
        fld = field64 if pp.precision == fq.F64 else field
        fld.update(Bsrc)
        fq.qmap_plane(fld, *plane, pp, out=out)
        fq.loss_logq_tw(out["Q"], out["Tw"], tgt["Q"], tgt["Tw"], out["status"], 0.1, out=lbuf)
        g.zero_()
        fq.backward(fld, lbuf["dQ"], lbuf["dTw"], g)

    def timed(pp, g, k):
        ms = []
        for _ in range(k):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(pp, Bd, g)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    def kernel_times(pp, g, k):
        field.set_timing(True)
        fwd, rev, curlt = [], [], []
        for _ in range(k):
            flush.fill_(1.0)
            field.update(Bd)
            fq.qmap_plane(field, *plane, pp, out=out)
            fwd.append(field.times()[0])
            fq.loss_logq_tw(out["Q"], out["Tw"], tgt["Q"], tgt["Tw"], out["status"], 0.1, out=lbuf)
            g.zero_()
            fq.backward(field, lbuf["dQ"], lbuf["dTw"], g)
            t = field.times()
            rev.append(t[0])
            curlt.append(t[2])
        field.set_timing(False)
        return float(np.mean(fwd)), float(np.mean(rev)), float(np.mean(curlt))

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for _ in range(args.warmup):
        step(p32, Bd, dB)
    torch.cuda.synchronize()
    clocks.mark()
    ms32 = timed(p32, dB, args.steps)
    clk = clocks.stop()
    loss32 = float(lbuf["loss"])
    g32 = dB.cpu().numpy().astype(np.float64)
    tape = fq.tape_export(field, n, cap=0)
    acc_steps = float(tape["nsteps"].to(torch.float64).sum())
    trials = float(out["steps"].to(torch.float64).sum())
    t_fwd, t_rev, t_curl = kernel_times(p32, dB, max(3, args.steps // 2))
    # FP64 beside it
    step(p64, Bd, dB64)
    torch.cuda.synchronize()
    ms64 = timed(p64, dB64, max(2, args.fp64_steps))
    loss64 = float(lbuf["loss"])
    g64 = dB64.cpu().numpy()
    # the fixed-step scheme (3/8 rule, Eq. step with step_perp = 3 cells): the
    # same differentiation step, FP32
    pfx = fq.params(precision="f32", tape=1, scheme=1)
    for _ in range(args.warmup):
        step(pfx, Bd, dB)
    torch.cuda.synchronize()
    msfx = timed(pfx, dB, args.steps)
    tfx_fwd, tfx_rev, _ = kernel_times(pfx, dB, max(3, args.steps // 2))
    accfx = float(fq.tape_export(field, n, cap=0)["nsteps"].to(torch.float64).sum())

    # end to end from pinned host memory: B in, loss and dB out
    Bh = torch.from_numpy(B).pin_memory()
    Bdev = torch.empty_like(Bd)
    dBh = torch.empty(Bd.shape, dtype=torch.float32).pin_memory()
    lh = torch.empty((), dtype=torch.float64).pin_memory()
    e2e = []
    for it in range(args.warmup + args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Bdev.copy_(Bh, non_blocking=True)
        step(p32, Bdev, dB)
        dBh.copy_(dB, non_blocking=True)
        lh.copy_(lbuf["loss"], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e.append(e0.elapsed_time(e1))

    # oracle checks on a seeded sample of seeds (weights only there): the
    # FP64 gradient, the float reverse sweep on the FP64 steps, and the FP32
    # gradient; timed as the CPU baseline
    rng = np.random.default_rng(SEED)
    sample = np.sort(rng.choice(n, ADJ_SAMPLE, replace=False))
    wq, wt = rng.standard_normal(ADJ_SAMPLE), rng.standard_normal(ADJ_SAMPLE)
    WQ = torch.zeros(n, dtype=torch.float64, device=dev)
    WT = torch.zeros(n, dtype=torch.float64, device=dev)
    WQ[torch.from_numpy(sample).to(dev)] = torch.from_numpy(wq).to(dev)
    WT[torch.from_numpy(sample).to(dev)] = torch.from_numpy(wt).to(dev)
    B64 = B.astype(np.float64)
    t0 = time.perf_counter()
    ref, info = oadj.vjp_sample(B64, grid, *plane, sample, wq, wt, oracle.params(tol=TOL))
    ora_s = time.perf_counter() - t0

    def gpu_vjp(pp):
        fieldx.update(Bd)
        fq.qmap_plane(fieldx, *plane, pp, out=out)
        g = torch.zeros(Bd.shape, dtype=torch.float64, device=dev)
        fq.backward(fieldx, WQ, WT, g)
        return g.cpu().numpy()

    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))  # noqa: E731
    # the same differentiation step on a stretched grid over the same box (the
    # same sources and tube; horizontal widths growing 1 % per cell from the
    # middle, vertical 2 % per cell upward): FP32 gradient time, FP64 gradient
    # against the oracle's stretched adjoint on the same seed sample
    Bs, Bts, grid_s = synth.adjoint_cubes(seed=SEED, n=ADJ_CUBE, ratios=(1.01, 1.01, 1.02))
    Bsd = torch.from_numpy(Bs).to(dev)
    hi = grid_s.hi
    plane_s = ((0.0, 0.0, 0.0), (hi[0] / ADJ_SEEDS, 0.0, 0.0), (0.0, hi[1] / ADJ_SEEDS, 0.0), ADJ_SEEDS, ADJ_SEEDS)
    fs32 = fq.Field(Bsd, coords=grid_s.coords, pack=("f32",))
    fs64 = fq.Field(Bsd, coords=grid_s.coords, pack=("f64",))
    ftgs = fq.Field(torch.from_numpy(Bts).to(dev), coords=grid_s.coords, pack=("f32",))
    tgs = fq.qmap_plane(ftgs, *plane_s, fq.params(precision="f32", tol=TOL))
    outs_ = fq.alloc_out(n, device=dev)

    def step_s(g):
        fs32.update(Bsd)
        fq.qmap_plane(fs32, *plane_s, p32, out=outs_)
        fq.loss_logq_tw(outs_["Q"], outs_["Tw"], tgs["Q"], tgs["Tw"], outs_["status"], 0.1, out=lbuf)
        g.zero_()
        fq.backward(fs32, lbuf["dQ"], lbuf["dTw"], g)

    for _ in range(args.warmup):
        step_s(dB)
    torch.cuda.synchronize()
    mss = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step_s(dB)
        e1.record(stream)
        torch.cuda.synchronize()
        mss.append(e0.elapsed_time(e1))
    fs64.update(Bsd)
    fq.qmap_plane(fs64, *plane_s, p64, out=outs_)
    gs = torch.zeros(Bsd.shape, dtype=torch.float64, device=dev)
    fq.backward(fs64, WQ, WT, gs)
    fs64.check()
    Bs64 = Bs.astype(np.float64)
    t0 = time.perf_counter()
    ref_s, _ = oadj.vjp_sample(Bs64, grid_s, *plane_s, sample, wq, wt, oracle.params(tol=TOL))
    ora_s_s = time.perf_counter() - t0
    stretched = {"value": float(np.mean(mss)) / 1000.0, "unit": "s/grad", "dtype": "f32",
                 "note": "the same step on a stretched grid over the same box (x, y widths x1.01 per cell from "
                         "the middle, z widths x1.02 per cell upward)",
                 "cell_width_range": [float(min(np.diff(grid_s.axis(a)).min() for a in range(3))),
                                      float(max(np.diff(grid_s.axis(a)).max() for a in range(3)))],
                 "error_vs_oracle": {"f64": rel(gs.cpu().numpy(), ref_s)}, "oracle_sample_s": ora_s_s}
    for fl in (fs32, fs64, ftgs):
        fl.close()
    t0 = time.perf_counter()
    ref_fx, _ = oadj.vjp_sample(B64, grid, *plane, sample, wq, wt, oracle.params(scheme=1))
    ora_fx_s = time.perf_counter() - t0
    errs_fx = {"f64": rel(gpu_vjp(fq.params(precision="f64", tape=1, scheme=1)), ref_fx),
               "f32": rel(gpu_vjp(fq.params(precision="f32", tape=1, scheme=1)), ref_fx)}
    fd = fd_directional(fq, field64, Bd, grid, plane, tgt, g32, g64, n, dev)
    errs = {"f64": rel(gpu_vjp(p64), ref),
            "f64_forward_f32_reverse": rel(gpu_vjp(fq.params(precision="f64", tol=TOL, tape=1,
                                                             reverse_precision="f32")), ref),
            "f32": rel(gpu_vjp(p32), ref),
            "f32_vs_f64_full_loss_gradient": rel(g32, g64),
            "scale_invariance_f32": float(abs(np.sum(g32 * B)) / (np.linalg.norm(g32) * np.linalg.norm(B))),
            "scale_invariance_f64": float(abs(np.sum(g64 * B)) / (np.linalg.norm(g64) * np.linalg.norm(B))),
            "sample_seeds": ADJ_SAMPLE, "sample_lines": int(len(info["lines"]))}
    peaks, peak_kind = _measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    achieved = trials * FLOPS_PER_TRIAL / (t_fwd / 1000.0) / 1e12
    rev_tflops = acc_steps * REV_FLOPS_PER_STEP / (t_rev / 1000.0) / 1e12
    ceil = getattr(args, "ceilings", None)
    # the taped tracer against the measured gather and FMA ceilings (the same
    # work per trial as the map's tracer), else the nominal FP32 issue rate
    if ceil:
        tg = trials * GATHER_BYTES_PER_TRIAL / (t_fwd / 1000.0) / 1e12
        fg, fa = tg / ceil["gather_walk_TBs"], achieved / ceil["fma_f32_TFLOPs"]
        adj_roof = {"bound": "gather" if fg >= fa else "alu", "achieved": tg if fg >= fa else achieved,
                    "peak": ceil["gather_walk_TBs"] if fg >= fa else ceil["fma_f32_TFLOPs"],
                    "unit": "TB/s" if fg >= fa else "TFLOP/s", "frac": max(fg, fa), "traffic": None,
                    "gather": {"achieved_TBs": tg, "ceiling_TBs": ceil["gather_walk_TBs"], "frac": fg},
                    "alu": {"achieved_TFLOPs": achieved, "ceiling_TFLOPs": ceil["fma_f32_TFLOPs"], "frac": fa},
                    "peak_source": "measured on this GPU by the probes (fqsl_probe_gather, fqsl_probe_fma)"}
    else:
        adj_roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved / alu_peak, "traffic": None,
                    "peak_source": "152 SMs x 128 FP32 lanes x 2 x %.0f MHz (%s sm_max_mhz)" % (sm_mhz, peak_kind)}
    adj_roof["kernel"] = "taped lattice tracer k_trace_tape_f32 (%d B, %d flops per trial)" % (
        GATHER_BYTES_PER_TRIAL, FLOPS_PER_TRIAL)
    adj_roof["note"] = ("latency-bound: the longest direction of a line is a chain of dependent gathers "
                        "(the longest line takes 236 trial steps against a mean of 14)")
    s32 = float(np.mean(ms32)) / 1000.0
    line = {"metric": ADJ_METRIC, "value": s32, "unit": "s/grad", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * s32, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": ADJ_WORKLOAD, "cube": list(ADJ_CUBE), "seeds": [ADJ_SEEDS, ADJ_SEEDS],
                       "tol_perp": TOL, "tape_chunk": 16, "loss": "mean (log10 Q - log10 Qt)^2 + 0.1 (Tw - Twt)^2",
                       "l2": "flushed between steps (256 MB write)", "inputs_resident": True},
            "loss": {"f32": loss32, "f64": loss64},
            "fp64": {"value": float(np.mean(ms64)) / 1000.0, "unit": "s/grad"},
            "kernels_ms": {"forward_taped_trace_f32": t_fwd, "reverse_sweep_f32": t_rev, "curl_transpose": t_curl},
            "work": {"trial_steps": trials, "accepted_steps": acc_steps, "accepted_per_half_line": acc_steps / (2 * n)},
            "roofline": adj_roof,
            "reverse_sweep": {"ms": t_rev, "passes": "A1 states, A2 Jacobians, B per-line recurrence, C VJP + scatter",
                              "achieved_TFLOPs": rev_tflops, "frac_of_alu_peak": rev_tflops / alu_peak,
                              "gather_TBs": acc_steps * REV_GATHER_BYTES_PER_STEP / (t_rev / 1000.0) / 1e12,
                              "scatter_GBs": acc_steps * REV_SCATTER_BYTES_PER_STEP / (t_rev / 1000.0) / 1e9},
            "error_vs_oracle": errs,
            "fd_directional": fd,
            "stretched": stretched,
            "fixed_step": {"value": float(np.mean(msfx)) / 1000.0, "unit": "s/grad", "dtype": "f32",
                           "note": "the same differentiation step with the 3/8-rule scheme (step_perp = 3 "
                                   "cells scaled per line by |Bn0/B|, step_min 0.15)",
                           "kernels_ms": {"forward_taped_trace_rk38_f32": tfx_fwd, "reverse_sweep_f32": tfx_rev},
                           "accepted_per_half_line": accfx / (2 * n), "error_vs_oracle": errs_fx,
                           "oracle_sample_s": ora_fx_s},
            "e2e": {"value": float(np.mean(e2e)) / 1000.0, "unit": "s/grad", "h2d_bytes_per_step": int(B.nbytes),
                    "d2h_bytes_per_step": int(B.nbytes + 8)},
            "gpu_launches": 12 * args.steps, "clocks": clk,
            "cpu_baseline": {"value": ora_s * n / ADJ_SAMPLE, "unit": "s/grad", "cores": oracle.max_threads(),
                             "kind": "oracle",
                             "sample": "%d seeded-random seeds (%d lines with their neighbours), %.1f s, scaled "
                                       "by %d" % (ADJ_SAMPLE, len(info["lines"]), ora_s, n // ADJ_SAMPLE)}}
    if emit:
        print(json.dumps(line), flush=True)
    for fl in (field, field64, fieldx, ftgt):
        fl.close()
    return line


def loss_masked(Q, Tw, Qt, Twt, mask, w_tw=0.1):
    """The differentiation workload's loss over a fixed set of seeds (numpy,
    float64): mean of (log10 Q - log10 Qt)^2 + w_tw (Tw - Twt)^2."""
    return float(np.mean((np.log10(Q[mask]) - np.log10(Qt[mask])) ** 2 + w_tw * (Tw[mask] - Twt[mask]) ** 2))


def fd_directional(fq, field64, Bd, grid, plane, tgt, g32, g64, n, dev, ndir=4, eps=(1e-3, 2e-3)):
    """The frozen-sequence gradients (FP32 and FP64 loss gradients of the
    differentiation workload) along smooth directions dB -- the field of one
    extra buried source pair, scaled to rms(dB) = rms(B) -- against central
    differences of the loss of freely re-traced FP64 maps at the same
    tolerance (B +- eps dB, each map traced afresh, its own step sequence),
    over the usable seeds of the unperturbed map."""
    import torch

    import synth

    p = fq.params(precision="f64", tol=TOL)
    B = Bd.double().cpu().numpy()
    Qt, Twt = tgt["Q"].cpu().numpy(), tgt["Tw"].cpu().numpy()

    def traced(Bx):
        field64.update(torch.from_numpy(Bx.astype(np.float32)).to(dev) if Bd.dtype == torch.float32
                       else torch.from_numpy(Bx).to(dev))
        o = fq.qmap_plane(field64, *plane, p)
        return {k: o[k].cpu().numpy() for k in ("Q", "Tw", "status")}

    o0 = traced(B)
    bad = fq.LINE_BAD | fq.LINE_MIXED
    mask = (np.isfinite(o0["Q"]) & np.isfinite(o0["Tw"]) & np.isfinite(Qt) & np.isfinite(Twt) & (o0["Q"] > 0)
            & (Qt > 0) & ((o0["status"] & bad) == 0))
    rng = np.random.default_rng(SEED + 11)
    nx, ny = grid.n[0], grid.n[1]
    rows = []
    for _ in range(ndir):
        ch = synth.random_charges(rng, 2, ((0.0, nx - 1.0), (0.0, ny - 1.0)), depth=(4.0, 16.0))
        dB = synth.monopole_cube(grid, ch, dtype=np.float64)
        dB *= np.sqrt(np.mean(B * B) / np.mean(dB * dB))
        fds = []
        for e in eps:
            op, om = traced(B + e * dB), traced(B - e * dB)
            ok = mask & np.isfinite(op["Q"]) & np.isfinite(om["Q"]) & (op["Q"] > 0) & (om["Q"] > 0)
            fds.append((loss_masked(op["Q"], op["Tw"], Qt, Twt, ok) - loss_masked(om["Q"], om["Tw"], Qt, Twt, ok))
                       / (2.0 * e))
        d64, d32 = float(np.sum(g64 * dB)), float(np.sum(g32 * dB))
        rows.append({"fd": fds, "f64": d64, "f32": d32,
                     "rel_err_f64": abs(d64 - fds[0]) / abs(fds[0]), "rel_err_f32": abs(d32 - fds[0]) / abs(fds[0]),
                     "fd_eps_spread": abs(fds[1] - fds[0]) / abs(fds[0]),
                     "f32_vs_f64": abs(d32 - d64) / abs(d64)})
    traced(B)  # leave the field holding B
    return {"directions": rows, "eps": list(eps), "usable_seeds": int(mask.sum()),
            "median_rel_err_f64": float(np.median([r["rel_err_f64"] for r in rows])),
            "median_rel_err_f32": float(np.median([r["rel_err_f32"] for r in rows])),
            "max_f32_vs_f64": float(max(r["f32_vs_f64"] for r in rows)),
            "stable_directions": [i for i, r in enumerate(rows) if r["fd_eps_spread"] < 0.05],
            "note": "directional derivative of the loss along the field of a buried source pair (rms = rms B); "
                    "central differences of FP64 maps re-traced afresh at the same tolerance, at eps and 2 eps "
                    "(their spread shows how far the free map is from smooth at this tolerance)"}


def run_reference_adjoint(args):
    """The FP64 CPU adjoint oracle on a bounded seeded sample of the
    differentiation workload, scaled to seconds per full gradient."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    import synth
    from oracle import adjoint as oadj

    oracle.build()
    B, _, grid = synth.adjoint_cubes(seed=SEED, n=ADJ_CUBE)
    B64 = B.astype(np.float64)
    plane = _adj_plane()
    n = ADJ_SEEDS * ADJ_SEEDS
    rng = np.random.default_rng(17)
    per_step = 16
    times = []
    for it in range(args.warmup + args.steps):
        sample = np.sort(rng.choice(n, per_step, replace=False))
        t0 = time.perf_counter()
        oadj.vjp_sample(B64, grid, *plane, sample, np.ones(per_step), np.ones(per_step), oracle.params(tol=TOL))
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = float(np.mean(times)) * n / per_step
    line = {"impl": "reference", "metric": ADJ_METRIC, "value": value, "unit": "s/grad", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": ADJ_WORKLOAD, "sample_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "s/grad", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": "%d seeded-random seeds per step, scaled by %d" % (per_step, n // per_step)},
            "e2e": {"value": value, "unit": "s/grad", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fqsl", choices=["fqsl", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="plane workload: skip the adjoint s/grad measurement embedded in its line")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--only-f32", action="store_true",
                    help="time only the FP32 map (no FP64, e2e or CPU legs); used for ncu captures")
    ap.add_argument("--probes-only", action="store_true",
                    help="run only the roofline probes and print their ceilings (for profiling them)")
    ap.add_argument("--no-probes", action="store_true",
                    help="plane workload: skip the roofline probes (the roofline then uses nominal peaks)")
    ap.add_argument("--only-f64", action="store_true",
                    help="time only the FP64 map (no other legs); used for ncu captures of the FP64 tracer")
    ap.add_argument("--no-batch", action="store_true",
                    help="plane workload: skip the 48-cube batch embedded in its line")
    ap.add_argument("--no-volume", action="store_true",
                    help="plane workload: skip the large volume embedded in its line")
    ap.add_argument("--no-stretched", action="store_true",
                    help="plane workload: skip the stretched-grid map embedded in its line")
    ap.add_argument("--workload", default="plane", choices=["plane", "volume", "batch", "adjoint", "stretched"],
                    help="plane: the benchmark line; volume: the large-volume configuration; "
                         "batch: 48 uneven cubes in one launch; adjoint: d(loss)/dB on the 128x128x64 cube; "
                         "stretched: the plane map on a stretched grid")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.workload == "adjoint":
            run_reference_adjoint(args)
        else:
            run_reference(args)
        return
    if args.probes_only:
        # the roofline probes alone (a small command for profiling them)
        import torch

        print(json.dumps({"ceilings": measure_ceilings(torch.device("cuda", 0))}), flush=True)
        return
    if args.workload == "adjoint":
        run_adjoint(args)
        return
    if args.workload == "volume":
        run_volume(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "stretched":
        run_stretched(args)
        return

    import torch

    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    import __graft_entry__

    # one rank builds (a no-op when the library is current); the others wait
    # rather than compile into the same build folder at once
    if rank == 0:
        __graft_entry__._builder().build()
    if dist:
        dist.barrier()
    import paper_2208_12569_gb300 as fq

    B, grid, u, v = monopole24_inputs(rank)
    Bd = torch.from_numpy(B).to(dev)
    field32 = fq.Field(Bd, grid.origin, grid.spacing, pack=("f32",))
    field64 = fq.Field(Bd, grid.origin, grid.spacing, pack=("f64",))
    field32.set_timing(True)
    field64.set_timing(True)
    n = NU * NV
    out = fq.alloc_out(n, device=dev)
    p32 = fq.params(precision="f32", tol=TOL)
    pacc = fq.params(precision="f32acc64", tol=TOL)
    p64 = fq.params(precision="f64", tol=TOL)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def step(p):
        fld = field64 if p.precision == fq.F64 else field32
        fq.qmap_plane(fld, (0.0, 0.0, 0.0), u, v, NU, NV, p, out=out)

    def timed(p, k):
        fld = field64 if p.precision == fq.F64 else field32
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        kern = []
        for e0, e1 in ev:
            flush.fill_(1.0)
            e0.record(stream)
            step(p)
            e1.record(stream)
            kern.append(fld.times())
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in ev], kern

    if args.only_f64:
        # the FP64 map alone (a small command for profiling its tracer)
        for _ in range(args.warmup):
            step(p64)
        torch.cuda.synchronize()
        ms, kern = timed(p64, args.steps)
        field64.check()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": n / (float(np.mean(ms)) / 1000.0), "unit": "Q+Tw values/s",
                              "ms_per_step": float(np.mean(ms)),
                              "kernels_ms": {"trace_f64": float(np.mean([k[0] for k in kern]))},
                              "config": {"workload": WORKLOAD}, "partial": "only-f64"}), flush=True)
        return
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for _ in range(args.warmup):
        step(p32)
    field32.check()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark()
    ms32, kern32 = timed(p32, args.steps)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    res32 = {k: t.cpu().numpy() for k, t in out.items() if t is not None}
    if args.only_f32:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": n * ws / (float(np.mean(ms32)) / 1000.0),
                              "unit": "Q+Tw values/s", "ms_per_step": float(np.mean(ms32)),
                              "kernels_ms": {"trace_f32": float(np.mean([k[0] for k in kern32]))},
                              "config": {"workload": WORKLOAD}, "partial": "only-f32"}), flush=True)
        return
    # Method II (deviation vectors) on the same map, both ways of grad(B/|B|)
    fieldg = fq.Field(Bd, grid.origin, grid.spacing, pack=("f32", "gradb"))
    m2, leg_res = {}, {}
    for way, qperp in ((1, 0), (2, 0), (1, 1)):
        pm2 = fq.params(precision="f32", tol=TOL, method=2, gradb_way=way, qperp=qperp)
        fq.qmap_plane(fieldg, (0.0, 0.0, 0.0), u, v, NU, NV, pm2, out=out)
        torch.cuda.synchronize()
        tms = []
        for _ in range(max(3, args.steps // 2)):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fq.qmap_plane(fieldg, (0.0, 0.0, 0.0), u, v, NU, NV, pm2, out=out)
            e1.record(stream)
            torch.cuda.synchronize()
            tms.append(e0.elapsed_time(e1))
        key = "way%d" % way + ("_qperp" if qperp else "")
        m2[key] = {"value": n / (float(np.mean(tms)) / 1000.0), "unit": "Q+Tw values/s",
                   "ms_per_step": float(np.mean(tms))}
        leg_res[("method2_f32", key)] = ({k: t.cpu().numpy() for k, t in out.items() if t is not None},
                                        dict(method=2, way=way, qperp=qperp))
    fieldg.close()
    # the paper's fixed-step scheme on the same map: 3/8-rule RK4, step_perp = 3 cells (Table 1), Eq. step
    rk = {}
    for prec in ("f32", "f64"):
        prk = fq.params(precision=prec, tol=TOL, scheme=1, step=3.0)
        fld = field64 if prec == "f64" else field32
        fq.qmap_plane(fld, (0.0, 0.0, 0.0), u, v, NU, NV, prk, out=out)
        torch.cuda.synchronize()
        tms = []
        for _ in range(max(3, (args.steps if prec == "f32" else args.fp64_steps))):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fq.qmap_plane(fld, (0.0, 0.0, 0.0), u, v, NU, NV, prk, out=out)
            e1.record(stream)
            torch.cuda.synchronize()
            tms.append(e0.elapsed_time(e1))
        rk[prec] = {"value": n / (float(np.mean(tms)) / 1000.0), "unit": "Q+Tw values/s",
                    "ms_per_step": float(np.mean(tms)),
                    "mean_trials_per_line": float(out["steps"].double().mean())}
        leg_res[("fixed_step_rk38", prec)] = ({k: t.cpu().numpy() for k, t in out.items() if t is not None},
                                             dict(scheme=1, step=3.0))
    step(pacc)
    torch.cuda.synchronize()
    msacc, kernacc = timed(pacc, args.steps)
    resacc = {k: t.cpu().numpy() for k, t in out.items() if t is not None}
    step(p64)
    torch.cuda.synchronize()
    ms64, kern64 = timed(p64, args.fp64_steps)
    res64 = {k: t.cpu().numpy() for k, t in out.items() if t is not None}

    ms_step, value = job_rate(float(np.mean(ms32)), n, dist, dev)
    value64 = n / (float(np.mean(ms64)) / 1000.0)

    # end to end through the C ABI from pinned host memory
    Bh = torch.from_numpy(B).pin_memory()
    Bdev = torch.empty_like(Bd)
    Qh = torch.empty(n, dtype=torch.float64).pin_memory()
    Twh = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Bdev.copy_(Bh, non_blocking=True)
        field32.update(Bdev)
        step(p32)
        Qh.copy_(out["Q"], non_blocking=True)
        Twh.copy_(out["Tw"], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_serial = n * ws / (float(np.mean(e2e_ms)) / 1000.0)
    assert np.array_equal(np.isnan(Qh.numpy()), np.isnan(res32["Q"]))

    # the same, pipelined as a serving loop would run it: two field handles,
    # two device copies of B and two output sets alternate. Step k's
    # host-to-device copy and repack (upload stream) overlap step k-1's map
    # (compute stream), and its device-to-host copy of Q and Tw (download
    # stream) overlaps step k+1's map. Every step still copies its B in,
    # repacks, maps and reads Q and Tw back; L2 is flushed before every map;
    # the timed region spans all K steps.
    fields = [field32, fq.Field(Bd, grid.origin, grid.spacing, pack=("f32",))]
    Bdevs = [Bdev, torch.empty_like(Bd)]
    outs = [out, fq.alloc_out(n, device=dev)]
    Qhs = [Qh, torch.empty(n, dtype=torch.float64).pin_memory()]
    Twhs = [Twh, torch.empty(n, dtype=torch.float64).pin_memory()]
    s_up, s_comp, s_down = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    mapped = [torch.cuda.Event(), torch.cuda.Event()]  # the map of fields[b] into outs[b] is done
    loaded = [torch.cuda.Event(), torch.cuda.Event()]  # fields[b] holds this step's records
    copied = [torch.cuda.Event(), torch.cuda.Event()]  # outs[b] has been read back
    for b in range(2):
        mapped[b].record(s_comp)
        copied[b].record(s_down)

    def pipe_step(k):
        b = k % 2
        with torch.cuda.stream(s_up):
            Bdevs[b].copy_(Bh, non_blocking=True)  # Bdevs[b]: last read by this stream's repack
            s_up.wait_event(mapped[b])  # the map two steps back is done with fields[b]
            fields[b].update(Bdevs[b], stream=s_up)
            loaded[b].record(s_up)
        with torch.cuda.stream(s_comp):
            s_comp.wait_event(loaded[b])
            s_comp.wait_event(copied[b])
            flush.fill_(1.0)
            fq.qmap_plane(fields[b], (0.0, 0.0, 0.0), u, v, NU, NV, p32, out=outs[b], stream=s_comp)
            mapped[b].record(s_comp)
        with torch.cuda.stream(s_down):
            s_down.wait_event(mapped[b])
            Qhs[b].copy_(outs[b]["Q"], non_blocking=True)
            Twhs[b].copy_(outs[b]["Tw"], non_blocking=True)
            copied[b].record(s_down)

    for k in range(args.warmup):
        pipe_step(k)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(s_up)
    s_comp.wait_event(p0)
    s_down.wait_event(p0)
    for k in range(args.warmup, args.warmup + args.steps):
        pipe_step(k)
    s_comp.wait_stream(s_up)
    s_comp.wait_stream(s_down)
    p1.record(s_comp)
    torch.cuda.synchronize()
    e2e_pipe_ms = p0.elapsed_time(p1) / args.steps
    e2e_value = n * ws / (e2e_pipe_ms / 1000.0)
    for b in range(2):
        assert np.array_equal(np.isnan(Qhs[b].numpy()), np.isnan(res32["Q"]))
    fields[1].close()

    # roofline of the dominant kernel (the FP32 tracer): its time, and the
    # ceilings of its gather and FMA work measured on this GPU by the probes
    trials = float(res32["steps"].astype(np.int64).sum())
    trace_ms = float(np.mean([k[0] for k in kern32]))
    trace64_ms = float(np.mean([k[0] for k in kern64]))
    asm_ms = float(np.mean([k[2] for k in kern32]))
    ceilings = None if args.no_probes else measure_ceilings(dev)

    line = {"metric": METRIC, "value": value, "unit": "Q+Tw values/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cube": list(CUBE), "seeds": [NU, NV], "tol_perp": TOL,
                       "method": 1, "l2": "flushed between steps (256 MB write)", "inputs_resident": True},
            "f32_acc64": {"value": n / (float(np.mean(msacc)) / 1000.0), "unit": "Q+Tw values/s",
                          "ms_per_step": float(np.mean(msacc)),
                          "trace_ms": float(np.mean([k[0] for k in kernacc])),
                          "note": "error norm and length/Tw sums accumulated in FP64 every step"},
            "method2_f32": dict(m2, note="deviation vectors (Method II), tol = tol_perp, same map; "
                                         "_qperp: Q_perp, end planes perpendicular to B"),
            "fixed_step_rk38": dict(rk, note="Method I, 3/8-rule RK4, step_perp = 3 cells scaled per line by "
                                             "Eq. step (step_min 0.15), same map"),
            "fp64": {"value": value64, "unit": "Q+Tw values/s", "ms_per_step": float(np.mean(ms64)),
                     "trace_ms": float(np.mean([k[0] for k in kern64])),
                     "speedup_fp32_over_fp64": value / ws / value64},
            "kernels_ms": {"trace_f32": trace_ms, "trace_f64": trace64_ms, "assemble": asm_ms},
            "work": {"trial_steps_per_map_f32_tracer": trials, "mean_trials_per_line_f32_tracer": trials / n,
                     "trial_steps_per_map_f64_tracer": float(res64["steps"].astype(np.int64).sum())},
            "e2e": {"value": e2e_value, "unit": "Q+Tw values/s", "ms_per_step": e2e_pipe_ms,
                    "h2d_bytes_per_step": int(B.nbytes), "d2h_bytes_per_step": int(2 * n * 8),
                    "note": "per step: H2D of B from pinned memory, repack (curl), map, D2H of Q and Tw; "
                            "pipelined over three streams (step k's copy and repack overlap step k-1's map, "
                            "its read-back step k+1's map), L2 flushed before each map",
                    "serial": {"value": e2e_serial, "ms_per_step": float(np.mean(e2e_ms))}},
            "gpu_launches": 3 * args.steps, "clocks": clk}
    if rank == 0 and ws == 1 and not args.no_adjoint:
        # the metric's second part: seconds per gradient of the differentiation workload
        a = run_adjoint(argparse.Namespace(steps=args.steps, warmup=args.warmup, fp64_steps=args.fp64_steps,
                                           ceilings=ceilings), emit=False)
        line["adjoint"] = {k: a[k] for k in ("metric", "value", "unit", "ms_per_step", "higher_is_better", "config",
                                             "fp64", "kernels_ms", "error_vs_oracle", "e2e", "cpu_baseline",
                                             "roofline", "reverse_sweep", "loss", "fixed_step", "stretched",
                                             "fd_directional")}
    if rank == 0 and ws == 1 and not args.no_batch:
        # the batched uneven workload (48 cubes, one graph-captured autotuned launch)
        bt = run_batch(argparse.Namespace(steps=args.steps, warmup=args.warmup), emit=False)
        line["batch"] = {k: bt[k] for k in ("value", "unit", "config", "per_cube_launches", "batch_run",
                                            "batch_graph", "batch_graph_autotuned", "fp64_batch_run",
                                            "error_vs_oracle_sample", "cpu_baseline")}
        line["batch"]["batch_graph_autotuned"] = {k: v for k, v in bt["batch_graph_autotuned"].items() if k != "table"}
        line["batch"]["speedup_over_per_cube_launches"] = bt["value"] / bt["per_cube_launches"]["value"]
    if rank == 0 and ws == 1 and not args.no_volume:
        # the large volume (1024^2 x 512 cube, 512^2 x 256 seeds, 4096^2 map)
        vl = run_volume(argparse.Namespace(no_cpu_baseline=args.no_cpu_baseline), emit=False)
        line["volume"] = {k: vl[k] for k in vl if k not in ("metric", "workload")}
    if rank == 0 and ws == 1 and not args.no_stretched:
        # the same map on a stretched grid (its oracle check runs in the tests and in --workload stretched)
        st = run_stretched(argparse.Namespace(steps=args.steps, warmup=args.warmup, fp64_steps=args.fp64_steps,
                                              no_cpu_baseline=True), emit=False)
        line["stretched"] = {k: st[k] for k in ("value", "unit", "ms_per_step", "config", "f32_acc64", "fp64",
                                                "kernels_ms", "work", "uniform_f32")}
    ref = sample = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb, sample, ref = cpu_baseline(B, grid, u, v)
        line["cpu_baseline"] = cb
        line["error_vs_oracle"] = {"f32": err_stats(res32, ref, sample), "f32_acc64": err_stats(resacc, ref, sample),
                                   "f64": err_stats(res64, ref, sample)}
        # the Method II and fixed-step legs against the oracle on a seeded
        # 4000-seed sample of the same lattice
        import oracle

        B64 = B.astype(np.float64)
        Jo, Go = oracle.curl(B64, grid), oracle.gradb(B64, grid)
        es = np.sort(np.random.default_rng(SEED + 7).choice(n, 4000, replace=False))
        # accuracy against the map itself: a converged oracle reference
        # (tol_perp = 1e-10) on the same 4000 seeds, so that FP32 rounding is
        # stated beside FP64's own integration error at the benchmark tolerance
        t0 = time.perf_counter()
        conv = oracle.plane(B64, grid, (0.0, 0.0, 0.0), u, v, NU, NV, oracle.params(tol=CONVERGED_TOL), sample=es,
                            J=Jo)
        conv_s = time.perf_counter() - t0
        acc = {"reference": "oracle at tol_perp = %g on %d seeded-random seeds (%.1f s)" % (CONVERGED_TOL, len(es),
                                                                                              conv_s),
               "f32": err_stats(res32, conv, es), "f32_acc64": err_stats(resacc, conv, es),
               "f64": err_stats(res64, conv, es)}
        acc["f32_p99_over_f64_p99"] = acc["f32"]["q_rel_p99"] / max(acc["f64"]["q_rel_p99"], 1e-300)
        line["accuracy_vs_converged"] = acc
        for (leg, key), (res, kw) in leg_res.items():
            ref_l = oracle.plane(B64, grid, (0.0, 0.0, 0.0), u, v, NU, NV, oracle.params(tol=TOL, **kw), sample=es,
                                 J=Jo, G=Go if kw.get("way") == 1 else None)
            e = err_stats(res, ref_l, es)
            e["bitwise"] = bool(all(np.array_equal(res[k][es], ref_l[k], equal_nan=True)
                                    for k in ("Q", "Tw", "face1", "face2", "status")))
            line[leg][key]["error_vs_oracle"] = e
    # the algorithmic trial count: the oracle's counters on its sample, scaled
    # to the map (the FP64 tracer's own counts, which equal the oracle's step
    # for step, without the CPU leg); GPU FP32 retries do not count
    if ref is not None:
        trials_alg = float(ref["steps"].astype(np.int64).sum()) * n / len(sample)
        work_src = "oracle trial counters on %d of %d seeds, scaled" % (len(sample), n)
    else:
        trials_alg = float(res64["steps"].astype(np.int64).sum())
        work_src = "FP64 tracer trial counters (equal to the oracle's)"
    line["work"]["trial_steps_per_map_algorithmic"] = trials_alg
    line["work"]["algorithmic_source"] = work_src
    line["roofline"] = roofline(trials_alg, trace_ms, trace64_ms, ceilings, work_src)
    if rank == 0:
        print(json.dumps(line), flush=True)
    field32.close()
    field64.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
