#!/usr/bin/env python3
"""Benchmark of RM synthesis on GB300: one JSON line on rank 0.

A step is one rms_synth call over the MWA-like large-phase cube (1024^2 LOS x
1536 channels 72-231 MHz x 4001 phi in [-2000, 2000] rad/m^2; FP32 Q/U
resident in HBM, complex64 F (33.6 GB) and the peak map written back to HBM)
with the plan built once beforehand (the phase matrix and RMSF are
per-dataset constants, Sec. 2.3).  The metric is G(LOS * active channel * phi)/s.
The same JSON line carries, as sub-objects, the LOFAR-HBA-like cube
(512^2 x 400 x 401, `lofar`) and the learned peak proposal on its 2048^2-LOS
workload (`learned`), each with its own error against the FP64 oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--path bf16x3] [--layout chan]
  python bench.py --config lofar | precision | lofar_lr | lofar_hr [--peak-only]
  python bench.py --config learned   (the learned peak proposal against the full grid alone)
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)

The cube is generated on the device by the seeded generator's device twin; the
rows the CPU oracle checks are regenerated on the host.

Multi-GPU (torchrun): every rank synthesises its own full cube (weak scaling,
no collective on the data path); value = all ranks' units / max rank time.
"""
from __future__ import annotations

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

METRIC = "RM-synth G(LOS*chan*phi)/s at stated error vs FP64"
UNIT = "G(LOS*chan*phi)/s"
CONFIG_NAME = "mwa"
# timed steps per workload when --steps is not given: about 5 s of timed work
DEFAULT_STEPS = {"mwa": 40, "precision": 60, "lofar_lr": 150, "lofar_hr": 3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="bf16x3")
    ap.add_argument("--layout", default="chan", choices=["chan", "los"])
    ap.add_argument("--config", default=CONFIG_NAME)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-paths", action="store_true", help="skip timing the other precision paths")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--nlos", type=int, default=None, help="override the workload's LOS count (profiling runs)")
    ap.add_argument("--peak-only", action="store_true", help="write the peak map only, no F cube")
    ap.add_argument("--no-clean", action="store_true", help="skip timing RM-CLEAN of the synthesised cube")
    ap.add_argument("--n-train", type=int, default=1 << 20, help="learned workload: training LOS")
    ap.add_argument("--epochs", type=int, default=8, help="learned workload: training epochs")
    ap.add_argument("--hidden", type=int, default=256, help="learned workload: hidden units")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the LOFAR and learned sub-objects of the default run")
    a = ap.parse_args()
    if a.steps is None:
        a.steps = DEFAULT_STEPS.get(a.config, 200 if a.config != "learned" else 20)
    return a


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="rms_clocks_%d_" % self.dev, suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()
        return False

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        # samples under load only: drop the idle head/tail below 50% of max
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        try:
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons), "samples": len(sm)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import dataclasses
    from paper_1810_06250_gb300 import inputs
    cfg = inputs.CONFIGS[args.config]
    if args.nlos is not None:
        cfg = dataclasses.replace(cfg, nlos=args.nlos)
    freq, w, phi = inputs.frequencies(cfg), inputs.weights(cfg), inputs.phi_grid(cfg)
    import oracle
    oracle.build()
    op = oracle.plan(freq, "freq", w)
    nact = int(np.count_nonzero(w))
    # each step = a bounded sample so that the whole run ends within a few minutes; the
    # sample's LOS are generated on the host as they are needed
    # the oracle deals LOS to its threads 16 at a time: calibrate and sample in whole
    # rounds of 16 LOS per thread, so that every host core works
    budget = 150.0
    rnd = 16 * max(1, oracle.num_threads())
    Q, U = inputs.make_cube(cfg, 0, min(cfg.nlos, rnd))
    t0 = time.perf_counter()
    oracle.synth(Q, U, op, phi)
    per_los = (time.perf_counter() - t0) / len(Q)
    n = int(budget / max(1, args.steps + args.warmup) / per_los) // rnd * rnd
    n = int(min(cfg.nlos, max(rnd, n)))
    pool = min(cfg.nlos, 4 * n)
    Q, U = inputs.make_cube(cfg, 0, pool)
    for i in range(args.warmup):
        oracle.synth(Q[:n], U[:n], op, phi)
    times = []
    for i in range(args.steps):
        s = (i * n) % max(1, pool - n)
        t0 = time.perf_counter()
        oracle.synth(Q[s:s + n], U[s:s + n], op, phi)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    units = n * nact * len(phi) * len(times)
    v = units / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(cfg, nact, args.layout, False, world),
            "sample_los_per_step": n,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d LOS per step of %d" % (n, cfg.nlos)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_value(kernel_src: str, summary: str, key: str):
    """A `key: value` line of a committed ncu summary, or None when the kernel source
    has changed since the counters were taken (sha256 prefix recorded there)."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
        m = re.search(r"%s: ([0-9.]+)" % re.escape(key), text)
        h = re.search(r"sha256\[:16\] ([0-9a-f]{16})", text)
        src = open(os.path.join(ROOT, "paper_1810_06250_gb300", "csrc", kernel_src), "rb").read()
        if m and h and hashlib.sha256(src).hexdigest()[:16] == h.group(1):
            return float(m.group(1))
    except OSError:
        pass
    return None


def measured_traffic(kernel_src: str, summary: str):
    """DRAM bytes per launch from a committed ncu summary (None when the source changed)."""
    v = profile_value(kernel_src, summary, "traffic_bytes_per_launch")
    return None if v is None else int(v)


def workload_config(cfg, nact, layout, peak_only=False, world=1):
    """The `config` object of a bench line: the workload, identical in both arms."""
    L = cfg.nlos
    return {"workload": workload_name(cfg, nact, layout, peak_only), "nlos_per_gpu": L,
            "nchan": cfg.nchan, "nchan_active": nact, "nphi": cfg.nphi, "layout": layout,
            "l2": "inputs larger than L2 (%.2f GB in%s per step)"
                  % (L * cfg.nchan * 8 / 1e9, "" if peak_only else ", %.2f GB out" % (L * cfg.nphi * 8 / 1e9)),
            "parallelism": "replicas" if world > 1 else "single GPU",
            "units_per_step_total_channels": L * cfg.nchan * cfg.nphi,
            "inputs": "device-generated by the seeded generator's device twin; the CPU sample is "
                      "regenerated on the host"}


def workload_name(cfg, nact, layout, peak_only=False):
    side = int(round(cfg.nlos ** 0.5))
    shape = "%dx%d LOS" % (side, side) if side * side == cfg.nlos else "%d LOS" % cfg.nlos
    return ("%s: %s x %d channels (%d active) %.3f-%.3f MHz x %d phi in [%g, %g] rad/m^2, FP32 Q/U %s-major, %s"
            % (cfg.name, shape, cfg.nchan, nact, cfg.nu0 / 1e6, cfg.nu1 / 1e6, cfg.nphi, cfg.phi_min, cfg.phi_max,
               layout, "peak map only" if peak_only else "complex64 F + peak map"))


def time_steps(fn, stream, steps, warmup, torch, barrier=None):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for i in range(steps):
        fn()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    total = ev[0].elapsed_time(ev[-1])
    if barrier:
        barrier()
    return total, per


def sample_rows(cfg, n, rng):
    """About n LOS in 64-row blocks spread over the cube: (rows, host Q, host U) regenerated on the
    host by the seeded generator (inputs.make_cube), as the oracle's input."""
    from paper_1810_06250_gb300 import inputs
    blk = 64
    nb = max(1, min(n // blk, cfg.nlos // blk))
    starts = np.sort(rng.choice(cfg.nlos // blk, nb, replace=False)) * blk
    Qs, Us = zip(*(inputs.make_cube(cfg, int(s0), blk) for s0 in starts))
    rows = (starts[:, None] + np.arange(blk)[None, :]).ravel()
    return rows, np.concatenate(Qs), np.concatenate(Us)


def oracle_sample(cfg, freq, w, phi, L, seconds):
    """The FP64 oracle, as it stands, on all host cores over a LOS sample of about `seconds` of
    work: the CPU baseline and the reference values of the error check."""
    import oracle
    from paper_1810_06250_gb300 import inputs
    oracle.build()
    op = oracle.plan(freq, "freq", w)
    nact = int(np.count_nonzero(w))
    # calibrate on enough LOS to keep every host core busy, then size the sample
    ncal = int(min(L, 64 * max(1, oracle.num_threads())))
    Qc, Uc = inputs.make_cube(cfg, 0, ncal)
    t0 = time.perf_counter()
    oracle.synth(Qc, Uc, op, phi)
    per_los = (time.perf_counter() - t0) / ncal
    n = int(min(L, max(256, seconds / per_los)))
    rows, Qs, Us = sample_rows(cfg, n, np.random.default_rng(12345))
    t0 = time.perf_counter()
    Fo = oracle.synth(Qs, Us, op, phi)
    dt = time.perf_counter() - t0
    base = {"value": len(rows) * nact * cfg.nphi / dt / 1e9, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "%d of %d LOS in 64-LOS blocks (all %d active channels x %d phi), FP64 C oracle, OpenMP over "
                      "LOS, %.1f s" % (len(rows), L, nact, cfg.nphi, dt)}
    return {"rows": rows, "Fo": Fo, "peak": oracle.peak(Fo), "plan": op, "baseline": base}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def tensor_roofline(path, useful_flops, kt, timed_s, peaks, traffic, step_ms, hbm_bytes):
    """Roofline of the contraction kernel (the dominant one): the method's own work,
    8 flop per (LOS, active channel, phi) unit, over the dense BF16 tensor peak.
    The split precisions issue three 16-bit products per useful flop, so they can
    reach at most 1/3 of that peak; the issued products are reported beside it."""
    terms = 1 if path == "bf16" else 3
    burst, sust = peaks.get("bf16_tflops"), peaks.get("bf16_tflops_sustained")
    kind = "measured"
    if not burst or not sust:
        burst, sust, kind = 1900.0, 1700.0, "fallback"
    long_region = timed_s >= 1.0
    peak = sust if long_region else burst
    split_ms, gemm_ms, ncalls = kt
    gemm_launch_ms = gemm_ms / max(1, ncalls)
    achieved = useful_flops / (gemm_launch_ms * 1e-3) / 1e12
    return {"kernel": "gemm_kernel (tensor-core contraction + fused epilogue)", "bound": "tensor",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "peak_source": "%s %s dense BF16 tensor peak (MEASURED_PEAKS.json %s): the timed region lasted %.2f s, %s"
                           % (kind, "sustained" if long_region else "burst",
                              "bf16_tflops_sustained" if long_region else "bf16_tflops", timed_s,
                              "seconds-long, so the sustained figure applies" if long_region
                              else "shorter than 1 s, so the burst figure applies"),
            "frac_of_burst": achieved / burst, "frac_of_sustained": achieved / sust,
            "issued_products_per_flop": terms, "issued_tflops": achieved * terms,
            "issued_frac": achieved * terms / peak, "split_ceiling_frac": 1.0 / terms,
            "launch_ms": gemm_launch_ms, "split_launch_ms": split_ms / max(1, ncalls), "timed_launches": ncalls,
            "step_frac": useful_flops / (step_ms * 1e-3) / 1e12 / peak,
            "hbm_gbs_step": hbm_bytes / (step_ms * 1e-3) / 1e9,
            "algorithmic": "8 flop per (LOS, active channel, phi) unit (one complex multiply-add); achieved = "
                           "algorithmic flop per launch / the contraction kernel's CUDA-event duration (the "
                           "library's event hook on the launching stream, averaged over the timed launches); "
                           "FP16 and BF16 share the dense tensor rate; a split precision issues %d 16-bit products "
                           "per flop, so split_ceiling_frac is its best possible frac" % terms}


def measure_cube(args, cfg_name, path, layout, steps, warmup, dev, local, world=1, barrier=None, nlos=None,
                 peak_only=False, with_paths=False, with_e2e=False, with_cpu=False, with_clean=False,
                 cpu_seconds=15.0):
    """Time rms_synth on one workload; return the result fields of a bench line."""
    import dataclasses
    import torch
    import paper_1810_06250_gb300 as rms
    from paper_1810_06250_gb300 import inputs, learned as Lm
    from paper_1810_06250_gb300.dist import throughput
    cfg = inputs.CONFIGS[cfg_name]
    if nlos is not None:
        cfg = dataclasses.replace(cfg, nlos=nlos)
    freq, w, phi = inputs.frequencies(cfg), inputs.weights(cfg), inputs.phi_grid(cfg)
    nact = int(np.count_nonzero(w))
    L = cfg.nlos
    peak_only = peak_only or L * cfg.nphi * 8 > 64e9     # F of the 4000^2 x 7000 cube is 0.9 TB
    stream = torch.cuda.Stream(dev)
    units = L * nact * cfg.nphi

    t_plan0 = time.perf_counter()
    plan = rms.Plan(freq, phi, path, weights=w, device=local)
    plan_ms = 1e3 * (time.perf_counter() - t_plan0)
    # the cube is generated on the device by the seeded generator's device twin
    q, u = Lm.generate(plan.handle, cfg, 0, L, layout)
    F = None if peak_only else torch.empty(L, cfg.nphi, 2, device=dev)
    pidx = torch.empty(L, dtype=torch.int32, device=dev)
    pabs = torch.empty(L, device=dev)
    pphi = torch.empty(L, device=dev)

    def step():
        plan.synth(q, u, L, layout, F, pidx, pabs, pphi, stream)

    tensor_path = path in ("bf16", "bf16x3", "fp16x3")
    with torch.cuda.stream(stream):
        with ClockSampler(local) as clk:
            for _ in range(warmup):
                step()
            # the library records events around its two kernels on this stream
            if tensor_path:
                rms.rms_plan_set_kernel_timing(plan.handle, True)
            total_ms, per = time_steps(step, stream, steps, 0, torch, barrier)
            if tensor_path:
                rms.rms_plan_set_kernel_timing(plan.handle, False)
    plan.sync(stream)
    kt = rms.rms_plan_kernel_times(plan.handle) if tensor_path else (0.0, 0.0, 0)
    sched = {k: rms.rms_plan_info(plan.handle, v) for k, v in
             (("ctas", rms.RMS_INFO_LAST_CTAS), ("cta_pairs", rms.RMS_INFO_LAST_PAIR),
              ("n_panels", rms.RMS_INFO_LAST_PANELS), ("kernels_per_step", rms.RMS_INFO_LAST_KERNELS))} \
        if tensor_path else None
    value, tmax = throughput(units, steps, total_ms, world, dev)
    avg_launch_ms = statistics.mean(per)

    peaks = load_peaks()
    useful_flops = 8.0 * units
    hbm_bytes = L * (8.0 * (nact if layout == "chan" else cfg.nchan) + (0 if peak_only else 8.0 * cfg.nphi) + 12.0)
    full_size = nlos is None and not peak_only
    if tensor_path:
        traffic = measured_traffic("gemm.cu", "gemm_%s_bf16x3.md" % cfg_name) \
            if (path == "bf16x3" and layout == "chan" and full_size) else None
        roof = tensor_roofline(path, useful_flops, kt, total_ms * 1e-3, peaks, traffic, avg_launch_ms, hbm_bytes)
        if traffic is not None:
            # the ncu counters of the same capture (a smaller case of this workload, same kernel source)
            roof["ncu"] = {"summary": "profiles/gemm_%s_bf16x3.md" % cfg_name,
                           "tensor_pipe_active_pct": profile_value("gemm.cu", "gemm_%s_bf16x3.md" % cfg_name,
                                                                   "tensor_pipe_active_pct"),
                           "dram_throughput_pct": profile_value("gemm.cu", "gemm_%s_bf16x3.md" % cfg_name,
                                                                "dram_throughput_pct"),
                           "hbm_gbs_full_size": traffic / (roof["launch_ms"] * 1e-3) / 1e9}
        roof["schedule"] = dict(sched, note="n_panels 0: each CTA runs every phase tile of its M tile; k > 0: "
                                            "single-tile jobs in k panels of the phase matrix, peaks merged by "
                                            "64-bit atomics and a finalize kernel")
    elif path == "fp32_czt":
        # FFT synthesis: algorithmic work counted the usual way for FFTs, 5 M log2 M flop per
        # complex length-M transform (two per LOS), 6 flop per complex product (the spectrum
        # times H, and the pre- and post-chirps); bytes are the cube in and F out
        props = torch.cuda.get_device_properties(dev)
        clk_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = props.multi_processor_count * 128 * 2 * clk_mhz * 1e6 / 1e12
        M = 1024
        while M < cfg.nchan + cfg.nphi - 1:
            M *= 2
        fft_flops = L * (2 * 5.0 * M * np.log2(M) + 6.0 * M + 6.0 * (nact + cfg.nphi))
        achieved = fft_flops / (avg_launch_ms * 1e-3) / 1e12
        hbm_peak = peaks.get("hbm_gbs") or 6800.0
        hbm_gbs = hbm_bytes / (avg_launch_ms * 1e-3) / 1e9
        traffic = measured_traffic("czt.cu", "czt_lofar_ul2.md") \
            if (cfg_name == "lofar_ul2" and layout == "chan" and full_size) else None
        roof = {"kernel": "czt_kernel", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "peak_source": "SMs x 128 FP32 lanes x 2 x max SM clock", "fft_length": M,
                "hbm_gbs": hbm_gbs, "hbm_frac": hbm_gbs / hbm_peak,
                "algorithmic": "per LOS 2 x 5 M log2 M + 6 M + 6 (active channels + nphi) flop; "
                               "achieved = that / the kernel's CUDA-event duration",
                "note": "an FFT is mostly additions, one flop per FP32 instruction against two for an FMA, so "
                        "the FMA-flop peak overstates what it can reach; ncu counts the issue slots instead "
                        "(profiles/czt_lofar_ul2.md)"}
    else:
        props = torch.cuda.get_device_properties(dev)
        clk_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = props.multi_processor_count * 128 * 2 * clk_mhz * 1e6 / 1e12
        achieved = useful_flops / (avg_launch_ms * 1e-3) / 1e12
        traffic = measured_traffic("simt.cu", "simt_lofar_fp32_table.md") \
            if (path == "fp32_table" and layout == "chan" and cfg_name == "lofar" and full_size) else None
        roof = {"kernel": "simt_kernel", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": traffic, "traffic_unit": "bytes per launch (ncu dram read + write)",
                "peak_source": "SMs x 128 FP32 lanes x 2 x max SM clock",
                "hbm_gbs": hbm_bytes / (avg_launch_ms * 1e-3) / 1e9}

    in_gb = L * cfg.nchan * 8 / 1e9
    res = {"value": value, "unit": UNIT, "ms_per_step": tmax / steps, "steps": steps, "warmup": warmup,
           "dtype": path,
           "config": workload_config(cfg, nact, layout, peak_only, world),
           "roofline": roof, "gpu_launches": steps * (sched["kernels_per_step"] if sched else 1), "plan_ms": plan_ms,
           "clocks": clk.summary()}

    # end to end through host buffers, right after the device-timed region (before the
    # CPU oracle and the other paths run)
    if with_e2e and in_gb < 32:
        # page-locked host buffers from the library's allocator (registered huge-page memory)
        hbufs = [rms.HostBuffer(q.shape), rms.HostBuffer(u.shape)] + \
                ([] if peak_only else [rms.HostBuffer((L, cfg.nphi, 2))]) + \
                [rms.HostBuffer(L, "int32"), rms.HostBuffer(L), rms.HostBuffer(L)]
        Qh, Uh = hbufs[0].tensor, hbufs[1].tensor
        Fh = None if peak_only else hbufs[2].tensor
        ih, ah, ph = (b.tensor for b in hbufs[-3:])
        Qh.copy_(q)
        Uh.copy_(u)

        def e2e_step():
            plan.synth_host(Qh, Uh, L, layout, Fh, ih, ah, ph, stream)
        n_e2e = max(10, min(50, steps // 4))
        e2e_step()
        per_e2e = []
        for _ in range(n_e2e):
            t0 = time.perf_counter()
            e2e_step()
            per_e2e.append(time.perf_counter() - t0)
        dt = sum(per_e2e) / n_e2e
        res["e2e"] = {"value": units / dt / 1e9, "unit": UNIT, "ms_per_step": dt * 1e3, "steps": n_e2e,
                      "ms_median_min_max": [1e3 * statistics.median(per_e2e), 1e3 * min(per_e2e), 1e3 * max(per_e2e)],
                      "note": "the median, minimum and maximum over the calls are beside the mean: host-link "
                              "throughput varies with what else runs on the host",
                      "h2d_bytes_per_step": int(Qh.numel() * 4 + Uh.numel() * 4),
                      "d2h_bytes_per_step": int((0 if Fh is None else Fh.numel() * 4) + L * 12),
                      "how": "rms_synth_host: Q/U in page-locked host buffers from rms_host_alloc -> device in "
                             "LOS chunks, synthesis, F and peak map -> host buffers, copies overlapped on three "
                             "streams, sync"}
        del Qh, Uh, Fh, ih, ah, ph
        for b in hbufs:
            b.close()

    if with_clean and F is not None and cfg.nphi <= 2048 and tensor_path:
        # RM-CLEAN of the synthesised cube (FP64 Hogbom iterations, one warp per LOS)
        sigma_f = cfg.sigma * float(np.sqrt(np.sum(w * w)) / np.sum(w))
        thr = 5.0 * sigma_f
        Lc = min(L, 262144)     # a bounded number of LOS per call keeps the run short on big cubes
        c = rms.rms_clean_create(plan.handle)
        Fc = torch.empty(Lc, cfg.nphi, 2, device=dev)
        nit = torch.empty(Lc, dtype=torch.int32, device=dev)

        def clean_step():
            rms.rms_clean(c, F, Lc, 0.1, 1000, thr, Fc, None, None, nit, stream)
        with torch.cuda.stream(stream):
            t_cl, _ = time_steps(clean_step, stream, 3, 1, torch)
        rms.rms_clean_destroy(c)
        mean_it = float(nit.double().mean().item())
        res["clean"] = {"los_per_call": Lc, "ms_per_call": t_cl / 3, "los_per_s": Lc / (t_cl / 3 * 1e-3),
                        "gain": 0.1, "max_iter": 1000, "threshold": thr, "threshold_rule": "5 sigma_F",
                        "mean_iterations": mean_it, "precision": "f64",
                        "component_updates_per_s": Lc * mean_it * cfg.nphi / (t_cl / 3 * 1e-3)}
        del Fc, nit

    # the FP64 oracle on a bounded LOS sample: the CPU baseline, and the error of every path
    cpu = None
    if with_cpu:
        cpu = oracle_sample(cfg, freq, w, phi, L, cpu_seconds)
        sel = torch.from_numpy(cpu["rows"]).to(dev)

    def error_vs_fp64(Fd, pidx_d, pabs_d):
        Fo = cpu["Fo"]
        if Fd is not None:
            Fg = Fd[sel].cpu().numpy()
            Fg = Fg[..., 0] + 1j * Fg[..., 1]
            d = np.abs(Fg - Fo)
            per_los = d.max(axis=1) / np.abs(Fo).max(axis=1)
            return {"per_los_max": float(per_los.max()), "per_los_p999": float(np.quantile(per_los, 0.999)),
                    "cube": float(d.max() / np.abs(Fo).max()), "sample_los": int(len(cpu["rows"]))}
        oi, oa = cpu["peak"]
        ga = pabs_d[sel].cpu().numpy()
        return {"peak_abs_rel_max": float(np.max(np.abs(ga - oa) / np.abs(Fo).max(axis=1))),
                "peak_idx_equal": float(np.mean(pidx_d[sel].cpu().numpy() == oi)), "sample_los": int(len(cpu["rows"]))}

    if with_paths:
        paths = {}
        for p in ("fp32_fly", "fp32_table", "bf16", "bf16x3", "fp16x3", "fp32_czt"):
            if p == path:
                paths[p] = {"value": value, "ms_per_step": tmax / steps}
                continue
            try:
                pl = rms.Plan(freq, phi, p, weights=w, device=local)
            except rms.RmsError as e:
                if e.status != rms.RMS_ERR_UNSUPPORTED:
                    raise
                paths[p] = {"unsupported": "channels not uniform in lambda^2, or nchan + nphi - 1 > 2048"}
                continue
            with pl:
                # about 2 s of timed work per path (the FP32 paths run ~10x longer per step)
                n = max(3, min(50, int(2000.0 / (tmax / steps) / (8 if p.startswith("fp32") else 1))))

                def st2(pl=pl):
                    pl.synth(q, u, L, layout, F, pidx, pabs, pphi, stream)
                with torch.cuda.stream(stream):
                    tot, _ = time_steps(st2, stream, n, 2, torch)
                pl.sync(stream)
                paths[p] = {"value": units * n / (tot * 1e-3) / 1e9, "ms_per_step": tot / n}
                if cpu is not None:
                    torch.cuda.synchronize()
                    paths[p]["error_vs_fp64"] = error_vs_fp64(F, pidx, pabs)
        res["paths"] = paths
        # restore this path's output for the error check below
        plan.synth(q, u, L, layout, F, pidx, pabs, pphi, stream)
        plan.sync(stream)

    if cpu is not None:
        res["cpu_baseline"] = cpu["baseline"]
        if "clean" in res:
            import oracle
            from oracle import clean as oclean
            dphi = float(phi[1] - phi[0])
            R2 = oracle.rmsf(cpu["plan"], (np.arange(2 * len(phi) - 1) - (len(phi) - 1)) * dphi)
            k = min(len(cpu["rows"]), 256)
            t0 = time.perf_counter()
            oclean.clean(cpu["Fo"][:k], R2, 0.1, 1000, res["clean"]["threshold"], oracle.fwhm_measured(cpu["plan"]),
                         dphi)
            res["clean"]["cpu_oracle_los_per_s"] = k / (time.perf_counter() - t0)
        res["error_vs_fp64"] = error_vs_fp64(F, pidx, pabs)
        if "paths" in res:
            res["paths"][path]["error_vs_fp64"] = res["error_vs_fp64"]
    plan.close()
    del q, u, F, pidx, pabs, pphi
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return res


def run_ours(args):
    import torch
    import paper_1810_06250_gb300 as rms
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rms.build()
    barrier = None
    if world > 1:
        import torch.distributed as dist
        barrier = dist.barrier
    solo = rank == 0 and world == 1
    res = measure_cube(args, args.config, args.path, args.layout, args.steps, args.warmup, dev, local, world,
                       barrier, nlos=args.nlos, peak_only=args.peak_only, with_paths=solo and not args.no_paths,
                       with_e2e=solo and not args.no_e2e, with_cpu=solo and not args.no_cpu,
                       with_clean=solo and not args.no_clean, cpu_seconds=args.cpu_seconds)
    line = {"metric": METRIC, "value": res.pop("value"), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res.pop("ms_per_step"), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.path, "data": "synthetic"}
    for k in ("steps", "warmup", "unit", "dtype"):
        res.pop(k, None)
    line.update(res)
    if solo and args.config == CONFIG_NAME and args.nlos is None and not args.no_secondary:
        # the LOFAR-HBA-like cube: a shorter, contraction-lighter workload (23 K blocks of
        # 16 channels against MWA's 96), BF16x3, channel-major
        lo = measure_cube(args, "lofar", "bf16x3", "chan", 200, 10, dev, local, with_cpu=not args.no_cpu,
                          cpu_seconds=5.0)
        line["lofar"] = {k: lo[k] for k in ("value", "unit", "ms_per_step", "dtype", "config", "roofline",
                                            "clocks", "error_vs_fp64", "cpu_baseline") if k in lo}
        # the learned peak proposal on its own workload (trained here, on the GPU)
        try:
            line["learned"] = measure_learned(args, dev, local, rank, world, None, 10, 3)[0]
        except Exception as e:   # reported, not hidden: the main line stands on its own
            line["learned"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


LEARNED_METRIC = "learned peak map: full-grid-equivalent G(LOS*chan*phi)/s at >=99.5% phi_peak agreement"


def measure_learned(args, dev, local, rank, world, barrier, steps, warmup):
    """The learned proposal on the learned workload (2048^2 LOS, LOFAR band, SNR 5-100).

    The network is trained here on the GPU (1M generated LOS labelled by the
    full grid), its confidence threshold calibrated on a separate validation set,
    then one step = one rms_peakmap_learned call over the cube (device-resident
    FP32 Q/U in, peak map out), timed next to the full-grid peak map
    (rms_synth, peak map only) at the same precision and at plain BF16.
    Returns (the `learned` result object, the fields of a bench line)."""
    import torch
    import paper_1810_06250_gb300 as rms
    from paper_1810_06250_gb300 import inputs, learned as Lm
    path = args.path if args.config == "learned" else "bf16x3"
    layout = args.layout if args.config == "learned" else "chan"
    cfg = inputs.CONFIGS["learned"]
    if args.nlos is not None:
        import dataclasses
        cfg = dataclasses.replace(cfg, nlos=args.nlos)
    freq, w, phi = inputs.frequencies(cfg), inputs.weights(cfg), inputs.phi_grid(cfg)
    nact = int(np.count_nonzero(w))
    L = cfg.nlos
    plan = rms.Plan(freq, phi, path, weights=w, device=local)
    t0 = time.perf_counter()
    net = Lm.Net(plan, hidden=args.hidden, max_batch=4096, seed=101)
    win = Lm.Window(plan, 64)
    hist = Lm.train(plan.handle, net, cfg, n_train=args.n_train, epochs=args.epochs, batch=4096, seed=5001 + rank)
    tau, cal = Lm.calibrate(plan.handle, net, win, cfg, n_val=1 << 18, seed=6001 + rank, layout=layout)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    Q, U = Lm.generate(plan.handle, cfg, 0, L, layout, seed=cfg.seed + 1000 * rank)
    stream = torch.cuda.Stream(dev)
    php = torch.empty(L, device=dev)
    pka = torch.empty(L, device=dev)
    fb = torch.empty(L, dtype=torch.int32, device=dev)
    nfb = torch.zeros(1, dtype=torch.int64, device=dev)
    fidx = torch.empty(L, dtype=torch.int32, device=dev)
    fphi = torch.empty(L, device=dev)
    fabs = torch.empty(L, device=dev)
    units = L * nact * cfg.nphi

    def learned_step():
        rms.rms_peakmap_learned(win.handle, net.handle, Q, U, L, layout, tau, php, pka, fb, nfb, stream)

    def full_step():
        plan.synth(Q, U, L, layout, None, fidx, fabs, fphi, stream)

    with torch.cuda.stream(stream):
        with ClockSampler(local) as clk:
            t_learn, per = time_steps(learned_step, stream, steps, warmup, torch, barrier)
        t_full, _ = time_steps(full_step, stream, max(3, steps // 2), 2, torch)
        with rms.Plan(freq, phi, "bf16", weights=w, device=local) as p1:
            def bf16_step():
                p1.synth(Q, U, L, layout, None, fidx, fabs, fphi, stream)
            t_bf16, _ = time_steps(bf16_step, stream, max(3, steps // 2), 2, torch)
        # the full grid at the window's resolution (step D/2 over the same range: the
        # fine grid every window is cut from), same precision
        phi_fine = cfg.phi_min + 0.5 * (phi[1] - phi[0]) * np.arange(2 * cfg.nphi - 1)
        gidx = torch.empty(L, dtype=torch.int32, device=dev)
        gphi = torch.empty(L, device=dev)
        gabs = torch.empty(L, device=dev)
        with rms.Plan(freq, phi_fine, path, weights=w, device=local) as p2:
            def fine_step():
                p2.synth(Q, U, L, layout, None, gidx, gabs, gphi, stream)
            t_fine, _ = time_steps(fine_step, stream, max(3, steps // 2), 2, torch)
            fine_step()
        full_step()
        learned_step()
    torch.cuda.synchronize()
    plan.sync(stream)
    ms_learn = t_learn / steps
    ms_full = t_full / max(3, steps // 2)
    ms_bf16 = t_bf16 / max(3, steps // 2)
    ms_fine = t_fine / max(3, steps // 2)
    agree = float(np.mean(np.abs(php.cpu().numpy().astype(np.float64) - fphi.cpu().numpy()) <= 0.5 * (1 + 1e-6)))
    dfine = np.abs(php.cpu().numpy().astype(np.float64) - gphi.cpu().numpy())
    agree_fine_point = float(np.mean(dfine <= 1e-3))
    agree_fine = float(np.mean(dfine <= 0.5 * (1 + 1e-6)))
    fbr = float(fb.cpu().numpy().mean())
    from paper_1810_06250_gb300.dist import throughput
    value, tmax = throughput(units, steps, t_learn, world, dev)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6701.0)
    in_bytes = L * 8.0 * (nact if layout == "chan" else cfg.nchan)
    alg = in_bytes + 8.0 * L
    line = {"metric": LEARNED_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": tmax / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": path, "data": "synthetic",
            "config": {"workload": "learned: 2048x2048 LOS x 400 channels (%d active) 115-178 MHz x 401 phi in "
                                   "[-100, 100], FP32 Q/U %s-major, peak map only; 1-3 thin/Burn-slab components, "
                                   "SNR 5-100; window 64 x 0.25 rad/m^2" % (nact, layout),
                       "nlos_per_gpu": L, "l2": "inputs larger than L2 (13.4 GB per step)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "learned": {"speedup_vs_full_grid_same_precision": ms_full / ms_learn,
                        "speedup_vs_full_grid_bf16": ms_bf16 / ms_learn,
                        "speedup_vs_fine_full_grid_same_precision": ms_fine / ms_learn,
                        "ms_learned": ms_learn, "ms_full_grid": ms_full, "ms_full_grid_bf16": ms_bf16,
                        "ms_fine_full_grid": ms_fine, "fine_grid_nphi": int(len(phi_fine)),
                        "agreement": agree, "agreement_fine_grid": agree_fine,
                        "same_fine_point": agree_fine_point, "fallback_frac": fbr, "tau": tau, "val_fallback_frac": cal["fallback_frac"],
                        "train_loss": hist, "train_s": train_s, "n_train": args.n_train, "epochs": args.epochs,
                        "hidden": args.hidden,
                        "params": int(net.nparams), "flop_per_los": 2 * (net.nparams - args.hidden - cfg.nphi)},
            "roofline": {"bound": "hbm", "achieved": alg / (ms_learn * 1e-3) / 1e9, "peak": hbm_peak,
                         "unit": "GB/s", "frac": alg / (ms_learn * 1e-3) / 1e9 / hbm_peak, "traffic": None,
                         "algorithmic": "cube read once (8 B per LOS x contraction channel) + 8 B peak map per LOS",
                         "peak_source": "measured HBM copy (MEASURED_PEAKS.json)"},
            "gpu_launches": steps * 9, "clocks": clk.summary()}
    solo = rank == 0 and world == 1 and args.config == "learned"
    if solo and not args.no_e2e:
        # page-locked host buffers from the library's allocator (registered huge-page memory)
        hbufs = [rms.HostBuffer(Q.shape), rms.HostBuffer(U.shape), rms.HostBuffer(L), rms.HostBuffer(L)]
        Qh, Uh, ph_h, pa_h = (b.tensor for b in hbufs)
        Qh.copy_(Q)
        Uh.copy_(U)

        def e2e():
            with torch.cuda.stream(stream):
                Q.copy_(Qh, non_blocking=True)
                U.copy_(Uh, non_blocking=True)
                learned_step()
                ph_h.copy_(php, non_blocking=True)
                pa_h.copy_(pka, non_blocking=True)
            stream.synchronize()
        e2e()
        n_e2e = 5
        per_e2e = []
        for _ in range(n_e2e):
            t0 = time.perf_counter()
            e2e()
            per_e2e.append(time.perf_counter() - t0)
        dt = sum(per_e2e) / n_e2e
        line["e2e"] = {"value": units / dt / 1e9, "unit": UNIT, "ms_per_step": dt * 1e3, "steps": n_e2e,
                       "ms_median_min_max": [1e3 * statistics.median(per_e2e), 1e3 * min(per_e2e),
                                             1e3 * max(per_e2e)],
                       "h2d_bytes_per_step": int(Qh.numel() * 8), "d2h_bytes_per_step": int(L * 8),
                       "how": "Q/U in page-locked host buffers from rms_host_alloc -> device, rms_peakmap_learned, "
                              "phi_peak and |F|_peak -> host buffers"}
        del Qh, Uh, ph_h, pa_h
        for b in hbufs:
            b.close()
    if solo and not args.no_cpu:
        import oracle
        oracle.build()
        op = oracle.plan(freq, "freq", w)
        Qc, Uc = inputs.make_cube(cfg, 0, 128)
        t0 = time.perf_counter()
        oracle.synth(Qc, Uc, op, phi)
        per_los = (time.perf_counter() - t0) / 128
        n = int(min(L, max(128, args.cpu_seconds / per_los)))
        Qc, Uc = inputs.make_cube(cfg, 0, n)
        t0 = time.perf_counter()
        oracle.peak(oracle.synth(Qc[:n], Uc[:n], op, phi))
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n * nact * cfg.nphi / dt / 1e9, "unit": UNIT, "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": "full-grid FP64 peak map of %d of %d LOS, %.1f s"
                                % (n, L, dt)}
    net.close()
    win.close()
    plan.close()
    del Q, U
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    learned = line.pop("learned")
    learned.update({"ms_per_step": line["ms_per_step"], "value_full_grid_equivalent": line["value"],
                    "unit": UNIT, "dtype": path, "workload": line["config"]["workload"],
                    "roofline": line["roofline"], "clocks": line["clocks"]})
    return learned, line


def run_learned(args):
    import torch
    import paper_1810_06250_gb300 as rms
    rank, world, local = dist_env()
    barrier = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        barrier = dist.barrier
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rms.build()
    learned, line = measure_learned(args, dev, local, rank, world, barrier, args.steps, args.warmup)
    line["learned"] = learned
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "learned":
        run_learned(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
