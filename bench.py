#!/usr/bin/env python3
"""Benchmark of the comb-spectrum hot path on GB300.

Default workload: 10^6 frames x 1100 int16 samples at 1.1 GS/s (the paper's
2.2 GB/s data rate, 1 MHz bins), 99 teeth at |51 + 10k| MHz, Lorentzian
cavity (FWHM 80 MHz) driven at 23.686 kHz with 20 MHz amplitude, SNR 30 dB,
12-bit samples; 2.2 GB resident on the device (larger than L2, so no flush is
needed between steps).  One step = cg_process over all frames: cast, FFT,
tooth readout, normalisation, moment initial guess and LM fit (20 iterations,
tol 1e-6).  The metric is fitted spectra/s at fixed fit error (the sampled
frames are checked against the FP64 oracle in the same run).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own 10^6 frames (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fitted spectra/s & input GB/s vs HBM peak at fixed fit error; p99 frame-to-fit"
FWHM_HZ = 80e6
FANO_Q = 0.3                 # asymmetry of the Fano workload's lineshape


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over the ranks of the process group (x itself with one
    rank): every rank's work is timed, the job is as slow as its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(frames_per_rank: int, world_size: int, seconds: float) -> float:
    """Whole-job throughput: every rank processes its own frames_per_rank
    frames (no collective on the data path), the job takes the slowest
    rank's time."""
    return frames_per_rank * world_size / seconds


GEOMETRIES = {
    # name: (synth geometry attribute, generator keywords)
    "paper_rate": ("PAPER_RATE", dict(snr_db=30.0, center_amp_hz=20e6)),
    # the learned-guess workload: per-frame centre U(+-100 MHz), FWHM U(60, 100) MHz,
    # SNR U(20, 40) dB on the wide geometry (held out from the network's training)
    "learned": ("WIDE", dict(learned=True)),
    "wide": ("WIDE", dict(snr_db=30.0, center_amp_hz=20e6)),
    "tiny": ("TINY", dict(sigma=0.01 * 2048, center_amp_hz=5e6)),
    "serve4096": ("SERVE_4096", dict(snr_db=30.0, center_amp_hz=20e6)),
    # the paper's digitiser frame: 8-bit samples at 2.2 GS/s, 2200 per frame
    "paper8": ("PAPER_8BIT", dict(snr_db=30.0, center_amp_hz=20e6, bits=8)),
    # the paper's fitted lineshape: Fano profile (q = 0.3, FWHM 80 MHz, depth 0.7)
    # at the paper rate, fitted with the centre free, scale and offset boxed
    "fano": ("PAPER_RATE", dict(snr_db=30.0, center_amp_hz=20e6, shape="fano", fano_q=FANO_Q)),
    # the paper's whole configuration: its 8-bit 2.2 GS/s digitiser frames and
    # its Fano fit (with --init median, its initial centre too)
    "fano8": ("PAPER_8BIT", dict(snr_db=30.0, center_amp_hz=20e6, bits=8, shape="fano", fano_q=FANO_Q)),
}


def is_fano(args) -> bool:
    return args.workload in ("fano", "fano8")


def fano_opts(args) -> dict:
    """Plan options of the Fano workload: q and gamma fixed at the generator's
    values, scale and offset boxed +-10 % around the lineshape's 0.7 / 0.3."""
    if not is_fano(args):
        return {}
    import paper_2307_12988_gb300 as cg
    return dict(model=cg.MODEL_FANO, fano_q=FANO_Q, fano_gamma=FWHM_HZ / 2.0, fano_A=0.7, fano_B=0.3,
                fano_box=0.1)


FIT_DESC = {False: "moment init, 20-iteration LM",
            True: "lowest-tooth init, 20-iteration box-constrained Fano LM"}


def oracle_fit(y, x, args, converged=False):
    """The oracle's fit of the workload's model on spectra y."""
    import oracle
    if is_fano(args):
        r = oracle.fano_fit_batch(y, x, FANO_Q, FWHM_HZ / 2.0, 0.7, 0.3, box=0.1, converged=converged)
        return dict(r, params=np.column_stack([r["params"][:, 0], np.full(len(y), FWHM_HZ / 2.0),
                                               r["params"][:, 1:]]))
    return oracle.fit_batch(y, x, converged=converged)


def oracle_process(frames, bins, ref, x, args):
    """The oracle's whole path (readout, initial guess, LM) for the workload."""
    import oracle
    if is_fano(args):
        _, y = oracle.readout(frames, bins, ref)
        return oracle_fit(y, x, args)
    return oracle.process(frames, bins, ref, x)


def workload_name(args, n):
    g = geometry(args)
    return (f"{args.workload}_{g.sample_rate / 1e9:g}GSps_N{g.frame_len}_T{g.n_teeth}_"
            f"{n}frames_{args.readout}")


def geometry(args):
    import synth
    return getattr(synth, GEOMETRIES[args.workload][0])


def build_workload(args, n_frames, n_ref, device, seed_offset=0):
    import synth
    g = geometry(args)
    kw = dict(GEOMETRIES[args.workload][1])
    stream = synth.make_stream(g, synth.BASE_SEED + 2 + seed_offset)
    if kw.pop("learned", False):
        lp = synth.learned_params(n_frames, seed=synth.BASE_SEED + 600 + seed_offset)
        kw = dict(centers=lp["c"], fwhm_hz=lp["fwhm"], snr_db=lp["snr_db"])
        noise = dict(snr_db=30.0)
    else:
        noise = {k: v for k, v in kw.items() if k in ("snr_db", "sigma", "bits")}
    fr = synth.frames(stream, n_frames, device=device, **kw)
    rf = synth.frames(stream, n_ref, cavity=False, noise_stream=1, device=device, **noise)
    return g, fr["frames"], rf["frames"]


MLP_BLOB = os.path.join(ROOT, "paper_2307_12988_gb300", "data", "mlp_wide_t221.cgmlp")

# DRAM bytes per frame (dram__bytes_read.sum + dram__bytes_write.sum) of one
# ncu capture of each kernel on the paper-rate workload, by the stage names
# of the per-kernel timing; a kernel changed since its capture has none
NCU_TRAFFIC_PER_FRAME = {("paper_rate", "fft", "moment"): {"readout": 2523.8, "init": 397.1, "fit": 414.4}}

# FP32 operations of one LM point evaluation (model, residual, Jacobian and
# the 14 running sums of J^T J, J^T r and chi^2): 11 + 10 FMA x 2 + 4 adds
LM_FLOP_PER_POINT = 35
# the Fano model's point: e, 1 + e^2, its reciprocal, (q + e)^2 / (1 + e^2),
# the residual, dm/dc (7) and 9 running sums (6 FMA + 3 adds)
LM_FLOP_PER_POINT_FANO = 33


def alu_peak_measured(cg) -> dict:
    """FP32 fused multiply-add throughput measured on this device now
    (cg_fp32_peak: scalar and packed FP32x2 chains, CUDA events); the larger
    of the two is the ALU roofline's denominator."""
    scalar = cg.cg_fp32_peak(False, 20)
    packed = cg.cg_fp32_peak(True, 20)
    return {"tflops": max(scalar, packed), "scalar_tflops": scalar, "packed_tflops": packed,
            "kind": "measured (cg_fp32_peak, FMA chains, CUDA events)"}


def kernel_rooflines(stage_ms, stage_launches, n, g, T, args, mean_iters, hbm, bf16, alu_peak):
    """Per-kernel figures from the timing pass: mean launch time and the
    roofline each is bound by (algorithmic work / launch time)."""
    out = {}
    for st, ms in stage_ms.items():
        cnt = stage_launches[st]
        per = ms / cnt / 1e3                       # s per launch
        frames = n * args.steps_timed / cnt
        r = {"launches": cnt, "ms_per_launch": per * 1e3}
        if st == "readout" and args.readout in ("fft", "fold"):
            b = (args.sample_bytes * g.frame_len + 4 * T) * frames
            r.update(bound="hbm", achieved=b / per / 1e9, peak=hbm, unit="GB/s")
        elif st == "readout":
            f = 2.0 * g.frame_len * 2 * T * frames
            r.update(bound="tensor", achieved=f / per / 1e12, peak=bf16, unit="TFLOP/s")
        elif st == "init":
            b = (4 * T + 16 + 2) * frames
            r.update(bound="hbm", achieved=b / per / 1e9, peak=hbm, unit="GB/s")
        elif st == "median":
            b = (4 * T + 4) * frames                  # y in, the centre out
            r.update(bound="hbm", achieved=b / per / 1e9, peak=hbm, unit="GB/s")
        elif st == "mlp":
            f = 2.0 * (T * 256 + 256 * 256) * frames
            r.update(bound="tensor", achieved=f / per / 1e12, peak=bf16, unit="TFLOP/s")
        elif st == "fit":
            fp = LM_FLOP_PER_POINT_FANO if is_fano(args) else LM_FLOP_PER_POINT
            f = fp * T * (mean_iters + 1.0) * frames
            r.update(bound="alu", achieved=f / per / 1e12, peak=alu_peak, unit="TFLOP/s")
        if "achieved" in r:
            r["frac"] = r["achieved"] / r["peak"]
        tr = NCU_TRAFFIC_PER_FRAME.get((args.workload, args.readout, args.init), {}).get(st)
        r["traffic"] = tr * frames if tr is not None else None
        out[st] = r
    return out


def cpu_baseline_leg(frames, params, status, iters, plan, ref, g, args) -> dict:
    """CPU-baseline leg: the oracle, as it stands, timed on the host cores on a
    bounded sample of the same frames; its outputs on a sample also give the
    fit error of the GPU results (centres vs the oracle's converged optimum)."""
    import oracle
    frames_host = frames[: args.check_frames].cpu().numpy()
    p_host = params[: args.check_frames].cpu().numpy()
    bins, x = plan.bins, g.tooth_x
    probe = min(512, frames_host.shape[0])
    t = time.perf_counter()
    oracle_process(frames_host[:probe], bins, ref, x, args)
    dt = time.perf_counter() - t
    n = int(min(frames_host.shape[0], max(probe, probe * args.cpu_seconds / max(dt, 1e-6))))
    t = time.perf_counter()
    oracle_process(frames_host[:n], bins, ref, x, args)
    dt = time.perf_counter() - t
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    cpu = {"value": n / dt, "unit": "spectra/s", "cores": cores, "kind": "oracle",
           "sample": f"first {n} of the workload's frames (FP64 direct-sum DFT at the "
                     f"{g.n_teeth} teeth, {FIT_DESC[is_fano(args)]}), {dt:.1f} s"}
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(frames_host.shape[0], size=min(256, frames_host.shape[0]),
                             replace=False))
    _, y_idx = oracle.readout(frames_host[idx], bins, ref)
    conv = oracle_fit(y_idx, x, args, converged=True)
    dc = np.abs(p_host[idx, 0] - conv["params"][:, 0])
    st = status.cpu().numpy()
    fe = {"frames_checked": int(idx.size), "center_err_max_hz": float(dc.max()),
          "center_err_p99_hz": float(np.percentile(dc, 99)),
          "frac_within_1e-4_fwhm": float(np.mean(dc <= 1e-4 * FWHM_HZ)),
          "status_counts": {int(k): int(v) for k, v in zip(*np.unique(st, return_counts=True))},
          "mean_iters": float(iters.float().mean().item())}
    return {"cpu_baseline": cpu, "fit_error": fe}


def run_ours(args):
    import torch
    import paper_2307_12988_gb300 as cg

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.frames
    g, frames, ref_frames = build_workload(args, n, args.ref_frames, dev, seed_offset=rank)
    args.sample_bytes = frames.element_size()
    process = cg.cg_process_i8 if frames.dtype == torch.int8 else cg.cg_process
    plan0 = cg.Plan(g.sample_rate, g.frame_len, g.tooth_freqs, g.tooth_x)
    ref = plan0.reference_accumulate(ref_frames.to(torch.int16))   # (8-bit samples widen exactly)
    plan0.close()
    del ref_frames
    plan = cg.Plan(g.sample_rate, g.frame_len, g.tooth_freqs, g.tooth_x, ref,
                   lanes_per_frame=args.lanes, path=args.path, chunk_frames=args.chunk,
                   readout={"fft": cg.READOUT_FFT, "gemm": cg.READOUT_GEMM_SPLIT,
                            "fold": cg.READOUT_FOLD_GEMM}[args.readout],
                   sample_bits=args.sample_bits,
                   init={"moment": cg.INIT_MOMENT, "mlp": cg.INIT_MLP, "median": cg.INIT_MEDIAN}[args.init],
                   polish_iter=args.polish, **fano_opts(args))
    if args.init == "mlp":
        with open(MLP_BLOB, "rb") as f:
            plan.mlp_load(f.read())
    T = plan.T
    amps = torch.empty((n, T), dtype=torch.float32, device=dev)
    params = torch.empty((n, 4), dtype=torch.float32, device=dev)
    rss = torch.empty(n, dtype=torch.float32, device=dev)
    iters = torch.empty(n, dtype=torch.int16, device=dev)
    status = torch.empty(n, dtype=torch.int16, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        process(plan.handle, frames, n, amps, None, params, rss, iters, status, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    ms_step = ms / args.steps

    # per-kernel timing pass (events on the launching streams), after the
    # timed region so that it does not disturb the step time
    plan.timing(True)
    args.steps_timed = max(1, min(args.steps, 20))
    for _ in range(args.steps_timed):
        step()
    torch.cuda.synchronize()
    stages = plan.timing_collect()
    plan.timing(False)
    mean_iters = float(iters.float().mean().item())

    hbm, bf16, peak_kind = _peaks()
    alu = alu_peak_measured(cg)
    sb = args.sample_bytes
    bytes_per_frame = sb * g.frame_len + 4 * T + 16 + 4 + 2 + 2
    kern = kernel_rooflines({k: v[0] for k, v in stages.items()}, {k: v[1] for k, v in stages.items()},
                            n, g, T, args, mean_iters, hbm, bf16, alu["tflops"])
    dominant = max(kern, key=lambda k: kern[k]["launches"] * kern[k]["ms_per_launch"])
    dom = kern[dominant]
    total_frames = n * ws
    value = weak_scaling_value(n, ws, ms_step / 1e3)
    achieved = bytes_per_frame * n / (ms_step / 1e3) / 1e9
    result = {
        "metric": METRIC, "value": value, "unit": "spectra/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": ("synthetic (seeded comb interferograms, 8-bit in int8)" if sb == 1 else
                                 "synthetic (seeded comb interferograms, 12-bit in int16)"),
        "config": {"workload": workload_name(args, n),
                   "frames_per_gpu": n, "frame_len": g.frame_len, "teeth": T,
                   "sample_rate_hz": g.sample_rate, "resident_bytes": sb * g.frame_len * n,
                   "l2": f"inputs ({sb * g.frame_len * n / 1e9:.1f} GB) larger than L2; no flush",
                   "lanes_per_frame": plan.info["lanes_per_frame"],
                   "path": ["auto", "fused", "split", "pipeline"][plan.info["path"]],
                   "fft_len": plan.info["fft_len"], "readout": args.readout,
                   "init": "lowest tooth" if (is_fano(args) and args.init == "moment") else args.init,
                   "model": "fano" if is_fano(args) else "lorentz",
                   "polish_iter": args.polish if args.init == "mlp" else None},
        "input_gbs": total_frames * sb * g.frame_len / (ms_step / 1e3) / 1e9,
        "roofline": {"kernel": dominant, "bound": dom.get("bound"), "achieved": dom.get("achieved"),
                     "peak": dom.get("peak"), "unit": dom.get("unit"), "frac": dom.get("frac"),
                     "traffic": dom.get("traffic"),
                     "peak_kind": alu["kind"] if dom.get("bound") == "alu" else peak_kind},
        "alu_peak": alu,
        "step_hbm": {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "algorithmic_bytes_per_frame": bytes_per_frame},
        "kernels": kern,
        "mean_iters": mean_iters,
        "gpu_launches": int(round(sum(v[1] for v in stages.values()) * args.steps / args.steps_timed)),
        "clocks": clocks,
    }
    torch.cuda.synchronize()
    if rank == 0 and not args.quick:
        result.update(cpu_baseline_leg(frames, params, status, iters, plan, ref, g, args))
    if not args.quick:
        result["e2e"] = run_e2e(plan, frames, n, T, dev, args, ws)
    if not args.quick and args.serve_seconds > 0 and rank == 0:
        del frames, amps, params, rss, iters, status
        torch.cuda.empty_cache()
        result["serving"] = run_serving(args, dev)
    if rank == 0:
        print(json.dumps(result), flush=True)
    plan.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_e2e(plan, frames_dev, n, T, dev, args, ws):
    """Same metric through cg_process with host buffers: every step copies the
    frames from pinned host memory and reads every result back, in chunks on
    two streams so copies overlap the kernel."""
    import torch
    import paper_2307_12988_gb300 as cg
    N = plan.N
    sdt = frames_dev.dtype
    process = cg.cg_process_i8 if sdt == torch.int8 else cg.cg_process
    host_in = torch.empty((n, N), dtype=sdt, pin_memory=True)
    host_in.copy_(frames_dev.cpu())
    chunk = args.e2e_chunk
    nch = (n + chunk - 1) // chunk
    streams = [torch.cuda.Stream(dev) for _ in range(2)]
    bufs = []
    for _ in range(2):
        bufs.append(dict(fr=torch.empty((chunk, N), dtype=sdt, device=dev),
                         amps=torch.empty((chunk, T), dtype=torch.float32, device=dev),
                         params=torch.empty((chunk, 4), dtype=torch.float32, device=dev),
                         rss=torch.empty(chunk, dtype=torch.float32, device=dev),
                         iters=torch.empty(chunk, dtype=torch.int16, device=dev),
                         status=torch.empty(chunk, dtype=torch.int16, device=dev)))
    host_out = dict(amps=torch.empty((n, T), dtype=torch.float32, pin_memory=True),
                    params=torch.empty((n, 4), dtype=torch.float32, pin_memory=True),
                    rss=torch.empty(n, dtype=torch.float32, pin_memory=True),
                    iters=torch.empty(n, dtype=torch.int16, pin_memory=True),
                    status=torch.empty(n, dtype=torch.int16, pin_memory=True))

    def one_pass():
        for c in range(nch):
            s = streams[c % 2]
            b = bufs[c % 2]
            a0, a1 = c * chunk, min(n, (c + 1) * chunk)
            m = a1 - a0
            with torch.cuda.stream(s):
                b["fr"][:m].copy_(host_in[a0:a1], non_blocking=True)
                process(plan.handle, b["fr"], m, b["amps"], None, b["params"], b["rss"],
                        b["iters"], b["status"], s)
                for k in ("amps", "params", "rss", "iters", "status"):
                    host_out[k][a0:a1].copy_(b[k][:m], non_blocking=True)

    for _ in range(2):
        one_pass()
    torch.cuda.synchronize()
    steps = max(1, args.e2e_steps)
    t0 = time.perf_counter()
    for _ in range(steps):
        one_pass()
    torch.cuda.synchronize()
    dt = max_over_ranks((time.perf_counter() - t0) / steps, dev)
    d2h = n * (4 * T + 16 + 4 + 2 + 2)
    sb = frames_dev.element_size()
    return {"value": weak_scaling_value(n, ws, dt), "unit": "spectra/s", "h2d_bytes_per_step": n * N * sb,
            "d2h_bytes_per_step": d2h, "chunk_frames": chunk, "steps": steps,
            "input_gbs": n * ws * N * sb / dt / 1e9}


SERVE_STREAMS = [   # (geometry attribute, generator keywords): the three instruments of the serving workload
    ("PAPER_RATE", dict(snr_db=30.0, center_amp_hz=20e6)),
    ("WIDE", dict(snr_db=30.0, center_amp_hz=20e6)),
    ("SERVE_4096", dict(snr_db=30.0, center_amp_hz=20e6)),
]


def run_serving(args, dev) -> dict:
    """Streaming leg: three instrument streams (1100 @ 1.1 GS/s, 2500 @ 2.5 GS/s,
    4096 @ 2.0 GS/s) pushed in real time from pinned pools of pre-generated
    frames (replayed with fresh sequence numbers) into one server; each
    result's latency is its poll-ready time minus the acquisition time of the
    first frame of its push.  Reports sustained rates and p50 / p99 latency."""
    import threading
    import torch
    import paper_2307_12988_gb300 as cg
    import synth
    server = cg.Server(args.serve_budget)
    streams, pools, plans = [], [], []
    for i, (gname, kw) in enumerate(SERVE_STREAMS):
        g = getattr(synth, gname)
        st = synth.make_stream(g, synth.BASE_SEED + 800 + i)
        pool = synth.frames(st, args.serve_pool, device=dev, **kw)["frames"].cpu().numpy()
        rf = synth.frames(st, 4096, cavity=False, noise_stream=1, device=dev, snr_db=30.0)["frames"]
        p0 = cg.Plan(g.sample_rate, g.frame_len, g.tooth_freqs, g.tooth_x)
        ref = p0.reference_accumulate(rf)
        p0.close()
        plan = cg.Plan(g.sample_rate, g.frame_len, g.tooth_freqs, g.tooth_x, ref)
        period = g.frame_len / g.sample_rate
        chunk = max(1, int(round(args.serve_push_s / period)))
        ring = 2 * g.frame_len * max(8 * args.serve_batch, int(args.serve_ring_s / period))
        s = cg.Stream(server, plan, ring_bytes=ring, batch_frames=args.serve_batch,
                      max_delay_s=args.serve_delay, avg_window=10_000)
        streams.append((g, s, period, chunk))
        pools.append(pool)
        plans.append(plan)
    stop = threading.Event()
    counts = [dict(pushed=0, overflow=0, polled=0) for _ in streams]
    t0 = cg.cg_clock() + 0.05

    def producer(i):
        g, s, period, chunk = streams[i]
        pool = pools[i]
        k, seq = 0, 0
        while not stop.is_set():
            t_acq = t0 + seq * period                      # acquisition time of the chunk's first frame
            t_ready = t_acq + chunk * period               # the chunk is complete
            while cg.cg_clock() < t_ready:
                time.sleep(max(0.0, min(2e-4, t_ready - cg.cg_clock())))
            if cg.cg_clock() - t0 > args.serve_seconds:
                break
            if k + chunk > pool.shape[0]:
                k = 0
            st = s.push(pool[k:k + chunk], seq, t_acq)
            if st == 0:
                counts[i]["pushed"] += chunk
            else:
                counts[i]["overflow"] += chunk
            k += chunk
            seq += chunk

    def consumer(i):
        _, s, _, _ = streams[i]
        while not stop.is_set() or s.stats()["frames_polled"] < s.stats()["frames_pushed"]:
            r, _, _ = s.poll(cap=65536, timeout_s=0.05)
            counts[i]["polled"] += len(r)
            if stop.is_set() and len(r) == 0 and s.flush(5.0) != 0:
                break

    threads = [threading.Thread(target=producer, args=(i,)) for i in range(len(streams))]
    threads += [threading.Thread(target=consumer, args=(i,)) for i in range(len(streams))]
    for t in threads:
        t.start()
    for t in threads[:len(streams)]:
        t.join()
    stop.set()
    for t in threads[len(streams):]:
        t.join()
    out = {"seconds": args.serve_seconds, "batch_frames": args.serve_batch, "max_delay_s": args.serve_delay,
           "push_s": args.serve_push_s, "device_budget_bytes": args.serve_budget, "streams": []}
    tot_frames, tot_bytes = 0, 0.0
    for (g, s, period, chunk), c in zip(streams, counts):
        st = s.stats()
        out["streams"].append({
            "frame_len": g.frame_len, "teeth": g.n_teeth, "sample_rate_hz": g.sample_rate,
            "offered_gbs": 2 * g.frame_len / period / 1e9, "input_gbs": st["input_bytes_per_s"] / 1e9,
            "frames_done": st["frames_done"], "frames_dropped": st["frames_dropped"],
            "latency_p50_ms": st["latency_p50_s"] * 1e3, "latency_p99_ms": st["latency_p99_s"] * 1e3,
            "latency_max_ms": st["latency_max_s"] * 1e3, "batches": st["batches"],
            "windows_completed": st["window_index"] + 1})
        tot_frames += st["frames_done"]
        tot_bytes += st["input_bytes_per_s"]
        s.close()
    for p in plans:
        p.close()
    server.close()
    out["spectra_per_s"] = tot_frames / args.serve_seconds
    out["input_gbs"] = tot_bytes / 1e9
    out["latency_p99_ms_max"] = max(x["latency_p99_ms"] for x in out["streams"])
    return out


def run_reference(args):
    """The oracle as it stands on the host cores, on the same metric."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    import oracle
    import synth
    g = synth.PAPER_RATE
    stream = synth.make_stream(g, synth.BASE_SEED + 2)
    n = args.ref_impl_frames
    fr = synth.frames(stream, n, snr_db=30.0, center_amp_hz=20e6)["frames"]
    rf = synth.frames(stream, 2000, cavity=False, snr_db=30.0, noise_stream=1)["frames"]
    bins = oracle.tooth_bins(g.sample_rate, g.frame_len, g.tooth_freqs)
    ref = oracle.reference(rf, bins)
    for _ in range(args.warmup):
        oracle.process(fr[: max(1, n // 8)], bins, ref, g.tooth_x)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.process(fr, bins, ref, g.tooth_x)
        times.append(time.perf_counter() - t)
    dt = sum(times) / len(times)
    value = n / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "spectra/s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "paper_rate_1.1GSps_N1100_T99_1e6frames",
                      "sample_frames_per_step": n},
           "cpu_baseline": {"value": value, "unit": "spectra/s", "cores": cores,
                            "kind": "oracle",
                            "sample": f"{n} frames of the workload per step"},
           "e2e": {"value": value, "unit": "spectra/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_psd(args):
    """The displacement-PSD leg: Welch PSD (Hann segments of --psd-seg samples,
    half overlap) of a fitted-centre series of --psd-seconds at the paper's
    frame rate (1 MHz), resident on the device, then the resonance fit; a
    step is both.  The series is a thermally driven resonator (23.7 kHz,
    Q = 120, 2 MHz RMS) over a white floor; 2^24 samples are synthesised and
    tiled to the requested length."""
    import torch
    import paper_2307_12988_gb300 as cg
    import synth
    from oracle import psd as opsd

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fs, M = 1e6, args.psd_seg
    base = synth.oscillator_series(1 << 24, fs, 23.7e3, 120.0, rms=2e6, floor=2e4, seed=31 + rank)
    n = int(args.psd_seconds * fs)
    reps = (n + base.size - 1) // base.size
    x = torch.from_numpy(base.astype(np.float32)).to(dev).repeat(reps)[:n].contiguous()
    hbm, bf16, peak_kind = _peaks()
    psd = cg.Psd(M)
    stream = torch.cuda.current_stream()

    def step():
        S, K = psd.welch(x, fs)
        out = torch.empty(12, dtype=torch.float64, device=dev)
        cg.cg_resonance_fit(S, S.numel(), fs / M, 21e3, 26.5e3, 200, 1e-12, out)
        return S, K, out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    clocks = ClockSampler(local)
    clocks.start()
    ev[0].record(stream)
    for _ in range(args.steps):
        S, K, out = step()
    ev[1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    res = out.cpu().numpy()
    value = n / (ms / 1e3)
    L = M // 2
    flops = K * 5.0 * L * math.log2(L)                    # the complex transform of every segment
    achieved = flops / (ms / 1e3) / 1e12
    alu = alu_peak_measured(cg)
    alu_peak = alu["tflops"]
    # end to end: the series from pinned host memory, the PSD and fit back
    xh = x.cpu().pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(1, args.e2e_steps)):
        xd = xh.to(dev, non_blocking=True)
        S2, _ = psd.welch(xd, fs)
        o2 = torch.empty(12, dtype=torch.float64, device=dev)
        cg.cg_resonance_fit(S2, S2.numel(), fs / M, 21e3, 26.5e3, 200, 1e-12, o2)
        S2.cpu()
        o2.cpu()
    e2e_s = (time.perf_counter() - t0) / max(1, args.e2e_steps)
    # the oracle on a bounded sample of the same series
    sample = base[: min(base.size, int(args.cpu_seconds * 2.5e6))]
    t0 = time.perf_counter()
    f, So, Ko = opsd.welch(sample, fs, M)
    fb, Sb = opsd.band(f, So, 21e3, 26.5e3)
    opsd.fit(fb, Sb)
    cpu_s = time.perf_counter() - t0
    line = {
        "metric": "displacement PSD samples/s (Welch, Hann, half overlap) + resonance fit",
        "value": value, "unit": "samples/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 transform, f64 averages and fit", "data": "synthetic",
        "config": {"workload": f"psd_{args.psd_seconds:g}s_at_1MHz_seg{M}", "samples": n, "segments": K,
                   "l2": f"input ({4 * n / 1e9:.2f} GB) larger than L2; no flush"},
        "resonance": {"f0_hz": res[0], "f0_sigma_hz": res[4], "Q": res[1], "Q_sigma": res[5],
                      "steps": int(res[9]), "status": int(res[10])},
        "roofline": {"kernel": "psd_welch_kernel", "bound": "alu", "achieved": achieved, "peak": alu_peak,
                     "unit": "TFLOP/s", "frac": achieved / alu_peak, "traffic": None,
                     "peak_kind": alu["kind"]},
        "alu_peak": alu,
        "input_gbs": 4.0 * n / (ms / 1e3) / 1e9,
        "input_hbm_frac": 4.0 * n / (ms / 1e3) / 1e9 / hbm,
        "cpu_baseline": {"value": sample.size / cpu_s, "unit": "samples/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {sample.size} samples (numpy FP64 Welch + LM fit), {cpu_s:.1f} s"},
        "e2e": {"value": n / e2e_s, "unit": "samples/s", "h2d_bytes_per_step": 4 * n,
                "d2h_bytes_per_step": 8 * (M // 2 + 1) + 96},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_train(args):
    """The learned-guess training leg: epochs of ``cg_mlp_train_epoch`` (gather,
    forward, MSE, backward, Adam on the device) over --train-rows standardised
    spectra of --train-in teeth, hidden width --train-hidden, minibatches of
    --train-batch; a step is one epoch.  Throughput does not depend on the
    values, so rows and targets are seeded normal draws."""
    import torch
    import paper_2307_12988_gb300 as cg
    from oracle import mlp as omlp

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n, ni, H, no, B = args.train_rows, args.train_in, args.train_hidden, 4, args.train_batch
    g = torch.Generator(device="cpu").manual_seed(5)
    xh = torch.randn(n, ni, generator=g)
    th = torch.randn(n, no, generator=g)
    perm_h = torch.randperm(n, generator=g).to(torch.int32)
    x, t, perm = xh.to(dev), th.to(dev), perm_h.to(dev)
    net = cg.Mlp(ni, H, no, max_batch=B, seed=1)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        net.train_epoch(x, t, perm, B, 1e-4)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    clocks = ClockSampler(0)
    clocks.start()
    ev[0].record(stream)
    for _ in range(args.steps):
        losses = net.train_epoch(x, t, perm, B, 1e-4)
    ev[1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    net.params()   # raises if a product block gave up a bounded wait
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    value = n / (ms / 1e3)
    per_row = 2.0 * (ni * H + H * H + H * no)          # forward multiply-adds x 2
    flops = 3.0 * per_row * n                           # forward + the two backward products
    hbm, bf16, peak_kind = _peaks()
    tf32_peak = bf16 * (1.1 / 2.25)                     # nominal TF32 : BF16 dense ratio
    achieved = 3.0 * flops / (ms / 1e3) / 1e12          # three TF32 products per FP32 product
    # end to end: the epoch's rows and targets from pinned host memory, the
    # losses back
    xp, tp = xh.pin_memory(), th.pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(1, args.e2e_steps)):
        xd, td = xp.to(dev, non_blocking=True), tp.to(dev, non_blocking=True)
        lo = net.train_epoch(xd, td, perm, B, 1e-4)
        lo.cpu()
    e2e_s = (time.perf_counter() - t0) / max(1, args.e2e_steps)
    # the oracle (FP64 NumPy) on a bounded sample: whole minibatch gradients
    theta = net.params().astype(np.float64)
    xb, tb = xh[:B].numpy().astype(np.float64), th[:B].numpy().astype(np.float64)
    t0, rows_cpu = time.perf_counter(), 0
    while time.perf_counter() - t0 < min(args.cpu_seconds, 10.0):
        omlp.loss_and_grad(theta, xb, tb, ni, H, no)
        rows_cpu += B
    cpu_s = time.perf_counter() - t0
    line = {
        "metric": "learned-guess training rows/s (forward, MSE, backward, Adam)",
        "value": value, "unit": "rows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (products as three TF32 tensor-core products)", "data": "synthetic",
        "config": {"workload": f"mlp_train_{ni}x{H}x{H}x{no}_batch{B}", "rows": n,
                   "l2": "epoch inputs resident; no flush (each minibatch is read once per epoch)"},
        "final_batch_loss": float(losses[-1].item()),
        "roofline": {"kernel": "tgemm_kernel", "bound": "tensor", "achieved": achieved, "peak": tf32_peak,
                     "unit": "TFLOP/s", "frac": achieved / tf32_peak, "traffic": None,
                     "peak_kind": f"{peak_kind} bf16 x nominal tf32/bf16 ratio",
                     "note": "whole epoch time, small kernels included; three TF32 products counted"},
        "e2e": {"value": n / e2e_s, "unit": "rows/s", "h2d_bytes_per_step": 4 * n * (ni + no),
                "d2h_bytes_per_step": 4 * ((n + B - 1) // B)},
        "cpu_baseline": {"value": rows_cpu / cpu_s, "unit": "rows/s",
                         "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
                         "kind": "oracle", "sample": f"{rows_cpu} rows: FP64 NumPy minibatch gradients, no Adam"},
        "clocks": clk,
        # per minibatch: 2 gathers, 8 products, MSE + loss, 3 column sums,
        # Adam (+ one sum per K-split product, not counted)
        "gpu_launches": 16 * ((n + B - 1) // B) * args.steps,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=1_000_000)
    ap.add_argument("--ref-frames", type=int, default=10_000)
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--path", type=int, default=0, help="0 auto, 1 fused, 2 split, 3 pipeline")
    ap.add_argument("--chunk", type=int, default=0, help="frames per pipelined chunk (0: default)")
    ap.add_argument("--workload", choices=sorted(GEOMETRIES), default="paper_rate")
    ap.add_argument("--readout", choices=["fft", "gemm", "fold"], default="fft",
                    help="fft: pruned transform on the CUDA cores; gemm: DFT-at-teeth product on the "
                         "tensor cores; fold: coset fold on the CUDA cores + DFT at the teeth on the "
                         "tensor cores")
    ap.add_argument("--init", choices=["moment", "mlp", "median"], default="moment",
                    help="initial guess; mlp loads the trained network (221 teeth)")
    ap.add_argument("--polish", type=int, default=0, help="LM polish steps after the MLP guess (0: 2)")
    ap.add_argument("--sample-bits", type=int, default=12,
                    help="declared sample range for the GEMM readout (the workloads are 12-bit)")
    ap.add_argument("--quick", action="store_true", help="skip fit check, CPU baseline and e2e")
    ap.add_argument("--check-frames", type=int, default=200_000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--e2e-chunk", type=int, default=65536)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--ref-impl-frames", type=int, default=20000)
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="streaming leg duration (the serving workload runs 60 s per stream)")
    ap.add_argument("--serve-only", action="store_true", help="run only the streaming leg")
    ap.add_argument("--serve-batch", type=int, default=4096)
    ap.add_argument("--serve-delay", type=float, default=5e-4)
    ap.add_argument("--serve-push-s", type=float, default=2.5e-4, help="acquisition time per push")
    ap.add_argument("--serve-ring-s", type=float, default=0.25, help="ring length in seconds of data")
    ap.add_argument("--serve-pool", type=int, default=32768, help="pre-generated frames replayed per stream")
    ap.add_argument("--serve-budget", type=int, default=4 << 30)
    ap.add_argument("--psd-only", action="store_true", help="run only the displacement-PSD leg")
    ap.add_argument("--train-only", action="store_true", help="run only the learned-guess training leg")
    ap.add_argument("--train-rows", type=int, default=200_000)
    ap.add_argument("--train-in", type=int, default=221)
    ap.add_argument("--train-hidden", type=int, default=256)
    ap.add_argument("--train-batch", type=int, default=1024)
    ap.add_argument("--psd-seconds", type=float, default=600.0, help="series length (the paper's longest PSD: 10 min)")
    ap.add_argument("--psd-seg", type=int, default=32768, help="Welch segment length")
    args = ap.parse_args()
    if args.psd_only:
        run_psd(args)
    elif args.train_only:
        run_train(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.serve_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"serving": run_serving(args, torch.device("cuda", 0))}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
