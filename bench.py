"""AS-TAX throughput benchmark (frames/s) on the 128-element workload.

Workload: 128-element linear array, 0.3 mm pitch, 4096 samples at 40 MHz,
c = 1540 m/s, 1-6 seeded sources, 128 lateral x 512 depth pixels over
5-60 mm, 300 bins over 0.5-8 MHz, 3 Pattern-16 apodizations.
One step = one frame through the whole path: time FFT, apodized lateral
FFTs, propagate + inverse lateral FFT + correlate, NCC/TAX epilogue. Steps
alternate over --streams plans on as many CUDA streams (default 2), so that
one frame's small latency-bound kernels overlap another frame's fused kernel;
the timed region is bracketed by events that span every stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one rank per GPU. Frames are independent, so
every rank processes its own frames (weak scaling) and the only
collectives are a barrier and the max over ranks of the timed region.
Rank 0 prints one JSON line.

`--impl reference` times the FP64 CPU oracle on the host cores, on a bounded
sample of the same workload (bins x depth rows), scaled to frames/s.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "AS-TAX frames/s (128 el, 128×512 grid), plain vs chosen form at stated err"
SMS = 152
FP32_LANES_PER_SM = 128
POOL_FRAMES = 96        # 96 distinct frames x 2 MiB = 201 MB > 129 MB L2


def fused_flops_per_frame(n_bins, nz, nx, n_apod=3):
    """Algorithmic FP32 flops of the fused propagate-and-correlate kernel per
    frame: per (bin, row) and aperture, one phasor multiply (6 nx) and one
    nx-point inverse FFT (5 nx log2 nx); per pixel 6 accumulations of 4 flops."""
    import math
    n_acc = {1: 1, 2: 3, 3: 6}[n_apod]
    per_row = n_apod * (6 * nx + 5 * nx * math.log2(nx)) + 4 * n_acc * nx
    return float(n_bins * nz * per_row)


def workload_config(w, frames_per_step):
    """The workload part of the JSON line's config, shared by both arms."""
    return {"workload": w.name, "frames_per_step": frames_per_step, "n_elem": w.n_elem, "n_samples": w.nt,
            "nx": w.nx, "nz": w.nz, "n_bins": int(len(w.bins())), "n_apod": 3}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_mhz):
    """FP32 CUDA-core peak from unit counts: SMs x FP32 lanes x 2 flops (FMA) x clock."""
    return SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def prop_source_hash():
    h = hashlib.sha256()
    for f in ("pam_prop.cu", "pam_internal.h", "pam_ptx.h"):
        with open(os.path.join(ROOT, "paper_2412_02413_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def committed_traffic():
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    or None when the kernel source changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "prop_seg_traffic_astax_128el_128x512.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    if d.get("source_sha256") != prop_source_hash():
        return None
    return d.get("dram_bytes_per_launch")


def fp32_fma_rates(iters=2048):
    """(scalar, packed two-wide) FP32 FMA rates in TFLOP/s from the bench-side
    probe library, or (None, None) when it is missing."""
    import ctypes
    from paper_2412_02413_gb300 import build
    if not os.path.exists(build.PROBE_LIB):
        return None, None
    lib = ctypes.CDLL(build.PROBE_LIB)
    lib.pam_probe_fp32_fma_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.pam_probe_fp32_fma_rate.restype = ctypes.c_int
    out = []
    for packed in (0, 1):
        v = ctypes.c_double(0.0)
        out.append(v.value if lib.pam_probe_fp32_fma_rate(iters, packed, ctypes.byref(v)) == 0 else None)
    return tuple(out)


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"pam_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu_index)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.remove(self.path)
        if not rows:
            return None
        import statistics
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_index_for(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


# ------------------------------------------------------------------- pool --
def _make_frame(args):
    wid, f = args
    from paper_2412_02413_gb300 import synth
    return synth.make_frame(synth.workload(wid), f)[0]


def make_pool(wid, first, n):
    """Seeded synthetic frames, generated in spawned worker processes (before any CUDA call)."""
    import multiprocessing as mp

    import numpy as np
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=max(1, min(16, os.cpu_count() or 1))) as pool:
        frames = pool.map(_make_frame, [(wid, first + i) for i in range(n)])
    return np.stack(frames)


# --------------------------------------------------------- oracle timing --
def oracle_time(w, rf, nb, nzs, threads):
    """Seconds of one oracle AS-TAX call on the first nb bins of Omega x the
    first nzs depth rows of workload w's frame rf, with `threads` threads."""
    import oracle
    bins = w.bins()
    A = oracle.pattern(w.n_elem, 3, w.pattern_m)
    g = oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, nzs, w.z0, w.dz, bins[:nb])
    t0 = time.perf_counter()
    oracle.as_tax(g, rf, A, threads=threads)
    return time.perf_counter() - t0


def oracle_runs(w, rf, nb, nzs, threads, runs):
    """frames/s of `runs` oracle calls on a (bins x rows) sample, each scaled to
    a whole frame by the sampled fraction of (bin, row) units: mean, sd."""
    import statistics
    frac = (nb * nzs) / float(len(w.bins()) * w.nz)
    fps = [frac / oracle_time(w, rf, nb, nzs, threads) for _ in range(runs)]
    return {"value": statistics.mean(fps), "sd": statistics.stdev(fps) if len(fps) > 1 else 0.0, "runs": runs,
            "unit": "frames/s", "threads": threads, "extrapolated": frac < 1.0, "sampled_fraction": frac,
            "sample": f"{nb} of {len(w.bins())} bins x {nzs} of {w.nz} depth rows of one frame"}


def cpu_baseline(pool_np, runs=10):
    """The oracle on the host cores (the CPU baseline plan): the 128-element
    workload on a fixed sample, all threads and one thread, and whole frames of
    the 64-element workload on all threads; `runs` runs each, mean and sd."""
    from paper_2412_02413_gb300 import synth
    cores = os.cpu_count() or 1
    w2 = synth.workload(2)
    rf2 = pool_np[0]
    allt = oracle_runs(w2, rf2, min(2 * cores, len(w2.bins())), 128, cores, runs)
    one = oracle_runs(w2, rf2, 4, 32, 1, runs)
    w1 = synth.workload(1)
    rf1, _ = synth.make_frame(w1, 0)
    whole1 = oracle_runs(w1, rf1, len(w1.bins()), w1.nz, cores, runs)
    return {"value": allt["value"], "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": allt["sample"] + f", {cores} threads, {runs} runs (mean; sd in 'sd'), scaled to whole frames",
            "sd": allt["sd"], "runs": runs, "extrapolated": True, "sampled_fraction": allt["sampled_fraction"],
            "single_thread": one, "workload_64el_whole_frame": whole1}


def oracle_sample_rate(w, rf, budget_s, threads=None):
    """Times the oracle on a bounded sample of the workload (the first n_b bins
    of Omega x the first nz' depth rows) sized to about budget_s seconds, and
    scales it to frames/s. Returns (frames/s, seconds measured, sample
    description, threads, sampled fraction)."""
    threads = threads or (os.cpu_count() or 1)
    bins = w.bins()
    # calibrate on one bin per thread and 8 rows, then size the sample to the budget
    nb0 = min(len(bins), threads)
    t0 = oracle_time(w, rf, nb0, 8, threads)
    per_unit = t0 / (nb0 * 8)                               # s per (bin x row), all threads busy
    units = max(1, int(budget_s / max(per_unit, 1e-9)))
    nzs = int(min(w.nz, max(1, units // nb0)))
    nb = int(min(len(bins), max(nb0, units // max(nzs, 1))))
    t = oracle_time(w, rf, nb, nzs, threads)
    frac = (nb * nzs) / float(len(bins) * w.nz)
    sample = f"{nb} of {len(bins)} bins x {nzs} of {w.nz} depth rows of one frame, {threads} threads"
    return frac / t, t, sample, threads, frac


def run_reference(args):
    from paper_2412_02413_gb300 import dist, synth
    rank, _, world = dist.env_rank()
    if rank != 0:
        return 0
    w = synth.workload(args.workload)
    rf, _ = synth.make_frame(w, 0)
    budget = max(0.05, min(2.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample_rate(w, rf, budget)
    rates = []
    t_total = 0.0
    sample, threads, frac = "", 0, 1.0
    for _ in range(args.steps):
        fps, t, sample, threads, frac = oracle_sample_rate(w, rf, budget)
        rates.append(fps)
        t_total += t
    value = len(rates) / sum(1.0 / r for r in rates)   # frames per second of extrapolated time
    line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_config(w, 1), "streams": 1,
                       "sample": "oracle on a bounded sample of bins x depth rows, scaled to whole frames",
                       "extrapolated": True, "sampled_fraction": frac,
                       "measured_seconds": t_total},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": threads, "kind": "oracle",
                             "sample": sample + " per step", "extrapolated": True, "sampled_fraction": frac},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_forms(args, w, pool, stream, dev):
    """Frames/s of the batched forms (args.batch frames per call) on the frame pool;
    each tensor-core form's image is compared with the plain FP32 form's."""
    import torch
    from paper_2412_02413_gb300 import pam
    P = pool.shape[0]
    forms = {}
    ref_img = None
    names = [f for f in args.forms.split(",") if f]
    if names and names[0] != "fp32" and "fp32" in names:
        names.remove("fp32")
        names.insert(0, "fp32")
    from paper_2412_02413_gb300 import autotune
    tuner = autotune.Autotuner()
    for form in names:
        fp = pam.Plan.from_workload(w, max_frames=args.batch, form=form)
        fo = {"image": torch.empty(args.batch, w.nz, w.nx, device=dev),
              "rho_n": torch.empty(args.batch, w.nz, w.nx, device=dev)}
        nb = max(1, P // args.batch)
        tile = gframes = lane_rows = None
        if form != "fp32":   # the GEMM's M tile (one CTA per row, or CTA pairs) and frames per CTA
            if args.gemm_tile:
                tile = args.gemm_tile
                fp.set_gemm_tile(tile)
            else:
                tile = autotune.tune_gemm_tile(tuner, fp, pool[0:args.batch], form)
            if args.gemm_frames:
                gframes = args.gemm_frames
                fp.set_gemm_frames(gframes)
            else:
                gframes = autotune.tune_gemm_frames(tuner, fp, pool[0:args.batch], form)
        elif args.lane_rows:  # depth rows per lane of the fused kernel
            lane_rows = args.lane_rows
            fp.set_lane_rows(lane_rows)
        else:
            lane_rows = autotune.tune_lane_rows(tuner, [fp], pool[0:args.batch])

        def bstep(i):
            s0 = (i % nb) * args.batch
            fp.as_tax(pool[s0:s0 + args.batch], outs=fo, stream=stream)

        for i in range(3):
            bstep(i)
        torch.cuda.synchronize()
        fp.profile_enable(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.batch_steps):
            bstep(i)
        e1.record(stream)
        torch.cuda.synchronize()
        kms, kn, kl = fp.profile_read()
        fms = e0.elapsed_time(e1)
        bstep(0)
        torch.cuda.synchronize()
        img = fo["image"].double()
        entry = {"frames_per_call": args.batch, "gemm_tile_m": tile, "gemm_frames_per_cta": gframes,
                 "lane_rows": lane_rows,
                 "value": args.batch * args.batch_steps / (fms / 1000.0),
                 "unit": "frames/s", "ms_per_frame": fms / (args.batch * args.batch_steps),
                 "main_kernel_us_per_frame": 1000.0 * kms / max(kn, 1) / args.batch}
        if form != "fp32":
            # The method's work per frame: the per-bin propagation as a complex GEMM, (nz nx) x n_elem
            # by frames, 8 flops per complex MAC (20.1 GFLOP at 128 x 512, 128 elements, 300 bins).
            # The MMA work issued: M = nx, K = 2 n_elem (Re, Im), N = 2 per (bin, row), 2 flops per
            # MAC, three products (hi hi, hi lo, lo hi) in the split forms.
            method = 8.0 * w.nz * w.nx * w.n_elem * fp.n_bins
            mma = 2.0 * w.nx * (2 * w.n_elem) * 2 * fp.n_bins * w.nz * (3 if "split" in form else 1)
            peaks, kind = measured_peaks()
            sec = entry["main_kernel_us_per_frame"] * 1e-6
            entry["tensor"] = {"method_tflop_per_frame": method / 1e12, "achieved_tflops": method / sec / 1e12,
                               "frac_method": method / sec / 1e12 / peaks["bf16_tflops"],
                               "mma_tflop_per_frame": mma / 1e12, "mma_tflops": mma / sec / 1e12,
                               "frac_mma": mma / sec / 1e12 / peaks["bf16_tflops"],
                               "peak_tflops": peaks["bf16_tflops"],
                               "peak_basis": f"bf16_tflops ({kind}); FP16 dense rate equals BF16"}
        if form == "fp32":
            ref_img = img
        elif ref_img is not None:
            entry["rel_l2_vs_fp32"] = float(torch.linalg.norm(img - ref_img) / torch.linalg.norm(ref_img))
        forms[form] = entry
        fp.close()
    return forms


def run_batch(args, dev, stream):
    """Uneven batch (workload 3): args.batch_frames frames with their own
    sample counts and depth ranges in one graph-launched call, against a loop
    of one-frame calls of the same frames."""
    import numpy as np
    import torch
    from paper_2412_02413_gb300 import pam, synth
    ws = synth.batch_workload(args.batch_frames)
    frames = [(w.nt, w.nz) for w in ws]
    common = dict(n_elem=128, pitch=0.3e-3, fs=40e6, c=1540.0, z0=5e-3, dz=synth.BATCH_DZ, n_bins=300,
                  f_lo=0.5e6, f_hi=8e6, n_apod=3, pattern_m=16)
    b = pam.Batch(frames=frames, **common)
    rng = np.random.default_rng(20241203 + 3000 + 7)
    rf = torch.from_numpy(rng.standard_normal(b.rf_total, dtype=np.float32)).to(dev)
    img = torch.empty(b.map_total, device=dev)
    rn = torch.empty(b.map_total, device=dev)
    # persistent grid picked by the autotuner (cached; timed through the batch call itself)
    from paper_2412_02413_gb300 import autotune
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    tuner = autotune.Autotuner()
    tuned_grid = autotune.tune_batch_grid(tuner, b, rf, sms)
    tuned_key = autotune.make_key("batch_grid", b.n_elem, max(b.n_samples), max(b.nz), b.n_frames)
    for _ in range(3):
        b.as_tax(rf, image=img, rho_n=rn, stream=stream)
    torch.cuda.synchronize()
    k0 = b.info()[2]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.batch_calls):
        b.as_tax(rf, image=img, rho_n=rn, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    b.sync(stream)
    ms = e0.elapsed_time(e1) / args.batch_calls
    kernels = (b.info()[2] - k0) // args.batch_calls
    n_items, grid, _ = b.info()
    # loop of one-frame calls (direct launches, no graph) over the first frames
    nl = min(len(frames), args.batch_loop_frames)
    singles = []
    for i in range(nl):
        s1 = pam.Batch(frames=[frames[i]], **common)
        s1.configure(use_graph=False)
        r1 = rf[b.rf_offsets[i]:b.rf_offsets[i] + s1.rf_total].contiguous()
        singles.append((s1, r1, torch.empty(s1.map_total, device=dev), torch.empty(s1.map_total, device=dev)))
    for s1, r1, i1, n1 in singles:
        s1.as_tax(r1, image=i1, rho_n=n1, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for s1, r1, i1, n1 in singles:
        s1.as_tax(r1, image=i1, rho_n=n1, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    loop_ms = e0.elapsed_time(e1)
    for s1, *_ in singles:
        s1.close()
    # algorithmic FP32 work: the fused path per frame plus the direct time DFT (4 flops per sample, bin, channel)
    flops = sum(fused_flops_per_frame(len(b.bins[i]), nz, 128, 3) + 4.0 * len(b.bins[i]) * 128 * nt
                for i, (nt, nz) in enumerate(frames))
    peaks, _ = measured_peaks()
    peak_tf = fp32_peak_tflops(float(peaks.get("sm_max_mhz", 2070.0)))
    out = {"workload": "uneven_batch_128el_nt1024-8192_nz128-512_300bins", "frames_per_call": len(frames),
           "value": len(frames) / (ms / 1000.0), "unit": "frames/s", "ms_per_call": ms,
           "us_per_frame": 1000.0 * ms / len(frames), "kernels_per_call": kernels, "graph": True,
           "work_items": n_items, "persistent_ctas": grid,
           "autotuned": {"persistent_ctas": tuned_grid, "key": tuned_key,
                         "seconds": tuner.entries().get(tuned_key, {}).get("seconds")},
           "loop_frames": nl, "loop_value": nl / (loop_ms / 1000.0), "loop_us_per_frame": 1000.0 * loop_ms / nl,
           "achieved_tflops": flops / (ms / 1000.0) / 1e12, "fp32_peak_tflops": peak_tf,
           "frac_fp32_peak": flops / (ms / 1000.0) / 1e12 / peak_tf,
           "data": "synthetic Gaussian channel data of the workload's shapes"}
    out["speedup_vs_loop"] = out["value"] / out["loop_value"]
    b.close()
    return out


def run_learned(args, w, pool, stream, dev):
    """Learned AS-TAX (trained checkpoint, tensor-core network, error gate) on
    args.learned_batch frames per call, against the plain FP32 path on the
    same batch, at each error-gate bound of args.gate_tols. Accuracy of the
    learned image against the plain one over every pixel of the pool's
    distinct frames (learn.accuracy_rows: relative L2, brightest pixel, the
    1e-2 / exact-peak bar, ISNR and A_0.5 from pam_image_metrics)."""
    import torch
    from paper_2412_02413_gb300 import learn, pam
    if not os.path.exists(learn.CHECKPOINT):
        return {"unavailable": "no trained checkpoint (python -m paper_2412_02413_gb300.learn)"}
    params, meta = learn.load_checkpoint()
    B = args.learned_batch
    P = pool.shape[0]
    NS = max(1, args.streams)
    rf = pool[torch.arange(B, device=dev) % P].contiguous()
    # calls alternate over NS learned forms (and NS plain plans) on NS streams, as the
    # headline steps do: one batch's latency-bound gate and fallback overlap the next
    # batch's band energies
    Ls, plans = [], []
    for _ in range(NS):
        L_ = pam.Learned.from_workload(w, max_frames=B)
        L_.set_params(params)
        Ls.append(L_)
        plans.append(pam.Plan.from_workload(w, max_frames=B))
    streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(NS - 1)]
    imgs = [torch.empty(B, w.nz, w.nx, device=dev) for _ in range(NS)]
    rns = [torch.empty(B, w.nz, w.nx, device=dev) for _ in range(NS)]
    outss = [{"image": torch.empty(B, w.nz, w.nx, device=dev), "rho_n": torch.empty(B, w.nz, w.nx, device=dev),
              "image_as": torch.empty(B, w.nz, w.nx, device=dev)} for _ in range(NS)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for i in range(2 * NS):
            fn(i)
        torch.cuda.synchronize()
        e0.record(stream)
        for st_ in streams[1:]:
            st_.wait_event(e0)
        for i in range(args.learned_calls):
            fn(i)
        for st_ in streams[1:]:
            e_ = torch.cuda.Event()
            e_.record(st_)
            stream.wait_event(e_)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.learned_calls

    ms_p = timed(lambda i: plans[i % NS].as_tax(rf, outs=outss[i % NS], image_as=True, stream=streams[i % NS]))
    plan, outs = plans[0], outss[0]
    plan.as_tax(rf, outs=outs, image_as=True, stream=stream)
    n = min(B, P)
    gates = []
    for tol in [float(t) for t in args.gate_tols.split(",") if t]:
        for L_ in Ls:
            L_.configure(gate_tol=tol, tensor_cores=True)
            L_.info()
        ms_l = timed(lambda i: Ls[i % NS].as_tax(rf, image=imgs[i % NS], rho_n=rns[i % NS], stream=streams[i % NS]))
        kernels = sum(L_.info()["kernel_launches"] for L_ in Ls) // (args.learned_calls + 2 * NS)
        res = Ls[0].as_tax(rf, image=imgs[0], rho_n=rns[0], stream=stream)
        torch.cuda.synchronize()
        rows = learn.accuracy_rows(imgs[0][:n], outs["image"][:n], outs["image_as"][:n], res["gate_err"][:n],
                                   res["gate_pass"][:n], w)
        gates.append({"gate_tol": tol, "value": B / (ms_l / 1000.0), "unit": "frames/s",
                      "us_per_frame": 1000.0 * ms_l / B, "speedup_vs_plain": ms_p / ms_l, "kernels_per_call": kernels,
                      "accuracy_vs_plain": learn.summarize(rows)})
    for L_, p_ in zip(Ls, plans):
        L_.close()
        p_.close()
    return {"workload": w.name, "frames_per_call": B, "streams": NS, "plain_value": B / (ms_p / 1000.0),
            "plain_us_per_frame": 1000.0 * ms_p / B, "strict_bar": {"rel_l2": learn.STRICT_REL_L2, "peak": "exact"},
            "gates": gates,
            "checkpoint": {"frames": meta.get("frames"), "epochs": meta.get("epochs"),
                           "held_out": meta.get("held_out")}}


# -------------------------------------------------------------- our arm --
def run_ours(args):
    import numpy as np

    from paper_2412_02413_gb300 import dist, synth
    rank, local, world = dist.env_rank()
    w = synth.workload(args.workload)
    F = args.frames_per_step
    pool_np = make_pool(args.workload, 1000 * rank, args.pool)   # before any CUDA call

    import torch
    from paper_2412_02413_gb300 import pam
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist.init("nccl")
    plan = pam.Plan.from_workload(w, max_frames=F)
    pool = torch.from_numpy(pool_np).to(dev)
    P = pool.shape[0]
    outs = {"image": torch.empty(F, w.nz, w.nx, device=dev), "rho_n": torch.empty(F, w.nz, w.nx, device=dev)}
    stream = torch.cuda.current_stream()
    if args.batch_only:
        print(json.dumps({"batch": run_batch(args, dev, stream)}), flush=True)
        dist.finalize()
        return 0
    if args.learned_only:
        print(json.dumps({"learned": run_learned(args, w, pool, stream, dev), "config": {"workload": w.name}}),
              flush=True)
        dist.finalize()
        return 0
    if args.forms_only:
        # profiling aid: only the batched forms, one JSON line
        print(json.dumps({"forms": run_forms(args, w, pool, stream, dev), "config": {"workload": w.name}}),
              flush=True)
        dist.finalize()
        return 0

    # Steps alternate over args.streams plans, one per stream, so that one frame's
    # small kernels (time FFT, lateral FFT, epilogue) overlap another frame's fused
    # kernel; every step is still one whole frame through the path.
    NS = max(1, args.streams)
    plans = [plan] + [pam.Plan.from_workload(w, max_frames=F) for _ in range(NS - 1)]
    streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(NS - 1)]
    outs_k = [outs] + [{"image": torch.empty(F, w.nz, w.nx, device=dev),
                        "rho_n": torch.empty(F, w.nz, w.nx, device=dev)} for _ in range(NS - 1)]

    def step(i):
        s = (i * F) % (P - F + 1)
        k = i % NS
        plans[k].as_tax(pool[s:s + F], outs=outs_k[k], stream=streams[k])

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    # CTAs of the fused kernel in the multi-stream loop: with fewer than one per
    # SM the other streams' small kernels run beside it. Picked by the autotuner
    # on short runs of this loop (cached), before the timed region.
    from paper_2412_02413_gb300 import autotune
    if args.fft_radix:
        radix_choice = args.fft_radix
        for p_ in plans:
            p_.set_fft_radix(args.fft_radix)
    else:
        radix_choice = autotune.tune_time_fft_radix(autotune.Autotuner(), plans, pool[0:F])
    if args.lane_rows:
        lane_rows_choice = args.lane_rows
        for p_ in plans:
            p_.set_lane_rows(args.lane_rows)
    else:
        lane_rows_choice = autotune.tune_lane_rows(autotune.Autotuner(), plans, pool[0:F])
    grid_choice = None
    if NS > 1 and args.grid < 0:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        grid_choice = autotune.tune_stream_grid(autotune.Autotuner(), plans, step, sms, NS, w, F, streams)
    elif args.grid > 0:
        grid_choice = args.grid
    if grid_choice:
        for p_ in plans:
            p_.set_grid(int(grid_choice))
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    clocks = ClockSampler(gpu_index_for(local))
    clocks.start()
    time.sleep(0.3)
    dist.barrier()
    torch.cuda.synchronize()
    for p_ in plans:
        p_.profile_enable(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for st_ in streams[1:]:
        st_.wait_event(ev0)
    for i in range(args.steps):
        step(args.warmup + i)
    for st_ in streams[1:]:
        e_ = torch.cuda.Event()
        e_.record(st_)
        stream.wait_event(e_)
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prop_ms, prop_launches, launches = 0.0, 0, 0
    for p_ in plans:
        a_, b_, c_ = p_.profile_read()
        prop_ms, prop_launches, launches = prop_ms + a_, prop_launches + b_, launches + c_
        p_.profile_enable(False)
    ms_max = dist.max_over_ranks(ms, device=dev)
    frames_total = dist.sum_over_ranks(args.steps * F, device=dev)
    value = frames_total / (ms_max / 1000.0)

    # The dominant kernel alone: a single-stream run right after the timed region,
    # one CTA per SM (with several streams its launches share the SMs with the
    # other streams' kernels, which lengthens each launch beyond a step). The
    # roofline is taken from this per-launch time.
    iso_steps = max(1, min(args.steps, 500))
    plan.set_grid(0)
    for i in range(10):
        plan.as_tax(pool[i % P:i % P + F], outs=outs, stream=stream)
    torch.cuda.synchronize()
    plan.profile_enable(True)
    for i in range(iso_steps):
        s_ = (i * F) % (P - F + 1)
        plan.as_tax(pool[s_:s_ + F], outs=outs, stream=stream)
    torch.cuda.synchronize()
    iso_ms, iso_n, _ = plan.profile_read()
    plan.profile_enable(False)
    if grid_choice:
        plan.set_grid(int(grid_choice))

    # End to end through the host-buffer entry points: every step uploads its frame
    # from pinned memory and downloads its image and rho_n into pinned memory.
    # Pipelined (the value reported): max(2, --streams) plans on as many streams with
    # pam_as_xcorr_host_async, so one frame's copies overlap another's kernels; a
    # step's host buffers are reused that many steps later, after its download landed.
    # Blocking: pam_as_xcorr_host, which returns with the results in host memory.
    n_host = min(8, P)
    rf_host = torch.from_numpy(pool_np[: n_host * F].reshape(n_host, F, w.n_elem, w.nt).copy()).pin_memory()
    NE = max(2, NS)                      # frames in flight
    outs_host = [(torch.empty(F, w.nz, w.nx).pin_memory(), torch.empty(F, w.nz, w.nx).pin_memory())
                 for _ in range(NE)]
    outs_np = [(a.numpy(), b.numpy()) for a, b in outs_host]
    extra = [pam.Plan.from_workload(w, max_frames=F) for _ in range(NE - NS)]
    for p_ in extra:   # the tuned choices of the timed plans
        p_.set_fft_radix(int(radix_choice))
        p_.set_lane_rows(int(lane_rows_choice))
        if grid_choice:
            p_.set_grid(int(grid_choice))
    plans2 = plans + extra
    streams2 = streams + [torch.cuda.Stream(device=dev) for _ in range(NE - NS)]
    done = [torch.cuda.Event() for _ in range(NE)]
    e2e_steps = max(1, min(args.steps, 500))

    def e2e_pipelined(n):
        for i in range(n):
            k = i % NE
            if i >= NE:
                done[k].synchronize()
            plans2[k].as_xcorr_host_async(rf_host[i % n_host].numpy(), outs_np[k][0], outs_np[k][1],
                                          stream=streams2[k])
            done[k].record(streams2[k])
        torch.cuda.synchronize()

    e2e_pipelined(4)
    dist.barrier()
    t0 = time.perf_counter()
    e2e_pipelined(e2e_steps)
    t_e2e = dist.max_over_ranks(time.perf_counter() - t0, device=dev)
    e2e_value = dist.sum_over_ranks(e2e_steps * F, device=dev) / t_e2e
    for i in range(3):
        plan.as_xcorr_host(rf_host[i % n_host].numpy(), outs_np[0][0], outs_np[0][1], stream=stream)
    dist.barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        plan.as_xcorr_host(rf_host[i % n_host].numpy(), outs_np[0][0], outs_np[0][1], stream=stream)
    t_blk = dist.max_over_ranks(time.perf_counter() - t0, device=dev)
    e2e_blocking = dist.sum_over_ranks(e2e_steps * F, device=dev) / t_blk
    for p_ in extra:
        p_.close()

    # Batched forms: 64 frames per call, the plain FP32 path and the tensor-core forms.
    forms = {} if args.no_forms else run_forms(args, w, pool, stream, dev)
    batch = run_batch(args, dev, stream) if args.batch_frames > 0 and rank == 0 else {}
    learned = run_learned(args, w, pool, stream, dev) if args.learned_batch > 0 and rank == 0 else {}

    peaks, peak_kind = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tf = fp32_peak_tflops(sm_max)
    fma_tf, fma2_tf = (fp32_fma_rates() if rank == 0 else (None, None))   # after the timed region
    flops = fused_flops_per_frame(plan.n_bins, w.nz, w.nx, 3) * F
    live_launch_s = prop_ms / max(prop_launches, 1) / 1000.0
    alone_launch_s = iso_ms / max(iso_n, 1) / 1000.0
    achieved_tf = flops / alone_launch_s / 1e12
    traffic = committed_traffic()

    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(pool_np, runs=args.cpu_runs)
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Green's-function point sources, 20 dB channel SNR)",
            "config": {**workload_config(w, F), "streams": NS,
                       "fused_ctas": int(grid_choice) if grid_choice else "one per SM",
                       "time_fft_radix": int(radix_choice), "lane_rows": int(lane_rows_choice),
                       "l2": f"rotating pool of {P} distinct input frames ({P * w.n_elem * w.nt * 4 / 1e6:.0f} MB)"
                             " > 129 MB L2", "parallelism": f"frames sharded over {world} GPU(s)"},
            "e2e": {"value": e2e_value, "unit": "frames/s",
                    "h2d_bytes_per_step": F * w.n_elem * w.nt * 4, "d2h_bytes_per_step": 2 * F * w.nz * w.nx * 4,
                    "mode": f"pam_as_xcorr_host_async, {NE} plans on {NE} streams (copies overlap kernels)",
                    "blocking_value": e2e_blocking},
            "gpu_launches": int(launches),
            "avg_launch_us_alone": alone_launch_s * 1e6,
            "roofline": {"bound": "alu", "kernel": f"prop_seg_kernel<3,128,{int(lane_rows_choice)}> (fused propagate + "
                                                   "inverse lateral FFT + cross-spectra; rows per lane)",
                         "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s", "frac": achieved_tf / peak_tf,
                         "traffic": traffic,
                         "peak_basis": f"{SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz "
                                       f"(sm_max_mhz, {peak_kind})",
                         "flops_per_launch": flops, "avg_launch_us": alone_launch_s * 1e6,
                         "launch_timing": f"{iso_n} launches on one stream right after the timed region, one CTA "
                                          "per SM, CUDA events on the launch stream",
                         "share_of_step": alone_launch_s * 1e3 / (ms_max / args.steps),
                         "live": {"avg_launch_us": live_launch_s * 1e6, "launches": prop_launches,
                                  "achieved": flops / live_launch_s / 1e12,
                                  "frac": flops / live_launch_s / 1e12 / peak_tf,
                                  "share_of_step": (prop_ms / ms) if ms > 0 else None,
                                  "note": f"inside the timed region: {NS} streams, so each launch shares the SMs "
                                          "with the other streams' kernels and lasts longer than alone"},
                         "peak_fp32_measured": {"value": fma_tf, "unit": "TFLOP/s",
                                                "frac_of_peak": fma_tf / peak_tf if fma_tf else None,
                                                "packed_fma2_value": fma2_tf,
                                                "how": "libpam_probe.so (bench-side probe): independent FMA chains "
                                                       "on every SM, scalar and packed two-wide, after the timed "
                                                       "region"}},
            "clocks": ck,
            "forms": forms,
            "batch": batch,
            "learned": learned,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    for p_ in plans:
        p_.close()
    dist.finalize()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--frames-per-step", type=int, default=1)
    ap.add_argument("--streams", type=int, default=3, help="plans / streams the steps alternate over")
    ap.add_argument("--grid", type=int, default=-1,
                    help="CTAs of the fused kernel in the multi-stream loop (-1: autotuned, 0: one per SM)")
    ap.add_argument("--fft-radix", type=int, default=0, choices=[0, 4, 8],
                    help="largest radix of the time FFT (0: autotuned)")
    ap.add_argument("--lane-rows", type=int, default=0, choices=[0, 1, 2],
                    help="depth rows per lane of the fused kernel (0: autotuned)")
    ap.add_argument("--gemm-tile", type=int, default=0, choices=[0, 128, 256],
                    help="M tile of the tensor-core forms (0: autotuned)")
    ap.add_argument("--gemm-frames", type=int, default=0, choices=[0, 16, 32],
                    help="frames per CTA of the tensor-core forms (0: autotuned)")
    ap.add_argument("--pool", type=int, default=POOL_FRAMES)
    ap.add_argument("--cpu-runs", type=int, default=10, help="runs of each cpu_baseline measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched plain / tensor-core forms")
    ap.add_argument("--batch", type=int, default=64, help="frames per call of the batched forms")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--forms", default="fp32,bf16,fp16,bf16split,fp16split", help="comma list of batched forms to time")
    ap.add_argument("--forms-only", action="store_true", help="time only the batched forms (profiling aid)")
    ap.add_argument("--batch-frames", type=int, default=256, help="frames of the uneven batch (0: skip)")
    ap.add_argument("--batch-calls", type=int, default=10)
    ap.add_argument("--batch-loop-frames", type=int, default=32, help="frames of the one-frame-call loop")
    ap.add_argument("--batch-only", action="store_true", help="time only the uneven batch (profiling aid)")
    ap.add_argument("--learned-batch", type=int, default=256, help="frames per learned-form call (0: skip)")
    ap.add_argument("--learned-calls", type=int, default=6)
    ap.add_argument("--gate-tols", default="0.25,0.05,0.01", help="error-gate bounds of the learned form to time")
    ap.add_argument("--learned-only", action="store_true", help="time only the learned form (profiling aid)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
