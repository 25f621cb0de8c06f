"""Measured choice of launch parameters, cached as JSON.

Knobs with no closed-form best value on a given GPU:
* the largest radix of the time FFT's Stockham stages, 8 or 4
  (``Plan.set_fft_radix``);
* the depth rows per lane of the fused kernel, 1 or 2 (``Plan.set_lane_rows``);
* the number of CTAs of the fused kernel when several plans run on several
  streams (``Plan.set_grid``): fewer than one per SM leaves room for the other
  streams' small kernels;
* the bin split of the fused kernel (``Plan.set_split``; 0 is the even
  division);
* the persistent grid of a batch (``Batch.configure(persistent_ctas=...)``);
* the M tile of the tensor-core form's MMAs, 128 (one CTA per row) or 256
  (CTA pairs, ``Plan.set_gemm_tile``), and its frames per CTA, 32 or 16 (the
  MMA's N tile, ``Plan.set_gemm_frames``).
The tuner times each candidate through the library's own calls, keeps the
fastest, and caches it under a key made of the problem's shape: (kind,
n_elem, nt bucket, nz bucket, frames). nt and nz are bucketed to the next
power of 2 so that frames of similar size share an entry.

The selection and caching logic is plain Python and takes any timing
function, so it is tested without a GPU.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Callable, Dict, Iterable, Optional


def bucket(v: int) -> int:
    """Next power of 2 >= v (v >= 1)."""
    v = max(1, int(v))
    return 1 << (v - 1).bit_length()


def make_key(kind: str, n_elem: int, nt: int, nz: int, frames: int) -> str:
    return f"{kind}:ne{int(n_elem)}:nt{bucket(nt)}:nz{bucket(nz)}:F{int(frames)}"


def default_cache_path() -> str:
    p = os.environ.get("PAM_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "pam_gb300_autotune.json")


class Autotuner:
    """Keeps {key: {"best": value, "seconds": {str(value): s}}} in a JSON file."""

    def __init__(self, path: Optional[str] = None):
        self.path = path or default_cache_path()
        self._lock = threading.Lock()
        self._db: Dict[str, dict] = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as fh:
                    db = json.load(fh)
                if isinstance(db, dict):
                    self._db = {k: v for k, v in db.items() if isinstance(v, dict) and "best" in v}
            except (OSError, ValueError):
                self._db = {}

    def lookup(self, key: str):
        e = self._db.get(key)
        return None if e is None else e["best"]

    def entries(self) -> Dict[str, dict]:
        return dict(self._db)

    def tune(self, key: str, candidates: Iterable, run: Callable[[object], float], repeats: int = 3,
             force: bool = False):
        """Times ``run(c)`` (seconds per call) ``repeats`` times per candidate and
        keeps the candidate with the smallest median. Cached unless ``force``."""
        if not force:
            hit = self.lookup(key)
            if hit is not None:
                return hit
        cands = list(candidates)
        if not cands:
            raise ValueError("no candidates")
        times = {}
        for c in cands:
            ts = sorted(float(run(c)) for _ in range(max(1, repeats)))
            times[c] = ts[len(ts) // 2]
        best = min(cands, key=lambda c: (times[c], cands.index(c)))
        with self._lock:
            self._db[key] = {"best": best, "seconds": {str(c): times[c] for c in cands}}
            self._save()
        return best

    def _save(self):
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = f"{self.path}.tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(self._db, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def _event_timer(call, warmup: int = 1, iters: int = 3) -> float:
    """Seconds per call of ``call()`` from CUDA events on the current stream."""
    import torch
    for _ in range(warmup):
        call()
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(iters):
        call()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0 / iters


def tune_plan_split(tuner: Autotuner, plan, rf, candidates=(0, 1, 2, 4, 8, 9, 12, 16), force: bool = False):
    """Best bin split for ``plan.as_tax(rf)`` (0 is the built-in heuristic); applied to the plan."""
    F = rf.shape[0] if rf.dim() == 3 else 1
    key = make_key("split", plan.n_elem, plan.n_samples, plan.nz, F)
    outs = {}

    def run(c):
        plan.set_split(int(c))
        return _event_timer(lambda: plan.as_tax(rf, outs=outs))

    best = tuner.tune(key, candidates, run, force=force)
    plan.set_split(int(best))
    return best


def tune_time_fft_radix(tuner: Autotuner, plans, rf, force: bool = False):
    """Best largest radix (8 or 4) of the time FFT for ``plans[0].as_tax(rf)``;
    applied to every plan of ``plans``."""
    plan = plans[0]
    F = rf.shape[0] if rf.dim() == 3 else 1
    key = make_key("fft_radix", plan.n_elem, plan.n_samples, plan.nz, F)
    outs = {}

    def run(c):
        plan.set_fft_radix(int(c))
        return _event_timer(lambda: plan.as_tax(rf, outs=outs), warmup=2, iters=20)

    best = tuner.tune(key, (8, 4), run, force=force)
    for p in plans:
        p.set_fft_radix(int(best))
    return best


def tune_lane_rows(tuner: Autotuner, plans, rf, force: bool = False):
    """Best depth rows per lane (1 or 2) of the fused kernel for
    ``plans[0].as_tax(rf)``; applied to every plan of ``plans``. The two agree
    to rounding (the sums over bins are grouped by row tile)."""
    plan = plans[0]
    F = rf.shape[0] if rf.dim() == 3 else 1
    key = make_key("lane_rows", plan.n_elem, plan.n_samples, plan.nz, F)
    outs = {}

    def run(c):
        plan.set_lane_rows(int(c))
        return _event_timer(lambda: plan.as_tax(rf, outs=outs), warmup=2, iters=20)

    best = tuner.tune(key, (1, 2), run, force=force)
    for p in plans:
        p.set_lane_rows(int(best))
    return best


def batch_grid_candidates(n_items: int, num_sms: int):
    """Persistent grids tried for a batch: one CTA per SM (the most that fit),
    three quarters and half of that, each capped at the number of work items."""
    return sorted({min(n_items, c) for c in (num_sms // 2, (3 * num_sms) // 4, num_sms)})


def tune_batch_grid(tuner: Autotuner, batch, rf, num_sms: int, force: bool = False):
    """Best persistent grid for ``batch.as_tax(rf)``; applied to the batch."""
    n_items, _, _ = batch.info()
    cands = batch_grid_candidates(n_items, num_sms)
    key = make_key("batch_grid", batch.n_elem, max(batch.n_samples), max(batch.nz), batch.n_frames)
    img = None

    def run(c):
        nonlocal img
        batch.configure(use_graph=True, persistent_ctas=int(c))
        return _event_timer(lambda: batch.as_tax(rf))

    best = tuner.tune(key, cands, run, force=force)
    batch.configure(use_graph=True, persistent_ctas=int(best))
    return best


def stream_grid_candidates(num_sms: int):
    """CTA counts of the fused kernel tried for several plans on several
    streams: every SM (0), or a few SMs left free for the other streams' small
    kernels."""
    return [0] + [num_sms - k for k in (4, 8, 12, 16, 24) if num_sms - k >= num_sms // 2]


def _streams_timer(step, streams, n: int = 200, warmup: int = 12) -> float:
    """Seconds per step of ``step(i)`` (which enqueues step i on its own
    stream) over n steps, from CUDA events that span every stream."""
    import torch
    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(streams[0])
    for st in streams[1:]:
        st.wait_event(e0)
    for i in range(n):
        step(i)
    for st in streams[1:]:
        e = torch.cuda.Event()
        e.record(st)
        streams[0].wait_event(e)
    e1.record(streams[0])
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0 / n


def tune_stream_grid(tuner: Autotuner, plans, step, num_sms: int, n_streams: int, w, frames: int, streams,
                     force: bool = False):
    """Best CTA count of the fused kernel when ``step`` alternates over
    ``plans`` on ``streams``; applied to every plan. 0 means one CTA per SM."""
    key = make_key(f"stream_grid_S{int(n_streams)}", w.n_elem, w.nt, w.nz, frames)

    def run(c):
        for p in plans:
            p.set_grid(int(c))
        return _streams_timer(step, streams)

    best = tuner.tune(key, stream_grid_candidates(num_sms), run, force=force)
    for p in plans:
        p.set_grid(int(best))
    return best


def tune_gemm_tile(tuner: Autotuner, plan, rf, form: str, force: bool = False):
    """Best M tile (128 or 256) of the tensor-core form for ``plan.as_tax(rf)``;
    applied to the plan. The two give identical results."""
    F = rf.shape[0] if rf.dim() == 3 else 1
    key = make_key(f"gemm_tile_{form}", plan.n_elem, plan.n_samples, plan.nz, F)
    outs = {}

    def run(c):
        plan.set_gemm_tile(int(c))
        return _event_timer(lambda: plan.as_tax(rf, outs=outs), warmup=2, iters=5)

    best = tuner.tune(key, (128, 256), run, force=force)
    plan.set_gemm_tile(int(best))
    return best


def tune_gemm_frames(tuner: Autotuner, plan, rf, form: str, force: bool = False):
    """Best frames per CTA (32 or 16) of the tensor-core form for
    ``plan.as_tax(rf)``; applied to the plan. The two give identical results."""
    F = rf.shape[0] if rf.dim() == 3 else 1
    key = make_key(f"gemm_frames_{form}", plan.n_elem, plan.n_samples, plan.nz, F)
    outs = {}

    def run(c):
        plan.set_gemm_frames(int(c))
        return _event_timer(lambda: plan.as_tax(rf, outs=outs), warmup=2, iters=5)

    best = tuner.tune(key, (32, 16), run, force=force)
    plan.set_gemm_frames(int(best))
    return best
