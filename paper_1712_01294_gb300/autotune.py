"""Autotuner for the launch-shape knobs of a context.

Two knobs decide how the density pass maps particles to lanes:
* the cell length (``cell_factor`` x H0 of each box) decides how many
  candidate cells the h-iteration scans and how evenly the per-cell loops of
  a warp are filled; the best value depends on the particle distribution (a
  lattice-aligned grid can be twice as fast as a misaligned one);
* the candidate cache per particle (``density_cache``, 40 or 48 entries)
  decides which particles get one lane and which a whole warp: a particle
  with more candidates within 1.05 H than its cache holds is iterated by a
  warp (a blast cavity, the smallest boxes of an ensemble), and the larger
  cache costs occupancy.
The tuner times full steps for each combination on a copy of the caller's
particles (through the C ABI, CUDA-event timed) and keeps the fastest.  The
steps timed should cover the run being tuned for: the best cache size moves
as the run evolves (in the 256-box Sod/Sedov ensemble the 40-entry cache is
fastest over steps 2-3 and the 48-entry one over the 20 steps of the run,
by 8 %, once the blast cavities form), so `tune(..., steps=20, warmup=0)`
tunes a 20-step run from its initial state.  Results are cached by
(particle counts, precision, distribution signature, steps) in a JSON file.  The other kernels' block shapes are fixed by
design (one thread per particle, sized for occupancy at their register
counts).
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

DEFAULT_CANDIDATES = (0.7, 0.85, 1.0, 1.2, 1.45)
DEFAULT_CACHES = (40, 48)


def _cache_path(path=None):
    if path:
        return path
    root = os.environ.get("GZ_AUTOTUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "gz_mfm", "autotune.json")
    return root


def signature(p, precision) -> str:
    """Key of a particle set: box sizes, precision and a coarse digest of the
    support-radius distribution (its quartiles relative to H0)."""
    counts = [int(c) for c in (p.counts if len(p.counts) else [p.N])]
    H = np.asarray(p.H, dtype=np.float64)
    q = np.quantile(H, [0.1, 0.5, 0.9]) / max(float(np.mean(H)), 1e-300)
    digest = hashlib.sha1(np.asarray(counts, dtype=np.int64).tobytes()).hexdigest()[:12]
    return f"{len(counts)}x{sum(counts)}:{digest}:p{int(precision)}:h{q[0]:.2f}-{q[1]:.2f}-{q[2]:.2f}"


def _key(cf, cache):
    return f"{float(cf)},{int(cache)}"


def tune(p, precision, candidates=DEFAULT_CANDIDATES, caches=DEFAULT_CACHES, steps: int = 8,
         warmup: int = 1, cache: str | None = None, use_cache: bool = True, **params):
    """Returns (best (cell_factor, density_cache), {(cell_factor, density_cache): ms
    per step}) for host particles p."""
    import torch

    import paper_1712_01294_gb300 as gz
    path = _cache_path(cache)
    key = (signature(p, precision) + ":c" + "-".join(str(int(c)) for c in caches)
           + f":s{int(warmup)}+{int(steps)}")
    db = {}
    if use_cache and os.path.exists(path):
        try:
            db = json.load(open(path))
        except Exception:
            db = {}
        if key in db:
            def parse(k):
                a, b = k.split(",")
                return float(a), int(b)
            return parse(db[key]["best"]), {parse(k): v for k, v in db[key]["ms"].items()}
    counts = [int(c) for c in (p.counts if len(p.counts) else [p.N])]
    stream = torch.cuda.Stream()
    ms = {}
    with torch.cuda.stream(stream):
        base = gz.to_device(p, precision)
        for cf in candidates:
            for dc in caches:
                ctx = gz.Context(counts, gz.default_params(precision=precision, cell_factor=cf,
                                                           density_cache=int(dc), **params), stream=stream)
                d = {k: v.clone() for k, v in base.items()}
                for _ in range(warmup):
                    ctx.step(d)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    ctx.step(d)
                e1.record(stream)
                torch.cuda.synchronize()
                if ctx.status(reset=True)["ok"]:
                    ms[(float(cf), int(dc))] = e0.elapsed_time(e1) / steps
                ctx.close()
    best = min(ms, key=ms.get)
    if use_cache:
        db[key] = {"best": _key(*best), "ms": {_key(*k): v for k, v in ms.items()}}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        json.dump(db, open(tmp, "w"), indent=1)
        os.replace(tmp, path)
    return best, ms
