"""Shared helpers for the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np

import oracle as O

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "u", "H")


def cast_state(p, precision):
    """Host particles in the working precision, and the same values in FP64 for
    the oracle (so both sides see bit-identical inputs)."""
    import paper_1712_01294_gb300 as gz
    dt = np.float64 if precision == gz.GZ_FP64 else np.float32
    q = p.copy()
    for k in FIELDS:
        v = getattr(q, k).astype(dt)
        if k in ("x", "y", "z"):
            v = np.where(v >= 1.0, v - dt(1.0), v).astype(dt)
        setattr(q, k, v.astype(np.float64))
    return q


def device(p, precision, H=None):
    import torch
    import paper_1712_01294_gb300 as gz
    d = gz.to_device(p, precision)
    if H is not None:
        d["h"] = torch.as_tensor(np.asarray(H), dtype=d["x"].dtype).cuda().contiguous()
    return d


def ostate(p):
    return O.State.from_any(p.__dict__)


def rms(a):
    a = np.asarray(a, dtype=np.float64)
    return float(np.sqrt(np.mean(a * a))) if a.size else 0.0


def field_err(gpu, ref):
    """(max |diff| / RMS(ref), RMS(diff) / RMS(ref)) along the last axis."""
    g = np.asarray(gpu, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    s = rms(r)
    if s == 0.0:
        s = 1.0
    d = g - r
    return float(np.max(np.abs(d))) / s, rms(d) / s


def min_image(d):
    return np.where(d >= 0.5, d - 1.0, np.where(d < -0.5, d + 1.0, d))


def gpu_sets(ctx, cap=128):
    cnt, ids = ctx.neighbours(cap)
    cnt = cnt.cpu().numpy()
    ids = ids.cpu().numpy()
    return cnt, [set(ids[:c, i].tolist()) for i, c in enumerate(cnt)]


def oracle_sets(s, H):
    off, nb = O.neighbours(s, H)
    return [set(s.id[nb[off[i]:off[i + 1]]].tolist()) for i in range(s.N)]
