"""gz_scan_stats, the work counts of the neighbour search: its neighbours equal
the lists' counts of the density pass, and its candidates equal a host count
of the same cell scan (per-box cells of length >= H0, the scan's cell range
around [x - 1.05 H, x + 1.05 H] and its nearest-point test), exactly on a
lattice and to within a few borderline cells on jittered boxes."""
import math

import numpy as np
import pytest
import torch

from paper_1712_01294_gb300 import inputs as I

from gpu_common import cast_state, device

pytestmark = pytest.mark.gpu


def host_counts(x, y, z, H, ngb=32.0, cell_factor=1.0, rf=1.05):
    """Candidates tested, those within 1.05 H and within H, for one box."""
    N = x.size
    H0 = math.cbrt(3.0 * ngb / (4.0 * math.pi * N))
    nc = min(max(int(math.floor(1.0 / (cell_factor * H0))), 1), 512)
    P = np.stack([x, y, z], 1)
    c = np.minimum(np.floor(P * nc).astype(np.int64), nc - 1)
    occ = np.bincount((c[:, 2] * nc + c[:, 1]) * nc + c[:, 0], minlength=nc ** 3).reshape(nc, nc, nc)
    cand = inr = inh = 0
    for i in range(N):
        R = rf * H[i]
        full = not (R < 0.5)
        lo, hi, wraps = [], [], full
        for a in range(3):
            l = 0 if full else math.floor((P[i, a] - R) * nc - 1e-3)
            h = nc - 1 if full else math.floor((P[i, a] + R) * nc + 1e-3)
            if h - l + 1 >= nc:
                l, h, wraps = 0, nc - 1, True
            lo.append(l)
            hi.append(h)
        R2 = R * R * 1.0001
        cl = 1.0 / nc
        for cz in range(lo[2], hi[2] + 1):
            gz = 0.0 if wraps else max(cz * cl - P[i, 2], P[i, 2] - (cz + 1) * cl, 0.0)
            for cy in range(lo[1], hi[1] + 1):
                gy = 0.0 if wraps else max(cy * cl - P[i, 1], P[i, 1] - (cy + 1) * cl, 0.0)
                for cx in range(lo[0], hi[0] + 1):
                    gx = 0.0 if wraps else max(cx * cl - P[i, 0], P[i, 0] - (cx + 1) * cl, 0.0)
                    if gz * gz + gy * gy + gx * gx > R2:
                        continue
                    cand += occ[cz % nc, cy % nc, cx % nc]
        cand -= 1  # the particle itself
        d = P - P[i]
        d -= np.round(d)
        r2 = (d * d).sum(1)
        r2[i] = np.inf
        inr += int((r2 < R * R).sum())
        inh += int((r2 < H[i] * H[i]).sum())
    return cand, inr, inh


def stats_case(m, boxes, prec):
    q = cast_state(boxes, prec)
    counts = [int(c) for c in q.counts] if q.counts.size else [q.N]
    ctx = m.Context(counts, m.default_params(precision=prec))
    d = device(q, prec)
    ctx.density(d)
    st = ctx.scan_stats()
    ncount, _ = ctx.neighbours(cap=0)
    status = ctx.status(reset=True)
    assert status["ok"], status
    H = d["h"].double().cpu().numpy()
    X = {k: d[k].double().cpu().numpy() for k in ("x", "y", "z")}
    host = [0, 0, 0]
    off = np.concatenate([[0], np.cumsum(counts)])
    for b in range(len(counts)):
        sl = slice(int(off[b]), int(off[b + 1]))
        for k, v in enumerate(host_counts(X["x"][sl], X["y"][sl], X["z"][sl], H[sl])):
            host[k] += v
    ctx.close()
    return st, host, ncount


def _cat(parts):
    id0 = 0
    for b in parts:
        b.id += id0
        id0 += b.N
    cat = {k: np.concatenate([getattr(b, k) for b in parts]) for k in I.FIELDS + ("id",)}
    return I.Particles(*(cat[k] for k in I.FIELDS + ("id",)),
                       counts=np.array([b.N for b in parts], dtype=np.int64))


@pytest.mark.parametrize("prec", [0, 1])
def test_lattice_counts_are_exact(prec):
    import paper_1712_01294_gb300 as m
    p = I.turbulence(12, seed=3, jitter=0.0, sigma_lnrho=0.0)
    st, host, ncount = stats_case(m, p, prec)
    assert st["candidates"] == host[0]
    assert st["within_cache_radius"] == host[1]
    assert st["neighbours"] == host[2]
    assert st["neighbours"] == int(ncount.sum())
    print(prec, st, "candidates per neighbour", round(st["candidates"] / st["neighbours"], 2))


@pytest.mark.parametrize("prec", [0, 1])
def test_jittered_batched_counts_match_the_host_scan(prec):
    import paper_1712_01294_gb300 as m
    p = _cat([I.turbulence(n, seed=s) for n, s in ((9, 1), (12, 2), (14, 3))])
    st, host, ncount = stats_case(m, p, prec)
    # the cell tests and distances of the host are FP64: a borderline cell or
    # pair may fall the other way in FP32
    tol = 0 if prec == 0 else 2e-4
    assert abs(st["candidates"] - host[0]) <= tol * host[0]
    assert abs(st["within_cache_radius"] - host[1]) <= tol * host[1]
    assert abs(st["neighbours"] - host[2]) <= tol * host[2]
    assert st["neighbours"] == int(ncount.sum())
    assert st["candidates"] > st["within_cache_radius"] > st["neighbours"] > 0


def test_scan_stats_refuses_before_a_density_pass():
    import paper_1712_01294_gb300 as m
    q = cast_state(I.turbulence(8, seed=1), 1)
    ctx = m.Context([q.N], m.default_params())
    with pytest.raises(m.GZError):
        ctx.scan_stats()
    ctx.close()
