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


# --------------------------------------------- FP32 tolerance, element-wise
# The FP32 path's tolerance read element by element:
#     |gpu_i - oracle_i| <= 2e-5 RMS(oracle) + K32 eps32 S_i,
# with S_i the scale an FP32 evaluation of element i can resolve: the sum of
# the absolute values of the terms it adds up (plus, for a limited gradient,
# the amplification of rounding through the limiter factor).  An element the
# size of the field's RMS needs only the first term; the second matters for
# elements many times the RMS (a blast centre) or whose terms cancel.  S_i is
# computed for the elements beyond the first term only.
EPS32 = 2.0 ** -24
K32 = 8.0
GAMMA = 5.0 / 3.0


def _prims(s, n):
    rho = s.m * n
    return [rho, s.vx, s.vy, s.vz, (GAMMA - 1.0) * rho * s.u]


def grad_scale(s, H, n, B, graw, alpha, row, i, lists):
    """S_i of limited-gradient row `row` (field row // 3, axis row % 3) at i:
    sum_b |B_ab| sum_j psi_j |W_j - W_i| |d_jb| over N_i, plus, when the
    limiter acts, |g_raw| (|f_ext| + |f_i|) / |f_ext - f_i| over the extremes."""
    off, nb = lists
    q, a = row // 3, row % 3
    W = _prims(s, n)[q]
    js = nb[off[i]:off[i + 1]]
    dd = np.stack([min_image(s.x[js] - s.x[i]), min_image(s.y[js] - s.y[i]),
                   min_image(s.z[js] - s.z[i])], 1)
    r = np.sqrt((dd ** 2).sum(1))
    psi = np.array([O.W(float(v), float(H[i])) for v in r]) / n[i]
    Bm = np.array([[B[0, i], B[1, i], B[2, i]], [B[1, i], B[3, i], B[4, i]], [B[2, i], B[4, i], B[5, i]]])
    S = float(np.abs(Bm[a]) @ (psi[:, None] * np.abs(W[js] - W[i])[:, None] * np.abs(dd)).sum(0))
    if alpha[q, i] < 1.0 and js.size:
        fi = W[i]
        C = 0.0
        for fe in (max(fi, W[js].max()), min(fi, W[js].min())):
            if fe != fi:
                C = max(C, (abs(fe) + abs(fi)) / abs(fe - fi))
        S += abs(graw[row, i]) * C
    return S


def flux_scale(s, H, n, grad, B, dt, comp, i, pairs, p=None):
    """S_i of rate component comp (0-2 momentum, 3 energy) at i: the sum of the
    absolute values of the face contributions of i's flux pairs."""
    off, nb = pairs
    p = p or O.params()
    W = _prims(s, n)

    def side(k):
        return dict(x=np.array([s.x[k], s.y[k], s.z[k]]), H=H[k], n=n[k],
                    W=np.array([w[k] for w in W]), g=grad[:, k], B=B[:, k])
    tot = 0.0
    for j in nb[off[i]:off[i + 1]]:
        L, R = (i, j) if s.id[i] < s.id[j] else (j, i)
        r = O.pair(side(L), side(R), dt, p)
        tot += abs(r["dE"] if comp == 3 else r["dp"][comp])
    return tot


def fp32_elementwise(gpu, ref, scale_of, tol=2e-5):
    """Elements of one field beyond the element-wise FP32 tolerance: returns
    (failures [(i, err/RMS, S_i/RMS)], elements needing the second term,
    largest K needed)."""
    g = np.asarray(gpu, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    R = rms(r) or 1.0
    e = np.abs(g - r)
    beyond = np.flatnonzero(e > tol * R)
    fails, kmax = [], 0.0
    for i in beyond:
        S = scale_of(int(i))
        k = (e[i] - tol * R) / (EPS32 * S) if S > 0 else np.inf
        kmax = max(kmax, k)
        if k > K32:
            fails.append((int(i), e[i] / R, S / R))
    return fails, int(beyond.size), kmax
