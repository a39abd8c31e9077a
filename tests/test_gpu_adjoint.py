"""Hand-written CUDA adjoints vs the derivative oracle (torch autograd of the
step written in plain PyTorch CPU ops), through the C ABI.

Inputs are smooth (no exactly uniform field, which would be a kink of the
limiter).  FP64 path: element-wise within 1e-9 of each adjoint field's RMS.
FP32 path: RMS error within 1e-3 of the FP64 oracle's adjoint (reported)."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import torch_step as TS
from paper_1712_01294_gb300 import inputs as I

from gpu_common import cast_state, device, ostate

pytestmark = pytest.mark.gpu

GAM = 5.0 / 3.0


def gz():
    import paper_1712_01294_gb300 as m
    return m


def rms(a):
    a = np.asarray(a, dtype=np.float64)
    return float(np.sqrt(np.mean(a * a)))


FAILS = []


def check(name, got, ref, prec, tol64=1e-9, tol32=1e-3):
    """Records (not asserts) the error of one adjoint field; see assert_all."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = rms(ref) or 1.0
    rel = np.abs(got - ref) / scale
    err = float(rel.max()) if prec == 0 else rms(got - ref) / scale
    if err > (tol64 if prec == 0 else tol32):
        bad = np.flatnonzero(rel > (tol64 if prec == 0 else tol32))
        FAILS.append((name, err, int(bad.size), bad[:5].tolist(), got[bad[:3]].tolist(),
                      ref[bad[:3]].tolist()))
    return err


def assert_all():
    msg = "\n".join(str(f) for f in FAILS)
    FAILS.clear()
    assert not msg, msg


def _vz_zero():
    """Smooth field with vz = 0 exactly: every pair's vz bounds tie (lo = hi =
    0), so the clamp's adjoint must go to one side only (L, as the oracle's
    where() does)."""
    q = I.smooth_turbulence(12, seed=3)
    q.vz[:] = 0.0
    return q


@pytest.mark.parametrize("case", ["smooth", "vz_tied"])
@pytest.mark.parametrize("prec", [0, 1])
def test_flux_adjoint_matches_autograd(prec, case):
    m = gz()
    q = cast_state(I.smooth_turbulence(12, seed=3) if case == "smooth" else _vz_zero(), prec)
    s = ostate(q)
    prm = O.params()
    Ho, no, _, _ = O.density(s, prm)
    g = O.gradients(s, Ho, no, prm)
    grad, B = g["grad"], g["B"]
    if prec == m.GZ_MIXED32:
        Ho, no, grad, B = (a.astype(np.float32).astype(np.float64) for a in (Ho, no, grad, B))
    _, dt = O.timestep(s, Ho, no, prm)
    poff, pnb = O.flux_pairs(s, Ho)
    L, R = TS.canonical_pairs(poff, pnb, s.id)
    rng = np.random.default_rng(5)
    dpbar = rng.normal(size=(3, s.N))
    dEbar = rng.normal(size=s.N)
    # oracle: autograd of the flux stage with every input a leaf
    T = lambda a: torch.tensor(np.asarray(a, dtype=np.float64), requires_grad=True)
    x, y, z = T(s.x), T(s.y), T(s.z)
    rho0 = s.m * no
    if prec == m.GZ_MIXED32:
        rho0 = (s.m.astype(np.float32) * no.astype(np.float32)).astype(np.float64)
        P0 = ((np.float32(GAM - 1.0) * rho0.astype(np.float32)) * s.u.astype(np.float32)).astype(np.float64)
    else:
        P0 = (GAM - 1.0) * rho0 * s.u
    prim = [T(rho0), T(s.vx), T(s.vy), T(s.vz), T(P0)]
    H, n = T(Ho), T(no)
    gl_leaves = [T(grad[k]) for k in range(15)]
    gl = [[gl_leaves[3 * f + k] for k in range(3)] for f in range(5)]
    Bl = [T(B[k]) for k in range(6)]
    dp, dE = TS.flux_stage(x, y, z, prim, H, n, gl, Bl, L, R, dt)
    J = sum((dp[k] * torch.tensor(dpbar[k])).sum() for k in range(3)) + (dE * torch.tensor(dEbar)).sum()
    leaves = [x, y, z] + prim + [H, n] + gl_leaves + Bl
    ref = [t.numpy() for t in torch.autograd.grad(J, leaves, allow_unused=True)]
    # CUDA adjoint
    ctx = m.Context([s.N], m.default_params(precision=prec))
    d = device(q, prec, H=Ho)
    Tt = d["x"].dtype
    out = ctx.hydro_fluxes_backward(d, torch.as_tensor(no, dtype=Tt).cuda(),
                                    torch.as_tensor(grad, dtype=Tt).cuda().contiguous(),
                                    torch.as_tensor(B, dtype=Tt).cuda().contiguous(), dt,
                                    torch.as_tensor(dpbar).cuda().contiguous(),
                                    torch.as_tensor(dEbar).cuda().contiguous())
    st = ctx.status(reset=True)
    assert st["ok"], st
    o = {k: v.cpu().numpy() for k, v in out.items()}
    errs = {}
    for k in range(3):
        errs[f"x{k}"] = check(f"x{k}", o["x"][k], ref[k], prec)
    for f in range(5):
        errs[f"W{f}"] = check(f"W{f}", o["W"][f], ref[3 + f], prec)
    errs["H"] = check("H", o["h"], ref[8], prec)
    errs["n"] = check("n", o["n"], ref[9], prec)
    for q_ in range(15):
        errs[f"g{q_}"] = check(f"g{q_}", o["grad"][q_], ref[10 + q_], prec)
    for q_ in range(6):
        errs[f"B{q_}"] = check(f"B{q_}", o["B"][q_], ref[25 + q_], prec)
    print("flux adjoint errors", prec, {k: f"{v:.2e}" for k, v in errs.items()})
    assert_all()


KEYS = ("x", "y", "z", "vx", "vy", "vz", "m", "u")
OUTK = ("x", "y", "z", "vx", "vy", "vz", "u")


def step_adjoint_case(make, prec, seed=7, tol=None):
    """(oracle gradient dict, CUDA gradient dict) of J = sum <gbar, state_after>
    with respect to the state before one step (dt and neighbour sets frozen)."""
    m = gz()
    q = cast_state(make(), prec)
    prm = O.params(tol=1e-12 if prec == 0 else 1e-6)
    fr, s, Hs, n = TS.freeze(q.__dict__, prm)
    st = TS.as_tensors(s, requires_grad=True)
    out = TS.step(st, fr)
    rng = np.random.default_rng(seed)
    gbar = {k: rng.normal(size=s.N) for k in OUTK}
    J = sum((out[k] * torch.tensor(gbar[k])).sum() for k in OUTK)
    ref = dict(zip(KEYS, (g.numpy() for g in torch.autograd.grad(J, [st[k] for k in KEYS]))))
    ctx = m.Context([s.N], m.default_params(precision=prec, tol=1e-12 if prec == 0 else 1e-6))
    d = device(q, prec)
    T = d["x"].dtype
    gend = {k: torch.as_tensor(gbar[k], dtype=T).cuda().contiguous() for k in OUTK}
    gstart = {k: torch.zeros(s.N, dtype=T, device="cuda") for k in KEYS}
    ctx.step_backward(d, fr.dt, gend, gstart)
    st_ = ctx.status(reset=True)
    assert st_["ok"], st_
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in gstart.items()}
    return ref, got


@pytest.mark.parametrize("prec", [0, 1])
def test_step_adjoint_matches_autograd(prec):
    ref, got = step_adjoint_case(lambda: I.smooth_turbulence(12, seed=3), prec)
    errs = {k: check(k, got[k], ref[k], prec) for k in KEYS}
    print("step adjoint errors", prec, {k: f"{v:.2e}" for k, v in errs.items()})
    assert_all()


@pytest.mark.parametrize("level,ngb", [(0, 32.0), (0, 80.0), (1, 32.0), (1, 80.0), (2, 32.0),
                                       (2, 80.0)])
@pytest.mark.parametrize("prec", [0, 1])
def test_checkpointed_backward_equals_full_recompute(prec, level, ngb):
    """gz_step_backward from a step checkpoint (saved rates, H, n and the
    kernel-derivative sums; at level 1 the gradient pass's outputs; at level
    2 also the sorted order and the neighbour lists' first 64 slots) equals
    the full recompute from the start state bit for bit: the saved values
    are the ones the recomputed passes would produce.  With N_ngb = 80 many
    particles outgrow the density pass's per-thread cache and are finished
    by the warp-per-particle kernel, whose sums a rescan at H would not
    reproduce (hence n and the sums are kept at every level), and most lists
    are longer than the slots kept, and are rebuilt by a scan."""
    m = gz()
    q = cast_state(I.smooth_turbulence(12, seed=5), prec)
    ctx = m.Context([q.N], m.default_params(precision=prec, ngb=ngb))
    start = device(q, prec)
    d = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in start.items()}
    ck = ctx.new_checkpoint(level)
    assert ck.numel() == ctx.checkpoint_bytes(level)
    assert ctx.checkpoint_bytes(2) > ctx.checkpoint_bytes(1) > ctx.checkpoint_bytes(0) >= 32 * q.N
    dtu = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.step(d, 0.0, dtu, ck, level)
    dt = float(dtu.item())
    # the checkpointing step advances the state exactly like gz_step
    d2 = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in start.items()}
    ctx.step(d2, dt)
    for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h"):
        assert torch.equal(d[k], d2[k]), k
    T = d["x"].dtype
    rng = np.random.default_rng(11)
    gend = {k: torch.as_tensor(rng.normal(size=q.N), dtype=T).cuda() for k in OUTK}
    g_full = {k: torch.zeros(q.N, dtype=T, device="cuda") for k in KEYS}
    g_ckpt = {k: torch.zeros(q.N, dtype=T, device="cuda") for k in KEYS}
    ctx.step_backward(start, dt, gend, g_full)
    st = dict(start)
    st["h"] = d["h"].clone()
    ctx.step_backward(st, dt, gend, g_ckpt, ck, level)
    st_ = ctx.status(reset=True)
    assert st_["ok"], st_
    for k in KEYS:
        assert torch.equal(g_full[k], g_ckpt[k]), k
    # saved momentum rates are pairwise antisymmetric: they sum to round-off
    # (FP32 pair terms are summed in FP32 in groups of 8 before the FP64 flush)
    r = ck[:32 * q.N].view(torch.float64).view(4, q.N).cpu().numpy()
    for k in range(3):
        assert abs(r[k].sum()) <= (1e-12 if prec == 0 else 1e-6) * np.abs(r[k]).sum(), k


def _boxes(sizes):
    """Smooth-turbulence boxes of the given sizes, concatenated box by box
    (ids running on across the boxes)."""
    parts, id0 = [], 0
    for n, seed in sizes:
        b = I.smooth_turbulence(n, seed=seed)
        b.id += id0
        id0 += b.N
        parts.append(b)
    cat = {k: np.concatenate([getattr(b, k) for b in parts]) for k in I.FIELDS + ("id",)}
    return I.Particles(*(cat[k] for k in I.FIELDS + ("id",)),
                       counts=np.array([b.N for b in parts], dtype=np.int64)), parts


def _fixed_dt_backward(m, q, counts, prec, dt, gend, level):
    ctx = m.Context(counts, m.default_params(precision=prec))
    start = device(q, prec)
    d = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in start.items()}
    ck = ctx.new_checkpoint(level)
    dtu = torch.zeros(len(counts), dtype=torch.float64, device="cuda")
    ctx.step(d, dt, dtu, ck, level)
    assert bool((dtu == dt).all())
    T = d["x"].dtype
    g = {k: torch.zeros(q.N, dtype=T, device="cuda") for k in KEYS}
    st = dict(start)
    st["h"] = d["h"].clone()
    ctx.step_backward(st, dt, {k: v.to(T) for k, v in gend.items()}, g, ck, level)
    st_ = ctx.status(reset=True)
    assert st_["ok"], st_
    ctx.close()
    return d, g


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_backward_equals_each_box_alone(prec):
    """A batched context of three uneven boxes stepped with one fixed dt: the
    backward from its level-2 checkpoint equals, box by box, the backward of
    a context holding that box alone, bit for bit (each pass treats the boxes
    independently; the sort keeps each box's particles in their own order)."""
    m = gz()
    q, parts = _boxes([(8, 21), (11, 22), (9, 23)])
    counts = [b.N for b in parts]
    q = cast_state(q, prec)
    dt = 2e-3
    rng = np.random.default_rng(17)
    gend = {k: torch.as_tensor(rng.normal(size=q.N), dtype=torch.float64).cuda() for k in OUTK}
    d, g = _fixed_dt_backward(m, q, counts, prec, dt, gend, m.GZ_CKPT_LISTS)
    off = np.concatenate([[0], np.cumsum(counts)])
    for b, pb in enumerate(parts):
        sl = slice(int(off[b]), int(off[b + 1]))
        db, gb = _fixed_dt_backward(m, cast_state(pb, prec), [pb.N], prec, dt,
                                    {k: v[sl] for k, v in gend.items()}, m.GZ_CKPT_LISTS)
        for k in ("x", "vx", "u", "h"):
            assert torch.equal(db[k], d[k][sl]), (b, k)
        for k in KEYS:
            assert torch.equal(gb[k], g[k][sl]), (b, k)


def region_ke(state, mask):
    v2 = state["vx"] ** 2 + state["vy"] ** 2 + state["vz"] ** 2
    return (0.5 * state["m"].to(torch.float64) * v2.to(torch.float64) * mask).sum()


def kh_rollout_grad(prec, n=20, nsteps=3, smooth=0.08, seed=1715):
    """Gradient of the KH loss (kinetic energy of the particles that start at
    y > 0.75) after nsteps, with respect to initial v and u, via MFMStep."""
    m = gz()
    from paper_1712_01294_gb300 import autograd as GA
    q = cast_state(I.kh(n, seed=seed, smooth=smooth), prec)
    ctx = m.Context([q.N], m.default_params(precision=prec, tol=1e-12 if prec == 0 else 1e-6))
    d = device(q, prec)
    for k in ("vx", "vy", "vz", "u"):
        d[k].requires_grad_(True)
    mask = torch.as_tensor(q.y > 0.75, dtype=torch.float64).cuda()
    fin, dts = GA.rollout(ctx, dict(d), nsteps)
    L = region_ke(fin, mask)
    L.backward()
    grads = {k: d[k].grad.detach().cpu().numpy().astype(np.float64) for k in ("vx", "vy", "vz", "u")}
    st_ = ctx.status(reset=True)
    assert st_["ok"], st_
    return q, ctx, mask, dts, float(L), grads


def test_rollout_gradient_matches_central_differences():
    """FP64 path: <dL/d(v0, u0), delta> against central differences of the CUDA
    forward with the same frozen step sequence (spec bar: 1e-4)."""
    q, ctx, mask, dts, L0, grads = kh_rollout_grad(0, n=24, smooth=0.1)
    # along the gradient itself: a random direction nearly cancels, and then
    # the O(eps) jumps of limiter extrema switching in the shear layer dominate
    norm = np.sqrt(sum(float(np.sum(g * g)) for g in grads.values()))
    delta = {k: g / norm for k, g in grads.items()}
    dd = sum(float(np.sum(grads[k] * delta[k])) for k in grads)

    def loss(eps):
        d = device(q, 0)
        for k in delta:
            d[k] = d[k] + eps * torch.as_tensor(delta[k]).cuda()
        for dt in dts:
            ctx.step(d, dt)
        return float(region_ke(d, mask))
    fds = []
    for eps in (1e-4, 1e-5, 1e-6):
        fds.append((loss(eps) - loss(-eps)) / (2 * eps))
    rel = min(abs(fd - dd) / abs(fd) for fd in fds)
    print("rollout FD check", dd, fds, rel)
    assert rel <= 1e-4, (dd, fds)


def test_rollout_fp32_gradient_close_to_fp64():
    _, _, _, _, L64, g64 = kh_rollout_grad(0)
    _, _, _, _, L32, g32 = kh_rollout_grad(1)
    assert abs(L32 - L64) <= 1e-5 * abs(L64)
    for k in g64:
        err = rms(g32[k] - g64[k]) / rms(g64[k])
        print("fp32 vs fp64 rollout gradient", k, err)
        assert err <= 1e-2, (k, err)


def test_rollout_gradient_matches_dual_number_oracle():
    """Two FP64 steps: directional derivative from the PyTorch oracle's dual
    numbers (neighbour sets frozen per step at the oracle's own states)."""
    import torch.autograd.forward_ad as fwAD
    prec, nsteps = 0, 2
    q, ctx, mask, dts, L0, grads = kh_rollout_grad(prec, n=12, nsteps=nsteps, smooth=0.12)
    rng = np.random.default_rng(9)
    delta = {k: rng.normal(size=q.N) for k in grads}
    dd = sum(float(np.sum(grads[k] * delta[k])) for k in grads)
    prm = O.params(tol=1e-12)
    s = ostate(q)
    with fwAD.dual_level():
        st = TS.as_tensors(s)
        st = {k: (fwAD.make_dual(v, torch.as_tensor(delta[k])) if k in delta else v) for k, v in st.items()}
        cur_np = s
        for k_step in range(nsteps):
            fr, _, _, _ = TS.freeze({**cur_np.__dict__}, prm)
            fr.dt = dts[k_step]
            out = TS.step(st, fr)
            out["m"] = st["m"]
            st = out
            vals = {k: fwAD.unpack_dual(v).primal.numpy() for k, v in st.items()}
            cur_np = O.State(vals["x"], vals["y"], vals["z"], vals["vx"], vals["vy"], vals["vz"],
                             vals["m"], vals["u"], fr.Hstar.numpy(), s.id)
        v2 = st["vx"] ** 2 + st["vy"] ** 2 + st["vz"] ** 2
        Lt = (0.5 * st["m"] * v2 * torch.as_tensor(mask.cpu().numpy())).sum()
        dual = fwAD.unpack_dual(Lt).tangent.item()
    print("rollout dual-number check", dd, dual)
    assert abs(dd - dual) <= 1e-9 * abs(dual), (dd, dual)
