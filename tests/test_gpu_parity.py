"""CUDA path vs the FP64 oracle, pass by pass, through the C ABI.

Each pass gets the same frozen inputs on both sides (for the gradient, step
and flux passes the oracle's own H, n and gradients), so errors do not
compound.  FP64 path: neighbour sets and h-iteration counts bit-exact, every
other output within 1e-10 of the field's RMS.  FP32 (mixed) path: within
2e-5 of each field's RMS, as an RMS error and element by element (an element
may exceed it only by 8 eps32 times the sum of the absolute values of the
terms it adds up: the scale FP32 resolves at that element), neighbour sets
equal except for pairs within the FP32 rounding margin of the support radius.
"""
import numpy as np
import pytest

import oracle as O
from paper_1712_01294_gb300 import inputs as I

from gpu_common import (cast_state, device, field_err, flux_scale, fp32_elementwise, grad_scale,
                        gpu_sets, min_image, ostate, oracle_sets)

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5


def gz():
    import paper_1712_01294_gb300 as m
    return m


def make(kind, n):
    return {"sod": I.sod, "turb": I.turbulence, "sedov": I.sedov, "kh": I.kh}[kind](n)


CASES = [("sod", 23), ("turb", 24), ("sedov", 21)]


def ctx_for(N, precision, **kw):
    m = gz()
    return m.Context([N], m.default_params(precision=precision, **kw))


def assert_status_ok(ctx):
    st = ctx.status(reset=True)
    assert st["ok"], st


# ------------------------------------------------------------------ density
@pytest.mark.parametrize("kind,n", CASES)
def test_density_fp64_bitexact_sets_and_iterations(kind, n):
    m = gz()
    q = cast_state(make(kind, n), m.GZ_FP64)
    s = ostate(q)
    Ho, no, ito, _ = O.density(s, O.params())
    ctx = ctx_for(s.N, m.GZ_FP64)
    d = device(q, m.GZ_FP64)
    n_g, it_g = ctx.density(d)
    assert_status_ok(ctx)
    it_g = it_g.cpu().numpy()
    assert np.array_equal(it_g, ito), np.flatnonzero(it_g != ito)[:10]
    Hg = d["h"].cpu().numpy()
    assert np.max(np.abs(Hg - Ho) / Ho) <= 1e-12
    assert np.max(np.abs(n_g.cpu().numpy() - no) / no) <= 1e-12
    cnt, gs = gpu_sets(ctx)
    os_ = oracle_sets(s, Ho)
    bad = [i for i in range(s.N) if gs[i] != os_[i]]
    assert not bad, bad[:10]


@pytest.mark.parametrize("kind,n", CASES)
def test_density_fp32_within_tolerance(kind, n):
    m = gz()
    q = cast_state(make(kind, n), m.GZ_MIXED32)
    s = ostate(q)
    Ho, no, ito, _ = O.density(s, O.params())
    ctx = ctx_for(s.N, m.GZ_MIXED32)
    d = device(q, m.GZ_MIXED32)
    n_g, it_g = ctx.density(d)
    assert_status_ok(ctx)
    Hg = d["h"].cpu().numpy().astype(np.float64)
    assert field_err(Hg, Ho)[1] <= TOL32
    assert field_err(n_g.cpu().numpy(), no)[1] <= TOL32
    # converged H agrees far better than the tolerance; iteration counts agree
    # except where an FP32 evaluation lands within its rounding of the stop test
    assert np.max(np.abs(Hg - Ho) / Ho) < 2e-6
    dit = it_g.cpu().numpy() - ito
    assert np.mean(dit == 0) > 0.97 and np.max(np.abs(dit)) <= 1, np.bincount(np.abs(dit))
    # neighbour sets: differences only for pairs within FP32 rounding of r = H
    _, gs = gpu_sets(ctx)
    os_ = oracle_sets(s, Ho)
    X = np.stack([s.x, s.y, s.z], 1)
    idx = {int(v): k for k, v in enumerate(s.id)}
    for i in range(s.N):
        for j in gs[i] ^ os_[i]:
            dd = min_image(X[idx[j]] - X[i])
            r = np.sqrt((dd * dd).sum())
            assert abs(r - Ho[i]) / Ho[i] < 5e-6, (i, j, r, Ho[i])


# ---------------------------------------------------------------- gradients
def oracle_frozen(q):
    s = ostate(q)
    p = O.params()
    Ho, no, _, _ = O.density(s, p)
    g = O.gradients(s, Ho, no, p)
    return s, Ho, no, g


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
@pytest.mark.parametrize("kind,n", CASES)
def test_gradients_vs_oracle(kind, n, prec, tol):
    m = gz()
    q = cast_state(make(kind, n), prec)
    s, Ho, no, g = oracle_frozen(q)
    if prec == m.GZ_MIXED32:  # the FP32 path reads H and n rounded to float
        Ho = Ho.astype(np.float32).astype(np.float64)
        no = no.astype(np.float32).astype(np.float64)
        g = O.gradients(s, Ho, no, O.params())
    ctx = ctx_for(s.N, prec)
    d = device(q, prec, H=Ho)
    import torch
    n_d = torch.as_tensor(no, dtype=d["x"].dtype).cuda()
    grad, B = ctx.gradients(d, n_d)
    assert_status_ok(ctx)
    grad = grad.cpu().numpy()
    B = B.cpu().numpy()
    lists = O.neighbours(s, Ho) if prec == m.GZ_MIXED32 else None
    for r in range(15):
        mx, rm = field_err(grad[r], g["grad"][r])
        assert (mx if prec == 0 else rm) <= tol, ("grad", r, mx, rm)
        if prec == m.GZ_MIXED32:  # element-wise, with each element's FP32 scale
            fails, _, _ = fp32_elementwise(grad[r], g["grad"][r], lambda i: grad_scale(
                s, Ho, no, g["B"], g["grad_raw"], g["alpha"], r, i, lists))
            assert not fails, ("grad", r, fails[:5])
    for r in range(6):
        mx, rm = field_err(B[r], g["B"][r])
        assert (mx if prec == 0 else rm) <= tol, ("B", r, mx, rm)
        assert prec == 0 or mx <= tol, ("B", r, mx)


@pytest.mark.parametrize("prec", [0, 1])
def test_timestep_vs_oracle(prec):
    m = gz()
    q = cast_state(I.turbulence(20), prec)
    s, Ho, no, _ = oracle_frozen(q)
    if prec == m.GZ_MIXED32:
        Ho = Ho.astype(np.float32).astype(np.float64)
        no = no.astype(np.float32).astype(np.float64)
    dti_o, dt_o = O.timestep(s, Ho, no, O.params())
    ctx = ctx_for(s.N, prec)
    d = device(q, prec, H=Ho)
    import torch
    dti, dtb = ctx.timestep(d, torch.as_tensor(no, dtype=d["x"].dtype).cuda())
    assert_status_ok(ctx)
    tol = 1e-12 if prec == 0 else 1e-6
    assert np.max(np.abs(dti.cpu().numpy() - dti_o) / dti_o) <= tol
    assert abs(dtb.cpu().numpy()[0] - dt_o) / dt_o <= tol


# ------------------------------------------------------------------- fluxes
@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
@pytest.mark.parametrize("kind,n", CASES)
def test_fluxes_vs_oracle(kind, n, prec, tol):
    m = gz()
    q = cast_state(make(kind, n), prec)
    s, Ho, no, g = oracle_frozen(q)
    grad, B = g["grad"], g["B"]
    if prec == m.GZ_MIXED32:
        Ho = Ho.astype(np.float32).astype(np.float64)
        no = no.astype(np.float32).astype(np.float64)
        grad = grad.astype(np.float32).astype(np.float64)
        B = B.astype(np.float32).astype(np.float64)
    _, dt = O.timestep(s, Ho, no, O.params())
    cnt = O.Counters()
    dp_o, dE_o = O.fluxes(s, Ho, no, grad, B, dt, O.params(), counters=cnt)
    ctx = ctx_for(s.N, prec)
    d = device(q, prec, H=Ho)
    import torch
    T = d["x"].dtype
    dp, dE = ctx.hydro_fluxes(d, torch.as_tensor(no, dtype=T).cuda(),
                              torch.as_tensor(grad, dtype=T).cuda().contiguous(),
                              torch.as_tensor(B, dtype=T).cuda().contiguous(), dt)
    st = ctx.status(reset=True)
    assert st["ok"], st
    if prec == 0:
        assert st["counters"]["fallback"] == cnt.fallback
    dp = dp.cpu().numpy()
    dE = dE.cpu().numpy()
    pairs = O.flux_pairs(s, Ho) if prec == m.GZ_MIXED32 else None
    for r, (a, b) in enumerate(((dp[0], dp_o[0]), (dp[1], dp_o[1]), (dp[2], dp_o[2]), (dE, dE_o))):
        mx, rm = field_err(a, b)
        assert (mx if prec == 0 else rm) <= tol, ("rates", r, mx, rm)
        if prec == m.GZ_MIXED32:  # element-wise, with each element's FP32 scale
            fails, _, _ = fp32_elementwise(a, b, lambda i: flux_scale(s, Ho, no, grad, B, dt, r, i, pairs))
            assert not fails, ("rates", r, fails[:5])


# ------------------------------------------------------------------ step
@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
@pytest.mark.parametrize("kind,n", [("turb", 22), ("sod", 20)])
def test_full_step_vs_oracle(kind, n, prec, tol):
    m = gz()
    q = cast_state(make(kind, n), prec)
    s = ostate(q)
    o, dt_o, n_o, dp_o, dE_o = O.step(s, O.params())
    ctx = ctx_for(s.N, prec)
    d = device(q, prec)
    import torch
    dtu = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.step(d, 0.0, dtu)
    assert_status_ok(ctx)
    dt_g = float(dtu.cpu()[0])
    assert abs(dt_g - dt_o) / dt_o <= (1e-12 if prec == 0 else 1e-6)
    for k in ("x", "y", "z"):
        before = getattr(s, k)
        disp_g = min_image(d[k].cpu().numpy().astype(np.float64) - before)
        disp_o = min_image(getattr(o, k) - before)
        mx, rm = field_err(disp_g, disp_o)
        assert (mx if prec == 0 else rm) <= tol * (1 if prec == 0 else 50), (k, mx, rm)
    for k in ("vx", "vy", "vz", "u"):
        dv_g = d[k].cpu().numpy().astype(np.float64) - getattr(s, k)
        dv_o = getattr(o, k) - getattr(s, k)
        mx, rm = field_err(dv_g, dv_o)
        assert (mx if prec == 0 else rm) <= tol * (1 if prec == 0 else 50), (k, mx, rm)
    Hg = d["h"].cpu().numpy()
    assert np.max(np.abs(Hg - o.H) / o.H) <= (1e-12 if prec == 0 else 2e-6)


# ------------------------------------------------- properties of the path
@pytest.mark.parametrize("prec", [0, 1])
def test_pair_contributions_are_bitwise_opposite(prec):
    """Two-particle boxes: each particle's rates are one pair contribution, so
    they must be exact negatives (pair evaluated in id order)."""
    m = gz()
    import torch
    rng = np.random.default_rng(77)
    T = torch.float64 if prec == 0 else torch.float32
    ctx = ctx_for(2, prec)
    for trial in range(40):
        x = rng.uniform(0, 1, (3, 2))
        x[:, 1] = (x[:, 0] + rng.uniform(-0.2, 0.2, 3)) % 1.0
        ids = rng.permutation(2) + int(rng.integers(0, 1000))
        d = {k: torch.as_tensor(v, dtype=T).cuda() for k, v in
             (("x", x[0]), ("y", x[1]), ("z", x[2]), ("vx", rng.normal(0, 1, 2)),
              ("vy", rng.normal(0, 1, 2)), ("vz", rng.normal(0, 1, 2)),
              ("m", rng.uniform(0.5, 2, 2)), ("u", rng.uniform(0.5, 2, 2)),
              ("h", rng.uniform(0.25, 0.45, 2)))}
        d["id"] = torch.as_tensor(ids, dtype=torch.int64).cuda()
        n = torch.as_tensor(rng.uniform(5, 10, 2), dtype=T).cuda()
        grad = torch.as_tensor(rng.normal(0, 0.5, (15, 2)), dtype=T).cuda().contiguous()
        Bm = np.zeros((6, 2))
        Bm[0] = Bm[3] = Bm[5] = rng.uniform(10, 20, 2)
        Bm[1] = rng.uniform(-2, 2, 2)
        B = torch.as_tensor(Bm, dtype=T).cuda().contiguous()
        dp, dE = ctx.hydro_fluxes(d, n, grad, B, float(rng.uniform(0, 0.01)))
        dp = dp.cpu().numpy()
        dE = dE.cpu().numpy()
        assert np.array_equal(dp[:, 0], -dp[:, 1]), (trial, dp)
        assert dE[0] == -dE[1], (trial, dE)
    ctx.status(reset=True)


@pytest.mark.parametrize("prec", [0, 1])
def test_step_is_deterministic(prec):
    m = gz()
    q = cast_state(I.turbulence(18), prec)
    outs = []
    for _ in range(2):
        ctx = ctx_for(q.N, prec)
        d = device(q, prec)
        ctx.step(d)
        ctx.step(d)
        outs.append({k: v.cpu().numpy() for k, v in d.items()})
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_boxes_equal_single_boxes(prec):
    """A multi-box context gives every box exactly the result of its own context."""
    m = gz()
    import torch
    boxes = [I.sod(9, seed=5), I.sedov(11, seed=6), I.turbulence(10, seed=7)]
    qs = [cast_state(b, prec) for b in boxes]
    off = 0
    for qb in qs:
        qb.id = qb.id + off
        off += qb.N
    singles = []
    for qb in qs:
        ctx = ctx_for(qb.N, prec)
        d = device(qb, prec)
        ctx.step(d)
        singles.append({k: v.cpu().numpy() for k, v in d.items()})
    cat = {k: np.concatenate([getattr(qb, k) for qb in qs]) for k in
           ("x", "y", "z", "vx", "vy", "vz", "m", "u", "H", "id")}
    T = torch.float64 if prec == 0 else torch.float32
    d = {k: torch.as_tensor(v, dtype=T).cuda() for k, v in cat.items() if k not in ("H", "id")}
    d["h"] = torch.as_tensor(cat["H"], dtype=T).cuda()
    d["id"] = torch.as_tensor(cat["id"], dtype=torch.int64).cuda()
    ctx = m.Context([qb.N for qb in qs], m.default_params(precision=prec))
    ctx.step(d)
    assert_status_ok(ctx)
    off = 0
    for b, qb in enumerate(qs):
        for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h"):
            got = d[k].cpu().numpy()[off:off + qb.N]
            assert np.array_equal(got, singles[b][k]), (b, k)
        off += qb.N


def test_status_reports_hconv_like_the_oracle():
    m = gz()
    q = cast_state(I.sod(12), m.GZ_FP64)
    s = ostate(q)
    cnt = O.Counters()
    O.density(s, O.params(max_iter=2), counters=cnt)
    ctx = ctx_for(s.N, m.GZ_FP64, max_iter=2)
    d = device(q, m.GZ_FP64)
    ctx.density(d)
    st = ctx.status(reset=True)
    assert not st["ok"] and "hconv" in st["bits"]
    assert st["counters"]["hconv"] == cnt.hconv > 0
    assert st["first_bad_id"] >= 0


def test_single_particle_box_flags_nonconvergence_without_fault():
    m = gz()
    import torch
    ctx = ctx_for(1, m.GZ_MIXED32, max_iter=20)
    d = {k: torch.full((1,), v, dtype=torch.float32, device="cuda") for k, v in
         (("x", 0.5), ("y", 0.5), ("z", 0.5), ("vx", 0.0), ("vy", 0.0), ("vz", 0.0),
          ("m", 1.0), ("u", 1.0), ("h", 0.1))}
    d["id"] = torch.zeros(1, dtype=torch.int64, device="cuda")
    ctx.density(d)
    st = ctx.status(reset=True)
    assert "hconv" in st["bits"]
    assert 0.0 < float(d["h"].cpu()[0]) < 0.5


def test_density_reads_only_positions_h_and_ids():
    m = gz()
    q = cast_state(I.sod(10), m.GZ_MIXED32)
    d = device(q, m.GZ_MIXED32)
    ref = {k: v.clone() for k, v in d.items()}
    ctx = ctx_for(q.N, m.GZ_MIXED32)
    n1, it1 = ctx.density(ref)
    for k in ("vx", "vy", "vz", "m", "u"):
        d[k] = None
    n2, it2 = ctx.density(d)
    assert_status_ok(ctx)
    import torch
    assert torch.equal(n1, n2) and torch.equal(it1, it2) and torch.equal(ref["h"], d["h"])


@pytest.mark.parametrize("prec", [0, 1])
def test_planar_particles_make_E_singular_as_in_the_oracle(prec):
    """The method's degenerate case: every particle on the plane z = 1/2, so
    no E_i has a z-extent.  Given H and n, the gradient pass flags every
    particle singular (status bit and counter) and returns B = 0 and zero
    gradients, as the oracle does for the same inputs."""
    m = gz()
    import torch
    p = I.sod(8)
    p.z[:] = 0.5
    p.x = (p.x * 4) % 1.0
    q = cast_state(p, prec)
    s = ostate(q)
    H = np.full(q.N, 0.2)
    n = np.full(q.N, float(q.N))
    cnt = O.Counters()
    ref = O.gradients(s, H, n, O.params(), counters=cnt)
    assert cnt.singular == q.N
    ctx = ctx_for(q.N, prec)
    d = device(q, prec, H=H)
    T = d["x"].dtype
    grad, B = ctx.gradients(d, torch.as_tensor(n, dtype=T).cuda())
    st = ctx.status(reset=True)
    assert "singular" in st["bits"] and st["counters"]["singular"] == q.N
    assert bool((B == 0).all()) and bool((grad == 0).all())
    assert np.all(ref["B"] == 0.0) and np.all(ref["grad"] == 0.0)


def test_invalid_positions_are_flagged():
    m = gz()
    q = cast_state(I.sod(8), m.GZ_MIXED32)
    d = device(q, m.GZ_MIXED32)
    d["x"][3] = 1.5
    d["y"][7] = float("nan")
    ctx = ctx_for(q.N, m.GZ_MIXED32)
    ctx.density(d)
    st = ctx.status(reset=True)
    assert "nonfinite" in st["bits"]
    assert st["first_bad_id"] == 3


@pytest.mark.parametrize("prec", [0, 1])
def test_density_with_wide_supports_matches_the_oracle(prec):
    """Half the box thinned to one particle in 27 (supports of up to 2.6 cells
    there, 156 candidates within 1.05 H against the density pass's 48-entry
    cache near the dense half): those particles go to the warp-per-particle
    kernel (both of its ways of sharing a scan: candidate by candidate, and
    cell by cell for ranges of 64 cells or more).  FP64: neighbour sets and
    iteration counts bit-exact; FP32: H within 2e-6."""
    import torch
    m = gz()
    p = I.turbulence(24, seed=21)
    rng = np.random.default_rng(5)
    keep = (p.x >= 0.5) | (rng.uniform(size=p.x.size) < 1 / 27)
    for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u", "H", "id"):
        setattr(p, k, getattr(p, k)[keep])
    p.id = np.arange(p.x.size, dtype=np.int64)
    q = cast_state(p, prec)
    s = ostate(q)
    Ho, no, ito, _ = O.density(s, O.params())
    off, _ = O.neighbours(s, 1.05 * Ho)
    assert np.diff(off).max() > 48  # candidates beyond the cache: the warp kernel's particles
    ctx = ctx_for(s.N, prec, max_ngb=256)  # (up to ~150 neighbours near the interface)
    d = device(q, prec)
    n_g, it_g = ctx.density(d)
    assert_status_ok(ctx)
    cnt, gs = gpu_sets(ctx, 256)
    Hg = d["h"].cpu().numpy().astype(np.float64)
    if prec == 0:
        assert np.array_equal(it_g.cpu().numpy(), ito)
        assert np.max(np.abs(Hg - Ho) / Ho) <= 1e-12
        os_ = oracle_sets(s, Ho)
        bad = [i for i in range(s.N) if gs[i] != os_[i]]
        assert not bad, bad[:10]
    else:
        assert np.max(np.abs(Hg - Ho) / Ho) <= 2e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_plain_and_checkpointing_steps_are_bitwise_equal(prec):
    """A plain step's gradient pass skips the adjoint's bookkeeping (which
    particles the limiter's bounds came from); the step's results must not
    change: the same state bit for bit as the checkpointing step's."""
    import torch
    m = gz()
    q = cast_state(I.sedov(20, seed=9), prec)
    out = []
    for ck in (False, True):
        ctx = ctx_for(q.N, prec)
        d = device(q, prec)
        buf = ctx.new_checkpoint(m.GZ_CKPT_GRADIENTS) if ck else None
        for _ in range(3):
            ctx.step(d, 0.0, None, buf, m.GZ_CKPT_GRADIENTS) if ck else ctx.step(d)
        assert_status_ok(ctx)
        out.append({k: d[k].clone() for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h")})
        ctx.close()
    for k in out[0]:
        assert torch.equal(out[0][k], out[1][k]), k
