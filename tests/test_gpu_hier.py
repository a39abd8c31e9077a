"""Hierarchical (power-of-two) timesteps on the CUDA path (gz_step_hier)
against gz_step and the FP64 oracle: K = 0 and a one-bin interval reproduce
gz_step bitwise; with mixed bins the FP64 path follows the oracle's interval
(same bins, same number of active particle-substeps, fields within 1e-9 of
their RMS) and the FP32 path within its tolerance; momentum and energy are
conserved; repeated runs are bitwise equal."""
import numpy as np
import pytest

import oracle as O
from paper_1712_01294_gb300 import inputs as I

from gpu_common import cast_state, device, field_err, min_image, ostate

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h")


def gz():
    import paper_1712_01294_gb300 as m
    return m


def make(kind, n):
    return {"turb": lambda k: I.turbulence(k, seed=6), "sedov": I.sedov}[kind](n)


def ctx_for(counts, prec, **kw):
    m = gz()
    return m.Context(counts if isinstance(counts, list) else [counts],
                     m.default_params(precision=prec, **kw))


def snap(d):
    return {k: d[k].cpu().numpy().copy() for k in FIELDS}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kind,n", [("turb", 18), ("sedov", 17)])
def test_k0_equals_gz_step_bitwise(kind, n, prec):
    import torch
    q = cast_state(make(kind, n), prec)
    a = device(q, prec)
    ctx = ctx_for(q.N, prec)
    dta = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.step(a, 0.0, dta)
    b = device(q, prec)
    ctx2 = ctx_for(q.N, prec)
    dtb = torch.zeros(1, dtype=torch.float64, device="cuda")
    bins = torch.full((q.N,), -1, dtype=torch.int32, device="cuda")
    na = ctx2.step_hier(b, 0, 0.0, dtb, bins)
    assert ctx.status(reset=True)["ok"] and ctx2.status(reset=True)["ok"]
    assert na == q.N and int(bins.abs().sum()) == 0
    assert float(dta.item()) == float(dtb.item())
    sa, sb = snap(a), snap(b)
    for k in FIELDS:
        assert np.array_equal(sa[k], sb[k]), k


@pytest.mark.parametrize("prec", [0, 1])
def test_one_bin_interval_is_one_fixed_step_bitwise(prec):
    import torch
    q = cast_state(make("turb", 16), prec)
    ctx = ctx_for(q.N, prec)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    probe = device(q, prec)
    ctx.step(probe, 0.0, dt)
    D = 0.5 * float(dt.item())  # within every particle's criterion: all in bin 0
    a = device(q, prec)
    ctx.step(a, D)
    b = device(q, prec)
    na = ctx.step_hier(b, 3, D)
    assert ctx.status(reset=True)["ok"]
    assert na == q.N
    sa, sb = snap(a), snap(b)
    for k in FIELDS:
        assert np.array_equal(sa[k], sb[k]), k


@pytest.mark.parametrize("kind,n,K,fixed", [("turb", 14, 2, 0.0), ("sedov", 15, 4, 0.0),
                                            ("turb", 13, 3, 0.02)])
def test_fp64_interval_follows_the_oracle(kind, n, K, fixed):
    """fixed > 0: the interval is given (0.02 is about four CFL steps of this
    box, so its particles spread over the deeper bins)."""
    import torch
    m = gz()
    q = cast_state(make(kind, n), m.GZ_FP64)
    s = ostate(q)
    o, D_o, bins_o, na_o = O.step_hier(s, O.params(), K, dt=fixed)
    assert len(np.unique(bins_o)) > 1
    ctx = ctx_for(q.N, m.GZ_FP64)
    d = device(q, m.GZ_FP64)
    D = torch.zeros(1, dtype=torch.float64, device="cuda")
    bins = torch.zeros(q.N, dtype=torch.int32, device="cuda")
    na = ctx.step_hier(d, K, fixed, D, bins)
    st = ctx.status(reset=True)
    assert st["ok"], st
    assert abs(float(D.item()) - D_o) <= 1e-12 * D_o
    assert np.array_equal(bins.cpu().numpy(), bins_o)
    assert na == na_o
    for k in ("x", "y", "z"):
        before = getattr(s, k)
        mx, _ = field_err(min_image(d[k].cpu().numpy() - before), min_image(getattr(o, k) - before))
        assert mx <= 1e-9, (k, mx)
    for k in ("vx", "vy", "vz", "u"):
        mx, _ = field_err(d[k].cpu().numpy() - getattr(s, k), getattr(o, k) - getattr(s, k))
        assert mx <= 1e-9, (k, mx)
    assert np.max(np.abs(d["h"].cpu().numpy() - o.H) / o.H) <= 1e-12


@pytest.mark.parametrize("riemann", [1, 2])
def test_fp64_interval_with_the_exact_riemann_options_follows_the_oracle(riemann):
    import torch
    m = gz()
    q = cast_state(I.sod(12, rho_l=1.0, p_l=0.4, rho_r=1.0, p_r=0.4, u_l=-2.0, u_r=2.0), m.GZ_FP64)
    s = ostate(q)
    o, D_o, bins_o, na_o = O.step_hier(s, O.params(riemann=riemann), 2)
    ctx = ctx_for(q.N, m.GZ_FP64, riemann=riemann)
    d = device(q, m.GZ_FP64)
    D = torch.zeros(1, dtype=torch.float64, device="cuda")
    bins = torch.zeros(q.N, dtype=torch.int32, device="cuda")
    na = ctx.step_hier(d, 2, 0.0, D, bins)
    assert ctx.status(reset=True)["ok"]
    assert abs(float(D.item()) - D_o) <= 1e-12 * D_o and na == na_o
    assert np.array_equal(bins.cpu().numpy(), bins_o)
    for k in ("vx", "vy", "vz", "u"):
        mx, _ = field_err(d[k].cpu().numpy() - getattr(s, k), getattr(o, k) - getattr(s, k))
        assert mx <= 1e-9, (k, mx)


def test_fp32_interval_within_tolerance_of_the_oracle():
    import torch
    m = gz()
    q = cast_state(make("sedov", 15), m.GZ_MIXED32)
    s = ostate(q)
    o, D_o, bins_o, _ = O.step_hier(s, O.params(), 3)
    ctx = ctx_for(q.N, m.GZ_MIXED32)
    d = device(q, m.GZ_MIXED32)
    D = torch.zeros(1, dtype=torch.float64, device="cuda")
    bins = torch.zeros(q.N, dtype=torch.int32, device="cuda")
    ctx.step_hier(d, 3, 0.0, D, bins)
    assert ctx.status(reset=True)["ok"]
    assert abs(float(D.item()) - D_o) <= 1e-5 * D_o
    # a bin is an integer decided in the path's precision: FP32 criteria can
    # land on the other side of a power-of-two boundary
    assert np.mean(bins.cpu().numpy() == bins_o) >= 0.99
    for k in ("vx", "vy", "vz", "u"):
        _, rm = field_err(d[k].cpu().numpy().astype(np.float64) - getattr(s, k), getattr(o, k) - getattr(s, k))
        assert rm <= 2e-3, (k, rm)


@pytest.mark.parametrize("prec", [0, 1])
def test_interval_conserves_momentum_and_energy(prec):
    import torch
    q = cast_state(make("sedov", 16), prec)
    ctx = ctx_for(q.N, prec)
    d = device(q, prec)

    def totals():
        m_ = d["m"].double()
        v = [d[k].double() for k in ("vx", "vy", "vz")]
        P = torch.stack([(m_ * x).sum() for x in v]).cpu().numpy()
        E = float((m_ * (d["u"].double() + 0.5 * sum(x * x for x in v))).sum())
        return P, E

    P0, E0 = totals()
    bins = torch.zeros(q.N, dtype=torch.int32, device="cuda")
    ctx.step_hier(d, 4, 0.0, None, bins)
    assert ctx.status(reset=True)["ok"]
    assert len(torch.unique(bins)) > 1
    P1, E1 = totals()
    scale = float((d["m"].double() * d["u"].double().sqrt()).sum())
    tol = 1e-12 if prec == 0 else 1e-5
    assert np.all(np.abs(P1 - P0) <= tol * scale), P1 - P0
    assert abs(E1 - E0) <= tol * E0


def test_interval_is_deterministic_and_refuses_bad_arguments():
    m = gz()
    q = cast_state(make("sedov", 14), m.GZ_MIXED32)
    outs = []
    for _ in range(2):
        ctx = ctx_for(q.N, m.GZ_MIXED32)
        d = device(q, m.GZ_MIXED32)
        ctx.step_hier(d, 3)
        ctx.step_hier(d, 3)
        outs.append(snap(d))
    for k in FIELDS:
        assert np.array_equal(outs[0][k], outs[1][k]), k
    with pytest.raises(m.GZError):
        ctx.step_hier(d, 21)


def test_batched_boxes_equal_single_boxes():
    import torch
    m = gz()
    boxes = [I.sedov(11, seed=6), I.turbulence(10, seed=7), I.sod(9, seed=5)]
    qs = [cast_state(b, 1) for b in boxes]
    off = 0
    for qb in qs:
        qb.id = qb.id + off
        off += qb.N
    singles = []
    for qb in qs:
        ctx = ctx_for(qb.N, 1)
        d = device(qb, 1)
        ctx.step_hier(d, 3)
        singles.append(snap(d))
    cat = {k: np.concatenate([getattr(qb, k) for qb in qs]) for k in
           ("x", "y", "z", "vx", "vy", "vz", "m", "u", "H", "id")}
    d = {k: torch.as_tensor(v, dtype=torch.float32).cuda() for k, v in cat.items() if k not in ("H", "id")}
    d["h"] = torch.as_tensor(cat["H"], dtype=torch.float32).cuda()
    d["id"] = torch.as_tensor(cat["id"], dtype=torch.int64).cuda()
    ctx = ctx_for([qb.N for qb in qs], 1)
    ctx.step_hier(d, 3)
    assert ctx.status(reset=True)["ok"]
    off = 0
    for b, qb in enumerate(qs):
        for k in FIELDS:
            assert np.array_equal(d[k].cpu().numpy()[off:off + qb.N], singles[b][k]), (b, k)
        off += qb.N


@pytest.mark.parametrize("scheme", [0, 1])
def test_lone_particle_box_beside_a_normal_box_without_fault(scheme):
    """A one-particle box (no neighbours: the h-iteration cannot converge, no
    flux pair, an infinite criterion) batched with a normal box: the flags
    are reported and the normal box steps as it does alone."""
    import torch
    m = gz()
    q = cast_state(I.turbulence(10, seed=12), m.GZ_MIXED32)
    lone = {k: torch.full((1,), v, dtype=torch.float32, device="cuda") for k, v in
            (("x", 0.5), ("y", 0.5), ("z", 0.5), ("vx", 0.0), ("vy", 0.0), ("vz", 0.0), ("m", 1.0),
             ("u", 1.0), ("h", 0.1))}
    alone = device(q, m.GZ_MIXED32)
    ctx1 = ctx_for(q.N, m.GZ_MIXED32, scheme=scheme, max_iter=20)
    if scheme == 0:
        ctx1.step_hier(alone, 2)
    else:
        ctx1.step(alone)
    assert ctx1.status(reset=True)["ok"]
    d = device(q, m.GZ_MIXED32)
    both = {k: torch.cat([d[k], lone[k]]) for k in lone}
    both["id"] = torch.cat([d["id"], torch.tensor([10 ** 6], dtype=torch.int64, device="cuda")])
    ctx = ctx_for([q.N, 1], m.GZ_MIXED32, scheme=scheme, max_iter=20)
    if scheme == 0:
        ctx.step_hier(both, 2)
    else:
        ctx.step(both)
    st = ctx.status(reset=True)
    assert "hconv" in st["bits"]
    for k in ("x", "vx", "u", "h"):
        assert torch.equal(both[k][:q.N], alone[k]), k


@pytest.mark.parametrize("prec", [0, 1])
def test_mfv_k0_equals_gz_step_bitwise(prec):
    import torch
    m = gz()
    q = cast_state(make("turb", 14), prec)
    a = device(q, prec)
    ctx = ctx_for(q.N, prec, scheme=m.GZ_MFV)
    ctx.step(a)
    b = device(q, prec)
    ctx2 = ctx_for(q.N, prec, scheme=m.GZ_MFV)
    ctx2.step_hier(b, 0)
    assert ctx.status(reset=True)["ok"] and ctx2.status(reset=True)["ok"]
    for k in FIELDS + ("m",):
        assert torch.equal(a[k], b[k]), k


def test_mfv_fp64_interval_follows_the_oracle_and_conserves_mass():
    import torch
    m = gz()
    q = cast_state(make("sedov", 13), m.GZ_FP64)
    s = ostate(q)
    o, D_o, bins_o, na_o = O.step_hier(s, O.params(scheme=O.MFV), 3)
    assert len(np.unique(bins_o)) > 1
    ctx = ctx_for(q.N, m.GZ_FP64, scheme=m.GZ_MFV)
    d = device(q, m.GZ_FP64)
    D = torch.zeros(1, dtype=torch.float64, device="cuda")
    bins = torch.zeros(q.N, dtype=torch.int32, device="cuda")
    na = ctx.step_hier(d, 3, 0.0, D, bins)
    assert ctx.status(reset=True)["ok"]
    assert abs(float(D.item()) - D_o) <= 1e-12 * D_o and na == na_o
    assert np.array_equal(bins.cpu().numpy(), bins_o)
    for k in ("vx", "vy", "vz", "u", "m"):
        mx, _ = field_err(d[k].cpu().numpy() - getattr(s, k), getattr(o, k) - getattr(s, k))
        assert mx <= 1e-9, (k, mx)
    assert float(d["m"].sum()) == pytest.approx(float(q.m.sum()), rel=1e-13)
