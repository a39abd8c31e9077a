"""The domain decomposition on one GPU: the box split into 2 or 3 slab
subdomains, each a gz subdomain context of its own (gz_create_subdomain),
exchanging ghosts and taking the minimum of their steps in one process, and
over two gloo ranks (two processes sharing the GPU; their kernels never wait
on each other, the exchanges go through host memory).
Owned particles must end bitwise where the undivided box's gz_step puts
them, in FP64 and FP32, over several steps with migration between slabs
(the Sod split at x = 1/2 lies on a slab boundary).  The split step
(gz_step_begin + gz_step_finish) must equal gz_step bitwise, and the
subdomain calls must refuse what they do not take (and a subdomain context the
calls laid out for one particle count)."""
import os
import socket

import numpy as np
import pytest

from paper_1712_01294_gb300 import inputs as I

from gpu_common import cast_state, device

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "z", "vx", "vy", "vz", "u", "h")


def undivided(m, q, prec, steps):
    import torch
    ctx = m.Context([q.N], m.default_params(precision=prec))
    d = device(q, prec)
    dtu = torch.zeros(1, dtype=torch.float64, device="cuda")
    dts = []
    for _ in range(steps):
        ctx.step(d, 0.0, dtu)
        dts.append(float(dtu.item()))
    st = ctx.status(reset=True)
    assert st["ok"], st
    ctx.close()
    return d, dts


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kind,n,nsub", [("turb", 40, 2), ("turb", 40, 3), ("sod", 40, 2)])
def test_split_box_equals_undivided_box(kind, n, nsub, prec):
    from paper_1712_01294_gb300 import decomp as D
    import paper_1712_01294_gb300 as m
    make = {"turb": I.turbulence, "sod": I.sod}[kind]
    q = cast_state(make(n), prec)
    steps = 6
    ref, dref = undivided(m, q, prec, steps)
    box = D.DecomposedBox(device(q, prec), q.N, nsub, D.LocalComm(nsub),
                          params=m.default_params(precision=prec))
    dts = [box.step() for _ in range(steps)]
    for c in box.ctx.values():
        st = c.status(reset=True)
        assert st["ok"], st
    assert dts == dref
    got = box.gather()
    assert np.array_equal(got["id"].cpu().numpy(), np.arange(q.N))
    moved = int((D.owner(got["x"], nsub) != D.owner(device(q, prec)["x"], nsub)).sum().item())
    for k in KEYS:
        assert np.array_equal(got[k].cpu().numpy(), ref[k].cpu().numpy()), k
    box.close()
    print(f"{kind} {n}^3 over {nsub} subdomains, prec {prec}: {steps} steps bitwise equal; "
          f"{moved} particles changed slab")


def _gloo_rank(rank, world, port, prec, steps, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_1712_01294_gb300 as m
        from paper_1712_01294_gb300 import decomp as D
        q = cast_state(I.turbulence(40), prec)
        box = D.DecomposedBox(device(q, prec), q.N, world, D.DistComm(),
                              params=m.default_params(precision=prec))
        dts = [box.step() for _ in range(steps)]
        ok = all(c.status(reset=True)["ok"] for c in box.ctx.values())
        got = box.gather()
        out[rank] = ({k: v.cpu().numpy() for k, v in got.items()}, dts, ok)
        box.close()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("prec", [0, 1])
def test_two_gloo_ranks_equal_undivided_box(prec):
    import torch.multiprocessing as mp

    import paper_1712_01294_gb300 as m
    q = cast_state(I.turbulence(40), prec)
    steps, world = 4, 2
    ref, dref = undivided(m, q, prec, steps)
    with mp.Manager() as man:
        out = man.dict()
        ctx = mp.get_context("spawn")
        port = _free_port()
        procs = [ctx.Process(target=_gloo_rank, args=(r, world, port, prec, steps, out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(600)
            assert p.exitcode == 0
        res = dict(out)
    assert set(res) == set(range(world))
    for r in range(world):
        assert res[r][1] == dref  # the same steps on every rank
        assert res[r][2]
    ids = np.concatenate([res[r][0]["id"] for r in range(world)])
    order = np.argsort(ids)
    assert np.array_equal(ids[order], np.arange(q.N))
    for k in KEYS:
        got = np.concatenate([res[r][0][k] for r in range(world)])[order]
        assert np.array_equal(got, ref[k].cpu().numpy()), k


@pytest.mark.parametrize("prec", [0, 1])
def test_split_step_equals_gz_step(prec):
    import torch

    import paper_1712_01294_gb300 as m
    q = cast_state(I.turbulence(24, seed=5), prec)
    ref, _ = undivided(m, q, prec, 3)
    ctx = m.Context([q.N], m.default_params(precision=prec))
    d = device(q, prec)
    for _ in range(3):
        dt = ctx.step_begin(d)
        ctx.step_finish(d, dt)
    assert ctx.status(reset=True)["ok"]
    for k in KEYS:
        assert torch.equal(d[k], ref[k]), k
    ctx.close()


def test_subdomain_calls_refuse_bad_use():
    import torch

    import paper_1712_01294_gb300 as m
    q = cast_state(I.turbulence(12, seed=2), 1)
    ctx = m.Context([q.N], m.default_params())
    with pytest.raises(m.GZError):
        ctx.set_subdomain(q.N, q.N)  # not a subdomain context
    d = device(q, 1)
    with pytest.raises(m.GZError):
        ctx.step_finish(d, torch.zeros(1, dtype=torch.float64, device="cuda"))  # no begin
    ctx.close()
    sub = m.Context([q.N], m.default_params(), grid_count=2 * q.N)
    with pytest.raises(m.GZError):
        sub.set_subdomain(q.N + 1, 1)  # beyond capacity
    with pytest.raises(m.GZError):
        sub.set_subdomain(q.N, q.N + 1)  # more owned than held
    sub.set_subdomain(q.N, q.N)
    d = device(q, 1)
    # calls laid out for one particle count refuse a subdomain context
    with pytest.raises(m.GZError):
        sub.checkpoint_bytes(1)
    with pytest.raises(m.GZError):
        sub.step_hier(d, 1)
    stream = torch.cuda.Stream()
    sub2 = m.Context([q.N], m.default_params(), stream=stream, grid_count=q.N)
    with pytest.raises(m.GZError):
        sub2.graph_capture(d, 1)
    sub2.close()
    sub.step(d)  # the plain step is taken
    assert sub.status(reset=True)["ok"]
    sub.close()
