"""The domain decomposition's bookkeeping on the CPU (no GPU): slab
ownership, halo selection, the ghost exchange, the minimum of the
subdomains' steps and migration, with a host-side stand-in for the library's
step.  The stand-in gives each particle a new state that depends on its own
data and on the number of particles within three support radii of it (so a
missing ghost changes the result), drifts it, and proposes as its step the
minimum over its owned particles of a per-particle criterion.  Split over
subdomains (in one process, and over two gloo ranks with one subdomain
each) the box must end bitwise where the undivided box ends."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1712_01294_gb300 import decomp as D


class HostStep:
    """Stands in for a gz subdomain context on the host."""

    def __init__(self, capacity, n_total):
        self.capacity = capacity
        self.held = []

    def set_subdomain(self, n, n_owned, owned):
        assert owned.dtype == torch.uint8 and owned.numel() == n and int(owned.sum()) == n_owned
        self.own = owned.bool()

    def step_begin(self, p):
        ids = p["id"]
        assert bool((ids[1:] > ids[:-1]).all())  # ascending id, no duplicates
        self.held.append(ids.clone())
        X = torch.stack([p["x"], p["y"], p["z"]], 1).double()
        d = X[:, None, :] - X[None, :, :]
        d = d - torch.floor(d + 0.5)
        r = d.pow(2).sum(-1).sqrt()
        reach = 3.0 * p["h"].double()[:, None]
        self.count = ((r < reach).sum(1) - 1).to(p["x"].dtype)
        crit = 0.02 / (1.0 + (p["vx"].double() ** 2 + p["vy"].double() ** 2).sqrt())
        c = crit[self.own]
        return (c.min() if c.numel() else torch.tensor(float("inf"), dtype=torch.float64)).reshape(1)

    def step_finish(self, p, dt):
        dtv = dt.to(p["x"].dtype)[0]
        for a, v in (("x", "vx"), ("y", "vy"), ("z", "vz")):
            p[a].copy_(torch.remainder(p[a] + dtv * p[v], 1.0))
        p["u"].copy_(p["u"] + 1e-3 * self.count)
        p["vx"].copy_(p["vx"] * (1.0 + 1e-4 * self.count))

    def close(self):
        pass


def box(n=14, seed=3):
    rng = np.random.default_rng(seed)
    N = n ** 3
    g = (np.arange(n) + 0.5) / n
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    X = np.mod(X + rng.uniform(-0.2, 0.2, X.shape) / n, 1.0)
    p = {"x": X[:, 0], "y": X[:, 1], "z": X[:, 2], "vx": rng.normal(0, 1.0, N),
         "vy": rng.normal(0, 1.0, N), "vz": rng.normal(0, 0.3, N), "m": np.full(N, 1.0 / N),
         "u": np.ones(N), "h": np.full(N, 0.6 / n)}
    p = {k: torch.as_tensor(v, dtype=torch.float64) for k, v in p.items()}
    p["id"] = torch.arange(N, dtype=torch.int64)
    perm = torch.as_tensor(rng.permutation(N))  # storage order is not id order
    return {k: v[perm].contiguous() for k, v in p.items()}, N


def run(parts, N, nsub, comm, steps):
    b = D.DecomposedBox(parts, N, nsub, comm, make_ctx=lambda cap, nt: HostStep(cap, nt))
    dts = [b.step() for _ in range(steps)]
    return b, dts


def test_slab_helpers():
    x = torch.tensor([0.0, 0.2499, 0.25, 0.7, 0.99999, 1.0], dtype=torch.float64)
    assert D.owner(x, 4).tolist() == [0, 0, 1, 2, 3, 3]
    # periodic distance to slab 0 = [0, 1/4)
    d = D.slab_distance(torch.tensor([0.1, 0.3, 0.95, 0.6], dtype=torch.float64), 0, 4)
    assert torch.allclose(d, torch.tensor([0.0, 0.05, 0.05, 0.35], dtype=torch.float64))


def test_three_subdomains_in_one_process_equal_the_undivided_box():
    parts, N = box()
    ref, dref = run(parts, N, 1, D.LocalComm(1), 3)
    got, dgot = run(parts, N, 3, D.LocalComm(3), 3)
    assert dgot == dref
    a, b = ref.gather(), got.gather()
    for k in a:
        assert torch.equal(a[k], b[k]), k
    # one more step: each subdomain holds exactly its owned particles and
    # every other particle within the halo width of its slab
    start = ref.gather()
    w = got.halo_width()
    got.step()
    ref.step()
    for r in range(3):
        near = (D.owner(start["x"], 3) == r) | (D.slab_distance(start["x"], r, 3) < w)
        assert set(got.ctx[r].held[-1].tolist()) == set(start["id"][near].tolist())
    a, b = ref.gather(), got.gather()
    for k in a:
        assert torch.equal(a[k], b[k]), k
    # every particle is owned exactly once, inside its own slab
    for r in range(3):
        assert bool((D.owner(got.owned[r]["x"], 3) == r).all())
    assert sum(got.owned[r]["id"].numel() for r in range(3)) == N


def test_empty_slab_is_skipped():
    # every particle in x < 1/4: with 4 slabs, slab 2 holds none and lies
    # beyond the halo of every particle (slabs 1 and 3 hold ghosts only)
    parts, N = box()
    parts["x"] = parts["x"] * 0.25
    ref, dref = run(parts, N, 1, D.LocalComm(1), 3)
    got, dgot = run(parts, N, 4, D.LocalComm(4), 3)
    assert dgot == dref
    assert 2 not in got.ctx or not got.ctx[2].held  # slab 2 never stepped
    a, b = ref.gather(), got.gather()
    for k in a:
        assert torch.equal(a[k], b[k]), k


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts, N = box()
        b, dts = run(parts, N, world, D.DistComm(), 4)
        mine = b.gather()
        out[rank] = ({k: v.numpy() for k, v in mine.items()}, dts)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2])
def test_gloo_ranks_equal_the_undivided_box(world):
    parts, N = box()
    ref, dref = run(parts, N, 1, D.LocalComm(1), 4)
    a = ref.gather()
    with mp.Manager() as m:
        out = m.dict()
        ctx = mp.get_context("spawn")
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert set(res) == set(range(world))
    for r in range(world):
        assert res[r][1] == dref  # the same steps on every rank
    ids = np.concatenate([res[r][0]["id"] for r in range(world)])
    order = np.argsort(ids)
    assert np.array_equal(ids[order], a["id"].numpy())
    for k in a:
        got = np.concatenate([res[r][0][k] for r in range(world)])[order]
        assert np.array_equal(got, a[k].numpy()), k
