"""Domain decomposition of one periodic box over subdomains.

The GPU form of the domain decomposition in the paper's hybrid MPI + OpenMP
runtime (Sec. 1, Sec. 3): the box is cut into R slabs along x; subdomain r
owns the particles with floor(R x) = r and holds, besides them, ghost copies
of the particles within a halo of width w around its slab.  Each subdomain
is a gz context of its own (gz_create_subdomain: the whole box's cell grid),
one per GPU under torch.distributed, or several on one GPU.  One step:

1. ghosts: each subdomain sends every other one the owned particles within
   w of that one's slab (periodic distance);
2. each subdomain puts owned and ghost particles in ascending id (the
   undivided box's order, so that its cells hold the same particles in the
   same order), marks the owned ones (gz_set_subdomain) and runs the first
   half of the step (gz_step_begin: sort, h-iteration, gradients, the CFL
   step over its owned particles);
3. the box's step is the minimum over the subdomains (a collective);
4. the second half (gz_step_finish: fluxes, update); the owned particles'
   new state is kept, the ghosts' dropped;
5. migration: owned particles whose new x lies in another slab move there.

The halo width is halo_factor times the largest support radius of the box:
the owned particles' fluxes read their partners' gradients (up to one
support radius beyond the slab), which read their neighbours' densities (up
to two), which need those neighbours' full candidate sets (three, and the
h-iteration's 5 % cache margin).  With halo_factor 4 the owned particles'
step equals the undivided box's bit for bit (the u floor excepted, whose
median each subdomain takes over its own particles).

Nothing here computes the method: selection, concatenation, ordering and the
exchange move data; every pass of the step runs in the CUDA library.
"""
from __future__ import annotations

import math

import torch

FLOATS = ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h")


# ------------------------------------------------------------------ slabs
def owner(x: torch.Tensor, nsub: int) -> torch.Tensor:
    """Subdomain of each position: floor(nsub x), clipped to [0, nsub)."""
    return torch.clamp((x * nsub).floor().to(torch.int64), 0, nsub - 1)


def slab_distance(x: torch.Tensor, q: int, nsub: int) -> torch.Tensor:
    """Periodic distance from each position to slab q, [q/nsub, (q+1)/nsub)."""
    half = 0.5 / nsub
    d = x.double() - (q + 0.5) / nsub
    d = d - torch.floor(d + 0.5)  # minimum image
    return torch.clamp(d.abs() - half, min=0.0)


def take(parts: dict, idx: torch.Tensor) -> dict:
    """The particles idx of a particle set (a new set)."""
    return {k: v[idx].contiguous() for k, v in parts.items()}


def concat(sets: list) -> dict:
    """The sets one after another (the first set itself when all are empty)."""
    full = [s for s in sets if s["id"].numel()]
    if not full:
        return sets[0]
    return {k: torch.cat([s[k] for s in full]).contiguous() for k in full[0]}


def by_id(parts: dict) -> dict:
    """The set in ascending id."""
    return take(parts, torch.argsort(parts["id"], stable=True))


# ------------------------------------------------------------ communicators
class LocalComm:
    """Every subdomain in this process (a split on one GPU, or several GPUs
    driven from one process): exchanges pass tensors between dictionaries."""

    def __init__(self, size: int):
        self.size = size

    def local_ranks(self):
        return list(range(self.size))

    def alltoall(self, outbox: dict, fdtype=None, device=None) -> dict:
        """outbox[src][dst] = particle set; returns inbox[dst][src]."""
        inbox = {r: {} for r in range(self.size)}
        for src, msgs in outbox.items():
            for dst, parts in msgs.items():
                inbox[dst][src] = parts
        return inbox

    def allreduce(self, values: dict, op: str) -> dict:
        """Element-wise min or max of the ranks' tensors, given to every rank."""
        it = iter(values.values())
        acc = next(it).clone()
        for v in it:
            acc = torch.minimum(acc, v) if op == "min" else torch.maximum(acc, v)
        return {r: acc for r in values}


class DistComm:
    """One subdomain per process over torch.distributed: NCCL moves CUDA
    tensors, gloo CPU tensors (the sets are moved to the host around the
    exchange)."""

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist
        self.rank = dist.get_rank()
        self.size = dist.get_world_size()
        self.host = dist.get_backend() == "gloo"

    def local_ranks(self):
        return [self.rank]

    def _wire(self, t):
        return t.cpu() if self.host else t

    def alltoall(self, outbox: dict, fdtype=torch.float32, device=None) -> dict:
        """outbox[rank][dst] = particle set (fdtype floats on device); returns
        {rank: {src: set}}."""
        dist = self.dist
        mine = outbox[self.rank]
        dev = torch.device(device) if device is not None else torch.device("cpu")
        wdev = torch.device("cpu") if self.host else dev
        counts = torch.zeros(self.size, dtype=torch.int64)
        for dst, parts in mine.items():
            counts[dst] = parts["id"].numel()
        table = [torch.zeros(self.size, dtype=torch.int64, device=wdev) for _ in range(self.size)]
        dist.all_gather(table, counts.to(wdev))
        table = [t.cpu() for t in table]
        ops, recv = [], {}
        for src in range(self.size):
            n = int(table[src][self.rank])
            if src == self.rank or n == 0:
                continue
            fb = torch.empty((len(FLOATS), n), dtype=fdtype, device=wdev)
            ib = torch.empty(n, dtype=torch.int64, device=wdev)
            recv[src] = (fb, ib)
            ops += [dist.P2POp(dist.irecv, fb, src), dist.P2POp(dist.irecv, ib, src)]
        for dst, parts in mine.items():
            if dst == self.rank or parts["id"].numel() == 0:
                continue
            fb = self._wire(torch.stack([parts[k] for k in FLOATS]).contiguous())
            ib = self._wire(parts["id"].contiguous())
            ops += [dist.P2POp(dist.isend, fb, dst), dist.P2POp(dist.isend, ib, dst)]
        if ops:  # one group of point-to-point operations (NCCL runs them together)
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        inbox = {}
        for src, (fb, ib) in recv.items():
            fb, ib = fb.to(dev), ib.to(dev)
            inbox[src] = {k: fb[j].contiguous() for j, k in enumerate(FLOATS)} | {"id": ib}
        return {self.rank: inbox}

    def allreduce(self, values: dict, op: str) -> dict:
        dist = self.dist
        t = values[self.rank].clone()
        w = self._wire(t)
        dist.all_reduce(w, op=dist.ReduceOp.MIN if op == "min" else dist.ReduceOp.MAX)
        return {self.rank: w.to(t.device)}


# --------------------------------------------------------------- the box
class DecomposedBox:
    """One periodic box of n_total particles over nsub slab subdomains, of
    which this process drives comm.local_ranks().

    parts: the particle set of the whole box or any superset of the local
    subdomains' particles (dict of tensors x..u, h, id); each local
    subdomain keeps the particles it owns.  make_ctx(capacity, n_total)
    (optional) makes the object that steps a subdomain in place of a gz
    subdomain context (same methods: set_subdomain, step_begin, step_finish,
    capacity, close), for host-side tests of the bookkeeping."""

    def __init__(self, parts: dict, n_total: int, nsub: int, comm, params=None, stream=None,
                 halo_factor: float = 4.0, headroom: float = 1.25, make_ctx=None):
        self.nsub, self.n_total, self.comm = nsub, int(n_total), comm
        self.params, self.stream = params, stream
        self.halo_factor, self.headroom = halo_factor, headroom
        self.make_ctx = make_ctx
        self.fdtype, self.device = parts["x"].dtype, parts["x"].device
        own = owner(parts["x"], nsub)
        self.owned = {r: by_id(take(parts, torch.nonzero(own == r).flatten())) for r in comm.local_ranks()}
        self.ctx = {}
        self.last = {}

    # -- halo and exchange ---------------------------------------------------
    def halo_width(self) -> float:
        hmax = {r: (self.owned[r]["h"].max().double().reshape(1) if self.owned[r]["id"].numel()
                    else torch.zeros(1, dtype=torch.float64, device=self.owned[r]["h"].device))
                for r in self.owned}
        h = float(next(iter(self.comm.allreduce(hmax, "max").values())).item())
        if self.nsub == 1:
            return 0.0  # one subdomain: the whole box, no ghosts
        w = self.halo_factor * h
        if not (w < 0.5 * (1.0 - 1.0 / self.nsub)):
            raise ValueError(f"halo {w:.4f} too wide for {self.nsub} slabs (support radius {h:.4f})")
        return w

    def ghosts_for(self, r: int, w: float) -> dict:
        """The sets subdomain r sends as ghosts to every other subdomain."""
        x = self.owned[r]["x"]
        out = {}
        for q in range(self.nsub):
            if q == r:
                continue
            sel = torch.nonzero(slab_distance(x, q, self.nsub) < w).flatten()
            out[q] = take(self.owned[r], sel)
        return out

    def assemble(self, r: int, ghosts: dict):
        """Owned and ghost particles of subdomain r in ascending id, and the owned flags."""
        own = self.owned[r]
        sets = [own] + [g for g in ghosts.values() if g["id"].numel()]
        flags = [torch.ones(own["id"].numel(), dtype=torch.uint8, device=own["id"].device)]
        flags += [torch.zeros(g["id"].numel(), dtype=torch.uint8, device=own["id"].device)
                  for g in ghosts.values() if g["id"].numel()]
        local = concat(sets)
        fl = torch.cat(flags)
        order = torch.argsort(local["id"], stable=True)
        return take(local, order), fl[order].contiguous()

    # -- the library side ----------------------------------------------------
    def context(self, r: int, n: int):
        import paper_1712_01294_gb300 as gz
        c = self.ctx.get(r)
        if c is None or c.capacity < n:
            if c is not None:
                c.close()
            cap = max(n, int(math.ceil(n * self.headroom)))
            if self.make_ctx is not None:
                c = self.make_ctx(cap, self.n_total)
            else:
                c = gz.Context([cap], self.params, stream=self.stream, grid_count=self.n_total)
            self.ctx[r] = c
        return c

    def step(self, dt_fixed: float = 0.0) -> float:
        """One step of the whole box; returns the step taken."""
        ranks = self.comm.local_ranks()
        w = self.halo_width()
        inbox = self.comm.alltoall({r: self.ghosts_for(r, w) for r in ranks}, self.fdtype, self.device)
        dts, local = {}, {}
        for r in ranks:
            parts, flags = self.assemble(r, inbox[r])
            n, nown = int(parts["id"].numel()), int(self.owned[r]["id"].numel())
            if n == 0:  # nothing in or near this slab: no step, no bound on the box's step
                dts[r] = torch.full((1,), math.inf, dtype=torch.float64, device=self.device)
                local[r] = None
                continue
            ctx = self.context(r, n)
            ctx.set_subdomain(n, nown, flags)
            dts[r] = ctx.step_begin(parts)
            local[r] = (parts, flags)
        if dt_fixed > 0.0:
            dt = {r: torch.full_like(dts[r], dt_fixed) for r in ranks}
        else:
            dt = self.comm.allreduce(dts, "min")
        for r in ranks:
            if local[r] is None:
                continue
            parts, flags = local[r]
            self.ctx[r].step_finish(parts, dt[r])
            self.owned[r] = take(parts, torch.nonzero(flags).flatten())
        self.migrate()
        self.last = {r: float(dt[r][0].item()) for r in ranks}
        return self.last[ranks[0]]

    def migrate(self):
        """Owned particles whose position left the slab go to its new owner."""
        ranks = self.comm.local_ranks()
        outbox, keep = {}, {}
        for r in ranks:
            own = owner(self.owned[r]["x"], self.nsub)
            keep[r] = take(self.owned[r], torch.nonzero(own == r).flatten())
            outbox[r] = {q: take(self.owned[r], torch.nonzero(own == q).flatten())
                         for q in range(self.nsub) if q != r}
        inbox = self.comm.alltoall(outbox, self.fdtype, self.device)
        for r in ranks:
            self.owned[r] = by_id(concat([keep[r]] + list(inbox[r].values())))

    def gather(self) -> dict:
        """The local subdomains' owned particles together, in ascending id."""
        return by_id(concat([self.owned[r] for r in self.comm.local_ranks()]))

    def close(self):
        for c in self.ctx.values():
            c.close()
        self.ctx = {}
