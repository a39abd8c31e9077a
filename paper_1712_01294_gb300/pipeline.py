"""Steps on particle sets that live in host memory, with the copies overlapped.

``pipelined_steps`` runs one ``gz_step`` per host input set (pinned CPU
tensors, one dict per step) and reads each result back into its host output
set.  Two device buffers alternate: while step k runs on the context's
stream, the inputs of step k+1 are copied in and the results of step k-1 are
copied out on a second stream, so at most the first copy-in and the last
copy-out are exposed.  Nothing here computes: the copies are
``cudaMemcpyAsync`` transfers issued by torch, ordering is by CUDA events.
"""
from __future__ import annotations

IN_FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h", "id")
OUT_FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h")


def device_buffers(host, count: int = 2):
    """Device tensors shaped like the host set (one dict per buffer)."""
    import torch
    return [{k: torch.empty(t.shape, dtype=t.dtype, device="cuda") for k, t in host.items()}
            for _ in range(count)]


def pipelined_steps(ctx, host_in, host_out, dt_fixed: float = 0.0, dt_used=None, bufs=None,
                    copy_stream=None):
    """For each k: host_in[k] -> device, gz_step, device -> host_out[k].

    host_in: list of dicts of pinned CPU tensors (fields IN_FIELDS, the dtype of
    the context's precision; id int64).  host_out: list of dicts of pinned CPU
    tensors for OUT_FIELDS (same length).  dt_used (device float64 [nboxes],
    optional) receives the last step's timesteps.  bufs: two device buffer
    dicts from device_buffers (allocated here when None).  Returns after the
    work is enqueued; synchronise (or wait on ctx.stream) before reading
    host_out."""
    import torch
    n = len(host_in)
    if n != len(host_out):
        raise ValueError("host_in and host_out differ in length")
    if n == 0:
        return
    bufs = bufs if bufs is not None else device_buffers(host_in[0])
    cs = copy_stream if copy_stream is not None else torch.cuda.Stream()
    main = ctx.stream
    loaded = [torch.cuda.Event() for _ in bufs]   # copy-in of a buffer done
    stepped = [torch.cuda.Event() for _ in bufs]  # step on a buffer done
    drained = [None for _ in bufs]                # copy-out of a buffer done

    def load(k):
        b = k % len(bufs)
        with torch.cuda.stream(cs):
            if drained[b] is not None:
                cs.wait_event(drained[b])
            for f, t in host_in[k].items():
                bufs[b][f].copy_(t, non_blocking=True)
            loaded[b].record(cs)

    load(0)
    for k in range(n):
        b = k % len(bufs)
        if k + 1 < n:
            load(k + 1)
        main.wait_event(loaded[b])
        ctx.step(bufs[b], dt_fixed, dt_used)
        stepped[b].record(main)
        with torch.cuda.stream(cs):
            cs.wait_event(stepped[b])
            for f, t in host_out[k].items():
                t.copy_(bufs[b][f], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(cs)
            drained[b] = ev
    main.wait_stream(cs)
