"""torch.autograd bridge for the MFM step: forward = gz_step, backward =
gz_step_backward (the hand-written adjoint in the CUDA library).

Per-step checkpointing: each MFMStep node keeps the state its step started
from (x, y, z, vx, vy, vz, m, u), the converged support radius the step
returned and the step's checkpoint buffer (gz_step_checkpoint): the
per-particle momentum and energy rates with n and the kernel-derivative sum
at the converged H, at GZ_CKPT_GRADIENTS also the gradient pass's
per-particle outputs (about 370 bytes a particle in FP32; GZ_CKPT_RATES
keeps 40), and at the default level GZ_CKPT_LISTS also the sort's order and
the neighbour lists' first 64 slots (about 640 bytes a
particle in all).  The backward pass re-runs inside gz_step_backward what the
checkpoint does not hold (at level 2: the reverse pair lists; at lower
levels the sort, the density pass at the converged H and the lists) and
recomputes every pair quantity: none is stored.  Every level gives the same
gradients bit for bit.  The step dt is frozen at the value the forward used: a CFL step is
read back once per step.

Differentiable inputs: x, y, z, vx, vy, vz, m, u.  The support radius h is
passed through (a converged H does not depend on its initial guess) and ids
are integers.
"""
from __future__ import annotations

import torch

STATE = ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h")
GRADS = ("x", "y", "z", "vx", "vy", "vz", "m", "u")
OUT = ("x", "y", "z", "vx", "vy", "vz", "u", "h")


class MFMStep(torch.autograd.Function):
    """One MFM step of a gz Context with autograd support."""

    @staticmethod
    def forward(fctx, gz_ctx, dt, level, ids, x, y, z, vx, vy, vz, m, u, h):
        cur = {"x": x.clone(), "y": y.clone(), "z": z.clone(), "vx": vx.clone(), "vy": vy.clone(),
               "vz": vz.clone(), "m": m, "u": u.clone(), "h": h.clone(), "id": ids}
        dtu = torch.empty(1, dtype=torch.float64, device=x.device)
        ckpt = gz_ctx.new_checkpoint(level)
        gz_ctx.step(cur, float(dt), dtu, ckpt, level)
        used = float(dt) if dt > 0 else float(dtu.item())
        fctx.save_for_backward(x, y, z, vx, vy, vz, m, u, cur["h"], ckpt)
        fctx.gz_ctx, fctx.ids, fctx.dt, fctx.level = gz_ctx, ids, used, level
        gz_ctx.last_dt = used
        fctx.mark_non_differentiable(cur["h"])
        return tuple(cur[k] for k in OUT)

    @staticmethod
    def backward(fctx, *gout):
        x, y, z, vx, vy, vz, m, u, h_conv, ckpt = fctx.saved_tensors
        start = {"x": x, "y": y, "z": z, "vx": vx, "vy": vy, "vz": vz, "m": m, "u": u,
                 "h": h_conv.clone(), "id": fctx.ids}
        gend = {}
        for k, g in zip(OUT[:-1], gout[:-1]):
            gend[k] = (g if g is not None else torch.zeros_like(x)).contiguous()
        gstart = {k: torch.zeros_like(x) for k in GRADS}
        fctx.gz_ctx.step_backward(start, fctx.dt, gend, gstart, ckpt, fctx.level)
        return (None, None, None, None, gstart["x"], gstart["y"], gstart["z"], gstart["vx"],
                gstart["vy"], gstart["vz"], gstart["m"], gstart["u"], None)


def step(gz_ctx, state: dict, dt: float = 0.0, level: int = 2) -> dict:
    """One differentiable step; state holds x..u, h (tensors) and id; level is
    the checkpoint level (2: also the sorted order and lists, 1: rates and
    gradient pass kept, 0: rates only)."""
    outs = MFMStep.apply(gz_ctx, float(dt), int(level), state["id"], *(state[k] for k in STATE))
    new = dict(zip(OUT, outs))
    new["m"] = state["m"]
    new["id"] = state["id"]
    return new


def rollout(gz_ctx, state: dict, nsteps: int, dts=None, level: int = 2):
    """nsteps differentiable steps (CFL steps unless dts gives them); returns
    the final state and the list of steps used."""
    used = []
    for k in range(nsteps):
        dt = 0.0 if dts is None else float(dts[k])
        state = step(gz_ctx, state, dt, level)
        used.append(gz_ctx.last_dt)
    return state, used
