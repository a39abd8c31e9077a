"""gz_density_noalloc: the density pass for callers that cannot allocate device
memory (their memory belongs to their own pool, or their loop cannot afford
the synchronisation of an allocation).  It runs the same kernels as
gz_density, so it must give what gz_density gives bit for bit, call after
call, although every call reuses the same fixed scratch array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1712_01294_gb300 import inputs as I

from gpu_common import cast_state, device, ostate

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    import paper_1712_01294_gb300 as gz
    lib = gz.load_library()
    fn = lib.gz_density_noalloc
    fn.restype = C.c_int32
    fn.argtypes = [C.POINTER(gz.Params), C.c_int64, C.POINTER(gz._Particles), C.c_void_p,
                   C.c_void_p, C.c_void_p, C.c_void_p]
    return gz, fn


def _both(gz, fn, q, prec, H=None):
    """gz_density on a fresh context, then gz_density_noalloc on a copy of the
    same input; returns both results (h, n, iters) and the call's status bits."""
    import torch
    params = gz.default_params(precision=prec)
    stream = torch.cuda.current_stream()
    ref = device(q, prec, H)
    ctx = gz.Context([q.N], params)
    n_ref, it_ref = ctx.density(ref)
    st = ctx.status(reset=True)
    ctx.close()
    d = device(q, prec, H)
    n_out = torch.empty(q.N, dtype=d["x"].dtype, device="cuda")
    it_out = torch.empty(q.N, dtype=torch.int32, device="cuda")
    bits = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    parts = gz._Particles()
    for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h", "id"):
        setattr(parts, k, d[k].data_ptr())
    rc = fn(C.byref(params), q.N, C.byref(parts), C.c_void_p(n_out.data_ptr()),
            C.c_void_p(it_out.data_ptr()), C.c_void_p(bits.data_ptr()),
            C.c_void_p(stream.cuda_stream))
    assert rc == gz.GZ_OK
    torch.cuda.synchronize()
    got = (d["h"].cpu().numpy(), n_out.cpu().numpy(), it_out.cpu().numpy())
    want = (ref["h"].cpu().numpy(), n_ref.cpu().numpy(), it_ref.cpu().numpy())
    return got, want, int(bits.cpu()[0]) & 0xFFFFFFFF, st


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_density_equals_gz_density_on_consecutive_calls(prec):
    gz, fn = _noalloc_fn()
    # calls in a row with different boxes: none may see the previous one's leftovers
    for kind, n, seed in (("turb", 20, 3), ("sedov", 23, 4), ("turb", 12, 5)):
        make = I.turbulence if kind == "turb" else I.sedov
        q = cast_state(make(n, seed=seed), prec)
        got, want, bits, st = _both(gz, fn, q, prec)
        assert st["ok"], st
        assert bits == 0
        for a, b in zip(got, want):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_density_deferred_particles_equal_gz_density(prec):
    # an initial guess of 2.6 H0 puts about 600 candidates inside the first
    # scan radius, far more than the per-thread cache holds: every particle
    # takes the warp-per-particle kernel, in both calls
    gz, fn = _noalloc_fn()
    q = cast_state(I.turbulence(14, seed=8), prec)
    H = np.full(q.N, 2.6 * I.h0(q.N))
    got, want, bits, st = _both(gz, fn, q, prec, H)
    assert st["ok"] and bits == 0, (st, bits)
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
    if prec == gz.GZ_FP64:
        # the iteration counts are those of the oracle from the same start
        s = ostate(q)
        Ho, _, it_o, _ = O.density(s, O.params(), H_in=H)
        assert np.array_equal(got[2], it_o)
        assert np.max(np.abs(got[0] - Ho) / Ho) <= 1e-12


def test_noalloc_density_reports_device_status():
    gz, fn = _noalloc_fn()
    q = cast_state(I.sod(10, seed=6), gz.GZ_MIXED32)
    q.x[17] = 1.25  # outside the unit box: flagged by the binning pass
    got, want, bits, st = _both(gz, fn, q, gz.GZ_MIXED32)
    assert "nonfinite" in st["bits"]
    # the same word as the context's (the list-overflow bit is never reported)
    assert bits & gz.STATUS_BITS["nonfinite"]
    assert bits == st["raw"] & ~gz.STATUS_BITS["nbr_overflow"]
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


def test_noalloc_density_rejects_sizes_beyond_its_limit():
    import torch
    gz, fn = _noalloc_fn()
    params = gz.default_params()
    q = cast_state(I.sod(8), gz.GZ_MIXED32)
    d = device(q, gz.GZ_MIXED32)
    parts = gz._Particles()
    for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h", "id"):
        setattr(parts, k, d[k].data_ptr())
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert fn(C.byref(params), 32769, C.byref(parts), None, None, None, s) == gz.GZ_E_INVAL
    assert fn(C.byref(params), 0, C.byref(parts), None, None, None, s) == gz.GZ_E_INVAL
    fine = gz.default_params(cell_factor=0.25)  # would need a 64^3-cell grid at 32768 particles
    assert fn(C.byref(fine), 32768, C.byref(parts), None, None, None, s) == gz.GZ_E_INVAL
