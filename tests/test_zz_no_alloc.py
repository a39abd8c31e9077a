"""gz_density_noalloc: the density pass for callers that cannot allocate device
memory (their memory belongs to their own pool, or their loop cannot afford
the synchronisation of an allocation).  It must give what gz_density gives,
call after call, although every call reuses the same fixed scratch array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1712_01294_gb300 import inputs as I

from gpu_common import cast_state, device

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    import paper_1712_01294_gb300 as gz
    lib = gz.load_library()
    fn = lib.gz_density_noalloc
    fn.restype = C.c_int32
    fn.argtypes = [C.POINTER(gz.Params), C.c_int64, C.POINTER(gz._Particles), C.c_void_p,
                   C.c_void_p, C.c_void_p]
    return gz, fn


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_density_matches_gz_density_on_consecutive_calls(prec):
    import torch
    gz, fn = _noalloc_fn()
    params = gz.default_params(precision=prec)
    stream = torch.cuda.current_stream()
    # two calls in a row with different boxes: the second must not see the first's leftovers
    for kind, n, seed in (("turb", 20, 3), ("sedov", 23, 4)):
        make = I.turbulence if kind == "turb" else I.sedov
        q = cast_state(make(n, seed=seed), prec)
        ref = device(q, prec)
        ctx = gz.Context([q.N], params)
        n_ref, it_ref = ctx.density(ref)
        st = ctx.status(reset=True)
        assert st["ok"], st

        d = device(q, prec)
        n_out = torch.empty(q.N, dtype=d["x"].dtype, device="cuda")
        it_out = torch.empty(q.N, dtype=torch.int32, device="cuda")
        parts = ctx._parts({k: d[k] for k in ctx.FIELDS})
        rc = fn(C.byref(params), q.N, C.byref(parts), C.c_void_p(n_out.data_ptr()),
                C.c_void_p(it_out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == gz.GZ_OK
        torch.cuda.synchronize()
        h_ref, h_new = ref["h"].cpu().numpy(), d["h"].cpu().numpy()
        tol = 1e-12 if prec == gz.GZ_FP64 else 2e-5
        rel = np.abs(h_new.astype(np.float64) - h_ref) / h_ref
        assert rel.max() <= tol
        nr = n_ref.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(n_out.cpu().numpy() - nr) / nr) <= tol
        assert np.array_equal(it_out.cpu().numpy(), it_ref.cpu().numpy())
        ctx.close()


def test_noalloc_density_rejects_sizes_beyond_its_limit():
    import torch
    gz, fn = _noalloc_fn()
    params = gz.default_params()
    q = cast_state(I.sod(8), gz.GZ_MIXED32)
    d = device(q, gz.GZ_MIXED32)
    ctx = gz.Context([q.N], params)
    parts = ctx._parts(d)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert fn(C.byref(params), 32769, C.byref(parts), None, None, s) == gz.GZ_E_INVAL
    assert fn(C.byref(params), 0, C.byref(parts), None, None, s) == gz.GZ_E_INVAL
    fine = gz.default_params(cell_factor=0.25)  # would need a 64^3-cell grid at 32768 particles
    assert fn(C.byref(fine), 32768, C.byref(parts), None, None, s) == gz.GZ_E_INVAL
    ctx.close()
