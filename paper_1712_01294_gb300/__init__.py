"""GB300-native meshless finite-mass (MFM) hydrodynamics hot path.

Thin Python binding over the C ABI of ``libgz.so`` (``include/gz.h``): it only
marshals torch tensors (device memory) and the current CUDA stream into the C
calls; every step of the path runs in the library's CUDA kernels.  There is no
CPU fallback: if the library cannot be loaded, every call raises.

Names follow the C ABI: ``Context.density`` -> ``gz_density``,
``Context.gradients`` -> ``gz_gradients``, ``Context.timestep`` ->
``gz_timestep``, ``Context.hydro_fluxes`` -> ``gz_hydro_fluxes``,
``Context.step`` -> ``gz_step``, ``Context.step_backward`` ->
``gz_step_backward``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

__all__ = ["GZ_FP64", "GZ_MIXED32", "GZ_MFM", "GZ_MFV", "GZ_RIEMANN_HLLC", "GZ_RIEMANN_EXACT",
           "GZ_RIEMANN_FALLBACK", "Params", "Context", "GZError", "load_library",
           "default_params", "status_names"]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgz.so")

GZ_OK, GZ_E_INVAL, GZ_E_NOMEM, GZ_E_CUDA, GZ_E_DEVICE = 0, 1, 2, 3, 4
GZ_FP64, GZ_MIXED32 = 0, 1
GZ_MFM, GZ_MFV = 0, 1
GZ_RIEMANN_HLLC, GZ_RIEMANN_EXACT, GZ_RIEMANN_FALLBACK = 0, 1, 2
GZ_CKPT_RATES, GZ_CKPT_GRADIENTS, GZ_CKPT_LISTS = 0, 1, 2
STATUS_BITS = {
    "hconv": 1 << 0, "singular": 1 << 1, "nonfinite": 1 << 2, "nbr_overflow": 1 << 3,
    "hlim": 1 << 4, "fallback": 1 << 8, "pstar_neg": 1 << 9, "ufloor": 1 << 10,
    "kappa_fp64": 1 << 11,
}
PASSES = ("sort", "density", "lists", "reverse", "prim", "gradients", "fluxes", "update")
COUNTERS = ("hconv", "singular", "nonfinite", "nbr_overflow", "fallback", "pstar_neg",
            "ufloor", "kappa_fp64")


class GZError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gz error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("ngb", C.c_double), ("tol", C.c_double),
                ("cfl", C.c_double), ("kappa_max", C.c_double), ("beta", C.c_double),
                ("u_floor_frac", C.c_double), ("h_lim", C.c_double),
                ("cell_factor", C.c_double), ("precision", C.c_int32), ("hancock", C.c_int32),
                ("max_iter", C.c_int32), ("max_ngb", C.c_int32), ("scheme", C.c_int32),
                ("riemann", C.c_int32), ("density_cache", C.c_int32)]


class _Particles(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h", "id")]


_lock = threading.Lock()
_lib = None


def load_library(build_if_missing: bool = True):
    """Loads libgz.so (building it with nvcc if absent or stale); raises if impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        if build_if_missing and _build.stale():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing; run "
                               "__graft_entry__.build() on a machine with nvcc")
        lib = C.CDLL(LIB_PATH)
        st, vp, i32, d = C.c_int32, C.c_void_p, C.c_int32, C.c_double
        P = C.POINTER(_Particles)
        sig = {
            "gz_default_params": (st, [C.POINTER(Params)]),
            "gz_create": (st, [C.POINTER(Params), i32, vp, vp, C.POINTER(vp)]),
            "gz_destroy": (st, [vp]),
            "gz_density": (st, [vp, P, vp, vp]),
            "gz_gradients": (st, [vp, P, vp, vp, vp]),
            "gz_timestep": (st, [vp, P, vp, vp, vp]),
            "gz_hydro_fluxes": (st, [vp, P, vp, vp, vp, d, vp, vp, vp]),
            "gz_step": (st, [vp, P, d, vp]),
            "gz_step_hier": (st, [vp, P, i32, d, vp, vp, vp]),
            "gz_hydro_fluxes_backward": (st, [vp, P, vp, vp, vp, d, vp, vp, vp, vp, vp, vp, vp, vp]),
            "gz_graph_capture": (st, [vp, P, i32, d, vp]),
            "gz_graph_launch": (st, [vp]),
            "gz_checkpoint_bytes": (st, [vp, i32, vp]),
            "gz_step_checkpoint": (st, [vp, P, d, vp, vp, i32]),
            "gz_step_backward": (st, [vp, P, d, vp, i32, P, P]),
            "gz_get_neighbours": (st, [vp, vp, vp, i32]),
            "gz_get_status": (st, [vp, vp, vp, vp, i32]),
            "gz_last_error": (C.c_char_p, [vp]),
            "gz_version": (C.c_char_p, []),
            "gz_get_info": (st, [vp, vp, i32]),
            "gz_pair_count": (st, [vp, vp]),
            "gz_scan_stats": (st, [vp, vp]),
            "gz_profile_enable": (st, [vp, i32]),
            "gz_profile_read": (st, [vp, vp, vp, i32]),
            "gz_measure_alu": (st, [i32, vp, vp]),
            "gz_step_begin": (st, [vp, P, vp]),
            "gz_step_finish": (st, [vp, P, vp]),
            "gz_create_subdomain": (st, [C.POINTER(Params), C.c_int64, C.c_int64, vp, C.POINTER(vp)]),
            "gz_set_subdomain": (st, [vp, C.c_int64, C.c_int64, vp]),
            "gz_checkpoint_limiters": (st, [vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def default_params(**kw) -> Params:
    p = Params()
    load_library().gz_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def measure_alu(stream=None):
    """gz_measure_alu on the current device: measured FP32 and FP64 fused
    multiply-add throughput (TFLOP/s) and FP32 reciprocal-square-root
    throughput (T operations/s)."""
    import torch
    lib = load_library()
    st = C.c_void_p((stream if stream is not None else torch.cuda.current_stream()).cuda_stream)
    out = {}
    for which, key in ((0, "fp32_fma_tflops"), (1, "fp64_fma_tflops"), (2, "mufu_rsqrt_tops")):
        v = C.c_double()
        rc = lib.gz_measure_alu(which, C.byref(v), st)
        if rc != GZ_OK:
            raise GZError(rc, "gz_measure_alu failed")
        out[key] = round(v.value / 1e12, 3)
    return out


def status_names(bits: int):
    return [k for k, b in STATUS_BITS.items() if bits & b]


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Context:
    """One gz_ctx: ``counts`` particles per box, params, bound to a CUDA stream.

    Particle sets are dicts (or objects) with torch CUDA tensors x, y, z, vx,
    vy, vz, m, u, h (float32 for GZ_MIXED32, float64 for GZ_FP64) and id
    (int64), all contiguous.
    """

    FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h", "id")

    def __init__(self, counts, params: Params | None = None, stream=None, grid_count: int = 0, **kw):
        """grid_count > 0: a subdomain context (gz_create_subdomain) of one box
        holding up to counts[0] particles, its cell grid that of a box of
        grid_count particles."""
        import torch
        self.torch = torch
        self.lib = load_library()
        self.params = params if params is not None else default_params(**kw)
        self.counts = [int(c) for c in counts]
        self.N = sum(self.counts)
        self.capacity = self.N
        self.dtype = torch.float64 if self.params.precision == GZ_FP64 else torch.float32
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        if grid_count > 0:
            if len(self.counts) != 1:
                raise ValueError("a subdomain context holds one box")
            rc = self.lib.gz_create_subdomain(C.byref(self.params), self.N, int(grid_count),
                                              C.c_void_p(self.stream.cuda_stream), C.byref(h))
        else:
            arr = (C.c_int64 * len(self.counts))(*self.counts)
            rc = self.lib.gz_create(C.byref(self.params), len(self.counts), C.cast(arr, C.c_void_p),
                                    C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != GZ_OK:
            raise GZError(rc, "gz_create failed")
        self.h = h

    # -- helpers ------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.gz_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != GZ_OK:
            msg = self.lib.gz_last_error(self.h).decode()
            raise GZError(rc, f"{what}: {msg}")

    def _parts(self, p) -> _Particles:
        get = (lambda k: p[k]) if isinstance(p, dict) else (lambda k: getattr(p, k))
        s = _Particles()
        for k in self.FIELDS:
            t = get(k)
            want = self.torch.int64 if k == "id" else self.dtype
            if t is None:
                setattr(s, k, None)
                continue
            if t.dtype != want or not t.is_cuda or not t.is_contiguous() or t.numel() != self.N:
                raise ValueError(f"field {k}: need contiguous CUDA {want} of {self.N} elements")
            setattr(s, k, t.data_ptr())
        return s

    def empty(self, *shape, dtype=None):
        return self.torch.empty(*shape, dtype=dtype or self.dtype, device="cuda")

    # -- C ABI calls -----------------------------------------------------------
    def density(self, p, n_out=None, iters_out=None):
        """gz_density: solves H in place (p['h']); returns (n, iters)."""
        n_out = self.empty(self.N) if n_out is None else n_out
        iters_out = self.empty(self.N, dtype=self.torch.int32) if iters_out is None else iters_out
        s = self._parts(p)
        self._check(self.lib.gz_density(self.h, C.byref(s), _ptr(n_out), _ptr(iters_out)),
                    "gz_density")
        return n_out, iters_out

    def gradients(self, p, n, grad_out=None, B_out=None):
        """gz_gradients: returns (grad [15,N], B [6,N])."""
        grad_out = self.empty(15, self.N) if grad_out is None else grad_out
        B_out = self.empty(6, self.N) if B_out is None else B_out
        s = self._parts(p)
        self._check(self.lib.gz_gradients(self.h, C.byref(s), _ptr(n), _ptr(grad_out), _ptr(B_out)),
                    "gz_gradients")
        return grad_out, B_out

    def timestep(self, p, n):
        """gz_timestep: returns (dt_i [N] float64, dt_box [nboxes] float64)."""
        dti = self.empty(self.N, dtype=self.torch.float64)
        dtb = self.empty(len(self.counts), dtype=self.torch.float64)
        s = self._parts(p)
        self._check(self.lib.gz_timestep(self.h, C.byref(s), _ptr(n), _ptr(dti), _ptr(dtb)),
                    "gz_timestep")
        return dti, dtb

    def hydro_fluxes(self, p, n, grad, B, dt, dpdt=None, dEdt=None, with_mass=False):
        """gz_hydro_fluxes: returns (dpdt [3,N], dEdt [N]) in float64, and dmdt [N]
        third when with_mass (zeros under GZ_MFM)."""
        dpdt = self.empty(3, self.N, dtype=self.torch.float64) if dpdt is None else dpdt
        dEdt = self.empty(self.N, dtype=self.torch.float64) if dEdt is None else dEdt
        dmdt = self.empty(self.N, dtype=self.torch.float64) if with_mass else None
        s = self._parts(p)
        self._check(self.lib.gz_hydro_fluxes(self.h, C.byref(s), _ptr(n), _ptr(grad), _ptr(B),
                                             float(dt), _ptr(dpdt), _ptr(dEdt), _ptr(dmdt)),
                    "gz_hydro_fluxes")
        return (dpdt, dEdt, dmdt) if with_mass else (dpdt, dEdt)

    def hydro_fluxes_backward(self, p, n, grad, B, dt, dpdt_bar, dEdt_bar):
        """gz_hydro_fluxes_backward: dict of float64 adjoints x [3,N], h, n, W [5,N],
        grad [15,N], B [6,N]."""
        f64 = self.torch.float64
        out = {"x": self.empty(3, self.N, dtype=f64), "h": self.empty(self.N, dtype=f64),
               "n": self.empty(self.N, dtype=f64), "W": self.empty(5, self.N, dtype=f64),
               "grad": self.empty(15, self.N, dtype=f64), "B": self.empty(6, self.N, dtype=f64)}
        s = self._parts(p)
        self._check(self.lib.gz_hydro_fluxes_backward(
            self.h, C.byref(s), _ptr(n), _ptr(grad), _ptr(B), float(dt), _ptr(dpdt_bar),
            _ptr(dEdt_bar), _ptr(out["x"]), _ptr(out["h"]), _ptr(out["n"]), _ptr(out["W"]),
            _ptr(out["grad"]), _ptr(out["B"])), "gz_hydro_fluxes_backward")
        return out

    def step(self, p, dt_fixed: float = 0.0, dt_used=None, ckpt=None, level: int = 1):
        """gz_step in place on p; dt_used (device float64 [nboxes]) receives the
        steps.  With ckpt (a device buffer from new_checkpoint(level)),
        gz_step_checkpoint also saves what gz_step_backward of this step reads."""
        s = self._parts(p)
        if ckpt is None:
            self._check(self.lib.gz_step(self.h, C.byref(s), float(dt_fixed), _ptr(dt_used)), "gz_step")
        else:
            self._ckpt_ok(ckpt, level)
            self._check(self.lib.gz_step_checkpoint(self.h, C.byref(s), float(dt_fixed), _ptr(dt_used),
                                                    _ptr(ckpt), int(level)), "gz_step_checkpoint")
        return dt_used

    def step_begin(self, p, dt_box=None):
        """gz_step_begin: S1-S3 on p; returns dt_box (device float64 [nboxes]),
        each box's CFL step over its owned particles."""
        dt_box = self.empty(len(self.counts), dtype=self.torch.float64) if dt_box is None else dt_box
        s = self._parts(p)
        self._check(self.lib.gz_step_begin(self.h, C.byref(s), _ptr(dt_box)), "gz_step_begin")
        return dt_box

    def step_finish(self, p, dt):
        """gz_step_finish: S4 and S6 on the particle set of step_begin with the
        steps dt (device float64 [nboxes])."""
        s = self._parts(p)
        self._check(self.lib.gz_step_finish(self.h, C.byref(s), _ptr(dt)), "gz_step_finish")

    def set_subdomain(self, n: int, n_owned: int, owned=None):
        """gz_set_subdomain: the next calls take n particles, of which the
        n_owned marked in owned (CUDA uint8 [n], 1 = owned; None = all) are owned."""
        if owned is not None and (owned.dtype != self.torch.uint8 or not owned.is_cuda
                                  or not owned.is_contiguous() or owned.numel() != n):
            raise ValueError("owned must be a contiguous CUDA uint8 tensor of n elements")
        self._check(self.lib.gz_set_subdomain(self.h, int(n), int(n_owned), _ptr(owned)),
                    "gz_set_subdomain")
        self.N = int(n)
        self.counts = [int(n)]

    def step_hier(self, p, K: int, dt_fixed: float = 0.0, dt_used=None, bins=None):
        """gz_step_hier: one sync interval of 2^K hierarchical substeps in place on
        p; dt_used (device float64 [nboxes]) receives the interval, bins (device
        int32 [N]) the final bins.  Returns the number of active
        particle-substeps."""
        s = self._parts(p)
        act = C.c_int64()
        self._check(self.lib.gz_step_hier(self.h, C.byref(s), int(K), float(dt_fixed), _ptr(dt_used),
                                          _ptr(bins), C.byref(act)), "gz_step_hier")
        return int(act.value)

    def checkpoint_bytes(self, level: int = 1) -> int:
        """gz_checkpoint_bytes: size of one step checkpoint at this level."""
        v = C.c_int64()
        self._check(self.lib.gz_checkpoint_bytes(self.h, int(level), C.byref(v)), "gz_checkpoint_bytes")
        return int(v.value)

    def new_checkpoint(self, level: int = 1):
        """A device buffer for one step checkpoint (GZ_CKPT_RATES = 0,
        GZ_CKPT_GRADIENTS = 1 or GZ_CKPT_LISTS = 2)."""
        return self.empty(self.checkpoint_bytes(level), dtype=self.torch.uint8)

    def checkpoint_limiters(self, ckpt):
        """gz_checkpoint_limiters: the limiter's choices of the step that wrote
        ckpt (level GZ_CKPT_GRADIENTS, the last one): int64 [10, N] of ids."""
        out = self.empty(10, self.N, dtype=self.torch.int64)
        self._check(self.lib.gz_checkpoint_limiters(self.h, _ptr(ckpt), _ptr(out)),
                    "gz_checkpoint_limiters")
        return out

    def _ckpt_ok(self, ckpt, level):
        if (ckpt.dtype != self.torch.uint8 or not ckpt.is_cuda or not ckpt.is_contiguous()
                or ckpt.numel() < self.checkpoint_bytes(level) or ckpt.data_ptr() % 256):
            raise ValueError("ckpt must be a contiguous, 256-byte aligned CUDA uint8 buffer of "
                             "checkpoint_bytes(level) bytes")

    def graph_capture(self, p, nsteps: int, dt_fixed: float = 0.0, dt_used=None):
        """gz_graph_capture: record nsteps steps on p as one CUDA graph (the
        context stream must be a created torch.cuda.Stream)."""
        s = self._parts(p)
        self._graph_parts = s  # the graph keeps these pointers
        self._check(self.lib.gz_graph_capture(self.h, C.byref(s), int(nsteps), float(dt_fixed),
                                              _ptr(dt_used)), "gz_graph_capture")

    def graph_launch(self):
        """gz_graph_launch: replay the captured steps."""
        self._check(self.lib.gz_graph_launch(self.h), "gz_graph_launch")

    def step_backward(self, p_start, dt, gbar_end, gbar_start, ckpt=None, level: int = 1):
        """gz_step_backward: adjoint of one step (see include/gz.h); ckpt is the
        step's checkpoint (from step(..., ckpt=, level=)) or None to recompute."""
        a, b, c = self._parts(p_start), self._grad_parts(gbar_end), self._grad_parts(gbar_start)
        if ckpt is not None:
            self._ckpt_ok(ckpt, level)
        self._check(self.lib.gz_step_backward(self.h, C.byref(a), float(dt), _ptr(ckpt), int(level),
                                              C.byref(b), C.byref(c)), "gz_step_backward")
        return gbar_start

    def _grad_parts(self, g) -> _Particles:
        get = (lambda k: g.get(k)) if isinstance(g, dict) else (lambda k: getattr(g, k, None))
        s = _Particles()
        for k in self.FIELDS:
            t = get(k)
            setattr(s, k, None if t is None else t.data_ptr())
        return s

    def neighbours(self, cap: int = 0):
        """gz_get_neighbours: (counts [N] int32, ids [cap, N] int64 or None)."""
        cnt = self.empty(self.N, dtype=self.torch.int32)
        ids = self.empty(cap, self.N, dtype=self.torch.int64) if cap > 0 else None
        self._check(self.lib.gz_get_neighbours(self.h, _ptr(cnt), _ptr(ids), int(cap)),
                    "gz_get_neighbours")
        return cnt, ids

    def info(self):
        """gz_get_info: dict of host-side facts (kernel launches issued so far, ...)."""
        v = (C.c_int64 * 6)()
        self._check(self.lib.gz_get_info(self.h, C.cast(v, C.c_void_p), 6), "gz_get_info")
        return dict(zip(("launches", "N", "nboxes", "cells", "cap", "rcap"), (int(x) for x in v)))

    def pair_count(self) -> int:
        """gz_pair_count: ordered flux pairs of the last pair-building pass."""
        v = C.c_int64()
        self._check(self.lib.gz_pair_count(self.h, C.byref(v)), "gz_pair_count")
        return int(v.value)

    def scan_stats(self) -> dict:
        """gz_scan_stats: candidates a 1.05 H cell scan tests, those within
        1.05 H and those within H, summed over the last density pass."""
        v = (C.c_int64 * 3)()
        self._check(self.lib.gz_scan_stats(self.h, C.cast(v, C.c_void_p)), "gz_scan_stats")
        return dict(zip(("candidates", "within_cache_radius", "neighbours"), (int(x) for x in v)))

    def profile(self, enable: bool = True):
        """gz_profile_enable: CUDA-event timing of every pass."""
        self._check(self.lib.gz_profile_enable(self.h, 1 if enable else 0), "gz_profile_enable")

    def profile_read(self, reset: bool = False):
        """gz_profile_read: {pass: (total_ms, calls)}."""
        ms = (C.c_double * len(PASSES))()
        calls = (C.c_int64 * len(PASSES))()
        self._check(self.lib.gz_profile_read(self.h, C.cast(ms, C.c_void_p), C.cast(calls, C.c_void_p),
                                             1 if reset else 0), "gz_profile_read")
        return {k: (float(ms[i]), int(calls[i])) for i, k in enumerate(PASSES)}

    def status(self, reset: bool = False):
        """gz_get_status: dict with bits (names), first_bad_id and counters."""
        bits = C.c_uint32()
        bad = C.c_int64()
        cnt = (C.c_int64 * len(COUNTERS))()
        rc = self.lib.gz_get_status(self.h, C.byref(bits), C.byref(bad), C.cast(cnt, C.c_void_p),
                                    1 if reset else 0)
        if rc not in (GZ_OK, GZ_E_DEVICE):
            self._check(rc, "gz_get_status")
        return {"bits": status_names(bits.value), "raw": bits.value, "first_bad_id": bad.value,
                "counters": dict(zip(COUNTERS, (int(v) for v in cnt))), "ok": rc == GZ_OK}


def to_device(p, precision=GZ_MIXED32):
    """Host particle set (numpy, see ``inputs``) -> dict of contiguous CUDA tensors."""
    import torch
    dt = torch.float64 if precision == GZ_FP64 else torch.float32
    out = {}
    for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u"):
        out[k] = torch.as_tensor(getattr(p, k), dtype=dt).contiguous().cuda()
    out["h"] = torch.as_tensor(p.H, dtype=dt).contiguous().cuda()
    out["id"] = torch.as_tensor(p.id, dtype=torch.int64).contiguous().cuda()
    return out
