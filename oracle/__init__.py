"""FP64 CPU oracle for the MFM hydrodynamics step (ctypes wrapper over gz_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_1712_01294_gb300``) never imports it and shares no code with it.

The C source is compiled on first import (gcc, ``-O2 -ffp-contract=off
-fopenmp``) into ``oracle/libgz_oracle.so``; it is rebuilt when the source is
newer than the library.  Every function follows one reading of the method
(labels O1..O14 in ``gz_oracle.h``): the paper (GIZMO public release,
"Hydrodynamics" item and "Arbitrary (Moving) Meshes" section) names the
Lagrangian meshless finite-volume Godunov scheme but prints no formula.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gz_oracle.c")
_HDR = os.path.join(_HERE, "gz_oracle.h")
_LIB = os.path.join(_HERE, "libgz_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library if missing or stale; return its path."""
    stale = (not os.path.exists(_LIB)) or force or (
        max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_LIB))
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
               "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("ngb", C.c_double), ("tol", C.c_double),
                ("cfl", C.c_double), ("kappa_max", C.c_double), ("beta", C.c_double),
                ("u_floor_frac", C.c_double), ("h_lim", C.c_double),
                ("hancock", C.c_int32), ("max_iter", C.c_int32), ("use_cells", C.c_int32),
                ("scheme", C.c_int32), ("riemann", C.c_int32), ("pad", C.c_int32)]


class Counters(C.Structure):
    _fields_ = [(k, C.c_int64) for k in
                ("hconv", "singular", "fallback", "pstar_neg", "ufloor", "nonfinite",
                 "kappa_big", "pairs", "bin_clamp")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


MFM, MFV = 0, 1
HLLC, EXACT, EXACT_FALLBACK = 0, 1, 2  # MFM face solver (riemann)


def params(gamma=5.0 / 3.0, ngb=32.0, tol=1e-6, cfl=0.2, kappa_max=100.0, beta=1.0,
           u_floor_frac=1e-10, h_lim=0.5, hancock=1, max_iter=64, use_cells=1,
           scheme=MFM, riemann=HLLC) -> Params:
    if riemann not in (HLLC, EXACT, EXACT_FALLBACK):
        raise ValueError("riemann must be HLLC, EXACT or EXACT_FALLBACK")
    if scheme == MFV and riemann != HLLC:
        raise ValueError("the exact Riemann solver option covers the MFM face only")
    return Params(gamma, ngb, tol, cfl, kappa_max, beta, u_floor_frac, h_lim, hancock,
                  max_iter, use_cells, scheme, riemann, 0)


_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_I32 = C.POINTER(C.c_int32)
_U8 = C.POINTER(C.c_uint8)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i64, vp = C.c_double, C.c_int64, C.c_void_p
            lib.gzo_kernel_w.restype = d
            lib.gzo_kernel_w.argtypes = [d]
            lib.gzo_kernel_dw.restype = d
            lib.gzo_kernel_dw.argtypes = [d]
            lib.gzo_W.restype = d
            lib.gzo_W.argtypes = [d, d]
            lib.gzo_dWdH.restype = d
            lib.gzo_dWdH.argtypes = [d, d]
            lib.gzo_min_image.restype = d
            lib.gzo_min_image.argtypes = [d]
            lib.gzo_neighbours.restype = i64
            lib.gzo_neighbours.argtypes = [i64, vp, vp, vp, vp, vp, C.c_int32, vp, vp, i64]
            lib.gzo_flux_pairs.restype = i64
            lib.gzo_flux_pairs.argtypes = [i64, vp, vp, vp, vp, vp, C.c_int32, vp, vp, i64]
            lib.gzo_density.restype = C.c_int
            lib.gzo_density.argtypes = [i64, vp, vp, vp, vp, vp, vp, C.POINTER(Params), vp, vp,
                                        vp, vp, C.POINTER(Counters)]
            lib.gzo_gradients.restype = C.c_int
            lib.gzo_gradients.argtypes = [i64] + [vp] * 11 + [vp, C.POINTER(Params)] + \
                [vp] * 5 + [C.POINTER(Counters)]
            lib.gzo_timestep.restype = C.c_int
            lib.gzo_timestep.argtypes = [i64] + [vp] * 11 + [vp, C.POINTER(Params), vp, _D]
            lib.gzo_fluxes.restype = C.c_int
            lib.gzo_fluxes.argtypes = [i64] + [vp] * 13 + [d, vp, C.POINTER(Params), vp, vp, vp,
                                                         C.POINTER(Counters)]
            lib.gzo_update.restype = C.c_int
            lib.gzo_update.argtypes = [i64] + [vp] * 11 + [d, C.POINTER(Params),
                                                         C.POINTER(Counters)]
            lib.gzo_step.restype = C.c_int
            lib.gzo_step.argtypes = [i64] + [vp] * 10 + [C.POINTER(Params), _D, vp, vp, vp, vp,
                                                       C.POINTER(Counters)]
            lib.gzo_step_hier.restype = C.c_int
            lib.gzo_step_hier.argtypes = [i64] + [vp] * 10 + [C.POINTER(Params), C.c_int32, _D, vp,
                                                            C.POINTER(C.c_int64), C.POINTER(Counters)]
            lib.gzo_exchange.restype = C.c_int
            lib.gzo_exchange.argtypes = [i64] + [vp] * 15 + [d, C.POINTER(Params), vp, vp, vp, vp,
                                                           C.POINTER(Counters)]
            lib.gzo_pair.restype = C.c_int
            lib.gzo_pair.argtypes = [vp, d, d, vp, vp, vp, vp, d, d, vp, vp, vp, d,
                                     C.POINTER(Params), vp, _D, _D, vp, vp, _D, _D,
                                     C.POINTER(C.c_int), vp]
            lib.gzo_hllc_flux.restype = None
            lib.gzo_hllc_flux.argtypes = [vp, vp, vp, vp, d, _D, vp, _D]
            lib.gzo_hllc.restype = None
            lib.gzo_hllc.argtypes = [d] * 7 + [_D, _D]
            lib.gzo_riemann_star.restype = C.c_int
            lib.gzo_riemann_star.argtypes = [d] * 7 + [_D, _D]
            lib.gzo_riemann_sample.restype = None
            lib.gzo_riemann_sample.argtypes = [d] * 10 + [_D, _D, _D]
            lib.gzo_num_threads.restype = C.c_int
            lib.gzo_set_threads.argtypes = [C.c_int]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().gzo_num_threads())


def set_threads(n: int) -> None:
    _load().gzo_set_threads(int(n))


# -- O2 -----------------------------------------------------------------------
def kernel_w(q: float) -> float:
    return _load().gzo_kernel_w(float(q))


def kernel_dw(q: float) -> float:
    return _load().gzo_kernel_dw(float(q))


def W(r: float, H: float) -> float:
    return _load().gzo_W(float(r), float(H))


def dWdH(r: float, H: float) -> float:
    return _load().gzo_dWdH(float(r), float(H))


def min_image(d: float) -> float:
    return _load().gzo_min_image(float(d))


@dataclass
class State:
    """Particle state in FP64 (the oracle's working precision)."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    m: np.ndarray
    u: np.ndarray
    H: np.ndarray
    id: np.ndarray

    @property
    def N(self) -> int:
        return int(self.x.shape[0])

    @classmethod
    def from_any(cls, s) -> "State":
        g = (lambda k: _f64(getattr(s, k)) if not isinstance(s, dict) else _f64(s[k]))
        ids = s["id"] if isinstance(s, dict) else s.id
        return cls(*(g(k) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u", "H")),
                   np.ascontiguousarray(ids, dtype=np.int64))

    def copy(self) -> "State":
        return State(*(np.array(getattr(self, k)) for k in
                       ("x", "y", "z", "vx", "vy", "vz", "m", "u", "H", "id")))


def _csr(fn, s: State, R, use_cells):
    N = s.N
    R = _f64(R)
    off = np.zeros(N + 1, dtype=np.int64)
    tot = fn(N, _p(s.x), _p(s.y), _p(s.z), _p(s.id), _p(R), int(use_cells), _p(off), None, 0)
    nbr = np.zeros(max(tot, 1), dtype=np.int64)
    tot2 = fn(N, _p(s.x), _p(s.y), _p(s.z), _p(s.id), _p(R), int(use_cells), _p(off), _p(nbr), nbr.size)
    assert tot2 == tot
    return off, nbr[:tot]


def neighbours(s: State, R, use_cells=1):
    """O3: CSR (offsets, indices) of {j != i : r_ij^2 < R_i^2}, ascending id."""
    return _csr(_load().gzo_neighbours, s, R, use_cells)


def flux_pairs(s: State, H, use_cells=1):
    """O10 pair sets {j != i : r^2 < H_i^2 or r^2 < H_j^2}, ascending id."""
    return _csr(_load().gzo_flux_pairs, s, H, use_cells)


def density(s: State, p: Params, H_in=None, mask=None, counters: Counters | None = None):
    """O4/O5: returns (H, n, iters, f)."""
    N = s.N
    H_in = _f64(s.H if H_in is None else H_in)
    H = np.array(H_in)
    n = np.zeros(N)
    it = np.zeros(N, dtype=np.int32)
    f = np.zeros(N)
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    cnt = counters if counters is not None else Counters()
    _load().gzo_density(N, _p(s.x), _p(s.y), _p(s.z), _p(s.id), _p(H_in), _p(mk), C.byref(p),
                        _p(H), _p(n), _p(it), _p(f), C.byref(cnt))
    return H, n, it, f


def gradients(s: State, H, n, p: Params, mask=None, counters: Counters | None = None):
    """O6-O9: returns dict grad [15,N] (limited), grad_raw, B [6,N], alpha [5,N], kappa."""
    N = s.N
    H, n = _f64(H), _f64(n)
    out = {k: np.zeros((c, N)) for k, c in (("grad", 15), ("grad_raw", 15), ("B", 6), ("alpha", 5))}
    out["kappa"] = np.zeros(N)
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    cnt = counters if counters is not None else Counters()
    _load().gzo_gradients(N, _p(s.x), _p(s.y), _p(s.z), _p(s.id), _p(s.m), _p(H), _p(n),
                          _p(s.vx), _p(s.vy), _p(s.vz), _p(s.u), _p(mk), C.byref(p),
                          _p(out["grad"]), _p(out["B"]), _p(out["grad_raw"]), _p(out["alpha"]),
                          _p(out["kappa"]), C.byref(cnt))
    return out


def timestep(s: State, H, n, p: Params, mask=None):
    """O13: returns (dt_i [N], dt = cfl * min dt_i)."""
    N = s.N
    dti = np.zeros(N)
    dt = C.c_double(0.0)
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    _load().gzo_timestep(N, _p(s.x), _p(s.y), _p(s.z), _p(s.id), _p(s.m), _p(_f64(H)),
                         _p(_f64(n)), _p(s.vx), _p(s.vy), _p(s.vz), _p(s.u), _p(mk), C.byref(p),
                         _p(dti), C.byref(dt))
    return dti, dt.value


def fluxes(s: State, H, n, grad, B, dt, p: Params, mask=None, counters: Counters | None = None,
           with_mass: bool = False):
    """O10-O12: returns (dpdt [3,N], dEdt [N]), and dmdt [N] with with_mass."""
    N = s.N
    dp = np.zeros((3, N))
    dE = np.zeros(N)
    dm = np.zeros(N)
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    cnt = counters if counters is not None else Counters()
    _load().gzo_fluxes(N, _p(s.x), _p(s.y), _p(s.z), _p(s.id), _p(s.m), _p(_f64(H)),
                       _p(_f64(n)), _p(s.vx), _p(s.vy), _p(s.vz), _p(s.u), _p(_f64(grad)),
                       _p(_f64(B)), float(dt), _p(mk), C.byref(p), _p(dp), _p(dE), _p(dm),
                       C.byref(cnt))
    return (dp, dE, dm) if with_mass else (dp, dE)


def update(s: State, dpdt, dEdt, dt, p: Params, counters: Counters | None = None,
           dmdt=None) -> State:
    """O14 on a copy of the state (masses too when dmdt is given); returns it."""
    o = s.copy()
    cnt = counters if counters is not None else Counters()
    _load().gzo_update(o.N, _p(o.x), _p(o.y), _p(o.z), _p(o.vx), _p(o.vy), _p(o.vz), _p(o.m),
                       _p(o.u), _p(_f64(dpdt)), _p(_f64(dEdt)),
                       None if dmdt is None else _p(_f64(dmdt)), float(dt), C.byref(p),
                       C.byref(cnt))
    return o


def step(s: State, p: Params, dt: float = 0.0, counters: Counters | None = None,
         with_mass: bool = False):
    """O4..O14 on a copy; returns (new_state, dt_used, n, dpdt, dEdt), and dmdt
    after them with with_mass (the MFV mass rates; zero under MFM)."""
    o = s.copy()
    N = o.N
    n = np.zeros(N)
    dp = np.zeros((3, N))
    dE = np.zeros(N)
    dm = np.zeros(N)
    dtc = C.c_double(float(dt))
    cnt = counters if counters is not None else Counters()
    _load().gzo_step(N, _p(o.x), _p(o.y), _p(o.z), _p(o.vx), _p(o.vy), _p(o.vz), _p(o.m),
                     _p(o.u), _p(o.H), _p(o.id), C.byref(p), C.byref(dtc), _p(n), _p(dp),
                     _p(dE), _p(dm), C.byref(cnt))
    if with_mass:
        return o, dtc.value, n, dp, dE, dm
    return o, dtc.value, n, dp, dE


def step_hier(s: State, p: Params, K: int, dt: float = 0.0, counters: Counters | None = None):
    """One sync interval of hierarchical (power-of-two) timesteps on a copy
    (reading HT); returns (new_state, interval, bins [N] int32, active
    particle-substeps).  K = 0 is step()."""
    o = s.copy()
    N = o.N
    bins = np.zeros(N, dtype=np.int32)
    act = C.c_int64()
    dtc = C.c_double(float(dt))
    cnt = counters if counters is not None else Counters()
    rc = _load().gzo_step_hier(N, _p(o.x), _p(o.y), _p(o.z), _p(o.vx), _p(o.vy), _p(o.vz),
                               _p(o.m), _p(o.u), _p(o.H), _p(o.id), C.byref(p), int(K),
                               C.byref(dtc), _p(bins), C.byref(act), C.byref(cnt))
    if rc != 0:
        raise ValueError("step_hier: 0 <= K <= 20, N >= 1")
    return o, dtc.value, bins, int(act.value)


def exchange(x, y, z, ids, m, H, n, vx, vy, vz, u, grad, B, bins, active, D, p: Params | None = None,
             counters: Counters | None = None, with_mass: bool = False):
    """One hierarchical substep's pair exchange (gzo_exchange): returns
    (accp [3,N], accE [N], touched [N]) for the given per-particle arrays."""
    p = p if p is not None else params()
    a = [_f64(v) for v in (x, y, z, m, H, n, vx, vy, vz, u)]
    N = a[0].size
    g = np.ascontiguousarray(grad, dtype=np.float64).reshape(15, N)
    Bm = np.ascontiguousarray(B, dtype=np.float64).reshape(6, N)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    act = np.ascontiguousarray(active, dtype=np.uint8)
    accp = np.zeros((3, N))
    accE = np.zeros(N)
    tch = np.zeros(N, dtype=np.uint8)
    cnt = counters if counters is not None else Counters()
    accm = np.zeros(N)
    _load().gzo_exchange(N, _p(a[0]), _p(a[1]), _p(a[2]), _p(ids), _p(a[3]), _p(a[4]), _p(a[5]),
                         _p(a[6]), _p(a[7]), _p(a[8]), _p(a[9]), _p(g), _p(Bm), _p(bins), _p(act),
                         float(D), C.byref(p), _p(accp), _p(accE), _p(accm), _p(tch), C.byref(cnt))
    return (accp, accE, tch, accm) if with_mass else (accp, accE, tch)


def pair(L: dict, R: dict, dt: float, p: Params):
    """One canonical face (L = lower id); dicts hold x[3], H, n, W[5], g[15], B[6].

    Also returns the face states of O11 (rho, vx, vy, vz, P per side):
    ``pred_L``/``pred_R`` after reconstruction and the Hancock half step,
    ``face_L``/``face_R`` after the clamp (what the Riemann solver sees)."""
    A = np.zeros(3)
    face = np.full(20, np.nan)
    vf = np.zeros(3)
    dp = np.zeros(3)
    ps, ss, dE, dm = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    fl = C.c_int()
    arrs = [_f64(L[k]) for k in ("x", "W", "g", "B")] + [_f64(R[k]) for k in ("x", "W", "g", "B")]
    ok = _load().gzo_pair(_p(arrs[0]), float(L["H"]), float(L["n"]), _p(arrs[1]), _p(arrs[2]),
                          _p(arrs[3]), _p(arrs[4]), float(R["H"]), float(R["n"]), _p(arrs[5]),
                          _p(arrs[6]), _p(arrs[7]), float(dt), C.byref(p), _p(A), C.byref(ps),
                          C.byref(ss), _p(vf), _p(dp), C.byref(dE), C.byref(dm), C.byref(fl),
                          _p(face))
    return {"ok": ok, "A": A, "pstar": ps.value, "sstar": ss.value, "vf": vf, "dp": dp,
            "dE": dE.value, "dm": dm.value, "flags": fl.value, "pred_L": face[0:5],
            "pred_R": face[5:10], "face_L": face[10:15], "face_R": face[15:20]}


def hllc_flux(FL, FR, vf, nh, gamma):
    """MFV face flux: (mass, momentum [3], energy) flux densities, lab frame."""
    Fp = np.zeros(3)
    Fm, FE = C.c_double(), C.c_double()
    a = [_f64(v) for v in (FL, FR, vf, nh)]
    _load().gzo_hllc_flux(_p(a[0]), _p(a[1]), _p(a[2]), _p(a[3]), float(gamma), C.byref(Fm), _p(Fp),
                          C.byref(FE))
    return Fm.value, Fp, FE.value


def hllc(rhoL, uL, PL, rhoR, uR, PR, gamma):
    """O12: returns (S*, P*)."""
    ss, ps = C.c_double(), C.c_double()
    _load().gzo_hllc(rhoL, uL, PL, rhoR, uR, PR, gamma, C.byref(ss), C.byref(ps))
    return ss.value, ps.value


def riemann_star(rhoL, uL, PL, rhoR, uR, PR, gamma):
    """Exact Riemann solver: returns (p*, u*)."""
    ps, us = C.c_double(), C.c_double()
    rc = _load().gzo_riemann_star(rhoL, uL, PL, rhoR, uR, PR, gamma, C.byref(ps), C.byref(us))
    if rc != 0:
        raise ValueError("vacuum generated")
    return ps.value, us.value


def riemann_sample(rhoL, uL, PL, rhoR, uR, PR, gamma, xi):
    """Exact Riemann solution (rho, u, P) at xi = x/t for an array of xi."""
    ps, us = riemann_star(rhoL, uL, PL, rhoR, uR, PR, gamma)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    out = np.zeros((3, xi.size))
    r, u, P = C.c_double(), C.c_double(), C.c_double()
    lib = _load()
    for k, v in enumerate(xi):
        lib.gzo_riemann_sample(rhoL, uL, PL, rhoR, uR, PR, gamma, ps, us, float(v),
                               C.byref(r), C.byref(u), C.byref(P))
        out[:, k] = (r.value, u.value, P.value)
    return out
