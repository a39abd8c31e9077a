"""Seeded synthetic particle sets for the MFM hot path.

This module generates inputs only: it holds none of the hydrodynamics step's
arithmetic and imports nothing else from this package, so both the CUDA path
and the FP64 CPU oracle can be fed the same arrays.  Every generator is
deterministic in its seed (numpy PCG64).

Workloads (periodic unit box, gamma = 5/3, N_ngb = 32):

* ``sod``        -- jittered cubic lattice, Sod split at x = 1/2 realised through
  particle masses (left rho = 1, P = 1; right rho = 0.125, P = 0.1), v = 0.
* ``sedov``      -- jittered lattice, rho = 1, P = 1e-6, energy E deposited into
  the 32 particles nearest the centre with cubic-spline weights of radius equal
  to the distance of the 33rd nearest.
* ``turbulence`` -- jittered lattice; solenoidal Gaussian velocity field with
  per-mode power |v_k|^2 ~ k^-4 on integer wavenumbers 2 <= |k| <= 16, scaled
  to rms Mach 0.5; log-normal density (sigma_lnrho = 0.3, same spectrum shape,
  independent seed) realised through masses; uniform P = 1.
* ``kh``         -- Kelvin-Helmholtz shear layer: rho = 2, vx = +0.5 inside
  |y - 1/2| < 1/4, rho = 1, vx = -0.5 outside, P = 2.5, and
  vy = 0.01 sin(4 pi (x + phi)) with a seeded phase phi.
* ``ensemble``   -- independent boxes of n^3 particles, n uniform in 8..24,
  each a Sod (density ratio 2-10, pressure ratio 2-20) or Sedov (E in 0.1-1)
  setup chosen with probability 1/2.

Lattice points sit at (k + 1/2)/n with a uniform jitter in [-0.1, 0.1]/n per
axis.  The initial support radius is H0 = (3 N_ngb / (4 pi N))^(1/3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 5.0 / 3.0
NGB = 32.0
FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "u", "H")


@dataclass
class Particles:
    """Structure-of-arrays particle set (FP64 on the host)."""
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
    counts: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int64))
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.x.shape[0])

    def copy(self) -> "Particles":
        return Particles(*(np.array(getattr(self, k)) for k in FIELDS + ("id", "counts")),
                         meta=dict(self.meta))

    def box(self, b: int) -> "Particles":
        """Particles of box b of a batched set (contiguous slice)."""
        off = np.concatenate([[0], np.cumsum(self.counts)])
        s = slice(int(off[b]), int(off[b + 1]))
        return Particles(*(np.array(getattr(self, k)[s]) for k in FIELDS + ("id",)),
                         counts=np.array([off[b + 1] - off[b]], dtype=np.int64),
                         meta=dict(self.meta))


def h0(N: int, ngb: float = NGB) -> float:
    """Initial support radius for N particles in the unit box."""
    return (3.0 * ngb / (4.0 * math.pi * N)) ** (1.0 / 3.0)


def lattice(n: int, rng: np.random.Generator, jitter: float = 0.1):
    """Jittered cubic lattice of n^3 points; returns x, y, z and lattice indices."""
    k = np.arange(n, dtype=np.float64)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    base = np.stack([kx.ravel(), ky.ravel(), kz.ravel()])
    jit = rng.uniform(-jitter, jitter, size=base.shape)
    pos = (base + 0.5 + jit) / n
    pos = np.where(pos < 0.0, pos + 1.0, pos)
    pos = np.where(pos >= 1.0, pos - 1.0, pos)
    return pos[0], pos[1], pos[2], base.astype(np.int64)


def _finish(x, y, z, vx, vy, vz, m, u, ngb=NGB, id0=0, meta=None) -> Particles:
    N = x.shape[0]
    H = np.full(N, h0(N, ngb))
    ids = np.arange(id0, id0 + N, dtype=np.int64)
    return Particles(x, y, z, vx, vy, vz, m, u, H, ids,
                     counts=np.array([N], dtype=np.int64), meta=meta or {})


def sod(n: int = 32, seed: int = 1712, gamma: float = GAMMA, rho_l=1.0, p_l=1.0, rho_r=0.125,
        p_r=0.1, jitter: float = 0.1, u_l: float = 0.0, u_r: float = 0.0) -> Particles:
    """Shock tube along x: (rho_l, p_l, u_l) for x < 1/2, (rho_r, p_r, u_r) above
    (u = x-velocity; u_l = -2, u_r = 2, rho = 1, p = 0.4 gives the strong double
    rarefaction at x = 1/2 and, through the periodic wrap, a collision at x = 0)."""
    rng = np.random.default_rng(seed)
    x, y, z, _ = lattice(n, rng, jitter)
    N = x.size
    left = x < 0.5
    rho = np.where(left, rho_l, rho_r)
    P = np.where(left, p_l, p_r)
    m = rho / N
    u = P / ((gamma - 1.0) * rho)
    zero = np.zeros(N)
    vx = np.where(left, u_l, u_r).astype(np.float64)
    return _finish(x, y, z, vx, zero.copy(), zero.copy(), m, u,
                   meta=dict(kind="sod", n=n, seed=seed, rho_l=rho_l, p_l=p_l, rho_r=rho_r,
                             p_r=p_r, gamma=gamma, u_l=u_l, u_r=u_r))


def _deposit_weights(r: np.ndarray, R: float) -> np.ndarray:
    """Cubic-spline shaped weights of radius R (input recipe only)."""
    q = r / R
    w = np.where(q <= 0.5, 1.0 - 6.0 * q ** 2 + 6.0 * q ** 3,
                 np.where(q < 1.0, 2.0 * (1.0 - q) ** 3, 0.0))
    return w / w.sum()


def sedov(n: int = 64, seed: int = 1713, gamma: float = GAMMA, E: float = 1.0,
          p_bg: float = 1e-6, rho: float = 1.0, jitter: float = 0.1, nblast: int = 32) -> Particles:
    rng = np.random.default_rng(seed)
    x, y, z, _ = lattice(n, rng, jitter)
    N = x.size
    m = np.full(N, rho / N)
    u = np.full(N, p_bg / ((gamma - 1.0) * rho))
    r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
    ids = np.arange(N)
    order = np.lexsort((ids, r))  # by distance, ties by id
    near = order[:nblast]
    Rc = r[order[nblast]]
    w = _deposit_weights(r[near], Rc)
    u[near] += w * E / m[near]
    zero = np.zeros(N)
    return _finish(x, y, z, zero, zero.copy(), zero.copy(), m, u,
                   meta=dict(kind="sedov", n=n, seed=seed, E=E, p_bg=p_bg, rho=rho, gamma=gamma))


def _kvec(n: int):
    k = np.fft.fftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    return kx, ky, kz


def gaussian_field(n: int, rng: np.random.Generator, kmin=2.0, kmax=16.0, slope=-4.0,
                   ncomp: int = 1, solenoidal: bool = False) -> np.ndarray:
    """Real Gaussian random field(s) on an n^3 grid with per-mode power k^slope on
    kmin <= |k| <= kmax (integer wavenumbers), zero mean.  Shape (ncomp, n, n, n)."""
    kx, ky, kz = _kvec(n)
    k2 = kx * kx + ky * ky + kz * kz
    kk = np.sqrt(k2)
    band = (kk >= kmin) & (kk <= kmax)
    amp = np.zeros_like(kk)
    amp[band] = kk[band] ** (slope / 2.0)
    comps = []
    for _ in range(ncomp):
        white = rng.standard_normal((n, n, n))
        comps.append(np.fft.fftn(white) * amp)
    if solenoidal:
        vx, vy, vz = comps
        k2s = np.where(k2 > 0, k2, 1.0)
        kd = (kx * vx + ky * vy + kz * vz) / k2s
        comps = [vx - kx * kd, vy - ky * kd, vz - kz * kd]
    out = np.stack([np.real(np.fft.ifftn(c)) for c in comps])
    return out - out.mean(axis=(1, 2, 3), keepdims=True)


def turbulence(n: int = 128, seed: int = 1714, gamma: float = GAMMA, mach: float = 0.5,
               sigma_lnrho: float = 0.3, P: float = 1.0, jitter: float = 0.1) -> Particles:
    rng = np.random.default_rng(seed)
    x, y, z, idx = lattice(n, rng, jitter)
    N = x.size
    vrng = np.random.default_rng(seed + 1_000_003)
    drng = np.random.default_rng(seed + 2_000_003)
    v = gaussian_field(n, vrng, ncomp=3, solenoidal=True)
    g = gaussian_field(n, drng, ncomp=1)[0]
    g *= sigma_lnrho / g.std()
    c0 = math.sqrt(gamma * P / 1.0)
    vrms = math.sqrt(float(np.mean(v[0] ** 2 + v[1] ** 2 + v[2] ** 2)))
    v *= mach * c0 / vrms
    ix, iy, iz = idx
    vx = v[0][iz, iy, ix]
    vy = v[1][iz, iy, ix]
    vz = v[2][iz, iy, ix]
    rho = np.exp(g[iz, iy, ix] - 0.5 * sigma_lnrho ** 2)
    rho /= rho.mean()
    m = rho / N
    u = P / ((gamma - 1.0) * rho)
    return _finish(x, y, z, vx, vy, vz, m, u,
                   meta=dict(kind="turbulence", n=n, seed=seed, mach=mach,
                             sigma_lnrho=sigma_lnrho, gamma=gamma))


def kh(n: int = 64, seed: int = 1715, gamma: float = GAMMA, amp: float = 0.01,
       jitter: float = 0.1, smooth: float = 0.0) -> Particles:
    """Kelvin-Helmholtz layer.  smooth > 0 gives the differentiable variant:
    tanh interfaces of that width, and 1 % smooth modulations of P and vz so
    that no field is exactly uniform (a uniform field is a kink of the slope
    limiter, where the step has no derivative)."""
    rng = np.random.default_rng(seed)
    x, y, z, _ = lattice(n, rng, jitter)
    N = x.size
    phi = float(rng.uniform(0.0, 1.0))
    if smooth > 0.0:
        inside = 0.5 * (np.tanh((y - 0.25) / smooth) - np.tanh((y - 0.75) / smooth))
    else:
        inside = (np.abs(y - 0.5) < 0.25).astype(np.float64)
    rho = 1.0 + inside
    vx = -0.5 + inside
    vy = amp * np.sin(4.0 * math.pi * (x + phi))
    vz = np.zeros(N)
    P = np.full(N, 2.5)
    if smooth > 0.0:
        P = P * (1.0 + 0.01 * np.sin(2 * math.pi * (x + 2 * z)) * np.cos(2 * math.pi * y))
        vz = 0.01 * np.sin(2 * math.pi * (y - z + phi))
    m = rho / N
    u = P / ((gamma - 1.0) * rho)
    return _finish(x, y, z, vx, vy, vz, m, u,
                   meta=dict(kind="kh", n=n, seed=seed, phi=phi, gamma=gamma, smooth=smooth))


def smooth_turbulence(n: int = 16, seed: int = 1717, gamma: float = GAMMA) -> Particles:
    """Turbulent box whose pressure carries a smooth 10 % modulation, so every
    field varies smoothly (no limiter kink from an exactly uniform field)."""
    p = turbulence(n, seed=seed, gamma=gamma)
    mod = 1.0 + 0.1 * np.sin(2 * math.pi * p.x) * np.cos(2 * math.pi * p.y + 0.3) + \
        0.05 * np.sin(2 * math.pi * (p.z + p.x))
    p.u = p.u * mod
    p.meta["kind"] = "smooth_turbulence"
    return p


def ensemble(nboxes: int = 256, seed: int = 1716, nmin: int = 8, nmax: int = 24,
             gamma: float = GAMMA) -> Particles:
    """Independent boxes concatenated box by box; ``counts`` gives the sizes."""
    rng = np.random.default_rng(seed)
    parts = []
    kinds = []
    id0 = 0
    for b in range(nboxes):
        n = int(rng.integers(nmin, nmax + 1))
        s = int(rng.integers(0, 2**31 - 1))
        if rng.uniform() < 0.5:
            dr = float(rng.uniform(2.0, 10.0))
            pr = float(rng.uniform(2.0, 20.0))
            p = sod(n, seed=s, gamma=gamma, rho_l=1.0, p_l=1.0, rho_r=1.0 / dr, p_r=1.0 / pr)
            kinds.append(("sod", dr, pr))
        else:
            E = float(rng.uniform(0.1, 1.0))
            p = sedov(n, seed=s, gamma=gamma, E=E)
            kinds.append(("sedov", E))
        p.id += id0
        id0 += p.N
        parts.append(p)
    cat = {k: np.concatenate([getattr(p, k) for p in parts]) for k in FIELDS + ("id",)}
    counts = np.array([p.N for p in parts], dtype=np.int64)
    return Particles(*(cat[k] for k in FIELDS + ("id",)), counts=counts,
                     meta=dict(kind="ensemble", nboxes=nboxes, seed=seed, boxes=kinds,
                               gamma=gamma))


WORKLOADS = {
    "sod32": lambda: sod(32, seed=1712),
    "sedov64": lambda: sedov(64, seed=1713),
    "turb128": lambda: turbulence(128, seed=1714),
    "kh64": lambda: kh(64, seed=1715),
    "kh64_smooth": lambda: kh(64, seed=1715, smooth=0.05),
    "ensemble256": lambda: ensemble(256, seed=1716),
}
