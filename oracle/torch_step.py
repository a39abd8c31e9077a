"""The MFM step written a second time in plain PyTorch CPU ops (FP64), for
derivatives: forward-mode dual numbers (torch.autograd.forward_ad) give exact
directional derivatives, reverse mode gives full gradients.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).  Same readings
O1-O14 as ``gz_oracle.c``; its forward values are pinned to that oracle and
its derivatives to central finite differences of it (tests).

Differentiation conventions (the same for the CUDA adjoint):
* neighbour sets and the flux pair set are frozen at their forward values;
* the step dt is a constant (not differentiated through the CFL minimum);
* H is the root of f(H; x) = 0: it enters as H = H* - f(H*; x) / f'(H*; x)
  with the converged H* held constant, whose derivative is the implicit one,
  -(df/dx) / f';
* the u floor value (a multiple of a median) is a constant;
* min/max/clamp pass the derivative of the branch they select; at an exact
  tie (a limited face value equal to its clamp bound, which happens wherever
  the limiter zeroes a gradient) the clamp passes it to the unclamped value.
"""
from __future__ import annotations

import math

import numpy as np
import torch

PI = math.pi


def _w(q):
    t = 1.0 - q
    a = 1.0 - 6.0 * q * q + 6.0 * q * q * q
    b = 2.0 * t * t * t
    return torch.where(q <= 0.5, a, torch.where(q < 1.0, b, torch.zeros_like(q)))


def _dw(q):
    t = 1.0 - q
    a = -12.0 * q + 18.0 * q * q
    b = -6.0 * t * t
    return torch.where(q <= 0.5, a, torch.where(q < 1.0, b, torch.zeros_like(q)))


def W(r, H):
    return 8.0 / (PI * H * H * H) * _w(r / H)


def min_image(d):
    d = torch.where(d >= 0.5, d - 1.0, d)
    return torch.where(d < -0.5, d + 1.0, d)


def dense_lists(off, nbr, N):
    """CSR lists -> padded [N, K] index tensor (pad = -1) and mask."""
    cnt = np.diff(off)
    K = int(cnt.max()) if N else 0
    idx = -np.ones((N, max(K, 1)), dtype=np.int64)
    for i in range(N):
        idx[i, :cnt[i]] = nbr[off[i]:off[i + 1]]
    t = torch.as_tensor(idx)
    return t.clamp(min=0), t >= 0


def canonical_pairs(off, nbr, ids):
    """Unordered flux pairs (L, R) with id_L < id_R from the ordered CSR pair lists."""
    L, R = [], []
    for i in range(len(off) - 1):
        for j in nbr[off[i]:off[i + 1]]:
            if ids[i] < ids[j]:
                L.append(i)
                R.append(int(j))
    return torch.as_tensor(L, dtype=torch.long), torch.as_tensor(R, dtype=torch.long)


class Frozen:
    """Everything the differentiated step holds fixed: converged H*, neighbour
    lists N_i(H*), the flux pair set and dt."""

    def __init__(self, Hstar, nb, nbmask, pL, pR, dt):
        self.Hstar = torch.as_tensor(Hstar, dtype=torch.float64)
        self.nb, self.nbmask, self.pL, self.pR, self.dt = nb, nbmask, pL, pR, float(dt)


def offsets(x, y, z, a, b):
    """d = x_b - x_a (min image) for index tensors a, b."""
    return (min_image(x[b] - x[a]), min_image(y[b] - y[a]), min_image(z[b] - z[a]))


def step(state, fr: Frozen, gamma=5.0 / 3.0, ngb=32.0, beta=1.0, hancock=True,
         u_floor=None, return_all=False):
    """One MFM step.  state: dict of FP64 tensors x y z vx vy vz m u (N each)."""
    x, y, z = state["x"], state["y"], state["z"]
    vx, vy, vz, m, u = state["vx"], state["vy"], state["vz"], state["m"], state["u"]
    N = x.shape[0]
    nb, mk = fr.nb, fr.nbmask
    ii = torch.arange(N).unsqueeze(1).expand_as(nb)
    dx, dy, dz = offsets(x, y, z, ii, nb)
    r2 = (dx * dx + dy * dy) + dz * dz
    r = torch.sqrt(torch.where(mk, r2, torch.ones_like(r2)))
    # O4: implicit H through one Newton correction at the converged root
    Hs = fr.Hstar
    q0 = r / Hs.unsqueeze(1)
    n0 = W(torch.zeros_like(Hs), Hs) + torch.where(mk, W(r, Hs.unsqueeze(1)), 0.0).sum(1)
    f = 4.0 * PI / 3.0 * Hs ** 3 * n0 - ngb
    fp = (4.0 * PI / 3.0) * (8.0 / PI) * torch.where(mk, -_dw(q0) * q0 / Hs.unsqueeze(1), 0.0).sum(1)
    H = Hs - f / fp
    # O5
    Hb = H.unsqueeze(1)
    Wn = torch.where(mk, W(r, Hb), 0.0)
    n = W(torch.zeros_like(H), H) + Wn.sum(1)
    rho = m * n
    P = (gamma - 1.0) * rho * u
    prim = [rho, vx, vy, vz, P]
    # O6-O8
    psi = Wn / n.unsqueeze(1)
    E = [(psi * dx * dx).sum(1), (psi * dx * dy).sum(1), (psi * dx * dz).sum(1),
         (psi * dy * dy).sum(1), (psi * dy * dz).sum(1), (psi * dz * dz).sum(1)]
    a, b, c, d, e, ff = E
    Cxx, Cxy, Cxz = d * ff - e * e, c * e - b * ff, b * e - c * d
    Cyy, Cyz, Czz = a * ff - c * c, b * c - a * e, a * d - b * b
    det = a * Cxx + b * Cxy + c * Cxz
    B = [Cxx / det, Cxy / det, Cxz / det, Cyy / det, Cyz / det, Czz / det]
    g = []
    for fld in prim:
        df = torch.where(mk, fld[nb] - fld.unsqueeze(1), 0.0)
        S = [(df * dx * psi).sum(1), (df * dy * psi).sum(1), (df * dz * psi).sum(1)]
        g.append([B[0] * S[0] + B[1] * S[1] + B[2] * S[2],
                  B[1] * S[0] + B[3] * S[1] + B[4] * S[2],
                  B[2] * S[0] + B[4] * S[1] + B[5] * S[2]])
    # O9 limiter
    s_ij = Hb / (Hb + H[nb])
    gl = []
    for q, fld in enumerate(prim):
        fn = fld[nb]
        big = torch.finfo(torch.float64).max
        fmax = torch.maximum(fld, torch.where(mk, fn, -big).max(1).values)
        fmin = torch.minimum(fld, torch.where(mk, fn, big).min(1).values)
        D = (g[q][0].unsqueeze(1) * (s_ij * dx) + g[q][1].unsqueeze(1) * (s_ij * dy)) + \
            g[q][2].unsqueeze(1) * (s_ij * dz)
        Ds = torch.where(D == 0, torch.ones_like(D), D)
        up = torch.minimum(torch.ones_like(D), beta * (fmax - fld).unsqueeze(1) / Ds)
        dn = torch.minimum(torch.ones_like(D), beta * (fmin - fld).unsqueeze(1) / Ds)
        aij = torch.where(D > 0, up, torch.where(D < 0, dn, torch.ones_like(D)))
        aij = torch.where(mk, aij, torch.ones_like(aij))
        alpha = torch.minimum(torch.ones_like(fld), aij.min(1).values)
        gl.append([alpha * g[q][k] for k in range(3)])
    # O10-O12 over unordered pairs in canonical order
    dp, dE = flux_stage(x, y, z, prim, H, n, gl, B, fr.pL, fr.pR, fr.dt, gamma, hancock)
    # O14
    dt = fr.dt
    px = m * vx + dt * dp[0]
    py = m * vy + dt * dp[1]
    pz = m * vz + dt * dp[2]
    v2 = (vx * vx + vy * vy) + vz * vz
    En = m * (u + 0.5 * v2) + dt * dE
    nx, ny, nz = px / m, py / m, pz / m

    def wrap(v):
        v = torch.where(v < 0, v + 1.0, v)
        return torch.where(v >= 1.0, v - 1.0, v)
    out = {"x": wrap(x + dt * (0.5 * (vx + nx))), "y": wrap(y + dt * (0.5 * (vy + ny))),
           "z": wrap(z + dt * (0.5 * (vz + nz))), "vx": nx, "vy": ny, "vz": nz}
    un = En / m - 0.5 * ((nx * nx + ny * ny) + nz * nz)
    if u_floor is not None:
        un = torch.where(un > 0, un, torch.full_like(un, float(u_floor)))
    out["u"] = un
    if return_all:
        out.update({"H": H, "n": n, "dpdt": torch.stack(dp), "dEdt": dE,
                    "grad": torch.stack([gl[q][k] for q in range(5) for k in range(3)]),
                    "B": torch.stack(B)})
    return out


def flux_stage(x, y, z, prim, H, n, gl, B, L, R, dt, gamma=5.0 / 3.0, hancock=True):
    """O10-O12: rates dp/dt (list of 3) and dE/dt over the unordered canonical
    pairs (L, R), given primitives prim = [rho, vx, vy, vz, P], support radii
    H, densities n, limited gradients gl[field][axis] and B (6 components)."""
    N = x.shape[0]
    pdx, pdy, pdz = offsets(x, y, z, L, R)
    pr2 = (pdx * pdx + pdy * pdy) + pdz * pdz
    pr = torch.sqrt(pr2)
    HL, HR, nL, nR = H[L], H[R], n[L], n[R]
    psiRL = torch.where(pr2 < HL * HL, W(pr, HL) / nL, 0.0)
    psiLR = torch.where(pr2 < HR * HR, W(pr, HR) / nR, 0.0)
    VL, VR = 1.0 / nL, 1.0 / nR

    def Bd(idx):
        return [B[0][idx] * pdx + B[1][idx] * pdy + B[2][idx] * pdz,
                B[1][idx] * pdx + B[3][idx] * pdy + B[4][idx] * pdz,
                B[2][idx] * pdx + B[4][idx] * pdy + B[5][idx] * pdz]
    BLd, BRd = Bd(L), Bd(R)
    A = [VL * psiRL * BLd[k] + VR * psiLR * BRd[k] for k in range(3)]
    Am = torch.sqrt((A[0] * A[0] + A[1] * A[1]) + A[2] * A[2])
    ok = Am > 0
    Ams = torch.where(ok, Am, torch.ones_like(Am))
    nh = [A[k] / Ams for k in range(3)]
    s = HL / (HL + HR)
    sR = HR / (HL + HR)
    vf = [prim[1 + k][L] + s * (prim[1 + k][R] - prim[1 + k][L]) for k in range(3)]
    sdL = [s * pdx, s * pdy, s * pdz]
    sdR = [sR * -pdx, sR * -pdy, sR * -pdz]
    FL, FR = [], []
    for q in range(5):
        FL.append(prim[q][L] + ((gl[q][0][L] * sdL[0] + gl[q][1][L] * sdL[1]) + gl[q][2][L] * sdL[2]))
        FR.append(prim[q][R] + ((gl[q][0][R] * sdR[0] + gl[q][1][R] * sdR[1]) + gl[q][2][R] * sdR[2]))
    if hancock:
        h = 0.5 * dt
        divL = (gl[1][0][L] + gl[2][1][L]) + gl[3][2][L]
        divR = (gl[1][0][R] + gl[2][1][R]) + gl[3][2][R]
        FL[0] = FL[0] + h * (-prim[0][L] * divL)
        FR[0] = FR[0] + h * (-prim[0][R] * divR)
        for k in range(3):
            FL[1 + k] = FL[1 + k] + h * (-gl[4][k][L] / prim[0][L])
            FR[1 + k] = FR[1 + k] + h * (-gl[4][k][R] / prim[0][R])
        FL[4] = FL[4] + h * (-gamma * prim[4][L] * divL)
        FR[4] = FR[4] + h * (-gamma * prim[4][R] * divR)
    for q in range(5):
        # clamp as v < lo ? lo : (v > hi ? hi : v): at a tie the derivative
        # follows v (min/max of torch would split it between the branches)
        lo = torch.where(prim[q][L] <= prim[q][R], prim[q][L], prim[q][R])
        hi = torch.where(prim[q][L] >= prim[q][R], prim[q][L], prim[q][R])
        FL[q] = torch.where(FL[q] < lo, lo, torch.where(FL[q] > hi, hi, FL[q]))
        FR[q] = torch.where(FR[q] < lo, lo, torch.where(FR[q] > hi, hi, FR[q]))
    bad = (FL[0] <= 0) | (FL[4] <= 0) | (FR[0] <= 0) | (FR[4] <= 0)
    for q in range(5):
        FL[q] = torch.where(bad, prim[q][L], FL[q])
        FR[q] = torch.where(bad, prim[q][R], FR[q])
    vfn = (vf[0] * nh[0] + vf[1] * nh[1]) + vf[2] * nh[2]
    uL = ((FL[1] - vf[0]) * nh[0] + (FL[2] - vf[1]) * nh[1]) + (FL[3] - vf[2]) * nh[2]
    uR = ((FR[1] - vf[0]) * nh[0] + (FR[2] - vf[1]) * nh[1]) + (FR[3] - vf[2]) * nh[2]
    rL, PL, rR, PR = FL[0], FL[4], FR[0], FR[4]
    cL = torch.sqrt(gamma * PL / rL)
    cR = torch.sqrt(gamma * PR / rR)
    SL = torch.where(uL - cL <= uR - cR, uL - cL, uR - cR)
    SR = torch.where(uL + cL >= uR + cR, uL + cL, uR + cR)
    num = PR - PL + rL * uL * (SL - uL) - rR * uR * (SR - uR)
    den = rL * (SL - uL) - rR * (SR - uR)
    ss = num / den
    ps = torch.clamp(PL + rL * (SL - uL) * (ss - uL), min=0.0)
    ps = torch.where(ok, ps, 0.0)
    Fp = [-ps * A[k] for k in range(3)]
    FE = -ps * (ss + vfn) * Am
    dp = [torch.zeros(N, dtype=torch.float64).index_add(0, L, Fp[k]).index_add(0, R, -Fp[k])
          for k in range(3)]
    dE = torch.zeros(N, dtype=torch.float64).index_add(0, L, FE).index_add(0, R, -FE)
    return dp, dE


def freeze(state_np, params, use_cells=1):
    """Converged H* (the C oracle's h-iteration), lists and pairs, and the CFL dt."""
    import oracle as O
    s = O.State.from_any(state_np)
    Hs, n, it, f = O.density(s, params)
    off, nbr = O.neighbours(s, Hs, use_cells=use_cells)
    nb, mk = dense_lists(off, nbr, s.N)
    poff, pnb = O.flux_pairs(s, Hs, use_cells=use_cells)
    L, R = canonical_pairs(poff, pnb, s.id)
    _, dt = O.timestep(s, Hs, n, params)
    return Frozen(Hs, nb, mk, L, R, dt), s, Hs, n


def as_tensors(s, requires_grad=False):
    keys = ("x", "y", "z", "vx", "vy", "vz", "m", "u")
    return {k: torch.tensor(np.asarray(getattr(s, k)), dtype=torch.float64,
                            requires_grad=requires_grad) for k in keys}
