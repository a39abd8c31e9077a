"""Writes sedov64_t005.npz: the FP64 oracle's Sedov-Taylor blast advanced to
t = 0.05, the stored reference of the Sedov configuration's comparison
(tests/test_gpu_sedov_config.py).  Calls only the oracle and the seeded input
generator; run from the repository root:

    python tests/golden/make_sedov64.py

Workload: 64^3 = 262,144 jittered-lattice particles, rho = 1, background
P = 1e-6, gamma = 5/3, E = 1 deposited into the 32 particles nearest the
centre (inputs.sedov, seed 1713); global CFL steps (CFL 0.2, the oracle's
default parameters).  When t + 2 dt_previous reaches t = 0.05, each step's
CFL dt is formed from the state first and clipped to 0.05 - t, so the last
step ends at t = 0.05 exactly.

Stored (FP64): the step count and every dt; for a sample of particles (every
64th id and the 256 nearest the centre at t = 0) their ids and x, y, z, vx,
vy, vz, u, H at t = 0.05; the radially binned density (64 shells out to 0.5,
from one density pass on the final state) and the radius of its peak."""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_1712_01294_gb300 import inputs as I  # noqa: E402

T_END = 0.05
NBINS = 64


def sample_ids(p):
    c = np.stack([p.x, p.y, p.z], 1) - 0.5
    near = np.argsort(np.sqrt((c ** 2).sum(1)), kind="stable")[:256]
    return np.union1d(np.flatnonzero(p.id % 64 == 0), p.id[near])


def radial_density(s, n):
    r = np.sqrt((s.x - 0.5) ** 2 + (s.y - 0.5) ** 2 + (s.z - 0.5) ** 2)
    edges = np.linspace(0.0, 0.5, NBINS + 1)
    b = np.clip(np.digitize(r, edges) - 1, 0, NBINS - 1)
    rho = s.m * n
    cnt = np.bincount(b, None, NBINS)
    prof = np.bincount(b, rho, NBINS) / np.maximum(cnt, 1)
    mid = 0.5 * (edges[1:] + edges[:-1])
    return mid, prof, float(mid[int(np.argmax(prof))])


def main(out=os.path.join(HERE, "sedov64_t005.npz")):
    p = I.sedov(64, seed=1713)
    s = O.State.from_any(p.__dict__)
    prm = O.params()
    ids = sample_ids(p)
    t, dts = 0.0, []
    t0 = time.time()
    while t < T_END:
        # the step's own CFL dt, except within reach of the end: then the CFL
        # dt of the current state is formed first and clipped to T_END - t
        dt = 0.0
        if dts and t + 2.0 * dts[-1] >= T_END:
            H, n, _, _ = O.density(s, prm)
            _, dtc = O.timestep(s, H, n, prm)
            dt = min(dtc, T_END - t)
        s, dt_used, _, _, _ = O.step(s, prm, dt=dt)
        t = T_END if dt > 0.0 and dt == T_END - t else t + dt_used
        dts.append(dt_used)
        if len(dts) % 50 == 0:
            print(f"step {len(dts)} t {t:.6f} dt {dt_used:.3e} ({time.time() - t0:.0f} s)", flush=True)
    H, n, _, _ = O.density(s, prm)
    mid, prof, r_peak = radial_density(s, n)
    order = np.argsort(s.id)
    pick = order[ids]
    np.savez_compressed(out, t_end=T_END, steps=len(dts), dt=np.array(dts), ids=ids,
                        **{k: getattr(s, k)[pick] for k in ("x", "y", "z", "vx", "vy", "vz", "u", "H")},
                        shell_r=mid, shell_rho=prof, r_peak=r_peak)
    print(f"wrote {out}: {len(dts)} steps, peak density at r = {r_peak:.4f}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
