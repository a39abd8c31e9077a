// Hydro passes of the MFM step in sorted particle order (steps S2-S6).
// One thread per particle; neighbour lists are stored in groups of four
// slots across the particles (lslot), so a warp reads one group of its lists
// as contiguous bytes.  Every pair quantity that mixes both particles of a
// pair is either symmetric in its operands or evaluated in one fixed order of
// the pair (pair_order), so both particles get bitwise-opposite
// contributions (no atomics on rates).
#include <algorithm>
#include <type_traits>

#include "gz_device.cuh"
#include "gz_launch.cuh"

namespace gz {

namespace {

inline int blocks(int n, int t) { return (n + t - 1) / t; }

// --------------------------------------------------------------- O4 / O5
// Bracketed Newton iteration on f(H) = (4 pi/3) H^3 n(H) - N_ngb, written as
// (32/3)(1 + sum_j w(q_j)) - N_ngb with f' = (32/3) sum_j (-w'(q_j)) q_j / H.
// The first evaluation scans the cells once with radius Rc = 1.05 H and keeps
// (r^2, j) of the candidates inside Rc in shared memory; later evaluations
// read only that cache (rebuilt if H grows past Rc).  A particle with more
// than kDensCache candidates falls back to scanning the cells at every
// evaluation.  The neighbour list of the returned H is written at the end.
constexpr int kDensBlock = 64;
// Cache entries per thread: 40 (the largest count within 1.05 H seen on the
// workloads with N_ngb = 32) for boxes of 32^3 particles or more, where the
// smaller cache buys occupancy; 48 for smaller boxes, whose strong contrasts
// (blasts in a few thousand particles) overflow 40 more often.
constexpr int kDensCacheLarge = 40, kDensCacheSmall = 48;

// Radius of the candidate cache for a support Ht: 5% headroom so that small
// growth of H during the iteration needs no rescan, never past h_lim.
template <typename T>
__device__ __forceinline__ T dens_cache_radius(T Ht, const KParams& p) {
    T R = Ht * T(1.05);
    if (!(R < (T)p.h_lim)) R = max(Ht, (T)p.h_lim);
    return R;
}

// Rescan into the thread's shared-memory cache (the support grew past the
// cache radius): kept out of line so that the iteration loop holds no scan
// state; returns the number of candidates within R.
template <typename T, int kDensCache>
__device__ __noinline__ int dens_fill(const Grid& g, const BoxInfo& bx, const P4<T>* __restrict__ pos, int i,
                                      T xi, T yi, T zi, T R, T (*c_r2)[kDensBlock],
                                      unsigned (*c_j)[kDensBlock], int t) {
    const T R2 = R * R;
    int n = 0;
    for_candidates<T>(g, bx, pos, i, xi, yi, zi, R, [&](int j, T, T, T, T r2) {
        if (r2 < R2) {
            if (n < kDensCache) {
                c_r2[n][t] = r2;
                c_j[n][t] = (unsigned)j;
            }
            ++n;
        }
    });
    return n;
}

// One evaluation straight from the cells (more candidates than the cache
// holds and no deferral): the sums and the neighbour list of Ht.
template <typename T>
__device__ __noinline__ void dens_eval_cells(const Grid& g, const BoxInfo& bx, const P4<T>* __restrict__ pos,
                                             int i, T xi, T yi, T zi, T Ht, unsigned* __restrict__ col, int cap,
                                             int N, Acc<T>& sw, T& sd, int& c) {
    const T H2 = Ht * Ht;
    const T iH = T(1) / Ht;
    for_candidates<T>(g, bx, pos, i, xi, yi, zi, Ht, [&](int j, T, T, T, T r2) {
        if (r2 < H2) {
            const T q = psqrt(r2) * iH;
            T w, qdw;
            dens_terms(q, w, qdw);
            sw.add(w);
            sd += qdw;
            if (c < cap) store_slot(col + lcol(c, N), (unsigned)j);
            ++c;
        }
    });
}

// FP32: held to 96 registers (10 blocks of 64 per SM; the cache of 40 allows
// 10 to 11), which measured faster than 119 unspilled registers at 8 blocks.
template <typename T, int kDensCache>
__global__ void __launch_bounds__(kDensBlock, sizeof(T) == 4 ? 10 : 1)
    k_density(int N, Sorted<T> s, Grid g, KParams p, unsigned* __restrict__ nbr,
              int* __restrict__ ncount, int* __restrict__ iters, DevStatus* st,
              const int* __restrict__ list, const int* __restrict__ nlist, int* __restrict__ defer,
              int* __restrict__ ndefer) {
    __shared__ T c_r2[kDensCache][kDensBlock];
    __shared__ unsigned c_j[kDensCache][kDensBlock];
    const int t = threadIdx.x;
    int i = blockIdx.x * kDensBlock + t;
    if (list) {  // the particles of an index list only (hierarchical steps)
        if (i >= *nlist) return;
        i = list[i];
    } else if (i >= N) {
        return;
    }
    const BoxInfo bx = g.boxes[s.box[i]];
    const P4<T> me = s.pos[i];
    const T xi = me.x, yi = me.y, zi = me.z;
    double H = (double)s.h[i];
    if (!(H > 0.0) || !(H < p.h_lim)) {
        set_status(st, GZ_S_NONFINITE, GZ_C_NONFINITE, s.id[i]);
        H = cbrt(3.0 * p.ngb / (4.0 * kPi * (double)bx.count));
        if (!(H < p.h_lim)) H = 0.5 * p.h_lim;
    }
    // the cache of the starting H, scanned before the iteration (few live
    // values here, the iteration's FP64 state not yet among them)
    T Rc;
    int ncache;
    bool cached;
    {
        Rc = dens_cache_radius<T>((T)H, p);
        const T R2 = Rc * Rc;
        int n = 0;
        for_candidates<T>(g, bx, s.pos, i, xi, yi, zi, Rc, [&](int j, T, T, T, T r2) {
            if (r2 < R2) {
                if (n < kDensCache) {
                    c_r2[n][t] = r2;
                    c_j[n][t] = (unsigned)j;
                }
                ++n;
            }
        });
        ncache = n;
        cached = n <= kDensCache;
        if (!cached && defer) {
            // more candidates than the cache holds (a support spanning many
            // cells): left to k_density_warp, where a whole warp scans for
            // it and runs the iteration from the starting H
            defer[atomicAdd(ndefer, 1)] = i;
            return;
        }
    }
    const double C = 32.0 / 3.0;
    double lo = 0.0, hi = 0.0, S = 0.0, Hev = H;
    bool has_lo = false, has_hi = false, conv = false, clamped = false;
    T sd_last = T(0);
    int it, cnt = 0;
    for (it = 1; it <= p.max_iter; ++it) {
        const T Ht = (T)H;
        const T H2 = Ht * Ht;
        const T iH = T(1) / Ht;
        if (!cached || Ht > Rc) {  // grew past the cache radius: rescan
            Rc = dens_cache_radius<T>(Ht, p);
            ncache = dens_fill<T, kDensCache>(g, bx, s.pos, i, xi, yi, zi, Rc, c_r2, c_j, t);
            cached = ncache <= kDensCache;
            if (!cached && defer) {
                defer[atomicAdd(ndefer, 1)] = i;
                return;
            }
        }
        Acc<T> sw;
        T sd = T(0);
        int c = 0;
        if (cached) {
            for (int k = 0; k < ncache; ++k) {
                const T r2 = c_r2[k][t];
                if (r2 < H2) {
                    const T q = psqrt(r2) * iH;
                    T w, qdw;
                    dens_terms(q, w, qdw);
                    sw.add(w);
                    sd += qdw;
                    ++c;
                }
            }
        } else {
            dens_eval_cells<T>(g, bx, s.pos, i, xi, yi, zi, Ht, nbr + 4 * (size_t)i, p.cap, N, sw, sd, c);
        }
        cnt = c;
        sd_last = sd;
        Hev = (double)Ht;
        // f = (32/3)(1 + S) - N_ngb.  FP32 path: in FP32 (its rounding, about
        // 4e-6, is well inside the stop tolerance 1e-6 N_ngb); H, the bracket
        // and the update below stay FP64
        double f;
        if constexpr (std::is_same<T, float>::value) {
            const float Sf = sw.fvalue();
            S = (double)Sf;
            f = (double)((32.f / 3.f) * (1.f + Sf) - (float)p.ngb);
        } else {
            S = sw.value();
            f = C * (1.0 + S) - p.ngb;
        }
        if (fabs(f) <= p.tol * p.ngb) {
            conv = true;
            break;
        }
        if (it == p.max_iter) break;
        if (f < 0.0) {
            lo = Hev;
            has_lo = true;
        } else {
            hi = Hev;
            has_hi = true;
        }
        const double lo_eff = has_lo ? lo : 0.5 * Hev;
        const double hi_eff = has_hi ? hi : 2.0 * Hev;
        double Hn = 0.0;
        bool ok = false;
        // Newton step H - f / f' with f' = C sd / H.  H and the update stay
        // FP64; on the FP32 path the quotient f / f' (only its leading digits
        // matter to the step) is formed in FP32, sparing two FP64 divisions
        // an iteration on a part whose FP64 rate is 1/64 of FP32.
        if (std::is_same<T, float>::value) {
            const float fpf = (float)C * (float)sd / Ht;
            if (fpf > 0.f) {
                Hn = Hev - (double)((float)f / fpf);
                ok = (Hn > lo_eff) && (Hn < hi_eff);
            }
        } else {
            const double fp = C * (double)sd / Hev;
            if (fp > 0.0) {
                Hn = Hev - f / fp;
                ok = (Hn > lo_eff) && (Hn < hi_eff);
            }
        }
        if (!ok) Hn = (has_lo && has_hi) ? 0.5 * (lo + hi) : (f < 0.0 ? 2.0 * Hev : 0.5 * Hev);
        if (Hn >= p.h_lim) {
            Hn = 0.5 * (Hev + p.h_lim);
            clamped = true;
        }
        H = Hn;
    }
    if (it > p.max_iter) it = p.max_iter;
    if (cached) {  // list of the returned H, in scan order
        const T Ht = (T)Hev;
        const T H2 = Ht * Ht;
        int c = 0;
        for (int k = 0; k < ncache; ++k) {
            if (c_r2[k][t] < H2) {
                if (c < p.cap) store_slot(nbr + lslot(c, i, N), c_j[k][t]);
                ++c;
            }
        }
    }
    s.h[i] = (T)Hev;
    if (std::is_same<T, float>::value) {  // FP32 path: no FP64 division per particle
        const float Hf = (float)Hev;
        s.n[i] = (T)(8.f * (float)(1.0 + S) / ((float)kPi * Hf * Hf * Hf));
    } else {
        s.n[i] = (T)(8.0 * (1.0 + S) / (kPi * Hev * Hev * Hev));
    }
    if (s.sd) s.sd[i] = sd_last;  // (absent in the allocation-free density call)
    iters[i] = it;
    ncount[i] = cnt;
    if (!conv) {
        set_status(st, GZ_S_HCONV, GZ_C_HCONV, s.id[i]);
        if (clamped) atomicOr(&st->bits, GZ_S_HLIM);
    }
    if (cnt > p.cap) set_status(st, GZ_S_NBR_OVERFLOW, GZ_C_NBR_OVERFLOW, s.id[i]);
}

// The particles k_density deferred (more candidates within 1.05 H than its
// cache holds): one warp per particle, the same bracketed Newton iteration,
// each evaluation a warp-cooperative scan (for_candidates_lanes; sums reduced
// across the warp in FP64, so every lane holds the same totals and takes the
// same steps); the neighbour list of the returned H lane by lane.  Grid-stride over the deferred
// list, whose length only the device knows.
constexpr int kWarpDensBlock = 128;

template <typename T>
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(kWarpDensBlock)
    k_density_warp(int N, Sorted<T> s, Grid g, KParams p, unsigned* __restrict__ nbr,
                   int* __restrict__ ncount, int* __restrict__ iters, DevStatus* st,
                   const int* __restrict__ defer, const int* __restrict__ ndefer) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (kWarpDensBlock / 32);
    const int nd = *ndefer;
    for (int w = blockIdx.x * (kWarpDensBlock / 32) + (threadIdx.x >> 5); w < nd; w += warps) {
        const int i = defer[w];
        const BoxInfo bx = g.boxes[s.box[i]];
        const P4<T> me = s.pos[i];
        const T xi = me.x, yi = me.y, zi = me.z;
        double H = (double)s.h[i];
        if (!(H > 0.0) || !(H < p.h_lim)) {  // (flagged by k_density)
            H = cbrt(3.0 * p.ngb / (4.0 * kPi * (double)bx.count));
            if (!(H < p.h_lim)) H = 0.5 * p.h_lim;
        }
        const double C = 32.0 / 3.0;
        double lo = 0.0, hi = 0.0, S = 0.0, Hev = H;
        bool has_lo = false, has_hi = false, conv = false, clamped = false;
        T sd_last = T(0);
        int it, cnt = 0;
        for (it = 1; it <= p.max_iter; ++it) {
            const T Ht = (T)H;
            const T H2 = Ht * Ht;
            const T iH = T(1) / Ht;
            Acc<T> sw;
            T sd = T(0);
            int c = 0;
            for_candidates_lanes<T>(g, bx, s.pos, i, xi, yi, zi, Ht, lane, [&](int, T, T, T, T r2) {
                if (r2 < H2) {
                    const T q = psqrt(r2) * iH;
                    T w, qdw;
                    dens_terms(q, w, qdw);
                    sw.add(w);
                    sd += qdw;
                    ++c;
                }
            });
            const double Sw = warp_sum<T>(sw.value());
            const T sdw = (T)warp_sum<T>((double)sd);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            cnt = c;
            sd_last = sdw;
            Hev = (double)Ht;
            double f;
            if constexpr (std::is_same<T, float>::value) {
                const float Sf = (float)Sw;
                S = (double)Sf;
                f = (double)((32.f / 3.f) * (1.f + Sf) - (float)p.ngb);
            } else {
                S = Sw;
                f = C * (1.0 + S) - p.ngb;
            }
            if (fabs(f) <= p.tol * p.ngb) {
                conv = true;
                break;
            }
            if (it == p.max_iter) break;
            if (f < 0.0) {
                lo = Hev;
                has_lo = true;
            } else {
                hi = Hev;
                has_hi = true;
            }
            const double lo_eff = has_lo ? lo : 0.5 * Hev;
            const double hi_eff = has_hi ? hi : 2.0 * Hev;
            double Hn = 0.0;
            bool ok = false;
            if (std::is_same<T, float>::value) {
                const float fpf = (float)C * (float)sdw / Ht;
                if (fpf > 0.f) {
                    Hn = Hev - (double)((float)f / fpf);
                    ok = (Hn > lo_eff) && (Hn < hi_eff);
                }
            } else {
                const double fp = C * (double)sdw / Hev;
                if (fp > 0.0) {
                    Hn = Hev - f / fp;
                    ok = (Hn > lo_eff) && (Hn < hi_eff);
                }
            }
            if (!ok) Hn = (has_lo && has_hi) ? 0.5 * (lo + hi) : (f < 0.0 ? 2.0 * Hev : 0.5 * Hev);
            if (Hn >= p.h_lim) {
                Hn = 0.5 * (Hev + p.h_lim);
                clamped = true;
            }
            H = Hn;
        }
        if (it > p.max_iter) it = p.max_iter;
        {  // list of the returned H, in the order a thread's scan writes it (the
           // order of k_density, k_dens_given and k_lists)
            const T Ht = (T)Hev;
            for_hits_lanes_ordered<T>(g, bx, s.pos, i, xi, yi, zi, Ht, Ht * Ht, lane, [&](int k, int j) {
                if (k < p.cap) store_slot(nbr + lslot(k, i, N), (unsigned)j);
            });
        }
        if (lane == 0) {
            s.h[i] = (T)Hev;
            if (std::is_same<T, float>::value) {
                const float Hf = (float)Hev;
                s.n[i] = (T)(8.f * (float)(1.0 + S) / ((float)kPi * Hf * Hf * Hf));
            } else {
                s.n[i] = (T)(8.0 * (1.0 + S) / (kPi * Hev * Hev * Hev));
            }
            if (s.sd) s.sd[i] = sd_last;
            iters[i] = it;
            ncount[i] = cnt;
            if (!conv) {
                set_status(st, GZ_S_HCONV, GZ_C_HCONV, s.id[i]);
                if (clamped) atomicOr(&st->bits, GZ_S_HLIM);
            }
            if (cnt > p.cap) set_status(st, GZ_S_NBR_OVERFLOW, GZ_C_NBR_OVERFLOW, s.id[i]);
        }
        __syncwarp();
    }
}

// Neighbour lists N_i = {j : r_ij < H_i} for given H (O3).  only_over > 0:
// only the particles whose count exceeds it (lists a checkpoint kept up to
// that many slots; the others are restored from it).
template <typename T>
__global__ void __launch_bounds__(128)
    k_lists(int N, Sorted<T> s, Grid g, KParams p, unsigned* __restrict__ nbr,
            int* __restrict__ ncount, DevStatus* st, int only_over) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (only_over > 0 && ncount[i] <= only_over) return;
    const BoxInfo bx = g.boxes[s.box[i]];
    const T Hi = s.h[i];
    const T H2 = Hi * Hi;
    int c = 0;
    const P4<T> me = s.pos[i];
    for_candidates<T>(g, bx, s.pos, i, me.x, me.y, me.z, Hi,
                      [&](int j, T, T, T, T r2) {
                          if (r2 < H2) {
                              if (c < p.cap) store_slot(nbr + lslot(c, i, N), (unsigned)j);
                              ++c;
                          }
                      });
    ncount[i] = c;
    if (c > p.cap) set_status(st, GZ_S_NBR_OVERFLOW, GZ_C_NBR_OVERFLOW, s.id[i]);
}

// Density pass for a known converged H (a step checkpoint's): the neighbour
// list of H, n and the sum of -w'(q) q in one cell scan of radius H.  The
// candidates inside H come in the h-iteration's scan order and are summed the
// same way, so n and the sums equal the h-iteration's last evaluation bit
// for bit.
template <typename T>
__global__ void __launch_bounds__(128)
    k_dens_given(int N, Sorted<T> s, Grid g, KParams p, unsigned* __restrict__ nbr,
                 int* __restrict__ ncount, DevStatus* st) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const BoxInfo bx = g.boxes[s.box[i]];
    const T Ht = s.h[i];
    const T H2 = Ht * Ht;
    const T iH = T(1) / Ht;
    const P4<T> me = s.pos[i];
    Acc<T> sw;
    T sd = T(0);
    int c = 0;
    for_candidates<T>(g, bx, s.pos, i, me.x, me.y, me.z, Ht,
                      [&](int j, T, T, T, T r2) {
                          if (r2 < H2) {
                              const T q = psqrt(r2) * iH;
                              T w, qdw;
                              dens_terms(q, w, qdw);
                              sw.add(w);
                              sd += qdw;
                              if (c < p.cap) store_slot(nbr + lslot(c, i, N), (unsigned)j);
                              ++c;
                          }
                      });
    double S;
    if constexpr (std::is_same<T, float>::value)
        S = (double)sw.fvalue();  // as the h-iteration forms it
    else
        S = sw.value();
    const double Hev = (double)Ht;
    if (std::is_same<T, float>::value) {
        const float Hf = (float)Hev;
        s.n[i] = (T)(8.f * (float)(1.0 + S) / ((float)kPi * Hf * Hf * Hf));
    } else {
        s.n[i] = (T)(8.0 * (1.0 + S) / (kPi * Hev * Hev * Hev));
    }
    s.sd[i] = sd;
    ncount[i] = c;
    if (c > p.cap) set_status(st, GZ_S_NBR_OVERFLOW, GZ_C_NBR_OVERFLOW, s.id[i]);
}

// Reverse pairs (O10): j in N_i with r_ij >= H_j is appended to j's list.
// Reads the packed positions, whose w component is the converged H.
template <typename T>
__global__ void k_reverse(int N, Sorted<T> s, KParams p, const unsigned* __restrict__ nbr,
                          const int* __restrict__ ncount, int* __restrict__ rcount,
                          unsigned* __restrict__ rnbr, DevStatus* st) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const P4<T> me = s.pos[i];
    const T xim1 = me.x - T(1), yim1 = me.y - T(1), zim1 = me.z - T(1);
    const int cnt = min(ncount[i], p.cap);
    const unsigned* L = nbr + 4 * (size_t)i;
    for (int k0 = 0; k0 < cnt; k0 += 4) {
        const uint4 jj = col4_once(L, k0, N);
        const unsigned js[4] = {jj.x, jj.y, jj.z, jj.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (k0 + u >= cnt) break;
            const int j = (int)js[u];
            const P4<T> q = s.pos[j];
            const T dx = mi_diff(q.x, me.x, xim1), dy = mi_diff(q.y, me.y, yim1),
                    dz = mi_diff(q.z, me.z, zim1);
            const T r2 = sep2(dx, dy, dz);
            if (!(r2 < q.w * q.w)) {
                const int slot = atomicAdd(&rcount[j], 1);
                if (slot < p.rcap)
                    rnbr[lslot(slot, j, N)] = (unsigned)i;
                else
                    set_status(st, GZ_S_NBR_OVERFLOW, GZ_C_NBR_OVERFLOW, s.id[j]);
            }
        }
    }
}

// Orders each reverse list by sorted index so the flux sums are deterministic.
__global__ void k_sort_rev(int N, const int* __restrict__ rcount, unsigned* __restrict__ rnbr,
                           int rcap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int n = min(rcount[i], rcap);
    unsigned* L = rnbr + 4 * (size_t)i;
    for (int a = 1; a < n; ++a) {
        const unsigned v = L[lcol(a, N)];
        int b = a - 1;
        while (b >= 0 && L[lcol(b, N)] > v) {
            L[lcol(b + 1, N)] = L[lcol(b, N)];
            --b;
        }
        L[lcol(b + 1, N)] = v;
    }
}

// O5 primitives: rho = m n, P = (gamma - 1) rho u, c = sqrt(gamma P / rho).
template <typename T>
__global__ void k_prim(int N, Sorted<T> s, KParams p, DevStatus* st) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const T g = (T)p.gamma;
    const T rho = s.m[i] * s.n[i];
    const T P = (g - T(1)) * rho * s.u[i];
    const T c = sqrt(g * P / rho);
    s.rho[i] = rho;
    s.P[i] = P;
    s.c[i] = c;
    s.pos[i].w = s.h[i];
    s.prim[i] = P4<T>{rho, s.vx[i], s.vy[i], s.vz[i]};
    s.prim2[i] = P2<T>{P, c};
    if (!(rho > T(0)) || !(P > T(0)) || !finite_(c) || !finite_(s.vx[i]) || !finite_(s.vy[i]) ||
        !finite_(s.vz[i]))
        set_status(st, GZ_S_NONFINITE, GZ_C_NONFINITE, s.id[i]);
}

// ---------------------------------------------------------- O6-O9, O13
// Gradients, limiter and packed flux record; optionally the per-particle
// signal-speed step (over N_i and the reverse list) and its per-box minimum.
// Record (32 values): x y z H | 1/H knorm rho P | vx vy vz g0 | g1..g14 | B0..B5
// with knorm = 8/(pi H^3 n^2) so that V_i psi_j(x_i) = knorm * w(r/H).
// Neighbours are read four at a time (one 16-byte load of indices, then the
// packed records of all four) so their loads are in flight together.
// kInfo: also track which particles the limiter's bounds came from and write
// what the adjoint reads (ginfo, lim); without it (a plain forward step) that
// bookkeeping takes no registers or instructions (3 % faster; capped at 5
// blocks per SM the FP32 kernel spills and gains nothing more).
template <typename T, bool kInfo>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1)
    k_gradients(int N, Sorted<T> s, const unsigned* __restrict__ nbr, const int* __restrict__ ncount,
                const unsigned* __restrict__ rnbr, const int* __restrict__ rcount, KParams p,
                T* __restrict__ rec, double* __restrict__ dti, unsigned long long* __restrict__ dtmin,
                DevStatus* st, int want_dt, T* __restrict__ ginfo, int* __restrict__ lim,
                const int* __restrict__ list, const int* __restrict__ nlist,
                const unsigned char* __restrict__ owned) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool active;
    if (list) {  // the particles of an index list only (hierarchical steps)
        active = i < *nlist;
        i = active ? list[i] : 0;
    } else {
        active = i < N;
    }
    double dt_i = INFINITY;
    int mybox = 0;
    if (active) {
        mybox = s.box[i];
        const P4<T> me = s.pos[i];
        const T xi = me.x, yi = me.y, zi = me.z, Hi = me.w;
        const T xim1 = xi - T(1), yim1 = yi - T(1), zim1 = zi - T(1);
        const T ni = s.n[i];
        const P4<T> pm = s.prim[i];
        const P2<T> pm2 = s.prim2[i];
        const T Wi[5] = {pm.x, pm.y, pm.z, pm.w, pm2.x};
        const T ci = pm2.y;
        const T iH = T(1) / Hi;
        const T norm = T(8.0 / kPi) * iH * iH * iH / ni;
        T E[6] = {0, 0, 0, 0, 0, 0};
        T Sg[15];
        T fmax[5], fmin[5];
        int kmax[5], kmin[5];  // particles holding the extremes (for the adjoint)
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            fmax[f] = fmin[f] = Wi[f];
            kmax[f] = kmin[f] = i;
            Sg[3 * f] = Sg[3 * f + 1] = Sg[3 * f + 2] = T(0);
        }
        T vmax = T(0);
        bool any = false;
        const int cnt = min(ncount[i], p.cap);
        const unsigned* L = nbr + 4 * (size_t)i;
        for (int k0 = 0; k0 < cnt; k0 += 4) {
            const uint4 jj = col4(L, k0, N);
            const unsigned js[4] = {jj.x, jj.y, jj.z, jj.w};
            P4<T> q[4], w[4];
            P2<T> w2[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (k0 + u < cnt) {
                    q[u] = s.pos[js[u]];
                    w[u] = s.prim[js[u]];
                    w2[u] = s.prim2[js[u]];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (k0 + u >= cnt) break;
                const T dx = mi_diff(q[u].x, xi, xim1), dy = mi_diff(q[u].y, yi, yim1),
                        dz = mi_diff(q[u].z, zi, zim1);
                const T r2 = sep2(dx, dy, dz);
                const T r = psqrt(r2);
                const T psi = norm * kern_w(r * iH);
                const T pdx = psi * dx, pdy = psi * dy, pdz = psi * dz;
                E[0] += pdx * dx;
                E[1] += pdx * dy;
                E[2] += pdx * dz;
                E[3] += pdy * dy;
                E[4] += pdy * dz;
                E[5] += pdz * dz;
                const T Wj[5] = {w[u].x, w[u].y, w[u].z, w[u].w, w2[u].x};
#pragma unroll
                for (int f = 0; f < 5; ++f) {
                    const T df = Wj[f] - Wi[f];
                    Sg[3 * f] += df * pdx;
                    Sg[3 * f + 1] += df * pdy;
                    Sg[3 * f + 2] += df * pdz;
                    if (Wj[f] > fmax[f]) {
                        fmax[f] = Wj[f];
                        if constexpr (kInfo) kmax[f] = (int)js[u];
                    }
                    if (Wj[f] < fmin[f]) {
                        fmin[f] = Wj[f];
                        if constexpr (kInfo) kmin[f] = (int)js[u];
                    }
                }
                if (want_dt) {
                    const T vd = ((Wj[1] - Wi[1]) * dx + (Wj[2] - Wi[2]) * dy) + (Wj[3] - Wi[3]) * dz;
                    const T vs = ci + w2[u].y - min(pdiv(vd, r), T(0));
                    vmax = any ? max(vmax, vs) : vs;
                    any = true;
                }
            }
        }
        // O7: B = E^-1; FP64 re-do of E and its inverse when kappa > kappa_max
        T B[6], det, kap;
        invert_sym<T>(E, B, det, kap);
        T gt[15];
        bool singular;
        if (sizeof(T) == 4 && !(kap <= (T)p.kappa_max)) {
            double E64[6] = {0, 0, 0, 0, 0, 0};
            const double xd = (double)xi, yd = (double)yi, zd = (double)zi;
            const double iHd = 1.0 / (double)Hi;
            const double normd = 8.0 / kPi * iHd * iHd * iHd / (double)ni;
            for (int k = 0; k < cnt; ++k) {
                const P4<T> q = s.pos[L[lcol(k, N)]];
                const double dx = mi_diff((double)q.x, xd, 0.0), dy = mi_diff((double)q.y, yd, 0.0),
                             dz = mi_diff((double)q.z, zd, 0.0);
                const double r = sqrt(sep2(dx, dy, dz));
                const double psi = normd * kern_w(r * iHd);
                E64[0] += psi * dx * dx;
                E64[1] += psi * dx * dy;
                E64[2] += psi * dx * dz;
                E64[3] += psi * dy * dy;
                E64[4] += psi * dy * dz;
                E64[5] += psi * dz * dz;
            }
            double B64[6], det64, kap64;
            invert_sym<double>(E64, B64, det64, kap64);
            atomicOr(&st->bits, GZ_S_KAPPA_FP64);
            atomicAdd(&st->counters[GZ_C_KAPPA_FP64], 1ull);
            singular = !(det64 > 0.0) || !(kap64 <= 1e8);
#pragma unroll
            for (int q = 0; q < 6; ++q) B[q] = (T)B64[q];
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                const double s0 = Sg[3 * f], s1 = Sg[3 * f + 1], s2 = Sg[3 * f + 2];
                gt[3 * f] = (T)(B64[0] * s0 + B64[1] * s1 + B64[2] * s2);
                gt[3 * f + 1] = (T)(B64[1] * s0 + B64[3] * s1 + B64[4] * s2);
                gt[3 * f + 2] = (T)(B64[2] * s0 + B64[4] * s1 + B64[5] * s2);
            }
        } else {
            singular = !(det > T(0)) || !(kap <= T(1e8));
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                const T s0 = Sg[3 * f], s1 = Sg[3 * f + 1], s2 = Sg[3 * f + 2];
                gt[3 * f] = B[0] * s0 + B[1] * s1 + B[2] * s2;
                gt[3 * f + 1] = B[1] * s0 + B[3] * s1 + B[4] * s2;
                gt[3 * f + 2] = B[2] * s0 + B[4] * s1 + B[5] * s2;
            }
        }
        if (singular) {
            set_status(st, GZ_S_SINGULAR, GZ_C_SINGULAR, s.id[i]);
#pragma unroll
            for (int q = 0; q < 6; ++q) B[q] = T(0);
#pragma unroll
            for (int q = 0; q < 15; ++q) gt[q] = T(0);
        }
        // O9 limiter: alpha_f = min_j min(1, beta (f_ext - f_i) / D_j), D_j = g . s_ij d.
        // The numerator is fixed per field and the quotient decreases as D
        // moves away from 0 on its side, so the minimum is taken by the
        // largest positive and the most negative D_j: one division per field
        // and side after the loop instead of one per neighbour
        T Dpos[5] = {T(0), T(0), T(0), T(0), T(0)}, Dneg[5] = {T(0), T(0), T(0), T(0), T(0)};
        int jpos[5] = {-1, -1, -1, -1, -1}, jneg[5] = {-1, -1, -1, -1, -1};
        const T beta = (T)p.beta;
        for (int k0 = 0; k0 < cnt; k0 += 4) {
            const uint4 jj = col4(L, k0, N);
            const unsigned js[4] = {jj.x, jj.y, jj.z, jj.w};
            P4<T> q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (k0 + u < cnt) q[u] = s.pos[js[u]];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (k0 + u >= cnt) break;
                const T dx = mi_diff(q[u].x, xi, xim1), dy = mi_diff(q[u].y, yi, yim1),
                        dz = mi_diff(q[u].z, zi, zim1);
                const T sij = pdiv(Hi, Hi + q[u].w);
                const T ox = sij * dx, oy = sij * dy, oz = sij * dz;
#pragma unroll
                for (int f = 0; f < 5; ++f) {
                    const T D = (gt[3 * f] * ox + gt[3 * f + 1] * oy) + gt[3 * f + 2] * oz;
                    if (D > Dpos[f]) {
                        Dpos[f] = D;
                        if constexpr (kInfo) jpos[f] = (int)js[u];
                    }
                    if (D < Dneg[f]) {
                        Dneg[f] = D;
                        if constexpr (kInfo) jneg[f] = (int)js[u];
                    }
                }
            }
        }
        T al[5];
        int jact[5], kact[5];
        T Dact[5];
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            T a = T(1);
            jact[f] = -1;
            kact[f] = i;
            Dact[f] = T(0);
            if (Dpos[f] > T(0)) {
                const T ap = min(T(1), pdiv(beta * (fmax[f] - Wi[f]), Dpos[f]));
                if (ap < a) {
                    a = ap;
                    jact[f] = jpos[f];
                    kact[f] = kmax[f];
                    Dact[f] = Dpos[f];
                }
            }
            if (Dneg[f] < T(0)) {
                const T am = min(T(1), pdiv(beta * (fmin[f] - Wi[f]), Dneg[f]));
                if (am < a) {
                    a = am;
                    jact[f] = jneg[f];
                    kact[f] = kmin[f];
                    Dact[f] = Dneg[f];
                }
            }
            al[f] = a;
        }
        if (want_dt) {
            const int rc = min(rcount[i], p.rcap);
            const unsigned* RL = rnbr + 4 * (size_t)i;
            for (int k = 0; k < rc; ++k) {
                const int j = (int)RL[lcol(k, N)];
                const P4<T> q = s.pos[j];
                const P4<T> w = s.prim[j];
                const T dx = mi_diff(q.x, xi, xim1), dy = mi_diff(q.y, yi, yim1),
                        dz = mi_diff(q.z, zi, zim1);
                const T r = psqrt(sep2(dx, dy, dz));
                const T vd = ((w.y - Wi[1]) * dx + (w.z - Wi[2]) * dy) + (w.w - Wi[3]) * dz;
                const T vs = ci + s.prim2[j].y - min(pdiv(vd, r), T(0));
                vmax = any ? max(vmax, vs) : vs;
                any = true;
            }
            if (std::is_same<T, float>::value)  // FP32 path: no FP64 cbrt / division per particle
                dt_i = (any && vmax > T(0)) ? (double)(2.f * cbrtf(1.f / (float)ni) / (float)vmax) : INFINITY;
            else
                dt_i = (any && vmax > T(0)) ? 2.0 * cbrt(1.0 / (double)ni) / (double)vmax : INFINITY;
            dti[i] = dt_i;
        }
        if (kInfo && ginfo) {  // what the adjoint of this pass needs (rows 32-byte aligned)
            T G[kGInfo];
#pragma unroll
            for (int q = 0; q < 15; ++q) {
                G[q] = gt[q];
                G[15 + q] = Sg[q];
            }
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                G[30 + f] = al[f];
                G[35 + f] = Dact[f];
            }
            store_row32<kGInfo>(ginfo + (size_t)i * kGInfo, G);
            // the limiting particles: jact[0..4] then kact[0..4], a 40-byte row
            // (8-byte aligned) written as five 8-byte stores
            const int Lv[10] = {jact[0], jact[1], jact[2], jact[3], jact[4],
                                kact[0], kact[1], kact[2], kact[3], kact[4]};
            int2* Lm = reinterpret_cast<int2*>(lim + (size_t)i * 10);
#pragma unroll
            for (int m = 0; m < 5; ++m) Lm[m] = make_int2(Lv[2 * m], Lv[2 * m + 1]);
        }
        // the flux record: one 128-byte (FP32) row, written with 32-byte stores
        T R[kRecord];
        R[0] = xi;
        R[1] = yi;
        R[2] = zi;
        R[3] = Hi;
        R[4] = iH;
        R[5] = norm / ni;
        R[6] = Wi[0];
        R[7] = Wi[4];
        R[8] = Wi[1];
        R[9] = Wi[2];
        R[10] = Wi[3];
#pragma unroll
        for (int q = 0; q < 15; ++q) R[11 + q] = al[q / 3] * gt[q];
#pragma unroll
        for (int q = 0; q < 6; ++q) R[26 + q] = B[q];
        store_row32<kRecord>(rec + (size_t)i * kRecord, R);
    }
    if (want_dt) {
        // warp-level minimum per box, one atomic per warp when the warp is in one box;
        // in a subdomain only its owned particles take part
        const unsigned full = 0xffffffffu;
        const bool counts = active && (!owned || owned[s.orig[i]]);
        unsigned long long v = counts ? dbits(dt_i) : dbits(INFINITY);
        const int b0 = __shfl_sync(full, mybox, 0);
        const bool same = __all_sync(full, !active || mybox == b0);
        if (same) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                unsigned long long w = __shfl_xor_sync(full, v, o);
                v = w < v ? w : v;
            }
            if ((threadIdx.x & 31) == 0) atomicMin(&dtmin[b0], v);
        } else if (counts) {
            atomicMin(&dtmin[mybox], v);
        }
    }
}

// Builds flux records from caller-supplied gradients and B (caller order).
// With a list: its particles only, skipping those flagged in skip (the
// inactive partners of a hierarchical substep, whose gradients and B are
// those of their last active time).
template <typename T>
__global__ void k_pack_given(int N, Sorted<T> s, const T* __restrict__ grad, const T* __restrict__ B,
                             T* __restrict__ rec, const int* __restrict__ list,
                             const int* __restrict__ nlist, const unsigned char* __restrict__ skip) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (list) {
        if (i >= *nlist) return;
        i = list[i];
        if (skip && skip[i]) return;
    } else if (i >= N) {
        return;
    }
    const unsigned o = s.orig[i];
    const T Hi = s.h[i], ni = s.n[i];
    const T iH = T(1) / Hi;
    T* R = rec + (size_t)i * kRecord;
    R[0] = s.x[i];
    R[1] = s.y[i];
    R[2] = s.z[i];
    R[3] = Hi;
    R[4] = iH;
    R[5] = T(8.0 / kPi) * iH * iH * iH / ni / ni;
    R[6] = s.rho[i];
    R[7] = s.P[i];
    R[8] = s.vx[i];
    R[9] = s.vy[i];
    R[10] = s.vz[i];
    for (int q = 0; q < 15; ++q) R[11 + q] = grad[(size_t)q * N + o];
    for (int q = 0; q < 6; ++q) R[26 + q] = B[(size_t)q * N + o];
}

template <typename T>
__global__ void k_grad_out(int N, const unsigned* __restrict__ orig, const T* __restrict__ rec,
                           T* __restrict__ grad, T* __restrict__ B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned o = orig[i];
    const T* R = rec + (size_t)i * kRecord;
    if (grad)
        for (int q = 0; q < 15; ++q) grad[(size_t)q * N + o] = R[11 + q];
    if (B)
        for (int q = 0; q < 6; ++q) B[(size_t)q * N + o] = R[26 + q];
}

// One thread per particle over its pairs N_i then R_i (both contiguous
// lists, read four indices per 16-byte load).  Contributions are summed in
// the working precision over runs of 8 pairs and each run is added to FP64
// accumulators.  kMFV: the MFV fluxes (O15), which add dm/dt.  kRiem: the
// MFM face's Riemann solver (pair_rates).
constexpr int kFluxBlock = 128;

template <typename T, bool kMFV, int kRiem>
__global__ void __launch_bounds__(kFluxBlock)
    k_fluxes(int N, const T* __restrict__ rec, const long long* __restrict__ sid,
             const int* __restrict__ sbox, const unsigned* __restrict__ nbr,
             const int* __restrict__ ncount, const unsigned* __restrict__ rnbr,
             const int* __restrict__ rcount, KParams p, const double* __restrict__ dt_use,
             double* __restrict__ dpdt, double* __restrict__ dEdt, double* __restrict__ dmdt,
             DevStatus* st) {
    constexpr int nq = kMFV ? 5 : 4;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    T a[kRecord];
    load_rec(rec + (size_t)i * kRecord, a);
    const long long idi = kMFV ? sid[i] : 0;  // (MFV pairs are oriented by id)
    const T hdt = (T)(0.5 * dt_use[sbox[i]]);
    const T gam = (T)p.gamma;
    const bool hancock = p.hancock != 0;
    T inca[5];
    hancock_inc(a, hdt, gam, hancock, inca);
    T part[nq];
    double acc[nq];
#pragma unroll
    for (int q = 0; q < nq; ++q) {
        part[q] = T(0);
        acc[q] = 0.0;
    }
    int np = 0, nfall = 0, nneg = 0;
#pragma unroll 1
    for (int list = 0; list < 2; ++list) {
        const unsigned* L = list == 0 ? nbr + 4 * (size_t)i : rnbr + 4 * (size_t)i;
        const int cnt = list == 0 ? min(ncount[i], p.cap) : min(rcount[i], p.rcap);
        for (int k0 = 0; k0 < cnt; k0 += 4) {
            const uint4 jj = col4_once(L, k0, N);
            const unsigned js[4] = {jj.x, jj.y, jj.z, jj.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (k0 + u >= cnt) break;
                const int j = (int)js[u];
                T b[kRecord];
                load_rec(rec + (size_t)j * kRecord, b);
                T dp[3], dE, dm;
                int fl = 0;
                if (pair_rates<T, kMFV, kRiem>(a, b, pair_order<kMFV>(i, j, idi, sid), hdt, gam, hancock, inca,
                                               dp, dE, dm, fl)) {
                    part[0] += dp[0];
                    part[1] += dp[1];
                    part[2] += dp[2];
                    part[3] += dE;
                    if constexpr (kMFV) part[4] += dm;
                }
                nfall += fl & 1;
                nneg += (fl >> 1) & 1;
                if (++np == 8) {
#pragma unroll
                    for (int q = 0; q < nq; ++q) {
                        acc[q] += (double)part[q];
                        part[q] = T(0);
                    }
                    np = 0;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < nq; ++q) acc[q] += (double)part[q];
    dpdt[i] = acc[0];
    dpdt[(size_t)N + i] = acc[1];
    dpdt[2 * (size_t)N + i] = acc[2];
    dEdt[i] = acc[3];
    if constexpr (kMFV) dmdt[i] = acc[4];
    if (nfall) {
        atomicOr(&st->bits, GZ_S_FALLBACK);
        atomicAdd(&st->counters[GZ_C_FALLBACK], (unsigned long long)nfall);
    }
    if (nneg) {
        atomicOr(&st->bits, GZ_S_PSTAR_NEG);
        atomicAdd(&st->counters[GZ_C_PSTAR_NEG], (unsigned long long)nneg);
    }
}

// dmdt (MFV, O15) non-null: the mass advances too and is written back.
template <typename T>
__global__ void k_update(int N, Sorted<T> s, const double* __restrict__ dpdt,
                         const double* __restrict__ dEdt, const double* __restrict__ dmdt,
                         const double* __restrict__ dt_use, gz_particles out,
                         int* __restrict__ box_hits, DevStatus* st, double* __restrict__ rates_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned o = s.orig[i];
    const int b = s.box[i];
    if (rates_out) {  // the step's conserved-variable rates, caller order
        rates_out[o] = dpdt[i];
        rates_out[(size_t)N + o] = dpdt[(size_t)N + i];
        rates_out[2 * (size_t)N + o] = dpdt[2 * (size_t)N + i];
        rates_out[3 * (size_t)N + o] = dEdt[i];
    }
    T x = s.x[i], y = s.y[i], z = s.z[i], vx = s.vx[i], vy = s.vy[i], vz = s.vz[i], u = s.u[i];
    bool mass_ok = true;
    if (dmdt) {
        T m = s.m[i];
        update_one_mfv(m, x, y, z, vx, vy, vz, u, dpdt[i], dpdt[(size_t)N + i],
                       dpdt[2 * (size_t)N + i], dEdt[i], dmdt[i], dt_use[b]);
        ((T*)out.m)[o] = m;
        mass_ok = m > T(0);
    } else {
        update_one(s.m[i], x, y, z, vx, vy, vz, u, dpdt[i], dpdt[(size_t)N + i],
                   dpdt[2 * (size_t)N + i], dEdt[i], dt_use[b]);
    }
    ((T*)out.x)[o] = x;
    ((T*)out.y)[o] = y;
    ((T*)out.z)[o] = z;
    ((T*)out.vx)[o] = vx;
    ((T*)out.vy)[o] = vy;
    ((T*)out.vz)[o] = vz;
    ((T*)out.u)[o] = u;
    ((T*)out.h)[o] = s.h[i];
    if (!(u > T(0))) {
        atomicAdd(&box_hits[b], 1);
        set_status(st, GZ_S_UFLOOR, GZ_C_UFLOOR, -1);
    }
    if (!(mass_ok && finite_(x) && finite_(y) && finite_(z) && finite_(vx) && finite_(vy) &&
          finite_(vz) && finite_(u)))
        set_status(st, GZ_S_NONFINITE, GZ_C_NONFINITE, s.id[i]);
}

template <typename T>
struct Bits;
template <>
struct Bits<float> {
    typedef unsigned U;
    static constexpr int nbits = 32;
    __device__ static U get(float v) { return __float_as_uint(v); }
    __device__ static float put(U b) { return __uint_as_float(b); }
};
template <>
struct Bits<double> {
    typedef unsigned long long U;
    static constexpr int nbits = 64;
    __device__ static U get(double v) { return (U)__double_as_longlong(v); }
    __device__ static double put(U b) { return __longlong_as_double((long long)b); }
};

// O14 floor: for each box with a hit, the lower median of u at step start
// (radix select on the bit patterns of positive values), then every
// non-positive updated u of the box is set to u_floor_frac * median.
template <typename T>
__global__ void k_ufloor(Sorted<T> s, const BoxInfo* __restrict__ boxes,
                         const int* __restrict__ box_hits, gz_particles out, double frac,
                         const unsigned char* __restrict__ owned, int nown) {
    typedef typename Bits<T>::U U;
    const int b = blockIdx.x;
    if (box_hits[b] == 0) return;
    const int first = boxes[b].first, count = boxes[b].count;
    // in a subdomain (owned non-null, one box) the median of its owned particles
    __shared__ unsigned hist[256];
    __shared__ U prefix_s;
    __shared__ int k_s;
    U prefix = 0, mask = 0;
    int k = ((owned ? nown : count) - 1) / 2;
    if (k < 0) return;
    for (int shift = Bits<T>::nbits - 8; shift >= 0; shift -= 8) {
        for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[t] = 0;
        __syncthreads();
        for (int e = threadIdx.x; e < count; e += blockDim.x) {
            if (owned && !owned[s.orig[first + e]]) continue;
            const U v = Bits<T>::get(s.u[first + e]);
            if ((v & mask) == prefix) atomicAdd(&hist[(unsigned)((v >> shift) & 255u)], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int d = 0;
            for (; d < 255; ++d) {
                if (k < (int)hist[d]) break;
                k -= (int)hist[d];
            }
            prefix_s = prefix | ((U)d << shift);
            k_s = k;
        }
        __syncthreads();
        prefix = prefix_s;
        k = k_s;
        mask |= ((U)255u << shift);
        __syncthreads();
    }
    const T fl = (T)(frac * (double)Bits<T>::put(prefix));
    T* u = (T*)out.u;
    for (int e = threadIdx.x; e < count; e += blockDim.x) {
        const int o = first + e;  // caller order and sorted order share box ranges
        if (!(u[o] > T(0))) u[o] = fl;
    }
}

__global__ void k_dt_init(int nb, unsigned long long* dtmin) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) dtmin[b] = dbits(INFINITY);
}
__global__ void k_dt_final(int nb, const unsigned long long* __restrict__ dtmin, double cfl,
                           double dt_fixed, double* __restrict__ dt_use, double* __restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const double raw = __longlong_as_double((long long)dtmin[b]);
    const double dt = dt_fixed > 0.0 ? dt_fixed : cfl * raw;
    dt_use[b] = dt;
    if (out) out[b] = dt;
}
__global__ void k_dt_set(int nb, double dt, double* __restrict__ dt_use) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) dt_use[b] = dt;
}
__global__ void k_dt_out(int nb, const unsigned long long* __restrict__ dtmin, double cfl,
                         double* __restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) out[b] = cfl * __longlong_as_double((long long)dtmin[b]);
}

__global__ void k_get_nbrs(int N, const unsigned* __restrict__ orig, const long long* __restrict__ sid,
                           const unsigned* __restrict__ nbr, const int* __restrict__ ncount, int cap_in,
                           int32_t* __restrict__ count_out, int64_t* __restrict__ ids_out, int cap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned o = orig[i];
    const int c = ncount[i];
    count_out[o] = c;
    if (!ids_out) return;
    const int m = min(min(c, cap_in), cap);
    for (int k = 0; k < cap; ++k)
        ids_out[(size_t)k * N + o] = k < m ? (int64_t)sid[nbr[lslot(k, i, N)]] : (int64_t)-1;
}

// The limiter's choices per particle (sorted-order indices, 10 per particle)
// as particle ids in caller order: rows 0-4 the neighbour whose face bound
// set alpha_f (-1: alpha_f = 1), rows 5-9 the particle holding the extreme.
__global__ void k_get_limiters(int N, const unsigned* __restrict__ orig, const long long* __restrict__ sid,
                               const int* __restrict__ lim, int64_t* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned o = orig[i];
    for (int f = 0; f < 10; ++f) {
        const int j = lim[(size_t)i * 10 + f];
        out[(size_t)f * N + o] = j >= 0 ? (int64_t)sid[j] : (int64_t)-1;
    }
}

__global__ void k_pairs(int N, const int* __restrict__ ncount, const int* __restrict__ rcount,
                        int cap, int rcap, long long* __restrict__ out) {
    long long v = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        v += min(ncount[i], cap) + min(rcount[i], rcap);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd((unsigned long long*)out, (unsigned long long)v);
}

// Work of the cell scan at the converged H: per particle, the candidates a
// scan of radius 1.05 H (the density cache's) tests, those inside 1.05 H and
// those inside H; summed over the particles (out[0..2]).
template <typename T>
__global__ void __launch_bounds__(128)
    k_scan_stats(int N, Sorted<T> s, Grid g, KParams p, unsigned long long* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v[3] = {0, 0, 0};
    if (i < N) {
        const BoxInfo bx = g.boxes[s.box[i]];
        const P4<T> me = s.pos[i];
        const T Ht = s.h[i];
        const T R = dens_cache_radius<T>(Ht, p);
        const T R2 = R * R, H2 = Ht * Ht;
        for_candidates<T>(g, bx, s.pos, i, me.x, me.y, me.z, R, [&](int, T, T, T, T r2) {
            if (r2 < T(1e29)) ++v[0];  // (slots past a cell's range read a far point)
            if (r2 < R2) ++v[1];
            if (r2 < H2) ++v[2];
        });
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        unsigned long long x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(out + k, x);
    }
}

}  // namespace

cudaError_t run_pair_count(Ctx& c, long long* out_dev) {
    c.launches += 1;
    cudaMemsetAsync(out_dev, 0, sizeof(long long), c.stream);
    k_pairs<<<304, 256, 0, c.stream>>>(c.N, c.ncount, c.rcount, c.cap, c.rcap, out_dev);
    return cudaGetLastError();
}

KParams kparams(const Ctx& c) {
    KParams k;
    k.gamma = c.params.gamma;
    k.ngb = c.params.ngb;
    k.tol = c.params.tol;
    k.cfl = c.params.cfl;
    k.kappa_max = c.params.kappa_max;
    k.beta = c.params.beta;
    k.u_floor_frac = c.params.u_floor_frac;
    k.h_lim = c.params.h_lim;
    k.hancock = c.params.hancock;
    k.scheme = c.params.scheme;
    k.max_iter = c.params.max_iter;
    k.cap = c.cap;
    k.rcap = c.rcap;
    return k;
}

static Grid grid_of(const Ctx& c) {
    Grid g;
    g.boxes = c.boxes;
    g.cells = c.cells;
    return g;
}

template <typename T>
cudaError_t run_scan_stats(Ctx& c, long long* out_dev) {
    c.launches += 1;
    cudaError_t e = cudaMemsetAsync(out_dev, 0, 3 * sizeof(long long), c.stream);
    if (e != cudaSuccess) return e;
    k_scan_stats<T><<<blocks(c.N, 128), 128, 0, c.stream>>>(c.N, sorted_view<T>(c), grid_of(c), kparams(c),
                                                             (unsigned long long*)out_dev);
    return cudaGetLastError();
}
template cudaError_t run_scan_stats<float>(Ctx&, long long*);
template cudaError_t run_scan_stats<double>(Ctx&, long long*);

template <typename T>
cudaError_t run_density(Ctx& c, const int* list, const int* nlist, int n) {
    if (!list) n = c.N;
    if (n < 1) return cudaSuccess;
    long long min_count = c.N;
    for (const BoxInfo& b : c.hboxes) min_count = std::min(min_count, (long long)b.count);
    if (c.grid_count > 0) min_count = c.grid_count;  // a subdomain: as the whole box
    if (c.params.density_cache == kDensCacheLarge) min_count = 32 * 32 * 32;
    if (c.params.density_cache == kDensCacheSmall) min_count = 0;
    const Sorted<T> sv = sorted_view<T>(c);
    c.launches += c.defer ? 2 : 1;
    if (c.defer) cudaMemsetAsync(c.ndefer, 0, sizeof(int), c.stream);
    if (min_count >= 32 * 32 * 32)
        k_density<T, kDensCacheLarge><<<blocks(n, kDensBlock), kDensBlock, 0, c.stream>>>(
            c.N, sv, grid_of(c), kparams(c), c.nbr, c.ncount, c.iters, c.status, list, nlist, c.defer,
            c.ndefer);
    else
        k_density<T, kDensCacheSmall><<<blocks(n, kDensBlock), kDensBlock, 0, c.stream>>>(
            c.N, sv, grid_of(c), kparams(c), c.nbr, c.ncount, c.iters, c.status, list, nlist, c.defer,
            c.ndefer);
    if (c.defer) {
        const int wb = std::max(1, std::min(blocks(n, kWarpDensBlock / 32), 152 * 4));
        k_density_warp<T><<<wb, kWarpDensBlock, 0, c.stream>>>(c.N, sv, grid_of(c), kparams(c), c.nbr, c.ncount,
                                                                c.iters, c.status, c.defer, c.ndefer);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_density_given(Ctx& c) {
    c.launches += 1;
    k_dens_given<T><<<blocks(c.N, 128), 128, 0, c.stream>>>(c.N, sorted_view<T>(c), grid_of(c), kparams(c),
                                                             c.nbr, c.ncount, c.status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_build_lists(Ctx& c) {
    c.launches += 1;
    k_lists<T><<<blocks(c.N, 128), 128, 0, c.stream>>>(c.N, sorted_view<T>(c), grid_of(c), kparams(c),
                                                        c.nbr, c.ncount, c.status, 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_lists_over(Ctx& c, int kept) {
    c.launches += 1;
    k_lists<T><<<blocks(c.N, 128), 128, 0, c.stream>>>(c.N, sorted_view<T>(c), grid_of(c), kparams(c),
                                                        c.nbr, c.ncount, c.status, kept);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_reverse(Ctx& c) {
    c.launches += 2;
    cudaMemsetAsync(c.rcount, 0, sizeof(int) * (size_t)c.N, c.stream);
    k_reverse<T><<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, sorted_view<T>(c), kparams(c), c.nbr,
                                                          c.ncount, c.rcount, c.rnbr, c.status);
    k_sort_rev<<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, c.rcount, c.rnbr, c.rcap);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_prim(Ctx& c) {
    c.launches += 1;
    k_prim<T><<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, sorted_view<T>(c), kparams(c), c.status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_gradients(Ctx& c, bool want_dt, bool with_info, const int* list, const int* nlist, int n) {
    c.launches += want_dt ? 2 : 1;
    if (!list) n = c.N;
    if (want_dt) k_dt_init<<<blocks(c.nboxes, 256), 256, 0, c.stream>>>(c.nboxes, (unsigned long long*)c.dt_box);
    if (n < 1) return cudaGetLastError();
    if (with_info)
        k_gradients<T, true><<<blocks(n, 128), 128, 0, c.stream>>>(
            c.N, sorted_view<T>(c), c.nbr, c.ncount, c.rnbr, c.rcount, kparams(c), (T*)c.rec, c.dti,
            (unsigned long long*)c.dt_box, c.status, want_dt ? 1 : 0, (T*)c.ginfo, c.lim, list, nlist, c.owned);
    else
        k_gradients<T, false><<<blocks(n, 128), 128, 0, c.stream>>>(
            c.N, sorted_view<T>(c), c.nbr, c.ncount, c.rnbr, c.rcount, kparams(c), (T*)c.rec, c.dti,
            (unsigned long long*)c.dt_box, c.status, want_dt ? 1 : 0, nullptr, nullptr, list, nlist, c.owned);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_pack_given(Ctx& c, const T* grad, const T* B, const int* list, const int* nlist, int n,
                           const unsigned char* skip) {
    c.launches += 1;
    if (list && n < 1) return cudaSuccess;
    k_pack_given<T><<<blocks(list ? n : c.N, 256), 256, 0, c.stream>>>(c.N, sorted_view<T>(c), grad, B,
                                                                     (T*)c.rec, list, nlist, skip);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_grad_out(Ctx& c, T* grad, T* B) {
    c.launches += 1;
    k_grad_out<T><<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, c.vals, (const T*)c.rec, grad, B);
    return cudaGetLastError();
}

template <typename T, bool kMFV, int kRiem>
static void launch_fluxes(Ctx& c) {
    k_fluxes<T, kMFV, kRiem><<<blocks(c.N, kFluxBlock), kFluxBlock, 0, c.stream>>>(
        c.N, (const T*)c.rec, c.sid, c.sbox, c.nbr, c.ncount, c.rnbr, c.rcount, kparams(c), c.dt_use,
        c.dpdt, c.dEdt, kMFV ? c.dmdt : nullptr, c.status);
}

template <typename T>
cudaError_t run_fluxes(Ctx& c) {
    c.launches += 1;
    if (c.params.scheme == GZ_MFV)
        launch_fluxes<T, true, GZ_RIEMANN_HLLC>(c);
    else if (c.params.riemann == GZ_RIEMANN_EXACT)
        launch_fluxes<T, false, GZ_RIEMANN_EXACT>(c);
    else if (c.params.riemann == GZ_RIEMANN_FALLBACK)
        launch_fluxes<T, false, GZ_RIEMANN_FALLBACK>(c);
    else
        launch_fluxes<T, false, GZ_RIEMANN_HLLC>(c);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_update(Ctx& c, gz_particles& p, double* rates_out) {
    c.launches += 2;
    int* hits = c.box_hits;
    cudaMemsetAsync(hits, 0, sizeof(int) * (size_t)c.nboxes, c.stream);
    k_update<T><<<blocks(c.N, 256), 256, 0, c.stream>>>(
        c.N, sorted_view<T>(c), c.dpdt, c.dEdt, c.params.scheme == GZ_MFV ? c.dmdt : nullptr, c.dt_use, p,
        hits, c.status, rates_out);
    k_ufloor<T><<<c.nboxes, 1024, 0, c.stream>>>(sorted_view<T>(c), c.boxes, hits, p,
                                                  c.params.u_floor_frac, c.owned, c.n_owned);
    return cudaGetLastError();
}

// The u floor of O14 alone (after a kick that flagged box_hits).
template <typename T>
cudaError_t run_ufloor(Ctx& c, gz_particles& p) {
    c.launches += 1;
    k_ufloor<T><<<c.nboxes, 1024, 0, c.stream>>>(sorted_view<T>(c), c.boxes, c.box_hits, p,
                                                  c.params.u_floor_frac, c.owned, c.n_owned);
    return cudaGetLastError();
}

// Rates saved by a forward step (caller order) into the sorted rate arrays.
__global__ void k_rates_in(int N, const unsigned* __restrict__ orig, const double* __restrict__ rates,
                           double* __restrict__ dpdt, double* __restrict__ dEdt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned o = orig[i];
    dpdt[i] = rates[o];
    dpdt[(size_t)N + i] = rates[(size_t)N + o];
    dpdt[2 * (size_t)N + i] = rates[2 * (size_t)N + o];
    dEdt[i] = rates[3 * (size_t)N + o];
}

cudaError_t run_rates_in(Ctx& c, const double* rates) {
    c.launches += 1;
    k_rates_in<<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, c.vals, rates, c.dpdt, c.dEdt);
    return cudaGetLastError();
}

cudaError_t run_dt_init(Ctx& c) {
    c.launches += 1;
    k_dt_init<<<blocks(c.nboxes, 256), 256, 0, c.stream>>>(c.nboxes, (unsigned long long*)c.dt_box);
    return cudaGetLastError();
}

cudaError_t run_dt_finalize(Ctx& c, double dt_fixed, double* dt_used_dev) {
    c.launches += 1;
    k_dt_final<<<blocks(c.nboxes, 256), 256, 0, c.stream>>>(
        c.nboxes, (const unsigned long long*)c.dt_box, c.params.cfl, dt_fixed, c.dt_use, dt_used_dev);
    return cudaGetLastError();
}

cudaError_t run_dt_set(Ctx& c, double dt) {
    c.launches += 1;
    k_dt_set<<<blocks(c.nboxes, 256), 256, 0, c.stream>>>(c.nboxes, dt, c.dt_use);
    return cudaGetLastError();
}

__global__ void k_dt_copy(int nb, const double* __restrict__ dt, double* __restrict__ dt_use) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) dt_use[b] = dt[b];
}

cudaError_t run_dt_copy(Ctx& c, const double* dt) {
    c.launches += 1;
    k_dt_copy<<<blocks(c.nboxes, 256), 256, 0, c.stream>>>(c.nboxes, dt, c.dt_use);
    return cudaGetLastError();
}

// One-box table of a subdomain, written from values passed by value.
__global__ void k_set_box(BoxInfo* boxes, BoxInfo b) {
    if (threadIdx.x == 0 && blockIdx.x == 0) boxes[0] = b;
}

cudaError_t run_set_box(Ctx& c) {
    c.launches += 1;
    k_set_box<<<1, 32, 0, c.stream>>>(c.boxes, c.hboxes[0]);
    return cudaGetLastError();
}

cudaError_t run_dt_out(Ctx& c, double* out) {
    c.launches += 1;
    k_dt_out<<<blocks(c.nboxes, 256), 256, 0, c.stream>>>(c.nboxes, (const unsigned long long*)c.dt_box,
                                                          c.params.cfl, out);
    return cudaGetLastError();
}

cudaError_t run_get_limiters(Ctx& c, const int* lim, int64_t* out) {
    c.launches += 1;
    k_get_limiters<<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, c.vals, c.sid, lim, out);
    return cudaGetLastError();
}

cudaError_t run_get_neighbours(Ctx& c, int32_t* count_out, int64_t* ids_out, int cap) {
    c.launches += 1;
    k_get_nbrs<<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, c.vals, c.sid, c.nbr, c.ncount, c.cap,
                                                       count_out, ids_out, cap);
    return cudaGetLastError();
}

#define GZ_INST(T)                                                   \
    template cudaError_t run_density<T>(Ctx&, const int*, const int*, int);                    \
    template cudaError_t run_density_given<T>(Ctx&);                                            \
    template cudaError_t run_build_lists<T>(Ctx&);                                              \
    template cudaError_t run_lists_over<T>(Ctx&, int);                                          \
    template cudaError_t run_reverse<T>(Ctx&);                                                  \
    template cudaError_t run_prim<T>(Ctx&);                                                     \
    template cudaError_t run_gradients<T>(Ctx&, bool, bool, const int*, const int*, int);      \
    template cudaError_t run_pack_given<T>(Ctx&, const T*, const T*, const int*, const int*, int, \
                                           const unsigned char*);                               \
    template cudaError_t run_grad_out<T>(Ctx&, T*, T*);                                         \
    template cudaError_t run_fluxes<T>(Ctx&);                                                   \
    template cudaError_t run_update<T>(Ctx&, gz_particles&, double*);                          \
    template cudaError_t run_ufloor<T>(Ctx&, gz_particles&);
GZ_INST(float)
GZ_INST(double)
#undef GZ_INST

}  // namespace gz
