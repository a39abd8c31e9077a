// Hierarchical (power-of-two) timesteps: one sync interval of 2^K substeps
// built on the step's passes.  Reading of the method's hierarchical adaptive
// timesteps (the paper gives no formula):
//   - particle i sits in bin k_i in [0, K], step dt_i = D/2^k_i, and is active
//     at substep s when s is a multiple of 2^(K - k_i);
//   - substep 0: every particle is active; D = dt_fixed, or
//     min(cfl max_i dtc_i, 2^K cfl min_i dtc_i) per box (dtc the O13 criterion);
//     k_i = smallest k with D/2^k <= cfl dtc_i (K at most).  Later active
//     times may only deepen a bin;
//   - the caller's x holds each particle's position at the start of its
//     current step; at substep s every particle is placed at
//     x + (s - s_a) D/2^K * v_bar, v_bar = (v_start + v)/2, and a step that
//     ends moves x by dt_i v_bar (the trapezoid drift of O14);
//   - active particles run O4-O9 and O13; the others keep H, n, gradients and
//     B of their last active time.  Every flux pair with an active particle
//     exchanges the O11/O12 face fluxes over dt_ij = D/2^max(k_i, k_j)
//     (Hancock with dt_ij/2): each side accumulates rate * 2^(k_a - k_ij)
//     (exact power-of-two scaling, so the two shares stay equal and opposite)
//     and kicks momentum and energy by dt_a times that sum.
// Any Riemann option of the MFM face, and MFV (the exchange uses pair_rates
// with them; under MFV the mass shares ride along and the kick advances m).
// K = 0 is gz_step bitwise.  Pair lists of an active particle: N_i from the
// density pass and the pairs with r >= H_i (r < H_j), written by the partner
// j from a scan of its own support; an inactive particle's list holds its
// active partners, written by them (atomic slot counters, then every such
// list sorted by index, so every sum runs in a fixed order).
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "gz_device.cuh"
#include "gz_launch.cuh"

namespace gz {

namespace {

inline int nblk(int n, int t) { return (n + t - 1) / t; }

constexpr int kCmpBlock = 1024;

template <typename T>
__device__ __forceinline__ T wrap_pos(T v) {
    if (v < T(0)) v += T(1);
    if (v >= T(1)) v -= T(1);
    return v;
}

// ------------------------------------------------------ interval start
template <typename T>
__global__ void k_h_init(int N, gz_particles p, T* __restrict__ hva, T* __restrict__ hdvs,
                         int* __restrict__ hsa, int* __restrict__ hbin) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= N) return;
    hva[o] = ((const T*)p.vx)[o];
    hva[(size_t)N + o] = ((const T*)p.vy)[o];
    hva[2 * (size_t)N + o] = ((const T*)p.vz)[o];
    hdvs[o] = hdvs[(size_t)N + o] = hdvs[2 * (size_t)N + o] = T(0);
    hsa[o] = 0;
    hbin[o] = 0;
}

// Mean velocity of the current step so far: (v_start + v)/2 (FP64), or
// v_start + dv/2 with the accumulated change dv (FP32, the increment form).
template <typename T>
__device__ __forceinline__ T vbar(T va, T v, T dvs) {
    if constexpr (std::is_same<T, float>::value)
        return va + 0.5f * dvs;
    else
        return 0.5 * (va + v);
}

// Predicted positions of every particle at substep s (caller order) and the
// number of particles active there.
template <typename T>
__global__ void k_h_predict(int N, int s, int K, gz_particles p, const T* __restrict__ hva,
                            const T* __restrict__ hdvs, const int* __restrict__ hsa,
                            const int* __restrict__ hbin, const int* __restrict__ box_of,
                            const double* __restrict__ D, T* __restrict__ xp, int* __restrict__ count) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    bool act = false;
    if (o < N) {
        act = s % (1 << (K - hbin[o])) == 0;
        const int steps = s - hsa[o];
        const T* X[3] = {(const T*)p.x, (const T*)p.y, (const T*)p.z};
        const T* V[3] = {(const T*)p.vx, (const T*)p.vy, (const T*)p.vz};
        if (steps == 0) {
#pragma unroll
            for (int r = 0; r < 3; ++r) xp[(size_t)r * N + o] = X[r][o];
        } else {
            const double tau = ldexp(D[box_of[o]], -K) * (double)steps;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const size_t q = (size_t)r * N + o;
                xp[q] = wrap_pos<T>(X[r][o] + (T)tau * vbar<T>(hva[q], V[r][o], hdvs[q]));
            }
        }
    }
    const int c = __syncthreads_count(act);
    if (threadIdx.x == 0 && c) atomicAdd(count, c);
}

// Sorted bins and active flags.
__global__ void k_h_flags(int N, int s, int K, const unsigned* __restrict__ orig,
                          const int* __restrict__ hbin, int* __restrict__ sbin,
                          unsigned char* __restrict__ aflag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int b = hbin[orig[i]];
    sbin[i] = b;
    aflag[i] = (unsigned char)(s % (1 << (K - b)) == 0);
}

// ------------------------------------------- ordered stream compaction
// flag -> list of the flagged indices in increasing order: per-block counts,
// one block scanning them, per-block writes (warp ballots within a block).
__global__ void __launch_bounds__(kCmpBlock)
    k_cmp_count(int N, const unsigned char* __restrict__ flag, int* __restrict__ bcount) {
    const int i = blockIdx.x * kCmpBlock + threadIdx.x;
    const int c = __syncthreads_count(i < N && flag[i]);
    if (threadIdx.x == 0) bcount[blockIdx.x] = c;
}

__global__ void __launch_bounds__(kCmpBlock) k_cmp_scan(int nb, int* __restrict__ bcount, int* __restrict__ total) {
    __shared__ int part[kCmpBlock];
    const int t = threadIdx.x;
    const int chunk = (nb + kCmpBlock - 1) / kCmpBlock;
    const int b0 = min(nb, t * chunk), b1 = min(nb, b0 + chunk);
    int sum = 0;
    for (int b = b0; b < b1; ++b) sum += bcount[b];
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < kCmpBlock; off <<= 1) {  // inclusive scan (Hillis-Steele)
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - sum;  // exclusive prefix of this thread's chunk
    for (int b = b0; b < b1; ++b) {
        const int c = bcount[b];
        bcount[b] = run;
        run += c;
    }
    if (t == kCmpBlock - 1) *total = part[t];
}

__global__ void __launch_bounds__(kCmpBlock)
    k_cmp_write(int N, const unsigned char* __restrict__ flag, const int* __restrict__ boff,
                int* __restrict__ list) {
    __shared__ int wsum[kCmpBlock / 32];
    const int i = blockIdx.x * kCmpBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool f = i < N && flag[i];
    const unsigned ball = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[w] = __popc(ball);
    __syncthreads();
    if (w == 0) {  // exclusive scan of the warp counts
        const int v = wsum[lane];
        int x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        wsum[lane] = x - v;
    }
    __syncthreads();
    if (f) list[boff[blockIdx.x] + wsum[w] + __popc(ball & ((1u << lane) - 1u))] = i;
}

// --------------------------------------------------------- pair lists
// Cells holding at least one active particle (sorted ranges).
__global__ void k_h_cellact(int ncells, const int2* __restrict__ cells, const unsigned char* __restrict__ aflag,
                            unsigned char* __restrict__ cellact) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const int2 se = cells[c];
    unsigned char any = 0;
    for (int i = se.x; i < se.y && !any; ++i) any = aflag[i];
    cellact[c] = any;
}

// Cells within two cells (per axis, periodic) of a cell holding an active
// particle, marked by the active cells themselves (near must start zeroed).
__global__ void k_h_dilate(int ncells, const BoxInfo* __restrict__ boxes, int nboxes,
                           const unsigned char* __restrict__ cellact, unsigned char* __restrict__ near) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells || !cellact[c]) return;
    int lo = 0, hi = nboxes - 1;  // box of the cell: last box with cell_off <= c
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].cell_off <= c)
            lo = mid;
        else
            hi = mid - 1;
    }
    const BoxInfo bx = boxes[lo];
    const int nc = bx.nc, l = c - bx.cell_off;
    const int cx = l % nc, cy = (l / nc) % nc, cz = l / (nc * nc);
    for (int dz = -2; dz <= 2; ++dz) {
        const int wz = ((cz + dz) % nc + nc) % nc;
        for (int dy = -2; dy <= 2; ++dy) {
            const int wy = ((cy + dy) % nc + nc) % nc;
            for (int dx = -2; dx <= 2; ++dx) {
                const int wx = ((cx + dx) % nc + nc) % nc;
                near[bx.cell_off + (wz * nc + wy) * nc + wx] = 1;
            }
        }
    }
}

template <typename T>
__device__ __forceinline__ int cell_of(T v, int nc) {
    T f = floor(v * (T)nc);
    if (!(f >= T(0))) return 0;
    if (f > (T)(nc - 1)) return nc - 1;
    return (int)f;
}

// The flux pairs of active i with r >= H_i (so r < H_j, O10), found from the
// partner's side: every particle j scans its own support (cells without an
// active particle skipped) and appends itself to the list of each active i
// there with r >= H_i; the lists are put in index order by k_h_sort.  r^2 is
// the bit pattern the density pass forms for the pair, so these lists and
// N_i split the flux pairs exactly.
template <typename T>
__global__ void __launch_bounds__(128)
    k_h_rscatter(int N, Sorted<T> s, Grid g, KParams p, const unsigned char* __restrict__ aflag,
                 const unsigned char* __restrict__ cellact, const unsigned char* __restrict__ near,
                 unsigned* __restrict__ rnbr, int* __restrict__ rcount, DevStatus* st) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const BoxInfo bx = g.boxes[s.box[j]];
    const P4<T> me = s.pos[j];
    const T Hj = me.w;
    // a support spanning under two cells lies within two cells of its own
    // (the scan's range floor((x -+ H) nc -+ 1e-3)): without an active cell
    // there, nothing to append
    if (Hj * (T)bx.nc < T(1.99)) {
        const int nc = bx.nc;
        if (!near[bx.cell_off + (cell_of(me.z, nc) * nc + cell_of(me.y, nc)) * nc + cell_of(me.x, nc)]) return;
    }
    const T H2 = Hj * Hj;
    const unsigned char* ca = cellact + bx.cell_off;
    for_candidates<T>(
        g, bx, s.pos, j, me.x, me.y, me.z, Hj,
        [&](int i, T, T, T, T r2) {
            if (r2 < H2 && aflag[i]) {
                const T Hi = s.pos[i].w;
                if (!(r2 < Hi * Hi)) {
                    const int slot = atomicAdd(&rcount[i], 1);
                    if (slot < p.rcap)
                        rnbr[lslot(slot, i, N)] = (unsigned)j;
                    else
                        set_status(st, GZ_S_NBR_OVERFLOW, GZ_C_NBR_OVERFLOW, s.id[i]);
                }
            }
        },
        [&](int lc) { return ca[lc] != 0; });
}

// Active i appends itself to the list of each inactive partner.
__global__ void k_h_inlist(const int* __restrict__ alist, const int* __restrict__ nA,
                           const unsigned char* __restrict__ aflag, unsigned* __restrict__ nbr,
                           int* __restrict__ ncount, const unsigned* __restrict__ rnbr,
                           const int* __restrict__ rcount, int cap, int rcap,
                           const long long* __restrict__ sid, int N, DevStatus* st) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *nA) return;
    const int i = alist[t];
    for (int list = 0; list < 2; ++list) {
        const unsigned* L = list == 0 ? nbr + 4 * (size_t)i : rnbr + 4 * (size_t)i;
        const int n = list == 0 ? min(ncount[i], cap) : min(rcount[i], rcap);
        for (int k = 0; k < n; ++k) {
            const int j = (int)L[lcol(k, N)];
            if (aflag[j]) continue;
            const int slot = atomicAdd(&ncount[j], 1);
            if (slot < cap)
                nbr[lslot(slot, j, N)] = (unsigned)i;
            else
                set_status(st, GZ_S_NBR_OVERFLOW, GZ_C_NBR_OVERFLOW, sid[j]);
        }
    }
}

// Index order for the lists written by other threads: the inactive
// particles' partner lists and the active particles' r >= H_i pairs.
__global__ void k_h_sort(int N, const unsigned char* __restrict__ aflag, int* __restrict__ ncount,
                         unsigned* __restrict__ nbr, int cap, const int* __restrict__ rcount,
                         unsigned* __restrict__ rnbr, int rcap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    unsigned* L;
    int n;
    if (aflag[i]) {
        L = rnbr + 4 * (size_t)i;
        n = min(rcount[i], rcap);
    } else {
        n = min(ncount[i], cap);
        ncount[i] = n;
        L = nbr + 4 * (size_t)i;
    }
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

__global__ void k_h_tflags(int N, const unsigned char* __restrict__ aflag, const int* __restrict__ ncount,
                           unsigned char* __restrict__ tflag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    tflag[i] = (unsigned char)(aflag[i] || ncount[i] > 0);
}

// ----------------------------------------------- per-particle bookkeeping
// Active particles keep what the inactive ones will read later: H (into the
// caller's h), n, the limited gradients and B (from the flux record).
template <typename T>
__global__ void k_h_persist(int N, const int* __restrict__ alist, const int* __restrict__ nA,
                            Sorted<T> s, const T* __restrict__ rec, gz_particles p, T* __restrict__ hn,
                            T* __restrict__ hgrad, T* __restrict__ hB) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *nA) return;
    const int i = alist[t];
    const unsigned o = s.orig[i];
    const T* R = rec + (size_t)i * kRecord;
    for (int q = 0; q < 15; ++q) hgrad[(size_t)q * N + o] = R[11 + q];
    for (int q = 0; q < 6; ++q) hB[(size_t)q * N + o] = R[26 + q];
    hn[o] = s.n[i];
    ((T*)p.h)[o] = s.h[i];
}

// Largest finite criterion of every box (substep 0): a warp's maximum in one
// atomic when the warp lies in one box (positive doubles order like their
// bit patterns).
__global__ void k_h_dtmax(const int* __restrict__ alist, const int* __restrict__ nA,
                          const int* __restrict__ box, const double* __restrict__ dti,
                          unsigned long long* __restrict__ dtmax) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = t < *nA;
    const int i = in ? alist[t] : 0;
    const double v = in ? dti[i] : 0.0;
    unsigned long long bits = (in && isfinite(v) && v > 0.0) ? (unsigned long long)__double_as_longlong(v) : 0ull;
    const int b = in ? box[i] : -1;
    const unsigned full = 0xffffffffu;
    const int b0 = __shfl_sync(full, b, 0);
    if (__all_sync(full, !in || b == b0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(full, bits, o);
            bits = w > bits ? w : bits;
        }
        if ((threadIdx.x & 31) == 0 && b0 >= 0 && bits) atomicMax(&dtmax[b0], bits);
    } else if (in && bits) {
        atomicMax(&dtmax[b], bits);
    }
}

// Interval per box: min(cfl max dtc, 2^K cfl min dtc).
__global__ void k_h_interval(int nb, const unsigned long long* __restrict__ dtmin,
                             const unsigned long long* __restrict__ dtmax, double cfl, int K,
                             double* __restrict__ D) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const double lo = __longlong_as_double((long long)dtmin[b]);
    const double hi = dtmax[b] ? __longlong_as_double((long long)dtmax[b]) : 0.0;
    const double a = cfl * hi, c = ldexp(cfl * lo, K);
    D[b] = a < c ? a : c;
}

__device__ __forceinline__ int bin_for(double D, double cfl_dtc, int K) {
    for (int k = 0; k <= K; ++k)
        if (ldexp(D, -k) <= cfl_dtc) return k;
    return K;
}

// Bins of the active particles: assigned at substep 0, deepened later.
__global__ void k_h_bins(const int* __restrict__ alist, const int* __restrict__ nA,
                         const unsigned* __restrict__ orig, const int* __restrict__ box,
                         const double* __restrict__ dti, const double* __restrict__ D, double cfl, int K,
                         int first, int* __restrict__ hbin, int* __restrict__ sbin) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *nA) return;
    const int i = alist[t];
    int k = bin_for(D[box[i]], cfl * dti[i], K);
    if (!first) k = max(k, sbin[i]);
    sbin[i] = k;
    hbin[orig[i]] = k;
}

// ------------------------------------------------------------ exchange
constexpr int kXBlock = 128;

// Touched particle i over its pair lists (an active particle: N_i then its
// r >= H_i pairs; an inactive one: its active partners): the pair's face
// fluxes with the Hancock half step of dt_ij, scaled by 2^(k_i - k_ij),
// summed like the flux pass (working precision over runs of 8 pairs, then
// FP64).  kRiem: the MFM face's Riemann solver; kMFV: the MFV fluxes, whose
// mass share is summed too (pair_rates).
template <typename T, int kRiem, bool kMFV>
__global__ void __launch_bounds__(kXBlock)
    k_h_exchange(const int* __restrict__ tlist, const int* __restrict__ nT, const T* __restrict__ rec,
                 const long long* __restrict__ sid, const int* __restrict__ sbox,
                 const int* __restrict__ sbin, const unsigned* __restrict__ nbr,
                 const int* __restrict__ ncount, const unsigned* __restrict__ rnbr,
                 const int* __restrict__ rcount, KParams p, const double* __restrict__ D,
                 double* __restrict__ dpdt, double* __restrict__ dEdt, double* __restrict__ dmdt, int N,
                 DevStatus* st) {
    constexpr int nq = kMFV ? 5 : 4;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *nT) return;
    const int i = tlist[t];
    T a[kRecord];
    load_rec(rec + (size_t)i * kRecord, a);
    const long long idi = kMFV ? sid[i] : 0;  // (MFV pairs are oriented by id)
    const int ka = sbin[i];
    const double Db = D[sbox[i]];
    const T gam = (T)p.gamma;
    const bool hancock = p.hancock != 0;
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
        for (int k = 0; k < cnt; ++k) {
            const int j = (int)L[lcol(k, N)];
            T b[kRecord];
            load_rec(rec + (size_t)j * kRecord, b);
            const int kab = max(ka, sbin[j]);
            const T hdt = (T)(0.5 * ldexp(Db, -kab));
            T inca[5];
            hancock_inc(a, hdt, gam, hancock, inca);
            T dp[3], dE, dm;
            int fl = 0;
            const bool aL = pair_order<kMFV>(i, j, idi, sid);
            if (pair_rates<T, kMFV, kRiem>(a, b, aL, hdt, gam, hancock, inca, dp, dE, dm, fl)) {
                const T sc = (T)ldexp(1.0, ka - kab);
                part[0] += dp[0] * sc;
                part[1] += dp[1] * sc;
                part[2] += dp[2] * sc;
                part[3] += dE * sc;
                if constexpr (kMFV) part[4] += dm * sc;
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

// Kick of a touched particle by dt_i times its scaled sums: the O14 momentum
// and energy update without the drift (FP64 literal form; FP32 increments,
// which also accumulate the step's velocity change for the drift).
template <typename T>
__global__ void k_h_kick(const int* __restrict__ tlist, const int* __restrict__ nT, int N, Sorted<T> s,
                         const int* __restrict__ sbin, const double* __restrict__ dpdt,
                         const double* __restrict__ dEdt, const double* __restrict__ dmdt,
                         const double* __restrict__ D, gz_particles out, T* __restrict__ hdvs,
                         int* __restrict__ box_hits, DevStatus* st) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *nT) return;
    const int i = tlist[t];
    const unsigned o = s.orig[i];
    const int b = s.box[i];
    const double dt = ldexp(D[b], -sbin[i]);
    const double dpx = dpdt[i], dpy = dpdt[(size_t)N + i], dpz = dpdt[2 * (size_t)N + i], dE = dEdt[i];
    T vx = s.vx[i], vy = s.vy[i], vz = s.vz[i], u = s.u[i];
    T m = s.m[i];
    if constexpr (std::is_same<T, float>::value) {
        float dvx, dvy, dvz;
        if (dmdt)
            kick_one_mfv(m, vx, vy, vz, u, dpx, dpy, dpz, dE, dmdt[i], dt, dvx, dvy, dvz);
        else
            kick_one(m, vx, vy, vz, u, dpx, dpy, dpz, dE, dt, dvx, dvy, dvz);
        hdvs[o] = __fadd_rn(hdvs[o], dvx);
        hdvs[(size_t)N + o] = __fadd_rn(hdvs[(size_t)N + o], dvy);
        hdvs[2 * (size_t)N + o] = __fadd_rn(hdvs[2 * (size_t)N + o], dvz);
    } else {
        if (dmdt)
            kick_one_mfv(m, vx, vy, vz, u, dpx, dpy, dpz, dE, dmdt[i], dt);
        else
            kick_one(m, vx, vy, vz, u, dpx, dpy, dpz, dE, dt);
    }
    if (dmdt) ((T*)out.m)[o] = m;
    ((T*)out.vx)[o] = vx;
    ((T*)out.vy)[o] = vy;
    ((T*)out.vz)[o] = vz;
    ((T*)out.u)[o] = u;
    if (!(u > T(0))) {
        atomicAdd(&box_hits[b], 1);
        set_status(st, GZ_S_UFLOOR, GZ_C_UFLOOR, -1);
    }
    if (!(m > T(0) && finite_(vx) && finite_(vy) && finite_(vz) && finite_(u)))
        set_status(st, GZ_S_NONFINITE, GZ_C_NONFINITE, s.id[i]);
}

// End of the steps that finish after substep s: drift by dt_i v_bar, new
// step start (caller order).
template <typename T>
__global__ void k_h_finalize(int N, int s, int K, gz_particles p, T* __restrict__ hva, T* __restrict__ hdvs,
                             int* __restrict__ hsa, const int* __restrict__ hbin,
                             const int* __restrict__ box_of, const double* __restrict__ D, DevStatus* st) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= N) return;
    const int k = hbin[o];
    if ((s + 1) % (1 << (K - k)) != 0) return;
    const double dt = ldexp(D[box_of[o]], -k);
    T* X[3] = {(T*)p.x, (T*)p.y, (T*)p.z};
    const T* V[3] = {(const T*)p.vx, (const T*)p.vy, (const T*)p.vz};
    bool ok = true;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const size_t q = (size_t)r * N + o;
        T x;
        if constexpr (std::is_same<T, float>::value)
            x = drift_onef(X[r][o], hva[q], hdvs[q], dt);
        else
            x = drift_one(X[r][o], hva[q], V[r][o], dt);
        X[r][o] = x;
        ok = ok && finite_(x);
        hva[q] = V[r][o];
        hdvs[q] = T(0);
    }
    hsa[o] = s + 1;
    if (!ok) set_status(st, GZ_S_NONFINITE, GZ_C_NONFINITE, (long long)p.id[o]);
}

template <typename T>
void launch_exchange(Ctx& c, const KParams& kp, int N) {
    const int r = c.params.riemann;
    auto go = [&](auto kernel) {
        kernel<<<nblk(N, kXBlock), kXBlock, 0, c.stream>>>(c.tlist, c.hcount + 2, (const T*)c.rec, c.sid, c.sbox,
                                                           c.sbin, c.nbr, c.ncount, c.rnbr, c.rcount, kp, c.dt_use,
                                                           c.dpdt, c.dEdt, c.dmdt, N, c.status);
    };
    if (c.params.scheme == GZ_MFV)
        go(k_h_exchange<T, GZ_RIEMANN_HLLC, true>);
    else if (r == GZ_RIEMANN_EXACT)
        go(k_h_exchange<T, GZ_RIEMANN_EXACT, false>);
    else if (r == GZ_RIEMANN_FALLBACK)
        go(k_h_exchange<T, GZ_RIEMANN_FALLBACK, false>);
    else
        go(k_h_exchange<T, GZ_RIEMANN_HLLC, false>);
}

}  // namespace

cudaError_t ensure_hier_scratch(Ctx& c) {
    if (c.hier_arena) return cudaSuccess;
    // sized for the context's capacity (a subdomain context's N changes)
    const size_t Nz = (size_t)c.capacity, sz = c.precision == GZ_FP64 ? 8 : 4;
    const size_t nb = (size_t)nblk(c.capacity, kCmpBlock);
    struct Item {
        void** ptr;
        size_t bytes;
    } items[] = {
        {&c.hxp, 3 * sz * Nz},         {&c.hva, 3 * sz * Nz},        {&c.hdvs, 3 * sz * Nz},
        {&c.hn, sz * Nz},              {&c.hgrad, 15 * sz * Nz},     {&c.hB, 6 * sz * Nz},
        {(void**)&c.hsa, 4 * Nz},      {(void**)&c.hbin, 4 * Nz},    {(void**)&c.sbin, 4 * Nz},
        {(void**)&c.alist, 4 * Nz},    {(void**)&c.tlist, 4 * Nz},   {(void**)&c.hcount, 4 * 4},
        {(void**)&c.bcount, 4 * nb},   {(void**)&c.aflag, Nz},       {(void**)&c.tflag, Nz},
        {(void**)&c.cellact, (size_t)c.total_cells}, {(void**)&c.cellnear, (size_t)c.total_cells},
        {(void**)&c.dtmax, 8 * (size_t)c.nboxes},
    };
    size_t total = 0;
    for (auto& it : items) total += (it.bytes + 255) & ~(size_t)255;
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, total);
    if (e != cudaSuccess) return e;
    e = cudaMallocHost((void**)&c.hcount_host, 4 * sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(base);
        return e;
    }
    char* q = (char*)base;
    for (auto& it : items) {
        *it.ptr = q;
        q += (it.bytes + 255) & ~(size_t)255;
    }
    c.hier_arena = base;
    return cudaSuccess;
}

static cudaError_t compact(Ctx& c, const unsigned char* flag, int* list, int* count) {
    const int nb = nblk(c.N, kCmpBlock);
    c.launches += 3;
    k_cmp_count<<<nb, kCmpBlock, 0, c.stream>>>(c.N, flag, c.bcount);
    k_cmp_scan<<<1, kCmpBlock, 0, c.stream>>>(nb, c.bcount, count);
    k_cmp_write<<<nb, kCmpBlock, 0, c.stream>>>(c.N, flag, c.bcount, list);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_step_hier(Ctx& c, gz_particles& p, int K, double dt_fixed, double* dt_used_dev,
                          int32_t* bins_out, long long* active_out, const PassTimer& timer) {
    cudaError_t e = ensure_hier_scratch(c);
    if (e != cudaSuccess) return e;
    const int N = c.N;
    cudaStream_t st = c.stream;
    const KParams kp = kparams(c);
    Grid g;
    g.boxes = c.boxes;
    g.cells = c.cells;
    T* hxp = (T*)c.hxp;
    gz_particles pp = p;  // predicted positions, everything else the caller's arrays
    pp.x = hxp;
    pp.y = hxp + N;
    pp.z = hxp + 2 * (size_t)N;
    c.launches += 1;
    k_h_init<T><<<nblk(N, 256), 256, 0, st>>>(N, p, (T*)c.hva, (T*)c.hdvs, c.hsa, c.hbin);
    long long active = 0;
    const int S = 1 << K;
    for (int s = 0; s < S && e == cudaSuccess; ++s) {
        cudaMemsetAsync(c.hcount, 0, 4 * sizeof(int), st);
        c.launches += 1;
        k_h_predict<T><<<nblk(N, 256), 256, 0, st>>>(N, s, K, p, (const T*)c.hva, (const T*)c.hdvs, c.hsa,
                                                      c.hbin, c.box_of, c.dt_use, hxp, c.hcount);
        cudaMemcpyAsync(c.hcount_host, c.hcount, sizeof(int), cudaMemcpyDeviceToHost, st);
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        const int nA = c.hcount_host[0];
        active += nA;
        if (nA > 0) {
            Sorted<T> sv = sorted_view<T>(c);
            timer.begin(GZ_PASS_SORT);
            e = sort_and_bin<T>(c, pp, c.hn);
            c.launches += 1;
            k_h_flags<<<nblk(N, 256), 256, 0, st>>>(N, s, K, c.vals, c.hbin, c.sbin, c.aflag);
            if (e == cudaSuccess) e = compact(c, c.aflag, c.alist, c.hcount + 1);
            timer.end(GZ_PASS_SORT);
            cudaMemsetAsync(c.ncount, 0, sizeof(int) * (size_t)N, st);
            cudaMemsetAsync(c.rcount, 0, sizeof(int) * (size_t)N, st);
            timer.begin(GZ_PASS_DENSITY);
            if (e == cudaSuccess) e = run_density<T>(c, c.alist, c.hcount + 1, nA);
            timer.end(GZ_PASS_DENSITY);
            timer.begin(GZ_PASS_PRIM);
            if (e == cudaSuccess) e = run_prim<T>(c);
            timer.end(GZ_PASS_PRIM);
            timer.begin(GZ_PASS_REVERSE);
            c.launches += 6;
            c.launches += 1;
            k_h_cellact<<<nblk(c.total_cells, 256), 256, 0, st>>>(c.total_cells, c.cells, c.aflag, c.cellact);
            cudaMemsetAsync(c.cellnear, 0, (size_t)c.total_cells, st);
            k_h_dilate<<<nblk(c.total_cells, 256), 256, 0, st>>>(c.total_cells, c.boxes, c.nboxes, c.cellact,
                                                                  c.cellnear);
            k_h_rscatter<T><<<nblk(N, 128), 128, 0, st>>>(N, sv, g, kp, c.aflag, c.cellact, c.cellnear, c.rnbr,
                                                           c.rcount, c.status);
            k_h_inlist<<<nblk(nA, 128), 128, 0, st>>>(c.alist, c.hcount + 1, c.aflag, c.nbr, c.ncount, c.rnbr,
                                                       c.rcount, c.cap, c.rcap, c.sid, c.N, c.status);
            k_h_sort<<<nblk(N, 128), 128, 0, st>>>(N, c.aflag, c.ncount, c.nbr, c.cap, c.rcount, c.rnbr,
                                                    c.rcap);
            k_h_tflags<<<nblk(N, 256), 256, 0, st>>>(N, c.aflag, c.ncount, c.tflag);
            if (e == cudaSuccess) e = compact(c, c.tflag, c.tlist, c.hcount + 2);
            timer.end(GZ_PASS_REVERSE);
            timer.begin(GZ_PASS_GRAD);
            if (e == cudaSuccess) e = run_gradients<T>(c, true, false, c.alist, c.hcount + 1, nA);
            if (e == cudaSuccess)
                e = run_pack_given<T>(c, (const T*)c.hgrad, (const T*)c.hB, c.tlist, c.hcount + 2, N, c.aflag);
            c.launches += 1;
            k_h_persist<T><<<nblk(nA, 256), 256, 0, st>>>(N, c.alist, c.hcount + 1, sv, (const T*)c.rec, p,
                                                           (T*)c.hn, (T*)c.hgrad, (T*)c.hB);
            if (s == 0) {
                if (dt_fixed > 0.0) {
                    if (e == cudaSuccess) e = run_dt_set(c, dt_fixed);
                } else {
                    cudaMemsetAsync(c.dtmax, 0, 8 * (size_t)c.nboxes, st);
                    c.launches += 2;
                    k_h_dtmax<<<nblk(nA, 256), 256, 0, st>>>(c.alist, c.hcount + 1, c.sbox, c.dti, c.dtmax);
                    k_h_interval<<<nblk(c.nboxes, 256), 256, 0, st>>>(
                        c.nboxes, (const unsigned long long*)c.dt_box, c.dtmax, c.params.cfl, K, c.dt_use);
                }
            }
            c.launches += 1;
            k_h_bins<<<nblk(nA, 256), 256, 0, st>>>(c.alist, c.hcount + 1, c.vals, c.sbox, c.dti, c.dt_use,
                                                     c.params.cfl, K, s == 0 ? 1 : 0, c.hbin, c.sbin);
            timer.end(GZ_PASS_GRAD);
            timer.begin(GZ_PASS_FLUX);
            c.launches += 1;
            launch_exchange<T>(c, kp, N);
            timer.end(GZ_PASS_FLUX);
            timer.begin(GZ_PASS_UPDATE);
            cudaMemsetAsync(c.box_hits, 0, sizeof(int) * (size_t)c.nboxes, st);
            c.launches += 1;
            k_h_kick<T><<<nblk(N, 256), 256, 0, st>>>(c.tlist, c.hcount + 2, N, sv, c.sbin, c.dpdt, c.dEdt,
                                                       c.params.scheme == GZ_MFV ? c.dmdt : nullptr, c.dt_use,
                                                       p, (T*)c.hdvs, c.box_hits, c.status);
            if (e == cudaSuccess) e = run_ufloor<T>(c, p);
            timer.end(GZ_PASS_UPDATE);
        }
        c.launches += 1;
        k_h_finalize<T><<<nblk(N, 256), 256, 0, st>>>(N, s, K, p, (T*)c.hva, (T*)c.hdvs, c.hsa, c.hbin,
                                                       c.box_of, c.dt_use, c.status);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess && dt_used_dev)
        e = cudaMemcpyAsync(dt_used_dev, c.dt_use, sizeof(double) * (size_t)c.nboxes, cudaMemcpyDeviceToDevice,
                            st);
    if (e == cudaSuccess && bins_out)
        e = cudaMemcpyAsync(bins_out, c.hbin, sizeof(int) * (size_t)N, cudaMemcpyDeviceToDevice, st);
    c.nbr_valid = 0;  // the lists now mix active lists with partner lists
    if (active_out) *active_out = active;
    return e;
}

template cudaError_t run_step_hier<float>(Ctx&, gz_particles&, int, double, double*, int32_t*, long long*,
                                          const PassTimer&);
template cudaError_t run_step_hier<double>(Ctx&, gz_particles&, int, double, double*, int32_t*, long long*,
                                           const PassTimer&);

void free_hier_scratch(Ctx& c) {
    if (c.hier_arena) cudaFree(c.hier_arena);
    if (c.hcount_host) cudaFreeHost(c.hcount_host);
    c.hier_arena = nullptr;
    c.hcount_host = nullptr;
}

}  // namespace gz
