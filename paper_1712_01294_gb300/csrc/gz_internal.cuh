// Internal declarations of the GB300 MFM library: context layout, device
// status, kernel-side helpers.  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gz.h"

namespace gz {

constexpr double kPi = 3.14159265358979323846;
constexpr int kRecord = 32;  // values per packed particle record (flux pass)
constexpr int kAdj = 33;     // adjoint values per particle (see gz_adjoint.cu)
constexpr int kSeed = 56;    // gradient-pass adjoint record per particle (working precision):
                             // [0,15) S_bar, [15,21) E_bar, 21 psi norm, [22,27) W, 27 pad,
                             // [28,53) limiter seeds (5 per field), [53,56) pad
constexpr int kGInfo = 40;   // raw gradients, S sums, limiter factors, active limiter Delta

// Device status word (one per context).
struct DevStatus {
    unsigned int bits;
    unsigned int pad;
    unsigned long long first_bad_id;  // smallest id with an error bit (~0 = none)
    unsigned long long counters[GZ_NCOUNTERS];
};

// Per-box cell grid description (device table).
struct BoxInfo {
    int nc;          // cells per axis
    int cell_off;    // first cell of this box in the cell array
    int first;       // first particle (sorted order == caller order per box)
    int count;       // particles in the box
};

// Scalar parameters passed by value to kernels.
struct KParams {
    double gamma, ngb, tol, cfl, kappa_max, beta, u_floor_frac, h_lim;
    int hancock, max_iter, cap, rcap, scheme;
};

// Packed per-particle records (one 16-byte-aligned vector load each).
template <typename T>
struct alignas(16) P4 {
    T x, y, z, w;
};
template <typename T>
struct alignas(2 * sizeof(T)) P2 {
    T x, y;
};

// Sorted-order views the kernels share.
template <typename T>
struct Sorted {
    T *x, *y, *z, *vx, *vy, *vz, *m, *u, *h;
    long long* id;      // original ids, sorted order
    unsigned* orig;     // caller index of sorted particle
    int* box;           // box of sorted particle
    T *n, *rho, *P, *c;
    T* sd;              // sum over N_i of -w'(q) q at the converged H (density pass)
    P4<T>* pos;         // (x, y, z, H)
    P4<T>* prim;        // (rho, vx, vy, vz)
    P2<T>* prim2;       // (P, c)
};

struct Grid {
    const BoxInfo* boxes;  // device
    const int2* cells;     // (start, end) per cell, all boxes
};

struct Ctx {
    gz_params params;
    int precision;
    int N;
    int nboxes;
    std::vector<int64_t> counts;
    std::vector<BoxInfo> hboxes;
    int total_cells;
    int cbits;     // bits per axis of a cell coordinate
    int box_bits;  // bits of the box index in a key
    cudaStream_t stream;
    // a second stream for the step checkpoint's list copies, which overlap
    // the pair passes (created on the first checkpointing step)
    cudaStream_t side = nullptr;
    cudaEvent_t side_fork = nullptr, side_join = nullptr;
    std::string err;

    // device buffers
    void* arena;
    size_t arena_bytes;
    BoxInfo* boxes;
    int2* cells;
    unsigned *keys, *keys_alt, *vals, *vals_alt;
    unsigned* hist;
    int hist_len;
    int* box_of;  // caller order
    // sorted state (working precision) and derived per-particle data
    void *sx, *sy, *sz, *svx, *svy, *svz, *sm, *su, *sh, *sn, *srho, *sP, *sc, *ssd;
    void *spos, *sprim, *sprim2;  // packed records P4 (x y z H), P4 (rho v), P2 (P c)
    long long* sid;
    int* sbox;
    int* iters;
    int* ncount;
    unsigned* nbr;  // cap slots a particle, in groups of four across the particles (lslot)
    int* rcount;
    unsigned* rnbr;  // rcap slots a particle, laid out like nbr
    void* rec;       // [N][kRecord] working precision
    int* defer = nullptr;   // [N] particles the density pass leaves to its warp-per-particle kernel
    int* ndefer = nullptr;  // [1] their number
    double* dpdt;    // [3][N] sorted
    double* dEdt;    // [N] sorted
    double* dmdt;    // [N] sorted (GZ_MFV only, else null)
    double* dti;     // [N] sorted
    double* dt_box;  // [nboxes] CFL minimum (before the cfl factor is applied: raw min)
    double* dt_use;  // [nboxes] step used
    int* box_hits;   // [nboxes] u-floor hits of the current step
    DevStatus* status;
    int cap, rcap;
    int nbr_valid;  // neighbour lists of the last density pass are current
    long long launches;  // kernel launches issued
    // per-pass CUDA-event profile
    int prof;
    std::vector<cudaEvent_t> ev_pool;
    struct Pending {
        int pass;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    cudaEvent_t open_ev[GZ_NPASSES] = {};  // PassTimer::begin events awaiting their end
    double prof_ms[GZ_NPASSES];
    long long prof_calls[GZ_NPASSES];
    long long* pairs_dev;  // scratch for gz_pair_count
    // captured multi-step graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    long long graph_kernels = 0;
    // adjoint scratch, allocated on the first backward call
    void* adj_arena = nullptr;
    void* adj = nullptr;      // [N][kAdj] working precision
    void* wgt = nullptr;      // [N][4] rate adjoints (working precision); then kappa [N]
    void* seeds = nullptr;    // [N][kSeed] working precision
    unsigned long long* lbloom = nullptr;  // [N] bit (j & 63) set for each limiter target j
    int* lim = nullptr;       // [N][10] limiter: active neighbour, extreme particle per field
    void* ginfo = nullptr;    // [N][kGInfo] working precision
    // hierarchical-step scratch, allocated on the first gz_step_hier call
    void* hier_arena = nullptr;
    void* hxp = nullptr;      // [3][N] predicted positions (caller order)
    void* hva = nullptr;      // [3][N] velocity at the start of each particle's step
    void* hdvs = nullptr;     // [3][N] velocity change since then
    void* hn = nullptr;       // [N] n of each particle's last active time
    void* hgrad = nullptr;    // [15][N] limited gradients of that time
    void* hB = nullptr;       // [6][N] E^-1 of that time
    int* hsa = nullptr;       // [N] substep its current step started at
    int* hbin = nullptr;      // [N] bin (caller order)
    int* sbin = nullptr;      // [N] bin (sorted order)
    int* alist = nullptr;     // [N] active particles (sorted indices)
    int* tlist = nullptr;     // [N] particles with an exchange this substep
    int* hcount = nullptr;    // [4] device counters (predicted actives, |alist|, |tlist|)
    int* bcount = nullptr;    // per-block counts of the list compaction
    unsigned char* aflag = nullptr;  // [N] active (sorted order)
    unsigned char* tflag = nullptr;  // [N] touched (sorted order)
    unsigned char* cellact = nullptr;     // [cells] cell holds an active particle
    unsigned char* cellnear = nullptr;    // [cells] an active cell lies within two cells
    unsigned long long* dtmax = nullptr;  // [nboxes] largest finite criterion (bits)
    int* hcount_host = nullptr;           // pinned copy of hcount
    // subdomain of a decomposed box (gz_create_subdomain): the particles held
    // are the owned ones and ghost copies completing their neighbourhoods
    unsigned char* owned = nullptr;  // [capacity] 1 = owned (caller order); null: all owned
    int n_owned = 0;                 // owned particles held
    long long grid_count = 0;        // particle count the cell grid is built for (0: the box's own)
    int capacity = 0;                // particles the arrays hold (the context's creation count)
    int step_open = 0;               // gz_step_begin done, gz_step_finish pending
    const int* last_lim = nullptr;   // limiter indices of the last step checkpoint, in this sort
};

// ------------------------------------------------------------------ status
__device__ __forceinline__ void set_status(DevStatus* st, unsigned bit, int counter,
                                           long long id) {
    atomicOr(&st->bits, bit);
    atomicAdd(&st->counters[counter], 1ull);
    if ((bit & GZ_S_ERROR_MASK) && id >= 0)
        atomicMin(&st->first_bad_id, (unsigned long long)id);
}

// --------------------------------------------------------- O1 min image
// FP64: exactly the oracle's expression (difference, then shift by one).
__device__ __forceinline__ double mi_diff(double xj, double xi, double /*xim1*/) {
    double d = xj - xi;
    if (d >= 0.5)
        d = d - 1.0;
    else if (d < -0.5)
        d = d + 1.0;
    return d;
}
// FP32: shift the operand near 1 first (x - 1 is exact for x in [1/2, 1)),
// so the wrapped offset is correctly rounded like an unwrapped one.
__device__ __forceinline__ float mi_diff(float xj, float xi, float xim1) {
    float d = xj - xi;
    float dl = __fsub_rn(__fsub_rn(xj, 1.0f), xi);
    float dh = __fsub_rn(xj, xim1);
    return d >= 0.5f ? dl : (d < -0.5f ? dh : d);
}

// --------------------------------------------------------- O2 kernel
template <typename T>
__device__ __forceinline__ T kern_w(T q) {
    T t = T(1) - q;
    T a = T(1) + q * q * (T(-6) + T(6) * q);
    T b = T(2) * t * t * t;
    return q <= T(0.5) ? a : (q < T(1) ? b : T(0));
}
template <typename T>
__device__ __forceinline__ T kern_dw(T q) {
    T t = T(1) - q;
    T a = q * (T(-12) + T(18) * q);
    T b = T(-6) * t * t;
    return q <= T(0.5) ? a : (q < T(1) ? b : T(0));
}

// The two terms of the density sum at q = r / H (Eq. O2's kernel): W(q) and
// -q W'(q).  FP64: the pieces as above.  FP32: one cubic in x = q (q <= 1/2)
// or x = 1 - q (beyond), whose coefficients are selected, not both pieces
// evaluated:  W = 1 - 6x^2 + 6x^3 | 2x^3,  -q W' = 12x^2 - 18x^3 | 6x^2 - 6x^3
// (the outer piece in 1 - q, as in kern_w, so no cancellation near q = 1).
// Callers pass q < 1 up to rounding (entries with r^2 < H^2).
template <typename T>
__device__ __forceinline__ void dens_terms(T q, T& w, T& qdw) {
    w = kern_w(q);
    qdw = -kern_dw(q) * q;
}
template <>
__device__ __forceinline__ void dens_terms<float>(float q, float& w, float& qdw) {
    const bool in = q <= 0.5f;
    const float x = in ? q : 1.f - q;
    const float x2 = x * x;
    w = fmaf(fmaf(in ? 6.f : 2.f, x, in ? -6.f : 0.f), x2, in ? 1.f : 0.f);
    qdw = fmaf(in ? -18.f : -6.f, x, in ? 12.f : 6.f) * x2;
}

__device__ __forceinline__ bool finite_(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_(double v) { return isfinite(v); }

// r^2 = (dx dx + dy dy) + dz dz.  FP64 rounds after every operation (no FMA
// contraction), exactly like the oracle, so neighbour decisions agree bitwise.
__device__ __forceinline__ double sep2(double dx, double dy, double dz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}
// FP32: written with explicit fused multiply-adds so that every kernel forms
// r^2 of a pair with the same bits, whatever the compiler contracts elsewhere.
__device__ __forceinline__ float sep2(float dx, float dy, float dz) {
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Neighbour lists (N_i and the reverse lists) are stored in groups of four
// slots: slots 4g..4g+3 of sorted particle i are the 16 bytes at (g N + i) 4,
// N the context's particle count.  A warp, whose threads hold consecutive
// particles, reads one group of their lists as 512 contiguous bytes, one
// 16-byte load a thread.  A particle's list is the column nbr + 4 i; slot k
// of a column lies at lcol(k, N).  (Capacities are multiples of four.)
__device__ __forceinline__ size_t lcol(int k, int N) { return (size_t)(k >> 2) * 4 * (size_t)N + (size_t)(k & 3); }
__device__ __forceinline__ size_t lslot(int k, int i, int N) { return 4 * (size_t)i + lcol(k, N); }
// Slots k0..k0+3 (k0 a multiple of four) of the list column L; those at or
// past the list's count hold no particle.
__device__ __forceinline__ uint4 col4(const unsigned* __restrict__ L, int k0, int N) {
    return *reinterpret_cast<const uint4*>(L + lcol(k0, N));
}
// The same slots for a pass that reads each list once: not kept in L1, which
// stays for the records and positions the pass gathers (a pass that reads
// its lists twice, like the gradient pass, keeps col4).
__device__ __forceinline__ uint4 col4_once(const unsigned* __restrict__ L, int k0, int N) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(L + lcol(k0, N)));
    return r;
}

// A list slot written by the pass that builds the list: not allocated in
// L1, which stays for the candidates' positions the pass is scanning.
__device__ __forceinline__ void store_slot(unsigned* p, unsigned v) {
    asm volatile("st.global.L1::no_allocate.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ordered-integer image of a non-negative double (for atomicMin)
__device__ __forceinline__ unsigned long long dbits(double v) {
    return (unsigned long long)__double_as_longlong(v);
}

// Loop over all candidates j != self in the cells that overlap the cube
// [x - R, x + R] of particle self's box, calling fn(j, dx, dy, dz, r2).
// FP32 with a range well inside half the box: the periodic shift is chosen
// per cell row instead of per candidate, d = (x_j + a) - b with
// (a, b) = (0, x_i), (-1, x_i) for cells wrapped below 0 (x_j - 1 is exact
// there) or (0, x_i - 1) for cells wrapped above 1 (x_i - 1 is exact): the
// same correctly rounded offsets mi_diff gives, at a third of the cost.
// On that path fn is also called for the slots of the last group of four
// that lie past a cell's range, with r2 = +inf (j then names no candidate):
// every fn tests r2 against a finite radius before it uses j, so those calls
// do nothing, and the loop needs no per-candidate bounds test.  Candidates
// arrive in ascending j within each cell, as on the other path.
struct AllCells {
    __device__ __forceinline__ bool operator()(int) const { return true; }
};
template <typename T, typename F, typename CellOk = AllCells>
__device__ __forceinline__ void for_candidates(const Grid& g, const BoxInfo& bx,
                                               const P4<T>* __restrict__ pos, int self, T xi, T yi,
                                               T zi, T R, F&& fn, CellOk cell_ok = CellOk()) {
    const int nc = bx.nc;
    const int2* __restrict__ cells = g.cells + bx.cell_off;
    // positions outside [0, 1] (flagged by the binning pass) see no candidates
    if (!(xi >= T(0) && xi <= T(1) && yi >= T(0) && yi <= T(1) && zi >= T(0) && zi <= T(1) &&
          R >= T(0)))
        return;
    const bool full = !(R < T(0.5));  // (also catches non-finite R)
    const T c3[3] = {xi, yi, zi};
    int lo[3], hi[3];
    bool wraps_all = full;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = full ? 0 : (int)floor((c3[a] - R) * (T)nc - T(1e-3));
        hi[a] = full ? nc - 1 : (int)floor((c3[a] + R) * (T)nc + T(1e-3));
        if (hi[a] - lo[a] + 1 >= nc) {
            lo[a] = 0;
            hi[a] = nc - 1;
            wraps_all = true;
        }
    }
    const T xim1 = xi - T(1), yim1 = yi - T(1), zim1 = zi - T(1);
    const bool percell = sizeof(T) == 4 && !wraps_all && (T(2) * R + T(2) / (T)nc < T(0.5));
    // cells whose nearest point lies beyond R hold no candidate: skipped (the
    // gap of each axis from the cell's unwrapped extent; the margin covers the
    // rounding of the cell bounds; no pruning when the range wraps the box)
    const T cl = T(1) / (T)nc, R2m = R * R * T(1.0001);
    for (int cz = lo[2]; cz <= hi[2]; ++cz) {
        const int wz = cz < 0 ? cz + nc : (cz >= nc ? cz - nc : cz);
        const T az = cz < 0 ? T(-1) : T(0), bz = cz >= nc ? zim1 : zi;
        const T gz = wraps_all ? T(0) : max(max((T)cz * cl - zi, zi - (T)(cz + 1) * cl), T(0));
        const T gz2 = gz * gz;
        if (gz2 > R2m) continue;
        for (int cy = lo[1]; cy <= hi[1]; ++cy) {
            const int wy = cy < 0 ? cy + nc : (cy >= nc ? cy - nc : cy);
            const T ay = cy < 0 ? T(-1) : T(0), by = cy >= nc ? yim1 : yi;
            const T gy = wraps_all ? T(0) : max(max((T)cy * cl - yi, yi - (T)(cy + 1) * cl), T(0));
            const T gzy2 = gz2 + gy * gy;
            if (gzy2 > R2m) continue;
            const int row = (wz * nc + wy) * nc;
            for (int cx = lo[0]; cx <= hi[0]; ++cx) {
                const int wx = cx < 0 ? cx + nc : (cx >= nc ? cx - nc : cx);
                const T ax = cx < 0 ? T(-1) : T(0), bxx = cx >= nc ? xim1 : xi;
                const T gx = wraps_all ? T(0) : max(max((T)cx * cl - xi, xi - (T)(cx + 1) * cl), T(0));
                if (gzy2 + gx * gx > R2m) continue;
                if (!cell_ok(row + wx)) continue;  // (cell index within the box)
                const int2 se = cells[row + wx];
                if (percell) {
                    // four candidates' positions in flight at a time, their
                    // offsets formed before any is used (independent chains);
                    // slots past the range read a far-away point (r2 = +inf)
                    for (int j0 = se.x; j0 < se.y; j0 += 4) {
                        P4<T> q[4];
                        T dxs[4], dys[4], dzs[4], r2s[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            q[u] = j0 + u < se.y ? pos[j0 + u] : P4<T>{T(1e30), T(1e30), T(1e30), T(0)};
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            dxs[u] = (q[u].x + ax) - bxx;
                            dys[u] = (q[u].y + ay) - by;
                            dzs[u] = (q[u].z + az) - bz;
                            r2s[u] = sep2(dxs[u], dys[u], dzs[u]);
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (j0 + u != self) fn(j0 + u, dxs[u], dys[u], dzs[u], r2s[u]);
                    }
                } else {
                    for (int j0 = se.x; j0 < se.y; j0 += 4) {
                        P4<T> q[4];
                        T dxs[4], dys[4], dzs[4], r2s[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (j0 + u < se.y) q[u] = pos[j0 + u];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            dxs[u] = mi_diff(q[u].x, xi, xim1);
                            dys[u] = mi_diff(q[u].y, yi, yim1);
                            dzs[u] = mi_diff(q[u].z, zi, zim1);
                            r2s[u] = sep2(dxs[u], dys[u], dzs[u]);
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int j = j0 + u;
                            if (j >= se.y) break;
                            if (j == self) continue;
                            fn(j, dxs[u], dys[u], dzs[u], r2s[u]);
                        }
                    }
                }
            }
        }
    }
}

constexpr int kLaneCells = 16;

// Warp-cooperative candidate scan for one particle per warp (every lane
// passes the same particle): each lane calls fn(j, dx, dy, dz, r2) for its
// share of the candidates j != self in the cells overlapping [x - R, x + R]
// (cells whose nearest point lies beyond R skipped, as in for_candidates).
// Ranges of under kLaneCells cells are shared candidate by candidate (the
// lanes take start + lane, start + 32 + lane, ... of every cell); larger ones
// cell by cell (lane l takes cells l, l + 32, ... of the range, in row
// order), which keeps lanes busy where a support holds many cells and puts
// the cells' range and candidate loads in flight together instead of one
// cell after another.  Which lane
// sees which candidate depends only on the particle, so per-lane sums
// combined in a fixed order are deterministic.  Offsets from mi_diff.
template <typename T, typename F>
__device__ __forceinline__ void for_candidates_lanes(const Grid& g, const BoxInfo& bx,
                                                     const P4<T>* __restrict__ pos, int self, T xi, T yi,
                                                     T zi, T R, int lane, F&& fn) {
    const int nc = bx.nc;
    const int2* __restrict__ cells = g.cells + bx.cell_off;
    if (!(xi >= T(0) && xi <= T(1) && yi >= T(0) && yi <= T(1) && zi >= T(0) && zi <= T(1) &&
          R >= T(0)))
        return;
    const bool full = !(R < T(0.5));
    const T c3[3] = {xi, yi, zi};
    int lo[3], hi[3];
    bool wraps_all = full;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = full ? 0 : (int)floor((c3[a] - R) * (T)nc - T(1e-3));
        hi[a] = full ? nc - 1 : (int)floor((c3[a] + R) * (T)nc + T(1e-3));
        if (hi[a] - lo[a] + 1 >= nc) {
            lo[a] = 0;
            hi[a] = nc - 1;
            wraps_all = true;
        }
    }
    const T xim1 = xi - T(1), yim1 = yi - T(1), zim1 = zi - T(1);
    const T cl = T(1) / (T)nc, R2m = R * R * T(1.0001);
    auto gap = [&](int c, T v) { return wraps_all ? T(0) : max(max((T)c * cl - v, v - (T)(c + 1) * cl), T(0)); };
    auto cell_range = [&](int cx, int cy, int cz, int2& se) {
        const T gx = gap(cx, xi), gy = gap(cy, yi), gz = gap(cz, zi);
        if (gx * gx + gy * gy + gz * gz > R2m) return false;
        const int wx = cx < 0 ? cx + nc : (cx >= nc ? cx - nc : cx);
        const int wy = cy < 0 ? cy + nc : (cy >= nc ? cy - nc : cy);
        const int wz = cz < 0 ? cz + nc : (cz >= nc ? cz - nc : cz);
        se = cells[(wz * nc + wy) * nc + wx];
        return true;
    };
    auto visit = [&](int j) {
        const P4<T> q = pos[j];
        const T dx = mi_diff(q.x, xi, xim1), dy = mi_diff(q.y, yi, yim1), dz = mi_diff(q.z, zi, zim1);
        fn(j, dx, dy, dz, sep2(dx, dy, dz));
    };
    const int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
    const int ncube = ex * ey * ez;
    if (ncube >= kLaneCells) {
        for (int f = lane; f < ncube; f += 32) {
            const int cx = lo[0] + f % ex, cy = lo[1] + (f / ex) % ey, cz = lo[2] + f / (ex * ey);
            int2 se;
            if (!cell_range(cx, cy, cz, se)) continue;
            for (int j = se.x; j < se.y; ++j)
                if (j != self) visit(j);
        }
    } else {
        for (int cz = lo[2]; cz <= hi[2]; ++cz)
            for (int cy = lo[1]; cy <= hi[1]; ++cy)
                for (int cx = lo[0]; cx <= hi[0]; ++cx) {
                    int2 se;
                    if (!cell_range(cx, cy, cz, se)) continue;
                    for (int j = se.x + lane; j < se.y; j += 32)
                        if (j != self) visit(j);
                }
    }
}

// The candidates j != self with r^2 < R2 in the cells overlapping
// [x - R, x + R] (every lane passes the same particle), handed to
// emit(k, j) with k = 0, 1, ... in the order for_candidates visits them
// (cells in its loop order, j ascending within a cell), so a list written
// by a warp equals the one a thread's scan writes.  Cells are taken as
// for_candidates_lanes takes them: small ranges candidate by candidate (a
// ballot per 32 candidates places the hits), large ones 32 cells at a time
// (each lane counts its cell's hits, an exclusive prefix across the warp
// places them, the lane writes them).  Returns the number of hits.
template <typename T, typename E>
__device__ __forceinline__ int for_hits_lanes_ordered(const Grid& g, const BoxInfo& bx,
                                                      const P4<T>* __restrict__ pos, int self, T xi, T yi,
                                                      T zi, T R, T R2, int lane, E&& emit) {
    const int nc = bx.nc;
    const int2* __restrict__ cells = g.cells + bx.cell_off;
    if (!(xi >= T(0) && xi <= T(1) && yi >= T(0) && yi <= T(1) && zi >= T(0) && zi <= T(1) &&
          R >= T(0)))
        return 0;
    const bool full = !(R < T(0.5));
    const T c3[3] = {xi, yi, zi};
    int lo[3], hi[3];
    bool wraps_all = full;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = full ? 0 : (int)floor((c3[a] - R) * (T)nc - T(1e-3));
        hi[a] = full ? nc - 1 : (int)floor((c3[a] + R) * (T)nc + T(1e-3));
        if (hi[a] - lo[a] + 1 >= nc) {
            lo[a] = 0;
            hi[a] = nc - 1;
            wraps_all = true;
        }
    }
    const T xim1 = xi - T(1), yim1 = yi - T(1), zim1 = zi - T(1);
    const T cl = T(1) / (T)nc, R2m = R * R * T(1.0001);
    auto gap = [&](int c, T v) { return wraps_all ? T(0) : max(max((T)c * cl - v, v - (T)(c + 1) * cl), T(0)); };
    auto cell_range = [&](int cx, int cy, int cz, int2& se) {
        const T gx = gap(cx, xi), gy = gap(cy, yi), gz = gap(cz, zi);
        if (gx * gx + gy * gy + gz * gz > R2m) return false;
        const int wx = cx < 0 ? cx + nc : (cx >= nc ? cx - nc : cx);
        const int wy = cy < 0 ? cy + nc : (cy >= nc ? cy - nc : cy);
        const int wz = cz < 0 ? cz + nc : (cz >= nc ? cz - nc : cz);
        se = cells[(wz * nc + wy) * nc + wx];
        return true;
    };
    auto hit = [&](int j) {
        const P4<T> q = pos[j];
        const T dx = mi_diff(q.x, xi, xim1), dy = mi_diff(q.y, yi, yim1), dz = mi_diff(q.z, zi, zim1);
        return sep2(dx, dy, dz) < R2;
    };
    const unsigned full_mask = 0xffffffffu;
    int base = 0;
    const int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
    const int ncube = ex * ey * ez;
    if (ncube >= kLaneCells) {
        for (int f0 = 0; f0 < ncube; f0 += 32) {
            const int f = f0 + lane;
            int2 se = make_int2(0, 0);
            bool ok = false;
            if (f < ncube) ok = cell_range(lo[0] + f % ex, lo[1] + (f / ex) % ey, lo[2] + f / (ex * ey), se);
            int cnt = 0;
            if (ok)
                for (int j = se.x; j < se.y; ++j)
                    if (j != self && hit(j)) ++cnt;
            int pre = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(full_mask, pre, o);
                if (lane >= o) pre += y;
            }
            const int total = __shfl_sync(full_mask, pre, 31);
            int k = base + pre - cnt;
            if (ok)
                for (int j = se.x; j < se.y; ++j)
                    if (j != self && hit(j)) emit(k++, j);
            base += total;
        }
    } else {
        for (int cz = lo[2]; cz <= hi[2]; ++cz)
            for (int cy = lo[1]; cy <= hi[1]; ++cy)
                for (int cx = lo[0]; cx <= hi[0]; ++cx) {
                    int2 se;
                    if (!cell_range(cx, cy, cz, se)) continue;  // (the same for every lane)
                    for (int j0 = se.x; j0 < se.y; j0 += 32) {
                        const int j = j0 + lane;
                        const bool h = j < se.y && j != self && hit(j);
                        const unsigned m = __ballot_sync(full_mask, h);
                        if (h) emit(base + __popc(m & ((1u << lane) - 1u)), j);
                        base += __popc(m);
                    }
                }
    }
    return base;
}

}  // namespace gz
