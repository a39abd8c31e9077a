// Binning, device LSD radix sort and permutation (step S1: particles are
// Morton-sorted into a uniform cell grid per box; cell ranges are derived
// from the sorted keys).
#include <algorithm>

#include "gz_launch.cuh"

namespace gz {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kMaxDigitBits = 10;  // digits of up to 10 bits: 1024 buckets a pass
constexpr int kMaxDigits = 1 << kMaxDigitBits;
constexpr int kDigitsPerThread = kMaxDigits / kSortThreads;
constexpr int kSortTile = 4096;
constexpr int kSortPerWarp = kSortTile / kSortWarps;

// Spread the low 10 bits of v so that bit k lands on bit 3k.
__device__ __forceinline__ unsigned spread3(unsigned v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
// Inverse of spread3.
__device__ __forceinline__ unsigned compact3(unsigned v) {
    v &= 0x09249249u;
    v = (v ^ (v >> 2)) & 0x030C30C3u;
    v = (v ^ (v >> 4)) & 0x0300F00Fu;
    v = (v ^ (v >> 8)) & 0x030000FFu;
    v = (v ^ (v >> 16)) & 0x000003FFu;
    return v;
}

template <typename T>
__device__ __forceinline__ int cell_coord(T v, int nc) {
    T s = floor(v * (T)nc);
    if (!(s >= T(0))) return 0;  // also NaN
    if (s > (T)(nc - 1)) return nc - 1;
    return (int)s;
}

template <typename T>
__global__ void k_keys(int N, const T* __restrict__ x, const T* __restrict__ y,
                       const T* __restrict__ z, const int64_t* __restrict__ id,
                       const int* __restrict__ box_of, const BoxInfo* __restrict__ boxes, int cbits,
                       unsigned* __restrict__ keys, unsigned* __restrict__ vals, DevStatus* st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int b = box_of[i];
    const int nc = boxes[b].nc;
    const T xv = x[i], yv = y[i], zv = z[i];
    const bool ok = xv >= T(0) && xv < T(1) && yv >= T(0) && yv < T(1) && zv >= T(0) && zv < T(1);
    if (!ok) set_status(st, GZ_S_NONFINITE, GZ_C_NONFINITE, id[i]);
    unsigned mort = spread3(cell_coord(xv, nc)) | (spread3(cell_coord(yv, nc)) << 1) |
                    (spread3(cell_coord(zv, nc)) << 2);
    keys[i] = (cbits * 3 >= 32 ? 0u : ((unsigned)b << (3 * cbits))) | mort;
    vals[i] = (unsigned)i;
}

// Digit counts of one tile (nd = 2^bits digits, mask = nd - 1).
__global__ void k_rs_hist(const unsigned* __restrict__ keys, int N, int shift, unsigned mask, int nd,
                          unsigned* __restrict__ hist, int nblk) {
    __shared__ unsigned h[kMaxDigits];
    for (int t = threadIdx.x; t < nd; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortTile;
    for (int k = threadIdx.x; k < kSortTile; k += blockDim.x) {
        int e = base + k;
        if (e < N) atomicAdd(&h[(keys[e] >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nd; t += blockDim.x) hist[t * nblk + blockIdx.x] = h[t];
}

// Exclusive scan of one digit's row hist[d][0..nblk) (block d), and the row
// total into totals[d].
__global__ void k_rs_rows(unsigned* __restrict__ hist, int nblk, unsigned* __restrict__ totals) {
    __shared__ unsigned wsum[kSortWarps];
    __shared__ unsigned base_s;
    unsigned* row = hist + (size_t)blockIdx.x * nblk;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    unsigned running = 0;
    for (int b0 = 0; b0 < nblk; b0 += kSortThreads) {
        const int b = b0 + t;
        const unsigned v = b < nblk ? row[b] : 0u;
        unsigned x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (t == 0) {
            unsigned acc = 0;
            for (int w = 0; w < kSortWarps; ++w) {
                const unsigned ws = wsum[w];
                wsum[w] = acc;
                acc += ws;
            }
            base_s = acc;
        }
        __syncthreads();
        if (b < nblk) row[b] = running + wsum[warp] + x - v;
        running += base_s;
        __syncthreads();
    }
    if (t == 0) totals[blockIdx.x] = running;
}

// Stable scatter: each warp owns a contiguous sub-tile and walks it in order;
// lanes with equal digits are ranked with __match_any_sync.
__global__ void k_rs_scatter(const unsigned* __restrict__ kin, const unsigned* __restrict__ vin,
                             int N, int shift, unsigned mask, int nd, const unsigned* __restrict__ hist,
                             int nblk, const unsigned* __restrict__ totals, unsigned* __restrict__ kout,
                             unsigned* __restrict__ vout) {
    static_assert(kDigitsPerThread * kSortThreads == kMaxDigits, "whole digits per thread");
    __shared__ unsigned cnt[kSortWarps][kMaxDigits];
    __shared__ unsigned dbase[kMaxDigits];
    __shared__ unsigned wsum[kSortWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {  // the nd digits of this pass (nd a power of 2)
        const int lg = __ffs(nd) - 1;
        for (int t = threadIdx.x; t < kSortWarps * nd; t += blockDim.x) cnt[t >> lg][t & (nd - 1)] = 0;
    }
    {  // exclusive scan of the nd digit totals, kDigitsPerThread consecutive digits a thread
        const int d0 = kDigitsPerThread * threadIdx.x;
        unsigned v[kDigitsPerThread];
        unsigned tv = 0;
#pragma unroll
        for (int u = 0; u < kDigitsPerThread; ++u) {
            v[u] = d0 + u < nd ? totals[d0 + u] : 0u;
            tv += v[u];
        }
        unsigned incl = tv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        unsigned before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        unsigned run = before + incl - tv;
#pragma unroll
        for (int u = 0; u < kDigitsPerThread; ++u) {
            dbase[d0 + u] = run;
            run += v[u];
        }
    }
    __syncthreads();
    const int wbase = blockIdx.x * kSortTile + warp * kSortPerWarp;
    for (int c = 0; c < kSortPerWarp; c += 32) {
        int e = wbase + c + lane;
        if (e < N) atomicAdd(&cnt[warp][(kin[e] >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nd; d += blockDim.x) {
        unsigned run = dbase[d] + hist[d * nblk + blockIdx.x];
        for (int w = 0; w < kSortWarps; ++w) {
            unsigned v = cnt[w][d];
            cnt[w][d] = run;
            run += v;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int c = 0; c < kSortPerWarp; c += 32) {
        const int e = wbase + c + lane;
        const bool valid = e < N;
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        unsigned peers = 0, d = 0;
        if (valid) {
            const unsigned k = kin[e];
            d = (k >> shift) & mask;
            peers = __match_any_sync(vmask, d);
            const unsigned pos = cnt[warp][d] + __popc(peers & lt);
            kout[pos] = k;
            vout[pos] = vin[e];
        }
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) cnt[warp][d] += __popc(peers);
        __syncwarp();
    }
}

template <typename T>
__global__ void k_permute(int N, const unsigned* __restrict__ skeys,
                          const unsigned* __restrict__ svals, gz_particles p,
                          const void* __restrict__ n_in, const int* __restrict__ box_of,
                          const BoxInfo* __restrict__ boxes, int cbits, Sorted<T> s,
                          int2* __restrict__ cells) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned src = svals[i];
    s.x[i] = ((const T*)p.x)[src];
    s.y[i] = ((const T*)p.y)[src];
    s.z[i] = ((const T*)p.z)[src];
    // velocities, mass and energy are optional (the density pass reads none)
    if (p.vx) s.vx[i] = ((const T*)p.vx)[src];
    if (p.vy) s.vy[i] = ((const T*)p.vy)[src];
    if (p.vz) s.vz[i] = ((const T*)p.vz)[src];
    if (p.m) s.m[i] = ((const T*)p.m)[src];
    if (p.u) s.u[i] = ((const T*)p.u)[src];
    s.h[i] = ((const T*)p.h)[src];
    s.pos[i] = P4<T>{s.x[i], s.y[i], s.z[i], s.h[i]};
    s.id[i] = (long long)p.id[src];
    if (n_in) s.n[i] = ((const T*)n_in)[src];
    s.orig[i] = src;
    const int b = box_of[src];
    s.box[i] = b;
    const unsigned key = skeys[i];
    const unsigned mort = cbits * 3 >= 32 ? key : (key & ((1u << (3 * cbits)) - 1u));
    const int nc = boxes[b].nc;
    const int cx = compact3(mort), cy = compact3(mort >> 1), cz = compact3(mort >> 2);
    const int lin = boxes[b].cell_off + (cz * nc + cy) * nc + cx;
    if (i == 0 || skeys[i - 1] != key) cells[lin].x = i;
    if (i == N - 1 || skeys[i + 1] != key) cells[lin].y = i + 1;
}

template <typename T>
__global__ void k_unpermute(int N, int rows, const unsigned* __restrict__ orig,
                            const T* __restrict__ src, T* __restrict__ dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned o = orig[i];
    for (int r = 0; r < rows; ++r) dst[(size_t)r * N + o] = src[(size_t)r * N + i];
}

inline int blocks(int n, int t) { return (n + t - 1) / t; }

}  // namespace

template <typename T>
Sorted<T> sorted_view(Ctx& c) {
    Sorted<T> s;
    s.x = (T*)c.sx;
    s.y = (T*)c.sy;
    s.z = (T*)c.sz;
    s.vx = (T*)c.svx;
    s.vy = (T*)c.svy;
    s.vz = (T*)c.svz;
    s.m = (T*)c.sm;
    s.u = (T*)c.su;
    s.h = (T*)c.sh;
    s.id = c.sid;
    s.orig = c.vals;  // filled by sort_and_bin
    s.box = c.sbox;
    s.n = (T*)c.sn;
    s.rho = (T*)c.srho;
    s.P = (T*)c.sP;
    s.c = (T*)c.sc;
    s.sd = (T*)c.ssd;
    s.pos = (P4<T>*)c.spos;
    s.prim = (P4<T>*)c.sprim;
    s.prim2 = (P2<T>*)c.sprim2;
    return s;
}
template Sorted<float> sorted_view<float>(Ctx&);
template Sorted<double> sorted_view<double>(Ctx&);

template <typename T>
cudaError_t sort_and_bin(Ctx& c, const gz_particles& p, const void* n_in) {
    c.last_lim = nullptr;  // a new sort: earlier sorted-order indices no longer apply
    const int N = c.N;
    cudaStream_t st = c.stream;
    k_keys<T><<<blocks(N, 256), 256, 0, st>>>(N, (const T*)p.x, (const T*)p.y, (const T*)p.z, p.id,
                                               c.box_of, c.boxes, c.cbits, c.keys, c.vals,
                                               c.status);
    const int nblk = blocks(N, kSortTile);
    const int total_bits = 3 * c.cbits + c.box_bits;
    // the fewest passes of at most kMaxDigitBits bits, the bits spread evenly
    const int npass = (total_bits + kMaxDigitBits - 1) / kMaxDigitBits;
    const int bits = npass ? (total_bits + npass - 1) / npass : 0;
    c.launches += 1 + 3 * npass;  // (and k_permute, counted by permute_and_bin)
    unsigned *ki = c.keys, *vi = c.vals, *ko = c.keys_alt, *vo = c.vals_alt;
    for (int shift = 0; shift < total_bits; shift += bits) {
        const int pb = std::min(bits, total_bits - shift);
        const int nd = 1 << pb;
        const unsigned mask = (unsigned)nd - 1u;
        unsigned* totals = c.hist + (size_t)nd * nblk;
        k_rs_hist<<<nblk, kSortThreads, 0, st>>>(ki, N, shift, mask, nd, c.hist, nblk);
        k_rs_rows<<<nd, kSortThreads, 0, st>>>(c.hist, nblk, totals);
        k_rs_scatter<<<nblk, kSortThreads, 0, st>>>(ki, vi, N, shift, mask, nd, c.hist, nblk, totals, ko, vo);
        unsigned* t = ki;
        ki = ko;
        ko = t;
        t = vi;
        vi = vo;
        vo = t;
    }
    if (ki != c.keys) {  // odd number of passes: keep the result in the primary buffers
        cudaMemcpyAsync(c.keys, ki, sizeof(unsigned) * N, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(c.vals, vi, sizeof(unsigned) * N, cudaMemcpyDeviceToDevice, st);
    }
    return permute_and_bin<T>(c, p, n_in);
}

template <typename T>
cudaError_t permute_and_bin(Ctx& c, const gz_particles& p, const void* n_in) {
    c.last_lim = nullptr;
    const int N = c.N;
    cudaStream_t st = c.stream;
    c.launches += 1;
    cudaMemsetAsync(c.cells, 0, sizeof(int2) * (size_t)c.total_cells, st);
    Sorted<T> s = sorted_view<T>(c);
    k_permute<T><<<blocks(N, 256), 256, 0, st>>>(N, c.keys, c.vals, p, n_in, c.box_of, c.boxes,
                                                  c.cbits, s, c.cells);
    return cudaGetLastError();
}
template cudaError_t sort_and_bin<float>(Ctx&, const gz_particles&, const void*);
template cudaError_t sort_and_bin<double>(Ctx&, const gz_particles&, const void*);
template cudaError_t permute_and_bin<float>(Ctx&, const gz_particles&, const void*);
template cudaError_t permute_and_bin<double>(Ctx&, const gz_particles&, const void*);

template <typename T>
cudaError_t unpermute_T(Ctx& c, const T* src, T* dst, int rows) {
    c.launches += 1;
    k_unpermute<T><<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, rows, c.vals, src, dst);
    return cudaGetLastError();
}
template cudaError_t unpermute_T<float>(Ctx&, const float*, float*, int);
template cudaError_t unpermute_T<double>(Ctx&, const double*, double*, int);

cudaError_t unpermute_d(Ctx& c, const double* src, double* dst, int rows) {
    return unpermute_T<double>(c, src, dst, rows);
}
cudaError_t unpermute_i(Ctx& c, const int* src, int* dst) {
    c.launches += 1;
    k_unpermute<int><<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, 1, c.vals, src, dst);
    return cudaGetLastError();
}

}  // namespace gz
