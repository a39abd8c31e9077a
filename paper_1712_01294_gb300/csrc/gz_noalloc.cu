// gz_density_noalloc: the density pass (binning, sort, h-iteration) of one
// periodic box with all of its scratch in a fixed array that the library
// holds in device memory from load to exit, so the call allocates nothing.
//
// Who needs it: host codes that hand all device memory to their own pool
// or budget and forbid any other allocation, and callers that cannot pay
// for cudaMalloc/cudaFree inside their loop (both may synchronise the whole
// device).  They pass their own input and output arrays; everything else
// lives in g_noalloc_scratch below.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "gz_launch.cuh"

using namespace gz;

namespace {

constexpr int kMaxN = 32768;      // largest particle count accepted
constexpr int kMaxCells = 32768;  // largest cell grid (32^3 cells)
constexpr int kCap = 32;          // neighbour-list slots (lists are not returned)
constexpr int kMaxDevices = 64;

constexpr size_t al(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kHistLen = 1024 * ((kMaxN + 4095) / 4096) + 1024;  // counts + digit totals
// Worst case (FP64) of every slice the density pass touches.
constexpr size_t kScratchBytes =
    4 * al(4 * (size_t)kMaxN)                          // keys, keys_alt, vals, vals_alt
    + al(4 * kHistLen)                                 // radix histogram
    + al(4 * (size_t)kMaxN)                            // box of each particle
    + al(sizeof(BoxInfo))                              // box table
    + al(sizeof(int2) * (size_t)kMaxCells)             // cell ranges
    + 5 * al(8 * (size_t)kMaxN)                        // sorted x, y, z, h, n
    + al(32 * (size_t)kMaxN)                           // packed positions (x, y, z, H)
    + al(8 * (size_t)kMaxN)                            // sorted ids
    + 3 * al(4 * (size_t)kMaxN)                        // sorted box, iterations, counts
    + al(4 * (size_t)kMaxN * kCap)                     // neighbour lists
    + al(4 * (size_t)kMaxN) + al(4)                    // deferred particles and their count
    + al(sizeof(DevStatus));

// The scratch itself: every GPU that loads the library holds these bytes
// (8,295,168 B, about 8.3 MB) until the process exits.  All calls share it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (the host-side symbol is not a device address).
cudaError_t scratch_on_current_device(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}

// The one-box table, written on the device from values passed by value (no
// host buffer is referenced by the enqueued work).
__global__ void k_noalloc_box(BoxInfo* boxes, int nc, int count) {
    if (threadIdx.x == 0 && blockIdx.x == 0) boxes[0] = BoxInfo{nc, 0, 0, count};
}

// Copies the status bits of this call to the caller's word.  The lists are
// not returned (and hold only kCap slots), so their overflow bit means nothing
// to the caller and is left out.
__global__ void k_noalloc_status(const DevStatus* st, uint32_t* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = st->bits & ~(unsigned)GZ_S_NBR_OVERFLOW;
}

int ceil_log2i(long long v) {
    int b = 0;
    while ((1ll << b) < v) ++b;
    return b;
}

template <typename T>
gz_status run(const gz_params* prm, int N, gz_particles* p, void* n_out, int32_t* iters_out,
              uint32_t* status_out, cudaStream_t stream) {
    void* base = nullptr;
    if (scratch_on_current_device(&base) != cudaSuccess) return GZ_E_CUDA;
    // same cell grid as a one-box context of this size
    const double H0 = cbrt(3.0 * prm->ngb / (4.0 * M_PI * (double)N));
    const double f = floor(1.0 / (prm->cell_factor * H0));
    const int nc = f < 1.0 ? 1 : (f > 512.0 ? 512 : (int)f);
    if ((long long)nc * nc * nc > kMaxCells) return GZ_E_INVAL;

    Ctx c;
    c.params = *prm;
    c.precision = prm->precision;
    c.N = N;
    c.nboxes = 1;
    c.stream = stream;
    c.cap = kCap;
    c.rcap = 0;
    c.total_cells = nc * nc * nc;
    c.cbits = ceil_log2i(nc);
    c.box_bits = 0;
    c.launches = 0;
    c.prof = 0;
    c.hist_len = (int)kHistLen;
    char* q = (char*)base;
    auto take = [&](size_t bytes) {
        void* r = q;
        q += al(bytes);
        return r;
    };
    const size_t Nz = (size_t)kMaxN;
    c.keys = (unsigned*)take(4 * Nz);
    c.keys_alt = (unsigned*)take(4 * Nz);
    c.vals = (unsigned*)take(4 * Nz);
    c.vals_alt = (unsigned*)take(4 * Nz);
    c.hist = (unsigned*)take(4 * kHistLen);
    c.box_of = (int*)take(4 * Nz);
    c.boxes = (BoxInfo*)take(sizeof(BoxInfo));
    c.cells = (int2*)take(sizeof(int2) * (size_t)kMaxCells);
    c.sx = take(8 * Nz);
    c.sy = take(8 * Nz);
    c.sz = take(8 * Nz);
    c.sh = take(8 * Nz);
    c.sn = take(8 * Nz);
    c.spos = take(32 * Nz);
    c.sid = (long long*)take(8 * Nz);
    c.sbox = (int*)take(4 * Nz);
    c.iters = (int*)take(4 * Nz);
    c.ncount = (int*)take(4 * Nz);
    c.nbr = (unsigned*)take(4 * Nz * kCap);
    // particles with more candidates than the per-thread cache go to the
    // warp-per-particle kernel, exactly as in gz_density
    c.defer = (int*)take(4 * Nz);
    c.ndefer = (int*)take(4);
    c.status = (DevStatus*)take(sizeof(DevStatus));
    // the density pass never touches these
    c.svx = c.svy = c.svz = c.sm = c.su = c.srho = c.sP = c.sc = c.ssd = nullptr;
    c.dmdt = nullptr;
    c.sprim = c.sprim2 = nullptr;
    c.rcount = nullptr;
    c.rnbr = nullptr;
    c.rec = nullptr;
    c.dpdt = c.dEdt = c.dti = c.dt_box = c.dt_use = nullptr;
    c.box_hits = nullptr;
    c.pairs_dev = nullptr;

    // the scratch keeps the previous call's contents: reset what must start
    // clean (the box of every particle, the box table, the status word; the
    // deferred count is reset by the density launcher)
    cudaError_t e = cudaMemsetAsync(c.box_of, 0, 4 * (size_t)N, stream);
    if (e == cudaSuccess) {
        k_noalloc_box<<<1, 32, 0, stream>>>(c.boxes, nc, N);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c.status, 0, sizeof(DevStatus), stream);
    gz_particles only = *p;
    only.vx = only.vy = only.vz = only.m = only.u = nullptr;
    if (e == cudaSuccess) e = sort_and_bin<T>(c, only, nullptr);
    if (e == cudaSuccess) e = run_density<T>(c);
    if (e == cudaSuccess) e = unpermute_T<T>(c, (const T*)c.sh, (T*)p->h, 1);
    if (e == cudaSuccess && n_out) e = unpermute_T<T>(c, (const T*)c.sn, (T*)n_out, 1);
    if (e == cudaSuccess && iters_out) e = unpermute_i(c, c.iters, iters_out);
    if (e == cudaSuccess && status_out) k_noalloc_status<<<1, 32, 0, stream>>>(c.status, status_out);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? GZ_OK : GZ_E_CUDA;
}

}  // namespace

extern "C" gz_status gz_density_noalloc(const gz_params* params, int64_t n, gz_particles* p,
                                        void* n_out, int32_t* iters_out, uint32_t* status_out,
                                        void* cuda_stream) {
    if (!params || !p || !p->x || !p->y || !p->z || !p->h || !p->id) return GZ_E_INVAL;
    if (n < 1 || n > kMaxN) return GZ_E_INVAL;
    if (params->precision != GZ_FP64 && params->precision != GZ_MIXED32) return GZ_E_INVAL;
    if (!(params->ngb >= 1.0) || !(params->tol > 0.0) || !(params->cell_factor > 0.0) ||
        !(params->h_lim > 0.0 && params->h_lim <= 0.5) || params->max_iter < 1 ||
        (params->density_cache != 0 && params->density_cache != 40 && params->density_cache != 48))
        return GZ_E_INVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    return params->precision == GZ_FP64
               ? run<double>(params, (int)n, p, n_out, iters_out, status_out, s)
               : run<float>(params, (int)n, p, n_out, iters_out, status_out, s);
}
