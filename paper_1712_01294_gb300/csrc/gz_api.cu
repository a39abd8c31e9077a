// C ABI of the library (declared in include/gz.h): context management and
// the orchestration of the passes on the context's stream.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "gz_launch.cuh"

using namespace gz;

struct gz_ctx {
    Ctx c;
};

namespace {

const char* kVersion = "gz-mfm 0.1 (sm_103a)";

gz_status fail(gz_ctx* ctx, gz_status code, const std::string& msg) {
    if (ctx) ctx->c.err = msg;
    return code;
}

gz_status cuda_check(gz_ctx* ctx, cudaError_t e, const char* where) {
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(ctx, GZ_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return GZ_OK;
}

bool params_ok(const gz_params* p, std::string& why) {
    if (!(p->gamma > 1.0)) return why = "gamma must be > 1", false;
    if (!(p->ngb >= 1.0)) return why = "ngb must be >= 1", false;
    if (!(p->tol > 0.0)) return why = "tol must be > 0", false;
    if (!(p->cfl > 0.0)) return why = "cfl must be > 0", false;
    if (!(p->kappa_max > 0.0)) return why = "kappa_max must be > 0", false;
    if (!(p->beta > 0.0)) return why = "beta must be > 0", false;
    if (!(p->u_floor_frac >= 0.0)) return why = "u_floor_frac must be >= 0", false;
    if (!(p->h_lim > 0.0 && p->h_lim <= 0.5)) return why = "h_lim must be in (0, 0.5]", false;
    if (!(p->cell_factor > 0.0)) return why = "cell_factor must be > 0", false;
    if (p->precision != GZ_FP64 && p->precision != GZ_MIXED32)
        return why = "precision must be GZ_FP64 or GZ_MIXED32", false;
    if (p->max_iter < 1) return why = "max_iter must be >= 1", false;
    if (p->max_ngb < 8 || p->max_ngb > 4096) return why = "max_ngb must be in [8, 4096]", false;
    if (p->scheme != GZ_MFM && p->scheme != GZ_MFV) return why = "scheme must be GZ_MFM or GZ_MFV", false;
    if (p->riemann != GZ_RIEMANN_HLLC && p->riemann != GZ_RIEMANN_EXACT && p->riemann != GZ_RIEMANN_FALLBACK)
        return why = "riemann must be GZ_RIEMANN_HLLC, _EXACT or _FALLBACK", false;
    if (p->scheme == GZ_MFV && p->riemann != GZ_RIEMANN_HLLC)
        return why = "GZ_MFV takes GZ_RIEMANN_HLLC only", false;
    if (p->density_cache != 0 && p->density_cache != 40 && p->density_cache != 48)
        return why = "density_cache must be 0, 40 or 48", false;
    return true;
}

// The hand-written adjoint differentiates the MFM face with the HLLC star.
bool adjoint_covers(const gz_params& p) { return p.scheme == GZ_MFM && p.riemann == GZ_RIEMANN_HLLC; }

int ceil_log2(long long v) {
    int b = 0;
    while ((1ll << b) < v) ++b;
    return b;
}

cudaEvent_t take_event(Ctx& c) {
    if (!c.ev_pool.empty()) {
        cudaEvent_t e = c.ev_pool.back();
        c.ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records an event pair around one pass when profiling is on.
struct Pass {
    Ctx& c;
    int id;
    cudaEvent_t a = nullptr;
    Pass(Ctx& c_, int id_) : c(c_), id(id_) {
        if (c.prof) {
            a = take_event(c);
            cudaEventRecord(a, c.stream);
        }
    }
    ~Pass() {
        if (c.prof && a) {
            cudaEvent_t b = take_event(c);
            cudaEventRecord(b, c.stream);
            c.pending.push_back({id, a, b});
        }
    }
};

}  // namespace

void gz::PassTimer::begin(int pass) const {
    if (!c->prof || pass < 0 || pass >= GZ_NPASSES) return;
    cudaEvent_t a = take_event(*c);
    cudaEventRecord(a, c->stream);
    c->open_ev[pass] = a;
}

void gz::PassTimer::end(int pass) const {
    if (!c->prof || pass < 0 || pass >= GZ_NPASSES || !c->open_ev[pass]) return;
    cudaEvent_t b = take_event(*c);
    cudaEventRecord(b, c->stream);
    c->pending.push_back({pass, c->open_ev[pass], b});
    c->open_ev[pass] = nullptr;
}

namespace {

gz_status check_particles(gz_ctx* ctx, const gz_particles* p, bool need_vel) {
    if (!p) return fail(ctx, GZ_E_INVAL, "null particle set");
    if (!p->x || !p->y || !p->z || !p->h || !p->id)
        return fail(ctx, GZ_E_INVAL, "null particle array");
    if (need_vel && (!p->vx || !p->vy || !p->vz || !p->m || !p->u))
        return fail(ctx, GZ_E_INVAL, "null velocity, mass or energy array");
    return GZ_OK;
}

template <typename T>
gz_status do_density(gz_ctx* ctx, gz_particles* p, void* n_out, int32_t* iters_out) {
    Ctx& c = ctx->c;
    cudaError_t e;
    {
        Pass t(c, GZ_PASS_SORT);
        e = sort_and_bin<T>(c, *p, nullptr);
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_DENSITY);
        e = run_density<T>(c);
    }
    if (e == cudaSuccess) e = unpermute_T<T>(c, (const T*)c.sh, (T*)p->h, 1);
    if (e == cudaSuccess && n_out) e = unpermute_T<T>(c, (const T*)c.sn, (T*)n_out, 1);
    if (e == cudaSuccess && iters_out) e = unpermute_i(c, c.iters, iters_out);
    c.nbr_valid = 1;
    return cuda_check(ctx, e, "gz_density");
}

template <typename T>
gz_status prepare_given(gz_ctx* ctx, const gz_particles* p, const void* n, bool reverse) {
    Ctx& c = ctx->c;
    cudaError_t e;
    {
        Pass t(c, GZ_PASS_SORT);
        e = sort_and_bin<T>(c, *p, n);
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_LISTS);
        e = run_build_lists<T>(c);
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_PRIM);
        e = run_prim<T>(c);
    }
    if (e == cudaSuccess && reverse) {
        Pass t(c, GZ_PASS_REVERSE);
        e = run_reverse<T>(c);
    }
    c.nbr_valid = 1;
    return cuda_check(ctx, e, "prepare");
}

template <typename T>
gz_status do_gradients(gz_ctx* ctx, const gz_particles* p, const void* n, void* grad_out, void* B_out) {
    gz_status s = prepare_given<T>(ctx, p, n, false);
    if (s) return s;
    Ctx& c = ctx->c;
    cudaError_t e;
    {
        Pass t(c, GZ_PASS_GRAD);
        e = run_gradients<T>(c, false);
    }
    if (e == cudaSuccess) e = run_grad_out<T>(c, (T*)grad_out, (T*)B_out);
    return cuda_check(ctx, e, "gz_gradients");
}

template <typename T>
gz_status do_timestep(gz_ctx* ctx, const gz_particles* p, const void* n, double* dt_i, double* dt_box) {
    gz_status s = prepare_given<T>(ctx, p, n, true);
    if (s) return s;
    Ctx& c = ctx->c;
    cudaError_t e = run_gradients<T>(c, true);
    if (e == cudaSuccess && dt_i) e = unpermute_d(c, c.dti, dt_i, 1);
    if (e == cudaSuccess && dt_box) e = run_dt_out(c, dt_box);
    return cuda_check(ctx, e, "gz_timestep");
}

template <typename T>
gz_status do_fluxes(gz_ctx* ctx, const gz_particles* p, const void* n, const void* grad,
                    const void* B, double dt, double* dpdt, double* dEdt, double* dmdt) {
    gz_status s = prepare_given<T>(ctx, p, n, true);
    if (s) return s;
    Ctx& c = ctx->c;
    cudaError_t e = run_pack_given<T>(c, (const T*)grad, (const T*)B);
    if (e == cudaSuccess) e = run_dt_set(c, dt);
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_FLUX);
        e = run_fluxes<T>(c);
    }
    if (e == cudaSuccess) e = unpermute_d(c, c.dpdt, dpdt, 3);
    if (e == cudaSuccess) e = unpermute_d(c, c.dEdt, dEdt, 1);
    if (e == cudaSuccess && dmdt) {
        if (c.dmdt)
            e = unpermute_d(c, c.dmdt, dmdt, 1);
        else
            e = cudaMemsetAsync(dmdt, 0, sizeof(double) * (size_t)c.N, c.stream);
    }
    return cuda_check(ctx, e, "gz_hydro_fluxes");
}

template <typename T>
gz_status do_fluxes_backward(gz_ctx* ctx, const gz_particles* p, const void* n, const void* grad,
                             const void* B, double dt, const double* dpbar, const double* dEbar,
                             double* xbar, double* hbar, double* nbar, double* Wbar, double* gbar,
                             double* Bbar) {
    gz_status s = prepare_given<T>(ctx, p, n, true);
    if (s) return s;
    Ctx& c = ctx->c;
    cudaError_t e = ensure_adjoint_scratch(c);
    if (e == cudaSuccess) e = run_pack_given<T>(c, (const T*)grad, (const T*)B);
    if (e == cudaSuccess) e = run_dt_set(c, dt);
    if (e == cudaSuccess) e = run_flux_adjoint<T>(c, dpbar, dEbar);
    if (e == cudaSuccess) e = run_adj_out_flux(c, xbar, hbar, nbar, Wbar, gbar, Bbar);
    return cuda_check(ctx, e, "gz_hydro_fluxes_backward");
}

// Step checkpoint blob (device, caller-owned): [rates: 4 N doubles, caller
// order] [converged H, sorted order] then, at GZ_CKPT_GRADIENTS, the
// gradient pass's per-particle outputs in sorted order: flux record
// [N][kRecord], adjoint info [N][kGInfo] (working precision) and limiter
// indices [N][10]; at GZ_CKPT_LISTS also the sorted keys and order [N] u32
// each, the neighbour counts [N] and the first kCkptSlots slots of the
// neighbour lists (a prefix of their grouped layout); slices start on
// 256-byte boundaries.  Every level also keeps n and sum(-w'q) at the
// converged H (sorted order, after H): the density pass of a particle the
// h-iteration left to the warp kernel sums them in another order than a
// rescan would.
// (The backward pass sorts the same start state, so sorted order is the
// same.)
constexpr int kCkptSlots = 64;
struct Ckpt {
    double* rates = nullptr;
    void* H = nullptr;
    void *n = nullptr, *sd = nullptr;
    void* rec = nullptr;
    void* ginfo = nullptr;
    int* lim = nullptr;
    unsigned *keys = nullptr, *vals = nullptr;  // GZ_CKPT_LISTS
    int* ncount = nullptr;
    unsigned* nbr = nullptr;
    int slots = 0;
};
size_t ckpt_slice(size_t b) { return (b + 255) & ~(size_t)255; }
int ckpt_slots(const Ctx& c) { return std::min(c.cap, kCkptSlots); }
size_t ckpt_bytes(const Ctx& c, int level) {
    const size_t N = (size_t)c.N, ts = c.precision == GZ_FP64 ? 8 : 4;
    size_t b = ckpt_slice(sizeof(double) * 4 * N) + 3 * ckpt_slice(ts * N);
    if (level >= GZ_CKPT_GRADIENTS)
        b += ckpt_slice(ts * N * kRecord) + ckpt_slice(ts * N * kGInfo) + ckpt_slice(sizeof(int) * N * 10);
    if (level >= GZ_CKPT_LISTS)
        b += 3 * ckpt_slice(4 * N) + ckpt_slice(4 * N * (size_t)ckpt_slots(c));
    return b;
}
Ckpt ckpt_view(const Ctx& c, void* base, int level) {
    Ckpt k;
    if (!base) return k;
    const size_t N = (size_t)c.N, ts = c.precision == GZ_FP64 ? 8 : 4;
    char* p = (char*)base;
    k.rates = (double*)p;
    p += ckpt_slice(sizeof(double) * 4 * N);
    k.H = p;
    p += ckpt_slice(ts * N);
    k.n = p;
    p += ckpt_slice(ts * N);
    k.sd = p;
    p += ckpt_slice(ts * N);
    if (level >= GZ_CKPT_GRADIENTS) {
        k.rec = p;
        p += ckpt_slice(ts * N * kRecord);
        k.ginfo = p;
        p += ckpt_slice(ts * N * kGInfo);
        k.lim = (int*)p;
        p += ckpt_slice(sizeof(int) * N * 10);
    }
    if (level >= GZ_CKPT_LISTS) {
        k.keys = (unsigned*)p;
        p += ckpt_slice(4 * N);
        k.vals = (unsigned*)p;
        p += ckpt_slice(4 * N);
        k.ncount = (int*)p;
        p += ckpt_slice(4 * N);
        k.nbr = (unsigned*)p;
        k.slots = ckpt_slots(c);
    }
    return k;
}

// The groups of four list slots (group g of particle i at uint4 g N + i)
// among the first `groups` that hold part of particle i's list, from src to
// dst; the groups past a particle's count are not copied (no pass reads
// them).
__global__ void k_copy_lists(int N, int groups, const int* __restrict__ ncount, const uint4* __restrict__ src,
                             uint4* __restrict__ dst) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * groups) return;
    const int g = (int)(idx / N);
    const int i = (int)(idx - (long long)g * N);
    if (4 * g < ncount[i]) dst[idx] = src[idx];
}

cudaError_t copy_lists(Ctx& c, const int* ncount, const unsigned* src, unsigned* dst, int slots,
                       cudaStream_t st) {
    const long long n = (long long)c.N * (slots / 4);
    if (n == 0) return cudaSuccess;
    c.launches += 1;
    k_copy_lists<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c.N, slots / 4, ncount, (const uint4*)src,
                                                              (uint4*)dst);
    return cudaGetLastError();
}

// What the sort and the density pass leave that the backward pass would
// otherwise recompute: the sort's keys and order, the neighbour counts and
// the lists' first slots (groups of four slots across the particles:
// the first slots/4 groups are one contiguous prefix).
template <typename T>
cudaError_t save_lists(Ctx& c, const Ckpt& k, cudaStream_t st) {
    const size_t N = (size_t)c.N;
    cudaError_t e = cudaMemcpyAsync(k.keys, c.keys, 4 * N, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(k.vals, c.vals, 4 * N, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(k.ncount, c.ncount, 4 * N, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = copy_lists(c, c.ncount, c.nbr, k.nbr, k.slots, st);
    return e;
}

// Makes the side stream wait for the work issued so far on the context's
// stream (creating the stream and its events on first use).
cudaError_t fork_side(Ctx& c) {
    cudaError_t e = cudaSuccess;
    if (!c.side) e = cudaStreamCreateWithFlags(&c.side, cudaStreamNonBlocking);
    if (e == cudaSuccess && !c.side_fork) e = cudaEventCreateWithFlags(&c.side_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !c.side_join) e = cudaEventCreateWithFlags(&c.side_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(c.side_fork, c.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c.side, c.side_fork, 0);
    return e;
}

// The backward pass's sort and density pass from a GZ_CKPT_LISTS checkpoint:
// the sorted order and cells from the saved keys, the saved H, n, sums,
// counts and list slots, and a scan for the lists longer than the saved
// slots; the same values the sort and k_dens_given give.
template <typename T>
cudaError_t restore_lists(Ctx& c, const gz_particles& p, const Ckpt& k) {
    const size_t N = (size_t)c.N;
    cudaStream_t st = c.stream;
    cudaError_t e = cudaMemcpyAsync(c.keys, k.keys, 4 * N, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.vals, k.vals, 4 * N, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = permute_and_bin<T>(c, p, nullptr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.sh, k.H, sizeof(T) * N, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.sn, k.n, sizeof(T) * N, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.ssd, k.sd, sizeof(T) * N, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.ncount, k.ncount, 4 * N, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = copy_lists(c, c.ncount, k.nbr, c.nbr, k.slots, st);
    if (e == cudaSuccess && k.slots < c.cap) e = run_lists_over<T>(c, k.slots);
    return e;
}

// Points the context's gradient-pass outputs at a checkpoint for one call.
struct GradOutputs {
    Ctx& c;
    void *rec, *ginfo;
    int* lim;
    GradOutputs(Ctx& c_, const Ckpt& k) : c(c_), rec(c_.rec), ginfo(c_.ginfo), lim(c_.lim) {
        if (k.rec) {
            c.rec = k.rec;
            c.ginfo = k.ginfo;
            c.lim = k.lim;
        }
    }
    ~GradOutputs() {
        c.rec = rec;
        c.ginfo = ginfo;
        c.lim = lim;
    }
};

// Adjoint of gz_step: the forward passes are re-run from the start state
// (neighbour sets, H and every pair quantity recomputed, not stored; the
// rates and, at GZ_CKPT_GRADIENTS, the gradient pass's per-particle outputs
// come from the step's checkpoint when one is given), then the adjoint
// passes run in reverse order.
template <typename T>
gz_status do_step_backward(gz_ctx* ctx, const gz_particles* p, double dt, const Ckpt& ck,
                           const gz_particles* gend, gz_particles* gstart) {
    Ctx& c = ctx->c;
    cudaError_t e = ensure_adjoint_scratch(c);
    GradOutputs outs(c, ck);
    if (e == cudaSuccess && ck.keys) {  // GZ_CKPT_LISTS: sorted order and lists kept
        Pass t(c, GZ_PASS_SORT);
        e = restore_lists<T>(c, *p, ck);
    }
    if (e == cudaSuccess && !ck.keys) {
        Pass t(c, GZ_PASS_SORT);
        e = sort_and_bin<T>(c, *p, nullptr);
    }
    if (e == cudaSuccess && !ck.keys) {
        Pass t(c, GZ_PASS_DENSITY);
        if (ck.H) {  // the forward's converged H: no h-iteration; its n and sums
            const size_t bytes = sizeof(T) * (size_t)c.N;
            e = cudaMemcpyAsync(c.sh, ck.H, bytes, cudaMemcpyDeviceToDevice, c.stream);
            if (e == cudaSuccess) e = run_density_given<T>(c);
            if (e == cudaSuccess) e = cudaMemcpyAsync(c.sn, ck.n, bytes, cudaMemcpyDeviceToDevice, c.stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(c.ssd, ck.sd, bytes, cudaMemcpyDeviceToDevice, c.stream);
        } else {
            e = run_density<T>(c);
        }
    }
    if (e == cudaSuccess) e = run_prim<T>(c);
    if (e == cudaSuccess) e = run_reverse<T>(c);
    if (e == cudaSuccess && !ck.rec) {
        Pass t(c, GZ_PASS_GRAD);
        e = run_gradients<T>(c, false, true);
    }
    if (e == cudaSuccess) e = run_dt_set(c, dt);
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_FLUX);
        e = ck.rates ? run_rates_in(c, ck.rates) : run_fluxes<T>(c);
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_UPDATE);
        e = run_step_adjoint<T>(c, *gend, *gstart);
    }
    c.nbr_valid = 1;
    return cuda_check(ctx, e, "gz_step_backward");
}

// The first half of a step (S1-S3 with the CFL criterion) and, apart, its
// second half (S4, S6) with a step given on the device: gz_step split where
// a decomposed box takes the minimum over its subdomains.
template <typename T>
gz_status do_step_begin(gz_ctx* ctx, gz_particles* p, double* dt_box_dev) {
    Ctx& c = ctx->c;
    cudaError_t e;
    {
        Pass t(c, GZ_PASS_SORT);
        e = sort_and_bin<T>(c, *p, nullptr);
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_DENSITY);
        e = run_density<T>(c);
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_PRIM);
        e = run_prim<T>(c);
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_REVERSE);
        e = run_reverse<T>(c);
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_GRAD);
        e = run_gradients<T>(c, true, false);
        if (e == cudaSuccess) e = run_dt_out(c, dt_box_dev);
    }
    c.nbr_valid = 1;
    c.step_open = e == cudaSuccess;
    return cuda_check(ctx, e, "gz_step_begin");
}

template <typename T>
gz_status do_step_finish(gz_ctx* ctx, gz_particles* p, const double* dt_dev) {
    Ctx& c = ctx->c;
    cudaError_t e = run_dt_copy(c, dt_dev);
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_FLUX);
        e = run_fluxes<T>(c);
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_UPDATE);
        e = run_update<T>(c, *p, nullptr);
    }
    c.step_open = 0;
    return cuda_check(ctx, e, "gz_step_finish");
}

template <typename T>
gz_status do_step(gz_ctx* ctx, gz_particles* p, double dt_fixed, double* dt_used_dev, const Ckpt& ck) {
    Ctx& c = ctx->c;
    GradOutputs outs(c, ck);
    cudaError_t e;
    bool forked = false;
    {
        Pass t(c, GZ_PASS_SORT);
        e = sort_and_bin<T>(c, *p, nullptr);
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_DENSITY);
        e = run_density<T>(c);
        const size_t bytes = sizeof(T) * (size_t)c.N;
        if (e == cudaSuccess && ck.H) e = cudaMemcpyAsync(ck.H, c.sh, bytes, cudaMemcpyDeviceToDevice, c.stream);
        if (e == cudaSuccess && ck.n) e = cudaMemcpyAsync(ck.n, c.sn, bytes, cudaMemcpyDeviceToDevice, c.stream);
        if (e == cudaSuccess && ck.sd) e = cudaMemcpyAsync(ck.sd, c.ssd, bytes, cudaMemcpyDeviceToDevice, c.stream);
        // the sort's order and the lists are not written again in this
        // step: their copies run on the side stream, beside the pair passes
        if (e == cudaSuccess && ck.keys) {
            e = fork_side(c);
            if (e == cudaSuccess) {
                forked = true;
                e = save_lists<T>(c, ck, c.side);
                const cudaError_t e2 = cudaEventRecord(c.side_join, c.side);
                if (e == cudaSuccess) e = e2;
            }
        }
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_PRIM);
        e = run_prim<T>(c);  // also stores the converged H in the packed positions
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_REVERSE);
        e = run_reverse<T>(c);
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_GRAD);
        e = run_gradients<T>(c, !(dt_fixed > 0.0), ck.rec != nullptr);
        if (e == cudaSuccess) e = run_dt_finalize(c, dt_fixed, dt_used_dev);
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_FLUX);
        e = run_fluxes<T>(c);
    }
    if (e == cudaSuccess) {
        Pass t(c, GZ_PASS_UPDATE);
        e = run_update<T>(c, *p, ck.rates);
    }
    if (forked) {  // the step ends when the side stream's copies are done
        const cudaError_t e2 = cudaStreamWaitEvent(c.stream, c.side_join, 0);
        if (e == cudaSuccess) e = e2;
    }
    c.nbr_valid = 1;
    c.last_lim = ck.lim;
    return cuda_check(ctx, e, "gz_step");
}

}  // namespace

extern "C" {

const char* gz_version(void) { return kVersion; }

gz_status gz_default_params(gz_params* out) {
    if (!out) return GZ_E_INVAL;
    memset(out, 0, sizeof(*out));
    out->gamma = 5.0 / 3.0;
    out->ngb = 32.0;
    out->tol = 1e-6;
    out->cfl = 0.2;
    out->kappa_max = 100.0;
    out->beta = 1.0;
    out->u_floor_frac = 1e-10;
    out->h_lim = 0.5;
    out->cell_factor = 1.0;
    out->precision = GZ_MIXED32;
    out->hancock = 1;
    out->max_iter = 64;
    out->max_ngb = 128;
    return GZ_OK;
}

// gz_create, with the cell grid of each box built for grid_counts[b]
// particles when grid_counts is given (a subdomain: the whole box's grid).
gz_status create_ctx(const gz_params* params, int32_t nboxes, const int64_t* counts,
                     const int64_t* grid_counts, void* cuda_stream, gz_ctx** out) {
    if (!out || !params || !counts || nboxes < 1) return GZ_E_INVAL;
    *out = nullptr;
    std::string why;
    if (!params_ok(params, why)) return GZ_E_INVAL;
    long long N = 0;
    for (int b = 0; b < nboxes; ++b) {
        if (counts[b] < 1) return GZ_E_INVAL;
        N += counts[b];
    }
    if (N >= (1ll << 31) - 1) return GZ_E_INVAL;
    gz_ctx* ctx = new (std::nothrow) gz_ctx();
    if (!ctx) return GZ_E_NOMEM;
    Ctx& c = ctx->c;
    c.params = *params;
    c.precision = params->precision;
    c.N = (int)N;
    c.nboxes = nboxes;
    c.counts.assign(counts, counts + nboxes);
    c.stream = (cudaStream_t)cuda_stream;
    // lists are read four indices at a time, and the first 32 entries of each
    // list by the 32 lanes of a warp
    c.cap = std::max(32, (params->max_ngb + 7) / 8 * 8);
    c.launches = 0;
    c.prof = 0;
    for (int k = 0; k < GZ_NPASSES; ++k) {
        c.prof_ms[k] = 0.0;
        c.prof_calls[k] = 0;
    }
    c.rcap = std::max(32, c.cap / 2 / 4 * 4);
    // per-box cell grids: cell length ~ cell_factor * H0 of the box
    int maxnc = 1;
    long long cells = 0;
    int first = 0;
    c.hboxes.resize(nboxes);
    for (int b = 0; b < nboxes; ++b) {
        const double gc = grid_counts ? (double)grid_counts[b] : (double)counts[b];
        const double H0 = cbrt(3.0 * params->ngb / (4.0 * M_PI * gc));
        double f = floor(1.0 / (params->cell_factor * H0));
        int nc = f < 1.0 ? 1 : (f > 512.0 ? 512 : (int)f);
        c.hboxes[b].nc = nc;
        c.hboxes[b].cell_off = (int)cells;
        c.hboxes[b].first = first;
        c.hboxes[b].count = (int)counts[b];
        first += (int)counts[b];
        cells += (long long)nc * nc * nc;
        maxnc = std::max(maxnc, nc);
    }
    if (cells >= (1ll << 30)) {
        delete ctx;
        return GZ_E_INVAL;
    }
    c.total_cells = (int)cells;
    c.cbits = ceil_log2(maxnc);
    c.box_bits = ceil_log2(nboxes);
    if (3 * c.cbits + c.box_bits > 32) {
        delete ctx;
        return GZ_E_INVAL;
    }
    // one arena for all scratch
    const size_t Nz = (size_t)N;
    const size_t sz = params->precision == GZ_FP64 ? 8 : 4;
    const int nblk = (int)((N + 4095) / 4096);
    c.hist_len = 1024 * nblk + 1024;  // per-block counts of up to 1024 digits, then the digit totals
    struct Item {
        void** ptr;
        size_t bytes;
    };
    std::vector<Item> items = {
        {(void**)&c.keys, 4 * Nz},        {(void**)&c.keys_alt, 4 * Nz},
        {(void**)&c.vals, 4 * Nz},        {(void**)&c.vals_alt, 4 * Nz},
        {(void**)&c.hist, 4 * (size_t)c.hist_len},
        {(void**)&c.box_of, 4 * Nz},      {(void**)&c.boxes, sizeof(BoxInfo) * (size_t)nboxes},
        {(void**)&c.cells, sizeof(int2) * (size_t)cells},
        {(void**)&c.sx, sz * Nz},         {(void**)&c.sy, sz * Nz},
        {(void**)&c.sz, sz * Nz},         {(void**)&c.svx, sz * Nz},
        {(void**)&c.svy, sz * Nz},        {(void**)&c.svz, sz * Nz},
        {(void**)&c.sm, sz * Nz},         {(void**)&c.su, sz * Nz},
        {(void**)&c.sh, sz * Nz},         {(void**)&c.sn, sz * Nz},
        {(void**)&c.ssd, sz * Nz},
        {(void**)&c.srho, sz * Nz},       {(void**)&c.sP, sz * Nz},
        {(void**)&c.sc, sz * Nz},         {(void**)&c.sid, 8 * Nz},
        {(void**)&c.spos, 4 * sz * Nz},   {(void**)&c.sprim, 4 * sz * Nz},
        {(void**)&c.sprim2, 2 * sz * Nz},
        {(void**)&c.sbox, 4 * Nz},        {(void**)&c.iters, 4 * Nz},
        {(void**)&c.ncount, 4 * Nz},      {(void**)&c.nbr, 4 * Nz * (size_t)c.cap},
        {(void**)&c.rcount, 4 * Nz},      {(void**)&c.rnbr, 4 * Nz * (size_t)c.rcap},
        {(void**)&c.rec, sz * Nz * kRecord},
        {(void**)&c.defer, 4 * Nz},       {(void**)&c.ndefer, 4},
        {(void**)&c.dpdt, 8 * 3 * Nz},    {(void**)&c.dEdt, 8 * Nz},
        {(void**)&c.dmdt, params->scheme == GZ_MFV ? 8 * Nz : 0},
        {(void**)&c.dti, 8 * Nz},         {(void**)&c.dt_box, 8 * (size_t)nboxes},
        {(void**)&c.dt_use, 8 * (size_t)nboxes},
        {(void**)&c.box_hits, 4 * (size_t)nboxes},
        {(void**)&c.status, sizeof(DevStatus)},
        {(void**)&c.pairs_dev, 3 * sizeof(long long)},
    };
    size_t total = 0;
    for (auto& it : items) total += (it.bytes + 255) & ~(size_t)255;
    c.arena_bytes = total;
    if (cudaMalloc(&c.arena, total) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return GZ_E_NOMEM;
    }
    char* base = (char*)c.arena;
    for (auto& it : items) {
        *it.ptr = it.bytes ? base : nullptr;
        base += (it.bytes + 255) & ~(size_t)255;
    }
    std::vector<int> box_of(Nz);
    for (int b = 0; b < nboxes; ++b)
        for (int k = 0; k < c.hboxes[b].count; ++k) box_of[c.hboxes[b].first + k] = b;
    cudaError_t e = cudaMemcpyAsync(c.box_of, box_of.data(), 4 * Nz, cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.boxes, c.hboxes.data(), sizeof(BoxInfo) * nboxes, cudaMemcpyHostToDevice,
                            c.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.status, 0, sizeof(DevStatus), c.stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(&c.status->first_bad_id, 0xFF, sizeof(unsigned long long), c.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.ncount, 0, 4 * Nz, c.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.rcount, 0, 4 * Nz, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);  // host vectors go out of scope
    if (e != cudaSuccess) {
        cudaFree(c.arena);
        delete ctx;
        return GZ_E_CUDA;
    }
    c.capacity = (int)N;
    *out = ctx;
    return GZ_OK;
}

gz_status gz_create(const gz_params* params, int32_t nboxes, const int64_t* counts,
                    void* cuda_stream, gz_ctx** out) {
    return create_ctx(params, nboxes, counts, nullptr, cuda_stream, out);
}

// Calls whose buffers or captured launches are laid out for one particle
// count (checkpoints, CUDA graphs, the hierarchical step's bins) refuse a
// subdomain context, whose count changes with every gz_set_subdomain.
static gz_status refuse_subdomain(gz_ctx* ctx, const char* what) {
    return fail(ctx, GZ_E_INVAL, std::string(what) + ": not taken on a subdomain context");
}

gz_status gz_create_subdomain(const gz_params* params, int64_t capacity, int64_t grid_count,
                              void* cuda_stream, gz_ctx** out) {
    if (!out || capacity < 1 || grid_count < 1) return GZ_E_INVAL;
    gz_status s = create_ctx(params, 1, &capacity, &grid_count, cuda_stream, out);
    if (s) return s;
    Ctx& c = (*out)->c;
    c.grid_count = grid_count;
    c.n_owned = c.N;
    if (cudaMalloc(&c.owned, (size_t)capacity) != cudaSuccess) {
        cudaGetLastError();
        gz_destroy(*out);
        *out = nullptr;
        return GZ_E_NOMEM;
    }
    if (cudaMemsetAsync(c.owned, 1, (size_t)capacity, c.stream) != cudaSuccess ||
        cudaStreamSynchronize(c.stream) != cudaSuccess) {
        gz_destroy(*out);
        *out = nullptr;
        return GZ_E_CUDA;
    }
    return GZ_OK;
}

gz_status gz_set_subdomain(gz_ctx* ctx, int64_t n, int64_t n_owned, const uint8_t* owned) {
    if (!ctx) return GZ_E_INVAL;
    Ctx& c = ctx->c;
    if (!c.owned) return fail(ctx, GZ_E_INVAL, "gz_set_subdomain: not a subdomain context");
    if (n < 1 || n > c.capacity || n_owned < 0 || n_owned > n)
        return fail(ctx, GZ_E_INVAL, "gz_set_subdomain: need 1 <= n <= capacity, 0 <= n_owned <= n");
    c.N = (int)n;
    c.counts[0] = n;
    c.hboxes[0].count = (int)n;
    c.n_owned = (int)n_owned;
    c.nbr_valid = 0;
    c.step_open = 0;
    cudaError_t e = owned ? cudaMemcpyAsync(c.owned, owned, (size_t)n, cudaMemcpyDeviceToDevice, c.stream)
                          : cudaMemsetAsync(c.owned, 1, (size_t)n, c.stream);
    if (e == cudaSuccess) e = run_set_box(c);
    return cuda_check(ctx, e, "gz_set_subdomain");
}

gz_status gz_destroy(gz_ctx* ctx) {
    if (!ctx) return GZ_E_INVAL;
    cudaStreamSynchronize(ctx->c.stream);
    if (ctx->c.side) {
        cudaStreamSynchronize(ctx->c.side);
        cudaStreamDestroy(ctx->c.side);
    }
    if (ctx->c.side_fork) cudaEventDestroy(ctx->c.side_fork);
    if (ctx->c.side_join) cudaEventDestroy(ctx->c.side_join);
    for (auto& pe : ctx->c.pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    for (auto ev : ctx->c.ev_pool) cudaEventDestroy(ev);
    cudaFree(ctx->c.arena);
    if (ctx->c.owned) cudaFree(ctx->c.owned);
    if (ctx->c.adj_arena) cudaFree(ctx->c.adj_arena);
    free_hier_scratch(ctx->c);
    if (ctx->c.graph_exec) cudaGraphExecDestroy(ctx->c.graph_exec);
    if (ctx->c.graph) cudaGraphDestroy(ctx->c.graph);
    delete ctx;
    return GZ_OK;
}

#define GZ_DISPATCH(call_f, call_d) \
    (ctx->c.precision == GZ_FP64 ? (call_d) : (call_f))

gz_status gz_density(gz_ctx* ctx, gz_particles* p, void* n_out, int32_t* iters_out) {
    if (!ctx) return GZ_E_INVAL;
    if (gz_status s = check_particles(ctx, p, false)) return s;
    return GZ_DISPATCH(do_density<float>(ctx, p, n_out, iters_out),
                       do_density<double>(ctx, p, n_out, iters_out));
}

gz_status gz_gradients(gz_ctx* ctx, const gz_particles* p, const void* n, void* grad_out, void* B_out) {
    if (!ctx) return GZ_E_INVAL;
    if (gz_status s = check_particles(ctx, p, true)) return s;
    if (!n) return fail(ctx, GZ_E_INVAL, "null n");
    return GZ_DISPATCH(do_gradients<float>(ctx, p, n, grad_out, B_out),
                       do_gradients<double>(ctx, p, n, grad_out, B_out));
}

gz_status gz_timestep(gz_ctx* ctx, const gz_particles* p, const void* n, double* dt_i_out,
                      double* dt_box_out) {
    if (!ctx) return GZ_E_INVAL;
    if (gz_status s = check_particles(ctx, p, true)) return s;
    if (!n) return fail(ctx, GZ_E_INVAL, "null n");
    return GZ_DISPATCH(do_timestep<float>(ctx, p, n, dt_i_out, dt_box_out),
                       do_timestep<double>(ctx, p, n, dt_i_out, dt_box_out));
}

gz_status gz_hydro_fluxes(gz_ctx* ctx, const gz_particles* p, const void* n, const void* grad,
                          const void* B, double dt, double* dpdt, double* dEdt, double* dmdt) {
    if (!ctx) return GZ_E_INVAL;
    if (gz_status s = check_particles(ctx, p, true)) return s;
    if (!n || !grad || !B || !dpdt || !dEdt) return fail(ctx, GZ_E_INVAL, "null input/output");
    if (!(dt >= 0.0) || !isfinite(dt)) return fail(ctx, GZ_E_INVAL, "dt must be finite and >= 0");
    return GZ_DISPATCH(do_fluxes<float>(ctx, p, n, grad, B, dt, dpdt, dEdt, dmdt),
                       do_fluxes<double>(ctx, p, n, grad, B, dt, dpdt, dEdt, dmdt));
}

gz_status gz_hydro_fluxes_backward(gz_ctx* ctx, const gz_particles* p, const void* n,
                                   const void* grad, const void* B, double dt,
                                   const double* dpdt_bar, const double* dEdt_bar, double* x_bar,
                                   double* h_bar, double* n_bar, double* W_bar, double* grad_bar,
                                   double* B_bar) {
    if (!ctx) return GZ_E_INVAL;
    if (gz_status s = check_particles(ctx, p, true)) return s;
    if (!n || !grad || !B || !dpdt_bar || !dEdt_bar) return fail(ctx, GZ_E_INVAL, "null input");
    if (!adjoint_covers(ctx->c.params))
        return fail(ctx, GZ_E_INVAL, "the adjoint covers GZ_MFM with GZ_RIEMANN_HLLC only");
    if (!(dt >= 0.0) || !isfinite(dt)) return fail(ctx, GZ_E_INVAL, "dt must be finite and >= 0");
    return GZ_DISPATCH(do_fluxes_backward<float>(ctx, p, n, grad, B, dt, dpdt_bar, dEdt_bar, x_bar, h_bar,
                                                 n_bar, W_bar, grad_bar, B_bar),
                       do_fluxes_backward<double>(ctx, p, n, grad, B, dt, dpdt_bar, dEdt_bar, x_bar,
                                                  h_bar, n_bar, W_bar, grad_bar, B_bar));
}

gz_status gz_step(gz_ctx* ctx, gz_particles* p, double dt_fixed, double* dt_used_dev) {
    if (!ctx) return GZ_E_INVAL;
    if (gz_status s = check_particles(ctx, p, true)) return s;
    if (!isfinite(dt_fixed)) return fail(ctx, GZ_E_INVAL, "dt_fixed must be finite");
    return GZ_DISPATCH(do_step<float>(ctx, p, dt_fixed, dt_used_dev, Ckpt()),
                       do_step<double>(ctx, p, dt_fixed, dt_used_dev, Ckpt()));
}

gz_status gz_step_begin(gz_ctx* ctx, gz_particles* p, double* dt_box_dev) {
    if (!ctx) return GZ_E_INVAL;
    if (gz_status s = check_particles(ctx, p, true)) return s;
    if (!dt_box_dev) return fail(ctx, GZ_E_INVAL, "null dt_box_dev");
    return GZ_DISPATCH(do_step_begin<float>(ctx, p, dt_box_dev), do_step_begin<double>(ctx, p, dt_box_dev));
}

gz_status gz_step_finish(gz_ctx* ctx, gz_particles* p, const double* dt_dev) {
    if (!ctx) return GZ_E_INVAL;
    if (gz_status s = check_particles(ctx, p, true)) return s;
    if (!dt_dev) return fail(ctx, GZ_E_INVAL, "null dt_dev");
    if (!ctx->c.step_open) return fail(ctx, GZ_E_INVAL, "gz_step_finish without gz_step_begin");
    return GZ_DISPATCH(do_step_finish<float>(ctx, p, dt_dev), do_step_finish<double>(ctx, p, dt_dev));
}

gz_status gz_step_hier(gz_ctx* ctx, gz_particles* p, int32_t K, double dt_fixed, double* dt_used_dev,
                       int32_t* bins_out, int64_t* active_out) {
    if (!ctx) return GZ_E_INVAL;
    if (gz_status s = check_particles(ctx, p, true)) return s;
    if (!isfinite(dt_fixed)) return fail(ctx, GZ_E_INVAL, "dt_fixed must be finite");
    if (K < 0 || K > 20) return fail(ctx, GZ_E_INVAL, "K must be in [0, 20]");
    if (ctx->c.owned) return refuse_subdomain(ctx, "gz_step_hier");
    Ctx& c = ctx->c;
    const PassTimer timer{&c};
    long long act = 0;
    cudaError_t e = c.precision == GZ_FP64
                        ? run_step_hier<double>(c, *p, K, dt_fixed, dt_used_dev, bins_out, &act, timer)
                        : run_step_hier<float>(c, *p, K, dt_fixed, dt_used_dev, bins_out, &act, timer);
    if (active_out) *active_out = (int64_t)act;
    if (e == cudaErrorMemoryAllocation) return fail(ctx, GZ_E_NOMEM, "gz_step_hier: scratch allocation failed");
    return cuda_check(ctx, e, "gz_step_hier");
}

gz_status gz_checkpoint_bytes(gz_ctx* ctx, int32_t level, int64_t* bytes) {
    if (!ctx || !bytes || level < GZ_CKPT_RATES || level > GZ_CKPT_LISTS) return GZ_E_INVAL;
    if (ctx->c.owned) return refuse_subdomain(ctx, "gz_checkpoint_bytes");
    *bytes = (int64_t)ckpt_bytes(ctx->c, level);
    return GZ_OK;
}

gz_status gz_step_checkpoint(gz_ctx* ctx, gz_particles* p, double dt_fixed, double* dt_used_dev,
                             void* ckpt, int32_t level) {
    if (!ctx) return GZ_E_INVAL;
    if (gz_status s = check_particles(ctx, p, true)) return s;
    if (!isfinite(dt_fixed)) return fail(ctx, GZ_E_INVAL, "dt_fixed must be finite");
    if (!ckpt || ((uintptr_t)ckpt & 255) || level < GZ_CKPT_RATES || level > GZ_CKPT_LISTS)
        return fail(ctx, GZ_E_INVAL, "checkpoint: need a 256-byte aligned buffer and a valid level");
    if (!adjoint_covers(ctx->c.params))
        return fail(ctx, GZ_E_INVAL, "the adjoint covers GZ_MFM with GZ_RIEMANN_HLLC only");
    if (ctx->c.owned) return refuse_subdomain(ctx, "gz_step_checkpoint");
    const Ckpt ck = ckpt_view(ctx->c, ckpt, level);
    return GZ_DISPATCH(do_step<float>(ctx, p, dt_fixed, dt_used_dev, ck),
                       do_step<double>(ctx, p, dt_fixed, dt_used_dev, ck));
}

gz_status gz_graph_capture(gz_ctx* ctx, gz_particles* p, int32_t nsteps, double dt_fixed,
                           double* dt_used_dev) {
    if (!ctx || nsteps < 1) return GZ_E_INVAL;
    if (gz_status s = check_particles(ctx, p, true)) return s;
    Ctx& c = ctx->c;
    if (!c.stream) return fail(ctx, GZ_E_INVAL, "graph capture needs a created (non-default) stream");
    if (c.owned) return refuse_subdomain(ctx, "gz_graph_capture");
    if (!isfinite(dt_fixed)) return fail(ctx, GZ_E_INVAL, "dt_fixed must be finite");
    if (c.graph_exec) cudaGraphExecDestroy(c.graph_exec);
    if (c.graph) cudaGraphDestroy(c.graph);
    c.graph_exec = nullptr;
    c.graph = nullptr;
    const int prof = c.prof;
    c.prof = 0;
    const long long l0 = c.launches;
    cudaError_t e = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        c.prof = prof;
        return fail(ctx, GZ_E_CUDA, std::string("gz_graph_capture: ") + cudaGetErrorString(e));
    }
    gz_status st = GZ_OK;
    for (int k = 0; k < nsteps && st == GZ_OK; ++k)
        st = GZ_DISPATCH(do_step<float>(ctx, p, dt_fixed, dt_used_dev, Ckpt()),
                         do_step<double>(ctx, p, dt_fixed, dt_used_dev, Ckpt()));
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c.stream, &g);
    c.prof = prof;
    c.graph_kernels = c.launches - l0;
    c.launches = l0;
    if (st != GZ_OK || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st != GZ_OK ? st : fail(ctx, GZ_E_CUDA, std::string("gz_graph_capture: ") + cudaGetErrorString(e2));
    }
    e = cudaGraphInstantiate(&c.graph_exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(ctx, GZ_E_CUDA, std::string("gz_graph_capture: ") + cudaGetErrorString(e));
    }
    c.graph = g;
    return GZ_OK;
}

gz_status gz_graph_launch(gz_ctx* ctx) {
    if (!ctx) return GZ_E_INVAL;
    Ctx& c = ctx->c;
    if (!c.graph_exec) return fail(ctx, GZ_E_INVAL, "no captured graph");
    c.launches += c.graph_kernels;
    return cuda_check(ctx, cudaGraphLaunch(c.graph_exec, c.stream), "gz_graph_launch");
}

gz_status gz_step_backward(gz_ctx* ctx, const gz_particles* p_start, double dt, const void* ckpt,
                           int32_t level, const gz_particles* gbar_end, gz_particles* gbar_start) {
    if (!ctx) return GZ_E_INVAL;
    if (gz_status s = check_particles(ctx, p_start, true)) return s;
    if (!gbar_end || !gbar_start) return fail(ctx, GZ_E_INVAL, "null adjoint set");
    if (!(dt > 0.0) || !isfinite(dt)) return fail(ctx, GZ_E_INVAL, "dt must be finite and > 0");
    if (!adjoint_covers(ctx->c.params))
        return fail(ctx, GZ_E_INVAL, "the adjoint covers GZ_MFM with GZ_RIEMANN_HLLC only");
    if (ckpt && (((uintptr_t)ckpt & 255) || level < GZ_CKPT_RATES || level > GZ_CKPT_LISTS))
        return fail(ctx, GZ_E_INVAL, "checkpoint: need a 256-byte aligned buffer and a valid level");
    if (ctx->c.owned) return refuse_subdomain(ctx, "gz_step_backward");
    const Ckpt ck = ckpt_view(ctx->c, const_cast<void*>(ckpt), level);
    return GZ_DISPATCH(do_step_backward<float>(ctx, p_start, dt, ck, gbar_end, gbar_start),
                       do_step_backward<double>(ctx, p_start, dt, ck, gbar_end, gbar_start));
}

gz_status gz_get_neighbours(gz_ctx* ctx, int32_t* count_out, int64_t* ids_out, int32_t cap) {
    if (!ctx || !count_out || cap < 0) return GZ_E_INVAL;
    if (!ctx->c.nbr_valid) return fail(ctx, GZ_E_INVAL, "no neighbour lists yet");
    return cuda_check(ctx, run_get_neighbours(ctx->c, count_out, ids_out, cap), "gz_get_neighbours");
}

gz_status gz_checkpoint_limiters(gz_ctx* ctx, const void* ckpt, int64_t* ids_out) {
    if (!ctx || !ckpt || !ids_out) return GZ_E_INVAL;
    Ctx& c = ctx->c;
    const Ckpt ck = ckpt_view(c, const_cast<void*>(ckpt), GZ_CKPT_GRADIENTS);
    if (!c.last_lim || c.last_lim != ck.lim)
        return fail(ctx, GZ_E_INVAL, "gz_checkpoint_limiters: ckpt is not the last step checkpoint "
                                     "(GZ_CKPT_GRADIENTS) of this context");
    return cuda_check(ctx, run_get_limiters(c, ck.lim, ids_out), "gz_checkpoint_limiters");
}

gz_status gz_get_status(gz_ctx* ctx, uint32_t* bits, int64_t* first_bad_id, int64_t* counters,
                        int32_t reset) {
    if (!ctx) return GZ_E_INVAL;
    Ctx& c = ctx->c;
    DevStatus h;
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e == cudaSuccess) e = cudaMemcpy(&h, c.status, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(ctx, GZ_E_CUDA, std::string("gz_get_status: ") + cudaGetErrorString(e));
    if (bits) *bits = h.bits;
    if (first_bad_id) *first_bad_id = h.first_bad_id == ~0ull ? -1 : (int64_t)h.first_bad_id;
    if (counters)
        for (int k = 0; k < GZ_NCOUNTERS; ++k) counters[k] = (int64_t)h.counters[k];
    if (reset) {
        e = cudaMemsetAsync(c.status, 0, sizeof(DevStatus), c.stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(&c.status->first_bad_id, 0xFF, sizeof(unsigned long long), c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        if (e != cudaSuccess) return fail(ctx, GZ_E_CUDA, "gz_get_status reset failed");
    }
    return (h.bits & GZ_S_ERROR_MASK) ? GZ_E_DEVICE : GZ_OK;
}

const char* gz_last_error(gz_ctx* ctx) { return ctx ? ctx->c.err.c_str() : ""; }

gz_status gz_get_info(gz_ctx* ctx, int64_t* info, int32_t n) {
    if (!ctx || !info || n < 0 || n > 6) return GZ_E_INVAL;
    const Ctx& c = ctx->c;
    const int64_t v[6] = {c.launches, c.N, c.nboxes, c.total_cells, c.cap, c.rcap};
    for (int k = 0; k < n; ++k) info[k] = v[k];
    return GZ_OK;
}

gz_status gz_pair_count(gz_ctx* ctx, int64_t* ordered_pairs) {
    if (!ctx || !ordered_pairs) return GZ_E_INVAL;
    Ctx& c = ctx->c;
    if (!c.nbr_valid) return fail(ctx, GZ_E_INVAL, "no pair lists yet");
    long long h = 0;
    cudaError_t e = run_pair_count(c, c.pairs_dev);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, c.pairs_dev, sizeof(h), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return fail(ctx, GZ_E_CUDA, std::string("gz_pair_count: ") + cudaGetErrorString(e));
    *ordered_pairs = h;
    return GZ_OK;
}

gz_status gz_scan_stats(gz_ctx* ctx, int64_t* out3) {
    if (!ctx || !out3) return GZ_E_INVAL;
    Ctx& c = ctx->c;
    if (!c.nbr_valid) return fail(ctx, GZ_E_INVAL, "gz_scan_stats: no density pass yet");
    long long h[3] = {0, 0, 0};
    cudaError_t e = GZ_DISPATCH(run_scan_stats<float>(c, c.pairs_dev), run_scan_stats<double>(c, c.pairs_dev));
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, c.pairs_dev, sizeof(h), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return fail(ctx, GZ_E_CUDA, std::string("gz_scan_stats: ") + cudaGetErrorString(e));
    for (int k = 0; k < 3; ++k) out3[k] = h[k];
    return GZ_OK;
}

gz_status gz_profile_enable(gz_ctx* ctx, int32_t enable) {
    if (!ctx) return GZ_E_INVAL;
    ctx->c.prof = enable ? 1 : 0;
    return GZ_OK;
}

gz_status gz_profile_read(gz_ctx* ctx, double* ms, int64_t* calls, int32_t reset) {
    if (!ctx) return GZ_E_INVAL;
    Ctx& c = ctx->c;
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return fail(ctx, GZ_E_CUDA, std::string("gz_profile_read: ") + cudaGetErrorString(e));
    for (auto& pe : c.pending) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, pe.a, pe.b) == cudaSuccess) {
            c.prof_ms[pe.pass] += t;
            c.prof_calls[pe.pass] += 1;
        }
        c.ev_pool.push_back(pe.a);
        c.ev_pool.push_back(pe.b);
    }
    c.pending.clear();
    for (int k = 0; k < GZ_NPASSES; ++k) {
        if (ms) ms[k] = c.prof_ms[k];
        if (calls) calls[k] = c.prof_calls[k];
        if (reset) {
            c.prof_ms[k] = 0.0;
            c.prof_calls[k] = 0;
        }
    }
    return GZ_OK;
}

}  // extern "C"
