// Host-side launchers shared between the translation units of the library.
#pragma once

#include "gz_internal.cuh"

namespace gz {

template <typename T>
Sorted<T> sorted_view(Ctx& c);

// Binning + radix sort + permutation into the context's sorted arrays, and
// cell ranges.  n_in (caller order, may be null) is permuted into the sorted
// n array as well.  Returns a CUDA error code.
template <typename T>
cudaError_t sort_and_bin(Ctx& c, const gz_particles& p, const void* n_in);
// The part of sort_and_bin after the radix sort, from c.keys and c.vals as a
// sort left them (a checkpoint's copy of them: the same start state).
template <typename T>
cudaError_t permute_and_bin(Ctx& c, const gz_particles& p, const void* n_in);

// Writes sorted-order arrays back to caller order.
template <typename T>
cudaError_t unpermute_T(Ctx& c, const T* src, T* dst, int rows);
cudaError_t unpermute_d(Ctx& c, const double* src, double* dst, int rows);
cudaError_t unpermute_i(Ctx& c, const int* src, int* dst);

// Hydro passes (sorted order).
// list (device, sorted indices) and nlist (device count, at most n): run on
// those particles only.
template <typename T>
cudaError_t run_density(Ctx& c, const int* list = nullptr, const int* nlist = nullptr, int n = 0);
template <typename T>
cudaError_t run_density_given(Ctx& c);
template <typename T>
cudaError_t run_build_lists(Ctx& c);
// Rebuilds the lists of the particles with more than `kept` neighbours (the
// others' lists and counts restored from a checkpoint).
template <typename T>
cudaError_t run_lists_over(Ctx& c, int kept);
template <typename T>
cudaError_t run_reverse(Ctx& c);
template <typename T>
cudaError_t run_prim(Ctx& c);
template <typename T>
cudaError_t run_gradients(Ctx& c, bool want_dt, bool with_info = false, const int* list = nullptr,
                          const int* nlist = nullptr, int n = 0);
template <typename T>
cudaError_t run_timestep_only(Ctx& c);
template <typename T>
cudaError_t run_pack_given(Ctx& c, const T* grad, const T* B, const int* list = nullptr,
                           const int* nlist = nullptr, int n = 0, const unsigned char* skip = nullptr);
template <typename T>
cudaError_t run_fluxes(Ctx& c);
template <typename T>
cudaError_t run_update(Ctx& c, gz_particles& p, double* rates_out = nullptr);
cudaError_t run_rates_in(Ctx& c, const double* rates);
template <typename T>
cudaError_t run_ufloor(Ctx& c, gz_particles& p);
template <typename T>
cudaError_t run_grad_out(Ctx& c, T* grad_out, T* B_out);

cudaError_t run_dt_init(Ctx& c);
cudaError_t run_dt_finalize(Ctx& c, double dt_fixed, double* dt_used_dev);
cudaError_t run_dt_set(Ctx& c, double dt);
cudaError_t run_dt_out(Ctx& c, double* out);
cudaError_t run_dt_copy(Ctx& c, const double* dt);
cudaError_t run_set_box(Ctx& c);
cudaError_t run_get_neighbours(Ctx& c, int32_t* count_out, int64_t* ids_out, int cap);
cudaError_t run_get_limiters(Ctx& c, const int* lim, int64_t* out);

cudaError_t run_pair_count(Ctx& c, long long* out_dev);
template <typename T>
cudaError_t run_scan_stats(Ctx& c, long long* out_dev);

// Adjoint passes.
cudaError_t ensure_adjoint_scratch(Ctx& c);
template <typename T>
cudaError_t run_flux_adjoint(Ctx& c, const double* dpbar, const double* dEbar);
template <typename T>
cudaError_t run_step_adjoint(Ctx& c, const gz_particles& gend, gz_particles& gstart);
cudaError_t run_adj_out_flux(Ctx& c, double* xbar, double* hbar, double* nbar, double* Wbar, double* gbar,
                             double* Bbar);

KParams kparams(const Ctx& c);

// Per-pass CUDA-event profile (gz_profile_*) for passes launched outside the
// API layer: begin/end record events on the context stream when profiling is
// on (implemented with the API layer's event pool).
struct PassTimer {
    Ctx* c;
    void begin(int pass) const;
    void end(int pass) const;
};

// Hierarchical timesteps: one sync interval of 2^K substeps in place on p
// (one host synchronisation per substep to read the number of active
// particles).  active_out (host) receives the active particle-substeps.
cudaError_t ensure_hier_scratch(Ctx& c);
void free_hier_scratch(Ctx& c);
template <typename T>
cudaError_t run_step_hier(Ctx& c, gz_particles& p, int K, double dt_fixed, double* dt_used_dev,
                          int32_t* bins_out, long long* active_out, const PassTimer& timer);

}  // namespace gz
