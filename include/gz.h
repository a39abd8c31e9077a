/*
 * gz.h -- C ABI of the GB300 meshless finite-mass (MFM) hydrodynamics library.
 *
 * Method: GIZMO's Lagrangian mesh-free finite-volume Godunov scheme in its
 * meshless finite-mass form (GIZMO public-release paper: "Hydrodynamics" item
 * of the physics list, and the "Arbitrary (Moving) Meshes" section, where the
 * mesh moves with the fluid), in a periodic unit box ("periodic ... boundary
 * conditions" item) with a gamma-law equation of state and one global CFL
 * timestep.  The paper prints no formula for the scheme; the readings used
 * here are labelled O1..O14 and restated at each call below:
 *
 *   O1  minimum-image offsets d = x_j - x_i in the unit box
 *   O2  cubic-spline kernel W(r, H) = 8/(pi H^3) w(r/H), support radius H
 *   O3  neighbour set N_i = {j != i : r_ij < H_i}
 *   O4  H_i solves (4 pi/3) H^3 n_i(H) = N_ngb (bracketed Newton)
 *   O5  n_i = sum_{N_i + i} W(r_ij, H_i); V_i = 1/n_i; rho_i = m_i n_i
 *   O6  psi_j(x_i) = W(r_ij, H_i) / n_i
 *   O7  E_i = sum psi_j d d^T, B_i = E_i^-1
 *   O8  least-squares gradients g = B_i sum (f_j - f_i) d psi_j
 *   O9  per-particle limiter alpha_i (beta = 1, face point at s_ij = H_i/(H_i+H_j))
 *   O10 flux pairs r < max(H_i, H_j); face area
 *       A_ij = V_i psi_j(x_i) B_i d + V_j psi_i(x_j) B_j d
 *   O11 linear reconstruction + Hancock half step + pairwise clamp
 *   O12 HLLC (Davis wave speeds) in the face frame; MFM rates
 *       dp_i/dt = -sum P* A_ij, dE_i/dt = -sum P* (S* + v_f . n) |A_ij|
 *   O13 dt = cfl * min_i 2 V_i^(1/3) / max_j v_sig,ij
 *   O14 kick, trapezoid drift, periodic wrap, u floor
 *
 * gz_params.scheme selects GZ_MFM (above) or GZ_MFV, the paper's meshless
 * finite-volume variant, where mass also moves across the faces:
 *   O15 HLLC flux of mass, momentum and total energy through the face moving
 *       with v_f (star states of the face frame, boosted back to the lab
 *       frame); dm_i/dt = -sum F_m |A_ij|, dp_i/dt = -sum F_p |A_ij|,
 *       dE_i/dt = -sum F_E |A_ij|; the update advances m too.
 *
 * Conventions
 *   - Every call returns a gz_status; no exception or abort crosses the ABI.
 *     Calls are asynchronous on the context's CUDA stream; conditions found
 *     on the device are recorded in a device status word read (with a stream
 *     synchronisation) by gz_get_status.  gz_last_error gives host-side text.
 *   - Particle arrays are device pointers owned by the caller, one contiguous
 *     array per field (structure of arrays).  Their element type is float for
 *     GZ_MIXED32 and double for GZ_FP64 (ids are always int64).  The library
 *     never frees or keeps them beyond a call.  Outputs are written in the
 *     caller's particle order; internal sorting is invisible.
 *   - The context owns all scratch memory (sort buffers, cell ranges,
 *     neighbour lists, gradients, rates) and frees it in gz_destroy.
 *   - Boxes: a context holds nboxes independent periodic unit boxes; box b's
 *     particles are the contiguous slice [sum_{c<b} counts[c], ...).  Every
 *     box has its own cell grid and its own CFL timestep.
 *   - Ids must be unique non-negative int64 (within each box).  Every pair
 *     quantity is evaluated in one fixed order of the pair, so both
 *     particles of a pair receive bitwise-opposite rate contributions: the
 *     lower sorted position first in the MFM flux passes, the lower id first
 *     under GZ_MFV and in the adjoint.
 */
#ifndef GZ_H
#define GZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gz_status;

/* Return codes. */
#define GZ_OK 0
#define GZ_E_INVAL 1     /* invalid argument (null pointer, bad size, bad params) */
#define GZ_E_NOMEM 2     /* device allocation failed                             */
#define GZ_E_CUDA 3      /* a CUDA runtime call failed (text in gz_last_error)    */
#define GZ_E_DEVICE 4    /* device status word has error bits set (gz_get_status) */

/* Device status bits (gz_get_status).  Error bits: */
#define GZ_S_HCONV (1u << 0)        /* h-iteration hit max_iter (O4)               */
#define GZ_S_SINGULAR (1u << 1)     /* det(E) <= 0 or kappa > 1e8 (O7); B = 0 used  */
#define GZ_S_NONFINITE (1u << 2)    /* non-finite input or output value            */
#define GZ_S_NBR_OVERFLOW (1u << 3) /* a neighbour list exceeded its capacity       */
#define GZ_S_HLIM (1u << 4)         /* support radius reached h_lim                 */
/* Informational bits (counted, not errors): */
#define GZ_S_FALLBACK (1u << 8)     /* first-order face states used (O11)           */
#define GZ_S_PSTAR_NEG (1u << 9)    /* HLLC P* < 0 (O12; clamped to 0, or exact star
                                       under GZ_RIEMANN_FALLBACK), or a vacuum face   */
#define GZ_S_UFLOOR (1u << 10)      /* u floored after the update (O14)             */
#define GZ_S_KAPPA_FP64 (1u << 11)  /* E re-inverted in FP64 (kappa > kappa_max)    */
#define GZ_S_ERROR_MASK 0xFFu

/* Counter slots of gz_get_status. */
#define GZ_C_HCONV 0
#define GZ_C_SINGULAR 1
#define GZ_C_NONFINITE 2
#define GZ_C_NBR_OVERFLOW 3
#define GZ_C_FALLBACK 4
#define GZ_C_PSTAR_NEG 5
#define GZ_C_UFLOOR 6
#define GZ_C_KAPPA_FP64 7
#define GZ_NCOUNTERS 8

/* Schemes (gz_params.scheme). */
#define GZ_MFM 0 /* meshless finite mass: particle masses fixed (O12)             */
#define GZ_MFV 1 /* meshless finite volume: mass fluxes between particles (O15)   */

/* Riemann solvers of the MFM face (gz_params.riemann; O12).  EXACT: the
 * exact star pressure and contact speed of the face-frame Riemann problem
 * (safeguarded Newton iteration on the pressure function of each side:
 * shock branch (p - P_K) sqrt(A_K/(p + B_K)), A_K = 2/((gamma+1) rho_K),
 * B_K = (gamma-1)/(gamma+1) P_K; rarefaction branch
 * 2 c_K/(gamma-1) ((p/P_K)^((gamma-1)/(2 gamma)) - 1)) replace HLLC's P* and
 * S* on every face; a face whose fans open a vacuum carries P* = 0 and sets
 * GZ_S_PSTAR_NEG.  FALLBACK: HLLC, and the exact star where HLLC's P* < 0
 * (such faces still set GZ_S_PSTAR_NEG). */
#define GZ_RIEMANN_HLLC 0
#define GZ_RIEMANN_EXACT 1
#define GZ_RIEMANN_FALLBACK 2

/* Precision modes. */
#define GZ_FP64 0    /* every step in double                                          */
#define GZ_MIXED32 1 /* float state and pair math; double for the Newton update of H,
                        the E inversion when kappa > kappa_max, and the per-particle
                        rate accumulation and update                                 */

typedef struct {
    double gamma;        /* adiabatic index (5/3)                                     */
    double ngb;          /* effective neighbour number N_ngb (32)                     */
    double tol;          /* h-iteration stops when |f| <= tol * ngb (1e-6)            */
    double cfl;          /* CFL factor (0.2)                                          */
    double kappa_max;    /* FP64 re-inversion threshold for cond(E) (100)            */
    double beta;         /* limiter factor (1)                                        */
    double u_floor_frac; /* floor = u_floor_frac * lower median of u at step start   */
    double h_lim;        /* support radius stays below this (0.5)                    */
    double cell_factor;  /* cell length = cell_factor * H0 of the box (1.0)          */
    int32_t precision;   /* GZ_FP64 or GZ_MIXED32                                     */
    int32_t hancock;     /* 1: half-step predictor on face states (1)                */
    int32_t max_iter;    /* cap on f evaluations of the h-iteration (64)             */
    int32_t max_ngb;     /* capacity of each particle's neighbour list (128)         */
    int32_t scheme;      /* GZ_MFM or GZ_MFV (GZ_MFM)                                 */
    int32_t riemann;     /* MFM face solver: GZ_RIEMANN_HLLC, _EXACT or _FALLBACK     */
                         /* (GZ_RIEMANN_HLLC); GZ_MFV takes GZ_RIEMANN_HLLC only      */
    int32_t density_cache; /* h-iteration candidate cache per particle: 40 or 48      */
                           /* entries, or 0 (40 when every box holds >= 32^3          */
                           /* particles, else 48); a particle with more candidates    */
                           /* within 1.05 H is iterated by a whole warp (0)            */
} gz_params;

/* Structure-of-arrays particle set; every pointer is device memory with N
 * elements (float or double per precision; id int64).  h is the support
 * radius H (kernel is zero for r >= H). */
typedef struct {
    void* x;
    void* y;
    void* z;
    void* vx;
    void* vy;
    void* vz;
    void* m;
    void* u; /* specific internal energy */
    void* h;
    const int64_t* id;
} gz_particles;

typedef struct gz_ctx gz_ctx;

/* Fills *out with the defaults listed in gz_params.  Never fails for a
 * non-null pointer. */
gz_status gz_default_params(gz_params* out);

/* Creates a context for nboxes boxes with counts[b] particles each (host
 * array).  cuda_stream is a cudaStream_t (NULL = default stream); all work is
 * enqueued on it.  Allocates all scratch on the current device.  Errors:
 * GZ_E_INVAL (null out/counts/params, nboxes < 1, a count < 1, invalid
 * params), GZ_E_NOMEM. */
gz_status gz_create(const gz_params* params, int32_t nboxes, const int64_t* counts,
                    void* cuda_stream, gz_ctx** out);

/* Frees the context and its scratch (synchronises its stream). */
gz_status gz_destroy(gz_ctx* ctx);

/* O3-O5.  Reads x, y, z, h (h = initial guess of H) and id (vx, vy, vz, m
 * and u are not read and may be NULL); solves the
 * h-iteration for every particle and writes the converged H back into h,
 * the kernel number density n into n_out, and the number of f evaluations
 * into iters_out (int32).  n_out and iters_out may be NULL.  The neighbour
 * lists of the final H are kept in the context (gz_get_neighbours). */
gz_status gz_density(gz_ctx* ctx, gz_particles* p, void* n_out, int32_t* iters_out);

/* O6-O9 with the given H (p->h) and n (device, N values): writes the
 * limited gradients of (rho, vx, vy, vz, P) to grad_out as [15][N]
 * (row = field*3 + axis) and B = E^-1 to B_out as [6][N] (xx, xy, xz, yy,
 * yz, zz).  Either output may be NULL. */
gz_status gz_gradients(gz_ctx* ctx, const gz_particles* p, const void* n, void* grad_out,
                       void* B_out);

/* O13 with the given H and n: writes the per-particle signal-speed step
 * 2 V_i^(1/3)/max_j v_sig,ij into dt_i_out ([N], double, may be NULL) and
 * cfl * min over each box into dt_box_out ([nboxes] doubles, device). */
gz_status gz_timestep(gz_ctx* ctx, const gz_particles* p, const void* n, double* dt_i_out,
                      double* dt_box_out);

/* O10-O12 (O15 under GZ_MFV) with the given H, n, limited gradients grad
 * ([15][N]) and B ([6][N]) and half-step time dt (the Hancock predictor uses
 * dt/2): writes dp/dt to dpdt ([3][N] doubles), dE/dt to dEdt ([N]
 * doubles) and, if dmdt is non-NULL, dm/dt to dmdt ([N] doubles; zeros
 * under GZ_MFM). */
gz_status gz_hydro_fluxes(gz_ctx* ctx, const gz_particles* p, const void* n, const void* grad,
                          const void* B, double dt, double* dpdt, double* dEdt, double* dmdt);

/* Adjoint of gz_hydro_fluxes with the same frozen inputs (H, n, grad, B,
 * dt; neighbour and pair sets of those H): given dpdt_bar ([3][N]) and
 * dEdt_bar ([N]) = dL/d(rates), writes dL/d(inputs) as double arrays:
 * x_bar [3][N] (positions), h_bar [N], n_bar [N], W_bar [5][N] (rho, vx,
 * vy, vz, P), grad_bar [15][N], B_bar [6][N].  Any output may be NULL.
 * min/max/clamp pass the adjoint to the branch the forward took.  The adjoint
 * covers GZ_MFM with GZ_RIEMANN_HLLC only: otherwise this call,
 * gz_step_checkpoint and gz_step_backward return GZ_E_INVAL. */
gz_status gz_hydro_fluxes_backward(gz_ctx* ctx, const gz_particles* p, const void* n,
                                   const void* grad, const void* B, double dt,
                                   const double* dpdt_bar, const double* dEdt_bar, double* x_bar,
                                   double* h_bar, double* n_bar, double* W_bar, double* grad_bar,
                                   double* B_bar);

/* One full step O4-O14 in place on p (x, y, z, vx, vy, vz, u, h updated;
 * under GZ_MFV m too (O15), where a mass that is not positive after the
 * update sets GZ_S_NONFINITE; id read only).  dt_fixed > 0 uses that step for every box;
 * otherwise each box takes its CFL step.  dt_used_dev (device, nboxes
 * doubles, may be NULL) receives the steps used.  No host synchronisation. */
gz_status gz_step(gz_ctx* ctx, gz_particles* p, double dt_fixed, double* dt_used_dev);

/* The step split in two around its timestep: gz_step_begin runs S1-S3 (bin
 * and sort, h-iteration, primitives, pair lists, gradients and limiter) and
 * writes to dt_box_dev (device, nboxes doubles) the CFL step of each box,
 * cfl * min_i dtc_i (O13) over the box's owned particles (all of them outside
 * a subdomain); gz_step_finish then runs S4 and S6 (fluxes, update) with the
 * steps in dt_dev (device, nboxes doubles, e.g. the minimum of dt_box_dev
 * over the subdomains of one box).  gz_step_finish takes the particle set
 * given to gz_step_begin, unchanged, with no other call on the context in
 * between; begin then finish with dt_dev = dt_box_dev is gz_step bit for bit.
 * No host synchronisation.  Errors: GZ_E_INVAL (null arrays, finish without
 * begin), GZ_E_CUDA. */
gz_status gz_step_begin(gz_ctx* ctx, gz_particles* p, double* dt_box_dev);
gz_status gz_step_finish(gz_ctx* ctx, gz_particles* p, const double* dt_dev);

/* Domain decomposition: one periodic box split into subdomains, each held by
 * its own context (one per GPU, or several on one GPU), the GPU form of the
 * domain decomposition of the paper's hybrid MPI + OpenMP runtime (Sec. 1
 * and Sec. 3).  A subdomain context holds its owned particles and ghost
 * copies of the particles whose data its owned particles' step reads (a
 * halo, several support radii deep, refreshed by the caller each step).
 * gz_create_subdomain: one box whose arrays hold up to capacity particles and
 * whose cell grid (cell length cell_factor * H0) and density cache are those
 * of a box of grid_count particles, the whole undivided box, so that its
 * cells hold the same particles in the same order as that box's.
 * gz_set_subdomain: the particles of the next calls are n <= capacity arrays
 * (caller order; the whole box's relative order of particles is kept when
 * the caller keeps them in ascending id), owned (device, n bytes, copied; 1 =
 * owned, 0 = ghost; NULL = all owned) marks the n_owned owned ones.  Ghosts
 * are stepped like the others but take no part in the box's CFL minimum, and
 * the u floor (O14) takes the lower median of the owned particles' u.  With a
 * halo deep enough that every particle the owned particles' density,
 * gradient and flux passes read sees its full neighbourhood, the owned
 * particles' step equals the undivided box's bit for bit (the u floor
 * excepted: a subdomain's median is its own).  A subdomain context takes
 * gz_step, gz_step_begin / gz_step_finish and the single passes; the calls
 * whose buffers or captured launches are laid out for one particle count
 * (gz_checkpoint_bytes, gz_step_checkpoint, gz_step_backward, gz_step_hier,
 * gz_graph_capture) refuse it with GZ_E_INVAL.  Errors: GZ_E_INVAL (not a
 * subdomain context, sizes out of range), GZ_E_NOMEM, GZ_E_CUDA. */
gz_status gz_create_subdomain(const gz_params* params, int64_t capacity, int64_t grid_count,
                              void* cuda_stream, gz_ctx** out);
gz_status gz_set_subdomain(gz_ctx* ctx, int64_t n, int64_t n_owned, const uint8_t* owned);

/* Hierarchical (individual, power-of-two) timesteps: advances every box of p
 * by one sync interval D split into 2^K substeps of D/2^K (K in [0, 20]).
 * Reading of the paper's hierarchical adaptive timesteps (it gives no
 * formula): particle i takes bin k_i (step D/2^k_i) and is active at the
 * substeps that start a step of its own.  At substep 0 all particles are
 * active; D = dt_fixed when dt_fixed > 0, else per box
 * min(cfl max_i dtc_i, 2^K cfl min_i dtc_i) with dtc_i = 2 V_i^(1/3)/max v_sig
 * (O13), and k_i is the smallest k with D/2^k <= cfl dtc_i (at most K; later
 * active times may only deepen a bin).  At each substep the active particles
 * run O4-O9 and O13 at positions predicted for all particles
 * (x_start + elapsed * (v_start + v)/2); the others keep H, n, gradients and B
 * of their last active time; every flux pair (O10) with an active particle
 * exchanges the O11/O12 face fluxes over D/2^max(k_i, k_j) (Hancock with half
 * of that), equal and opposite for its two particles; momentum and energy are
 * kicked at once, and a step that ends drifts its particle by
 * dt_i (v_start + v_end)/2.  K = 0 gives gz_step's result bitwise.  In place
 * on p like gz_step (x, y, z, vx, vy, vz, u, h, and m under GZ_MFV; id read only); h ends as
 * each particle's H of its last active time.  dt_used_dev (device, nboxes
 * doubles, may be NULL) receives D per box, bins_out (device, N int32, caller
 * order, may be NULL) the final bins, *active_out (host, may be NULL) the
 * number of active particle-substeps.  Host synchronisation: one per substep
 * (the number of active particles sizes the launches; substeps without one
 * only drift), so the call cannot be captured in a CUDA graph.  Scratch of
 * about 150 bytes a particle (FP32) is allocated on the first call.  Every
 * Riemann option of the MFM face applies, and GZ_MFV (O15: the mass shares are
 * exchanged with momentum and energy, m is updated too).  Errors: GZ_E_INVAL
 * (K out of range), GZ_E_NOMEM. */
gz_status gz_step_hier(gz_ctx* ctx, gz_particles* p, int32_t K, double dt_fixed, double* dt_used_dev,
                       int32_t* bins_out, int64_t* active_out);

/* Captures nsteps consecutive gz_step calls on p (same arguments as gz_step)
 * into a CUDA graph owned by the context, replacing any earlier one; nothing
 * is executed.  The context's stream must be a created (non-default) stream.
 * gz_graph_launch replays the captured steps on that stream (the graph
 * keeps p's pointers: replays advance the same arrays).  Host
 * synchronisation: none in either call. */
gz_status gz_graph_capture(gz_ctx* ctx, gz_particles* p, int32_t nsteps, double dt_fixed,
                           double* dt_used_dev);
gz_status gz_graph_launch(gz_ctx* ctx);

/* Step checkpoints for the adjoint (per-step checkpointing of a rollout).
 * A checkpoint is a caller-owned device buffer, 256-byte aligned, of
 * gz_checkpoint_bytes(level) bytes, written by gz_step_checkpoint and read
 * by gz_step_backward of the same step; its layout is private.  Level
 * GZ_CKPT_RATES keeps the step's conserved-variable rates (the momentum
 * and total-energy rates of the MFM update, O12), the converged support
 * radii (O4) and the number density and kernel-derivative sum at them (44
 * bytes a particle in FP32) so the backward pass skips the h-iteration and
 * the flux pass; GZ_CKPT_GRADIENTS also keeps the
 * gradient pass's per-particle outputs (limited gradients, E^-1, limiter
 * factors and the indices of the limiting particles; about 330 bytes a
 * particle in FP32) so the backward pass skips that pass too;
 * GZ_CKPT_LISTS also keeps the sort's order and the neighbour lists
 * (their first 64 slots: about 270 bytes a particle more in FP32) so the
 * backward pass skips the radix sort and the density rescan that rebuilds
 * them (lists longer than 64 are rebuilt by a scan).  No pair quantity is
 * ever stored: the backward pass recomputes every one.  Every level gives
 * the same backward result bit for bit. */
#define GZ_CKPT_RATES 0
#define GZ_CKPT_GRADIENTS 1
#define GZ_CKPT_LISTS 2
gz_status gz_checkpoint_bytes(gz_ctx* ctx, int32_t level, int64_t* bytes);

/* The choices of the O9 limiter in the step whose checkpoint is ckpt (level
 * GZ_CKPT_GRADIENTS, the last gz_step_checkpoint on this context, with no
 * call that sorts in between), as particle ids in caller order: ids_out
 * (device, [10][N] int64) rows 0-4 (fields rho, vx, vy, vz, P) the neighbour
 * whose face bound set alpha_f (-1 where alpha_f = 1), rows 5-9 the particle
 * holding the extreme that bound reached (the particle itself where alpha_f =
 * 1).  Two runs with the same choices crossed no limiter switch: the step is
 * smooth between them in the limiter (a derivative check needs that).
 * Errors: GZ_E_INVAL (null arguments, ckpt not that checkpoint), GZ_E_CUDA. */
gz_status gz_checkpoint_limiters(gz_ctx* ctx, const void* ckpt, int64_t* ids_out);

/* gz_step (same arguments and effect) that also fills the checkpoint ckpt
 * at the given level.  At GZ_CKPT_LISTS the list copies run on a second
 * stream of the context (created, with two events, on the first such call;
 * released by gz_destroy), forked from and joined back to the context's
 * stream by events within the call, so work issued on the context's stream
 * after the call sees a complete checkpoint.  Make the first such call
 * outside any stream capture.  Host synchronisation: none. */
gz_status gz_step_checkpoint(gz_ctx* ctx, gz_particles* p, double dt_fixed, double* dt_used_dev,
                             void* ckpt, int32_t level);

/* Adjoint of one gz_step (all of O4-O14 with the step dt held fixed and
 * neighbour sets frozen at their forward values).  p_start is the state the
 * forward step started from (it is not modified).  ckpt (with its level) is
 * that step's checkpoint from gz_step_checkpoint, or NULL to recompute
 * everything from p_start; without a checkpoint, p_start's h is the initial
 * guess of the h-iteration (passing the h the forward step returned makes it
 * accept that H at once, with the same H, lists and sums as the forward).
 * gbar_end holds dL/d(state after the step) for x, y, z, vx, vy, vz, u (m, h,
 * id ignored; arrays in the working precision); gbar_start receives
 * dL/d(state before the step) for x, y, z, vx, vy, vz, u and m.  dt is the
 * step the forward used (> 0).  Host synchronisation: none. */
gz_status gz_step_backward(gz_ctx* ctx, const gz_particles* p_start, double dt, const void* ckpt,
                           int32_t level, const gz_particles* gbar_end, gz_particles* gbar_start);

/* Copies the neighbour lists of the last gz_density / gz_step: count_out
 * ([N] int32, device) and, if ids_out is non-NULL, the neighbours' ids into
 * ids_out ([cap][N] int64, slot-major, device; unused slots = -1).  Lists are
 * in enumeration order, not sorted. */
gz_status gz_get_neighbours(gz_ctx* ctx, int32_t* count_out, int64_t* ids_out, int32_t cap);

/* Synchronises the context stream and returns the accumulated device status
 * bits, the smallest particle id involved in an error (-1 if none) and, if
 * counters is non-NULL, GZ_NCOUNTERS event counts.  reset != 0 clears them.
 * Returns GZ_E_DEVICE when any error bit is set, GZ_E_CUDA on a CUDA error. */
gz_status gz_get_status(gz_ctx* ctx, uint32_t* bits, int64_t* first_bad_id, int64_t* counters,
                        int32_t reset);

/* Pass indices of the per-pass profile. */
#define GZ_PASS_SORT 0      /* S1 binning, radix sort, permutation            */
#define GZ_PASS_DENSITY 1   /* S2 h-iteration and neighbour lists             */
#define GZ_PASS_LISTS 2     /* neighbour lists for a given H                  */
#define GZ_PASS_REVERSE 3   /* reverse flux pairs                             */
#define GZ_PASS_PRIM 4      /* primitives rho, P, c                           */
#define GZ_PASS_GRAD 5      /* S3 gradients, limiter (+ S5 signal speed)      */
#define GZ_PASS_FLUX 6      /* S4 pairwise HLLC fluxes                        */
#define GZ_PASS_UPDATE 7    /* S6 kick, drift, wrap, u floor (+ dt finalise) */
#define GZ_NPASSES 8

/* Host-side facts about the context: info[0] kernel launches issued so far,
 * info[1] N, info[2] nboxes, info[3] cells of all boxes, info[4] neighbour
 * list capacity, info[5] reverse list capacity.  n = entries wanted (<= 6). */
gz_status gz_get_info(gz_ctx* ctx, int64_t* info, int32_t n);

/* Ordered flux pairs sum_i |P_i| of the last pass that built pair lists
 * (device reduction; synchronises the stream). */
gz_status gz_pair_count(gz_ctx* ctx, int64_t* ordered_pairs);

/* Work of the neighbour search (a diagnostic; the paper has no counterpart):
 * over the particles of the last density pass, at their converged H and the
 * positions that pass sorted, out3[0] = candidates a cell scan of radius
 * 1.05 H tests (the density cache's radius; the cells whose nearest point
 * lies beyond it are skipped, as in the density pass), out3[1] = those
 * within 1.05 H, out3[2] = those within H (the neighbours, O3).  out3 is a
 * host array of 3.  One extra kernel; synchronises the stream.  Errors:
 * GZ_E_INVAL (null arguments, no density pass yet), GZ_E_CUDA. */
gz_status gz_scan_stats(gz_ctx* ctx, int64_t* out3);

/* enable != 0: record CUDA events on the context stream around every pass of
 * subsequent calls (a few microseconds per pass).  gz_profile_read
 * synchronises and returns the accumulated milliseconds and invocation
 * counts per pass (GZ_NPASSES entries each); reset != 0 clears them. */
gz_status gz_profile_enable(gz_ctx* ctx, int32_t enable);
gz_status gz_profile_read(gz_ctx* ctx, double* ms, int64_t* calls, int32_t reset);

/* Density pass that allocates nothing (the paper has no counterpart: this is
 * a library-interface addition).  For callers that cannot call cudaMalloc:
 * host codes whose device memory is all handed out by their own pool or
 * budget, and loops that cannot afford the device-wide synchronisation an
 * allocation may cause.  Runs the same kernels as gz_density on a one-box
 * context of n particles with these params, so h, n and the iteration counts
 * are bitwise the same: reads x, y, z, h (initial guess), id (device arrays
 * of the working precision; vx, vy, vz, m, u are ignored), writes the
 * converged H back into h, n into n_out and the f-evaluation counts into
 * iters_out (either may be NULL); enqueued on cuda_stream.  Neighbour lists
 * are not kept (max_ngb has no effect).  status_out (device pointer, may be
 * NULL) receives this call's device status bits (GZ_S_*: positions outside
 * the box, non-convergence, ...; never GZ_S_NBR_OVERFLOW, as no list is
 * kept) when the stream reaches the end of the call.
 * Scratch: a fixed array inside the library (about 8.3 MB, held on every GPU
 * that loads the library until exit).  Limits: 1 <= n <= 32768 and a cell
 * grid of at most 32^3 cells (cell_factor * H0 >= 1/32), else GZ_E_INVAL.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call reuses the same array, so calls that overlap on the
 * GPU (other streams, other host threads) race; serialise them. */
gz_status gz_density_noalloc(const gz_params* params, int64_t n, gz_particles* p, void* n_out,
                             int32_t* iters_out, uint32_t* status_out, void* cuda_stream);

/* Measured throughput of one SM pipe on the current device (a measurement
 * aid for the ALU roofline, not part of the method): which = 0 FP32 fused
 * multiply-add (FLOP/s, 2 per FMA), 1 FP64 fused multiply-add (FLOP/s), 2 FP32
 * reciprocal square root of the special-function unit (operations/s).
 * Independent dependency chains over 8 blocks of 256 threads per SM, best of
 * three timed launches (CUDA events) on cuda_stream; a few milliseconds.
 * Synchronises the stream.  Errors: GZ_E_INVAL, GZ_E_NOMEM, GZ_E_CUDA. */
gz_status gz_measure_alu(int32_t which, double* ops_per_s, void* cuda_stream);

/* Text of the last host-side error of this context ("" if none). */
const char* gz_last_error(gz_ctx* ctx);

/* Library version string. */
const char* gz_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GZ_H */
