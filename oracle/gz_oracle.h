/*
 * FP64 CPU oracle for the meshless finite-mass (MFM) hydrodynamics step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this code: only tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant with the
 * CUDA library under paper_1712_01294_gb300/csrc.
 *
 * Method: GIZMO's Lagrangian mesh-free finite-volume Godunov scheme in its
 * meshless finite-mass form ("Hydrodynamics" item of the physics list; the
 * "Arbitrary (Moving) Meshes" section: the mesh moves with the fluid), with a
 * periodic box (boundary-condition item).  The paper gives no formulas; the
 * readings this file implements (kernel, h-iteration, E-matrix gradients,
 * face areas, limiter, Hancock predictor, HLLC, CFL step, update) are listed
 * one by one in the design notes and cited at each function below by their
 * reading label (O1 ... O14).
 *
 * All arithmetic is FP64 with FMA contraction disabled (-ffp-contract=off).
 * Every neighbour sum runs over neighbours in ascending original particle id,
 * so results do not depend on the thread count or on the neighbour finder
 * (brute force or cell list).
 */
#ifndef GZ_ORACLE_H
#define GZ_ORACLE_H
#include <stdint.h>

typedef struct {
    double gamma;        /* adiabatic index of the gamma-law EOS              */
    double ngb;          /* target effective neighbour number N_ngb           */
    double tol;          /* h-iteration tolerance: |f| <= tol * N_ngb         */
    double cfl;          /* CFL factor of the global timestep                 */
    double kappa_max;    /* condition-number threshold (FP64 redo on GPU)     */
    double beta;         /* limiter factor                                     */
    double u_floor_frac; /* u floor = u_floor_frac * median(u at step start)  */
    double h_lim;        /* support radius must stay below this (<= 0.5)     */
    int32_t hancock;     /* 1: add the half-step predictor to face states     */
    int32_t max_iter;    /* cap on f-evaluations of the h-iteration           */
    int32_t use_cells;   /* 0: brute-force neighbours; 1: cell list           */
    int32_t scheme;      /* 0: MFM (faces move with the contact, no mass      */
                         /*    flux); 1: MFV (faces move with v_f, HLLC mass,  */
                         /*    momentum and energy fluxes; masses evolve)      */
    int32_t riemann;     /* MFM face solver: 0 HLLC; 1 exact (iterative star  */
                         /*    pressure) on every face; 2 HLLC, exact where    */
                         /*    HLLC's P* < 0                                   */
    int32_t pad;
} gzo_params;

typedef struct {
    int64_t hconv;       /* particles whose h-iteration hit max_iter          */
    int64_t singular;    /* particles with det(E) <= 0 or kappa > 1e8         */
    int64_t fallback;    /* pair evaluations that fell back to first order    */
    int64_t pstar_neg;   /* pair evaluations with HLLC P* < 0 (clamped to 0,  */
                         /*    or replaced by the exact solver's under         */
                         /*    riemann = 2) or a vacuum face (exact solver)    */
    int64_t ufloor;      /* particles whose u was floored in the update       */
    int64_t nonfinite;   /* non-finite inputs or outputs                      */
    int64_t kappa_big;   /* particles with kappa > kappa_max                  */
    int64_t pairs;       /* ordered flux pairs visited                        */
    int64_t bin_clamp;   /* hierarchical steps: bin assignments capped at K   */
} gzo_counters;

/* O2 */
double gzo_kernel_w(double q);
double gzo_kernel_dw(double q);
double gzo_W(double r, double H);
double gzo_dWdH(double r, double H);

/* O1: minimum-image offset of one component. */
double gzo_min_image(double d);

/* O3: neighbour sets {j != i : r_ij^2 < R_i^2}, ascending id.  Returns the
 * total count; writes offsets[N+1] and nbr[] (particle indices) when nbr is
 * non-null and cap is large enough (else returns -total). */
int64_t gzo_neighbours(int64_t N, const double* x, const double* y, const double* z,
                       const int64_t* id, const double* R, int32_t use_cells,
                       int64_t* offsets, int64_t* nbr, int64_t cap);

/* O10 pair set {j != i : r^2 < H_i^2 or r^2 < H_j^2}, ascending id. */
int64_t gzo_flux_pairs(int64_t N, const double* x, const double* y, const double* z,
                       const int64_t* id, const double* H, int32_t use_cells,
                       int64_t* offsets, int64_t* nbr, int64_t cap);

/* O4/O5: h-iteration and density for the particles with mask[i] != 0 (all
 * when mask is null).  f_out (optional) receives the final f value. */
int gzo_density(int64_t N, const double* x, const double* y, const double* z,
                const int64_t* id, const double* H_in, const uint8_t* mask,
                const gzo_params* p, double* H_out, double* n_out,
                int32_t* iters_out, double* f_out, gzo_counters* cnt);

/* O6-O9: gradients, B = E^-1, limiter.  grad/grad_raw are [15][N] laid out
 * as (field*3 + axis)*N + i with fields (rho, vx, vy, vz, P); B is [6][N]
 * (xx, xy, xz, yy, yz, zz); alpha is [5][N]; kappa is [N].  Optional outputs
 * may be null. */
int gzo_gradients(int64_t N, const double* x, const double* y, const double* z,
                  const int64_t* id, const double* m, const double* H, const double* n,
                  const double* vx, const double* vy, const double* vz, const double* u,
                  const uint8_t* mask, const gzo_params* p, double* grad, double* B,
                  double* grad_raw, double* alpha, double* kappa, gzo_counters* cnt);

/* O13: per-particle signal-speed timestep and dt = cfl * min_i dt_i. */
int gzo_timestep(int64_t N, const double* x, const double* y, const double* z,
                 const int64_t* id, const double* m, const double* H, const double* n,
                 const double* vx, const double* vy, const double* vz, const double* u,
                 const uint8_t* mask, const gzo_params* p, double* dt_i, double* dt_min);

/* O10-O12: fluxes summed into dp/dt [3][N], dE/dt [N] and (MFV; may be
 * NULL) dm/dt [N]. */
int gzo_fluxes(int64_t N, const double* x, const double* y, const double* z,
               const int64_t* id, const double* m, const double* H, const double* n,
               const double* vx, const double* vy, const double* vz, const double* u,
               const double* grad, const double* B, double dt, const uint8_t* mask,
               const gzo_params* p, double* dpdt, double* dEdt, double* dmdt,
               gzo_counters* cnt);

/* O14: kick, trapezoid drift, periodic wrap, u floor; with dmdt (MFV) the
 * masses are advanced too (m is then written). */
int gzo_update(int64_t N, double* x, double* y, double* z, double* vx, double* vy,
               double* vz, double* m, double* u, const double* dpdt, const double* dEdt,
               const double* dmdt, double dt, const gzo_params* p, gzo_counters* cnt);

/* Whole step O4..O14.  State arrays are updated in place (H becomes the
 * converged support radius used in this step; m changes under MFV).
 * *dt_inout <= 0 requests the CFL step; the step used is written back.
 * n_out, dpdt, dEdt, dmdt optional. */
int gzo_step(int64_t N, double* x, double* y, double* z, double* vx, double* vy,
             double* vz, double* m, double* u, double* H, const int64_t* id,
             const gzo_params* p, double* dt_inout, double* n_out, double* dpdt,
             double* dEdt, double* dmdt, gzo_counters* cnt);

/* Hierarchical timesteps (reading HT; MFV too): one sync interval of 2^K
 * substeps in place on the state; *dt_inout > 0 fixes the interval D, else
 * the CFL rule sets it; the interval used is written back.  bin_out ([N],
 * optional) receives every particle's final bin, active_out (optional) the
 * number of active particle-substeps.  K = 0 is gzo_step.  Returns -1 for
 * K outside [0, 20] or N < 1. */
int gzo_step_hier(int64_t N, double* x, double* y, double* z, double* vx, double* vy,
                  double* vz, double* m, double* u, double* H, const int64_t* id,
                  const gzo_params* p, int32_t K, double* dt_inout, int32_t* bin_out,
                  int64_t* active_out, gzo_counters* cnt);

/* Pair exchange of one hierarchical substep: for every particle, the sum over
 * its flux pairs with an active partner (or itself active) of
 * rate * 2^(bin_i - max(bin_i, bin_j)), faces evaluated over
 * D/2^max(bin_i, bin_j) (accm, optional: the mass rates of MFV);
 * touched[i] = 1 when i is active or has such a pair. */
int gzo_exchange(int64_t N, const double* x, const double* y, const double* z,
                 const int64_t* id, const double* m, const double* H, const double* n,
                 const double* vx, const double* vy, const double* vz, const double* u,
                 const double* grad, const double* B, const int32_t* bin, const uint8_t* active,
                 double D, const gzo_params* p, double* accp, double* accE, double* accm,
                 uint8_t* touched, gzo_counters* cnt);

/* One face evaluation in canonical (L, R) order for pins: inputs are the
 * two particles' positions, H, n, primitives (rho, vx, vy, vz, P), limited
 * gradients [15] and B [6].  Outputs the face area vector A[3], P*, S*,
 * the face-frame velocity vf[3], and the L-side rate contributions
 * dp[3], dE and dm (zero under MFM; R receives the negatives).  face (may be
 * NULL) receives the face states (rho, vx, vy, vz, P) of both sides at two
 * points of O11: [0,5) L and [5,10) R after the reconstruction and the
 * Hancock half step, before the clamp; [10,15) L and [15,20) R as handed to
 * the Riemann solver.  Returns 0 if |A| = 0 (face then untouched). */
int gzo_pair(const double* xL, double HL, double nL, const double* WL, const double* gL,
             const double* BL, const double* xR, double HR, double nR, const double* WR,
             const double* gR, const double* BR, double dt, const gzo_params* p,
             double* A, double* pstar, double* sstar, double* vf, double* dp, double* dE,
             double* dm, int* flags, double* face);

/* MFV face flux (HLLC, Davis speeds) for face states FL, FR (rho, v[3], P,
 * lab frame) through a face moving with vf, unit normal nh from L to R:
 * lab-frame mass, momentum [3] and energy flux densities. */
void gzo_hllc_flux(const double* FL, const double* FR, const double* vf, const double* nh,
                   double gamma, double* Fm, double* Fp, double* FE);

/* O12 HLLC (Davis wave speeds) on 1-D states along the face normal. */
void gzo_hllc(double rhoL, double uL, double PL, double rhoR, double uR, double PR,
              double gamma, double* sstar, double* pstar);

/* Exact Riemann solver (ideal gas): star-region pressure and velocity, and
 * sampled state (rho, u, P) at similarity coordinate xi = x/t. */
int gzo_riemann_star(double rhoL, double uL, double PL, double rhoR, double uR, double PR,
                     double gamma, double* pstar, double* ustar);
void gzo_riemann_sample(double rhoL, double uL, double PL, double rhoR, double uR, double PR,
                        double gamma, double pstar, double ustar, double xi,
                        double* rho, double* u, double* P);

int gzo_num_threads(void);
void gzo_set_threads(int n);

#endif
