/*
 * FP64 CPU oracle for the MFM hydrodynamics step.  TEST INFRASTRUCTURE ONLY:
 * tests, the smoke check and the benchmark's CPU-baseline leg are the only
 * users.  See gz_oracle.h for the reading labels O1..O14 cited below.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no -ffast-math).
 */
#include "gz_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GZO_PI 3.14159265358979323846

/* ---------------------------------------------------------------- O2 ---- */
/* Cubic spline with compact support H (zero for r >= H), q = r / H:
 *   w(q) = 1 - 6 q^2 + 6 q^3        0 <= q <= 1/2
 *        = 2 (1 - q)^3              1/2 < q < 1
 *        = 0                        q >= 1
 *   W(r, H) = 8 / (pi H^3) * w(r / H),   normalised so that its volume
 *   integral is 1. */
double gzo_kernel_w(double q) {
    if (q <= 0.5) return 1.0 - 6.0 * q * q + 6.0 * q * q * q;
    if (q < 1.0) {
        double t = 1.0 - q;
        return 2.0 * t * t * t;
    }
    return 0.0;
}

double gzo_kernel_dw(double q) {
    if (q <= 0.5) return -12.0 * q + 18.0 * q * q;
    if (q < 1.0) {
        double t = 1.0 - q;
        return -6.0 * t * t;
    }
    return 0.0;
}

double gzo_W(double r, double H) {
    return 8.0 / (GZO_PI * H * H * H) * gzo_kernel_w(r / H);
}

/* dW/dH at fixed r: -(8 / (pi H^4)) (3 w + q w'). */
double gzo_dWdH(double r, double H) {
    double q = r / H;
    return -(8.0 / (GZO_PI * H * H * H * H)) * (3.0 * gzo_kernel_w(q) + q * gzo_kernel_dw(q));
}

/* ---------------------------------------------------------------- O1 ---- */
/* Periodic unit box: d = x_j - x_i per component, then d >= 1/2 -> d - 1 and
 * d < -1/2 -> d + 1 (so d = 1/2 maps to -1/2).  r^2 = (dx dx + dy dy) + dz dz. */
double gzo_min_image(double d) {
    if (d >= 0.5) return d - 1.0;
    if (d < -0.5) return d + 1.0;
    return d;
}

static inline double sep(const double* x, const double* y, const double* z, int64_t i,
                         int64_t j, double d[3]) {
    d[0] = gzo_min_image(x[j] - x[i]);
    d[1] = gzo_min_image(y[j] - y[i]);
    d[2] = gzo_min_image(z[j] - z[i]);
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

/* ------------------------------------------------ neighbour candidates --- */
/* Two interchangeable finders return, for particle i and radius R, every
 * j != i with r_ij^2 < R^2 (strict), in ascending original id.  The brute
 * force one walks all particles in id order; the cell list gathers from the
 * cells overlapping the cube [x - R, x + R] widened by one cell each way and
 * sorts by id.  Both apply the same exact test, so their lists are equal. */
typedef struct {
    int64_t N;
    const double *x, *y, *z;
    const int64_t* id;
    int64_t* order; /* particle indices in ascending id */
    int use_cells;
    int nc;
    int64_t* cstart; /* nc^3 + 1 */
    int64_t* cidx;   /* N, grouped by cell */
} finder_t;

typedef struct {
    int64_t id, idx;
} idpair_t;

typedef struct {
    idpair_t* buf;
    int64_t n, cap;
    int64_t* out;
    int64_t out_cap;
} scratch_t;

static int cmp_id(const void* a, const void* b) {
    int64_t ia = ((const idpair_t*)a)->id, ib = ((const idpair_t*)b)->id;
    return (ia > ib) - (ia < ib);
}

static const int64_t* g_sort_id; /* only used single-threaded in finder_init */
static int cmp_by_gid(const void* a, const void* b) {
    int64_t ia = g_sort_id[*(const int64_t*)a], ib = g_sort_id[*(const int64_t*)b];
    return (ia > ib) - (ia < ib);
}

static int cell_of(double v, int nc) {
    if (!(v == v)) return 0;
    double s = floor(v * (double)nc);
    if (s < 0.0) return 0;
    if (s > (double)(nc - 1)) return nc - 1;
    return (int)s;
}

static void finder_init(finder_t* f, int64_t N, const double* x, const double* y,
                        const double* z, const int64_t* id, int use_cells, double cell_len) {
    memset(f, 0, sizeof(*f));
    f->N = N;
    f->x = x;
    f->y = y;
    f->z = z;
    f->id = id;
    f->use_cells = use_cells;
    f->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) f->order[i] = i;
    g_sort_id = id;
    qsort(f->order, (size_t)N, sizeof(int64_t), cmp_by_gid);
    if (!use_cells) return;
    int nc = 1;
    if (cell_len > 0.0 && cell_len < 1.0) {
        double c = floor(1.0 / cell_len);
        nc = c < 1.0 ? 1 : (c > 256.0 ? 256 : (int)c);
    }
    f->nc = nc;
    int64_t ncell = (int64_t)nc * nc * nc;
    f->cstart = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    f->cidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) {
        int cx = cell_of(x[i], nc), cy = cell_of(y[i], nc), cz = cell_of(z[i], nc);
        cell[i] = ((int64_t)cz * nc + cy) * nc + cx;
        f->cstart[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) f->cstart[c + 1] += f->cstart[c];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    memcpy(fill, f->cstart, sizeof(int64_t) * (size_t)ncell);
    for (int64_t i = 0; i < N; ++i) f->cidx[fill[cell[i]]++] = i;
    free(fill);
    free(cell);
}

static void finder_free(finder_t* f) {
    free(f->order);
    free(f->cstart);
    free(f->cidx);
}

static void scratch_push(scratch_t* s, int64_t id, int64_t idx) {
    if (s->n == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 256;
        s->buf = (idpair_t*)realloc(s->buf, sizeof(idpair_t) * (size_t)s->cap);
    }
    s->buf[s->n].id = id;
    s->buf[s->n].idx = idx;
    s->n++;
}

static void scratch_free(scratch_t* s) {
    free(s->buf);
    free(s->out);
}

/* Returns the list length; *list points to indices in ascending id. */
static int64_t gather(const finder_t* f, scratch_t* s, int64_t i, double R, const int64_t** list) {
    const double R2 = R * R;
    double d[3];
    s->n = 0;
    if (!f->use_cells || f->nc < 3) {
        for (int64_t k = 0; k < f->N; ++k) {
            int64_t j = f->order[k];
            if (j == i) continue;
            if (sep(f->x, f->y, f->z, i, j, d) < R2) scratch_push(s, f->id[j], j);
        }
    } else {
        const int nc = f->nc;
        int lo[3], hi[3];
        const double pos[3] = {f->x[i], f->y[i], f->z[i]};
        for (int a = 0; a < 3; ++a) {
            lo[a] = (int)floor((pos[a] - R) * nc) - 1;
            hi[a] = (int)floor((pos[a] + R) * nc) + 1;
            if (hi[a] - lo[a] + 1 >= nc) {
                lo[a] = 0;
                hi[a] = nc - 1;
            }
        }
        for (int cz = lo[2]; cz <= hi[2]; ++cz) {
            int wz = ((cz % nc) + nc) % nc;
            for (int cy = lo[1]; cy <= hi[1]; ++cy) {
                int wy = ((cy % nc) + nc) % nc;
                for (int cx = lo[0]; cx <= hi[0]; ++cx) {
                    int wx = ((cx % nc) + nc) % nc;
                    int64_t c = ((int64_t)wz * nc + wy) * nc + wx;
                    for (int64_t k = f->cstart[c]; k < f->cstart[c + 1]; ++k) {
                        int64_t j = f->cidx[k];
                        if (j == i) continue;
                        if (sep(f->x, f->y, f->z, i, j, d) < R2) scratch_push(s, f->id[j], j);
                    }
                }
            }
        }
        qsort(s->buf, (size_t)s->n, sizeof(idpair_t), cmp_id);
    }
    if (s->out_cap < s->n) {
        s->out_cap = s->n + 64;
        s->out = (int64_t*)realloc(s->out, sizeof(int64_t) * (size_t)s->out_cap);
    }
    for (int64_t k = 0; k < s->n; ++k) s->out[k] = s->buf[k].idx;
    *list = s->out;
    return s->n;
}

static double max_of(const double* a, int64_t N) {
    double m = 0.0;
    for (int64_t i = 0; i < N; ++i)
        if (a[i] > m) m = a[i];
    return m;
}

static double median_cell_len(const double* H, int64_t N) {
    /* any cell length gives the same lists; pick about half the largest H */
    double m = max_of(H, N);
    return 0.5 * m;
}

/* ---------------------------------------------------------------- O3 ---- */
int64_t gzo_neighbours(int64_t N, const double* x, const double* y, const double* z,
                       const int64_t* id, const double* R, int32_t use_cells,
                       int64_t* offsets, int64_t* nbr, int64_t cap) {
    finder_t f;
    finder_init(&f, N, x, y, z, id, use_cells, median_cell_len(R, N));
    int64_t* cnt = (int64_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(int64_t));
#pragma omp parallel
    {
        scratch_t s = {0};
        const int64_t* list;
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < N; ++i) cnt[i] = gather(&f, &s, i, R[i], &list);
        scratch_free(&s);
    }
    int64_t total = 0;
    offsets[0] = 0;
    for (int64_t i = 0; i < N; ++i) {
        total += cnt[i];
        offsets[i + 1] = total;
    }
    if (nbr && total <= cap) {
#pragma omp parallel
        {
            scratch_t s = {0};
            const int64_t* list;
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = 0; i < N; ++i) {
                int64_t n = gather(&f, &s, i, R[i], &list);
                memcpy(nbr + offsets[i], list, sizeof(int64_t) * (size_t)n);
            }
            scratch_free(&s);
        }
    }
    free(cnt);
    finder_free(&f);
    return (nbr && total > cap) ? -total : total;
}

/* ---------------------------------------------------------------- O10 --- */
int64_t gzo_flux_pairs(int64_t N, const double* x, const double* y, const double* z,
                       const int64_t* id, const double* H, int32_t use_cells,
                       int64_t* offsets, int64_t* nbr, int64_t cap) {
    finder_t f;
    finder_init(&f, N, x, y, z, id, use_cells, median_cell_len(H, N));
    const double Hmax = max_of(H, N);
    int64_t* cnt = (int64_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(int64_t));
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            int64_t total = 0;
            offsets[0] = 0;
            for (int64_t i = 0; i < N; ++i) {
                total += cnt[i];
                offsets[i + 1] = total;
            }
            if (!nbr || total > cap) break;
        }
#pragma omp parallel
        {
            scratch_t s = {0};
            const int64_t* list;
            double d[3];
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = 0; i < N; ++i) {
                int64_t n = gather(&f, &s, i, Hmax > H[i] ? Hmax : H[i], &list);
                int64_t c = 0;
                for (int64_t k = 0; k < n; ++k) {
                    int64_t j = list[k];
                    double r2 = sep(x, y, z, i, j, d);
                    if (r2 < H[i] * H[i] || r2 < H[j] * H[j]) {
                        if (pass == 1) nbr[offsets[i] + c] = j;
                        c++;
                    }
                }
                if (pass == 0) cnt[i] = c;
            }
            scratch_free(&s);
        }
    }
    int64_t total = offsets[N];
    free(cnt);
    finder_free(&f);
    return (nbr && total > cap) ? -total : total;
}

/* ---------------------------------------------------------- O4 / O5 ----- */
/* f(H) = (4 pi / 3) H^3 n(H) - N_ngb with n(H) = W(0, H) + sum_{j in N_i(H)}
 * W(r_ij, H), summed self first then neighbours in ascending id.
 * f'(H) = (4 pi / 3)(8 / pi) sum_j (-w'(q_j)) q_j / H  (analytic derivative
 * of each term H^3 W(r_j, H); the self term's derivative is zero).
 * Iteration: stop when |f| <= tol N_ngb; bracket lo (f < 0) / hi (f > 0);
 * Newton step H - f / f'; when f' <= 0 or the step leaves the open interval
 * (lo, hi) -- where an unset side is H/2 below or 2H above -- take (lo+hi)/2
 * if both sides are set, else 2H (f < 0) or H/2 (f > 0).  A step reaching
 * h_lim is replaced by (H + h_lim)/2.  The count is the number of f
 * evaluations, capped at max_iter. */
static void density_one(const finder_t* fd, scratch_t* s, int64_t i, double H0,
                        const gzo_params* p, double* Hout, double* nout, int32_t* itout,
                        double* fout, int* conv) {
    double H = H0, lo = 0.0, hi = 0.0;
    int has_lo = 0, has_hi = 0;
    double n = 0.0, f = 0.0;
    int it;
    *conv = 0;
    for (it = 1; it <= p->max_iter; ++it) {
        const int64_t* list;
        int64_t cnt = gather(fd, s, i, H, &list);
        double d[3];
        n = gzo_W(0.0, H);
        double S = 0.0;
        for (int64_t k = 0; k < cnt; ++k) {
            int64_t j = list[k];
            double r2 = sep(fd->x, fd->y, fd->z, i, j, d);
            if (r2 < H * H) {
                double r = sqrt(r2);
                double q = r / H;
                n += gzo_W(r, H);
                S += -gzo_kernel_dw(q) * q / H;
            }
        }
        f = (4.0 * GZO_PI / 3.0) * H * H * H * n - p->ngb;
        double fp = (4.0 * GZO_PI / 3.0) * (8.0 / GZO_PI) * S;
        if (fabs(f) <= p->tol * p->ngb) {
            *conv = 1;
            break;
        }
        if (it == p->max_iter) break;
        if (f < 0.0) {
            lo = H;
            has_lo = 1;
        } else {
            hi = H;
            has_hi = 1;
        }
        double lo_eff = has_lo ? lo : 0.5 * H;
        double hi_eff = has_hi ? hi : 2.0 * H;
        double Hn = 0.0;
        int newton_ok = 0;
        if (fp > 0.0) {
            Hn = H - f / fp;
            newton_ok = (Hn > lo_eff) && (Hn < hi_eff);
        }
        if (!newton_ok) {
            if (has_lo && has_hi)
                Hn = 0.5 * (lo + hi);
            else
                Hn = (f < 0.0) ? 2.0 * H : 0.5 * H;
        }
        if (Hn >= p->h_lim) Hn = 0.5 * (H + p->h_lim);
        H = Hn;
    }
    if (it > p->max_iter) it = p->max_iter;
    *Hout = H;
    *nout = n;
    *itout = it;
    if (fout) *fout = f;
}

int gzo_density(int64_t N, const double* x, const double* y, const double* z,
                const int64_t* id, const double* H_in, const uint8_t* mask,
                const gzo_params* p, double* H_out, double* n_out, int32_t* iters_out,
                double* f_out, gzo_counters* cnt) {
    finder_t fd;
    finder_init(&fd, N, x, y, z, id, p->use_cells, median_cell_len(H_in, N));
    int64_t hconv = 0;
#pragma omp parallel reduction(+ : hconv)
    {
        scratch_t s = {0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < N; ++i) {
            if (mask && !mask[i]) continue;
            int conv;
            density_one(&fd, &s, i, H_in[i], p, &H_out[i], &n_out[i], &iters_out[i],
                        f_out ? &f_out[i] : NULL, &conv);
            if (!conv) hconv++;
        }
        scratch_free(&s);
    }
    finder_free(&fd);
    if (cnt) cnt->hconv += hconv;
    return hconv ? 1 : 0;
}

/* ------------------------------------------------------- O6 - O9 -------- */
/* Primitive state of particle j: rho = m n, v, P = (gamma - 1) rho u. */
static inline void prim(int64_t j, const double* m, const double* n, const double* vx,
                        const double* vy, const double* vz, const double* u, double gamma,
                        double W[5]) {
    W[0] = m[j] * n[j];
    W[1] = vx[j];
    W[2] = vy[j];
    W[3] = vz[j];
    W[4] = (gamma - 1.0) * W[0] * u[j];
}

int gzo_gradients(int64_t N, const double* x, const double* y, const double* z,
                  const int64_t* id, const double* m, const double* H, const double* n,
                  const double* vx, const double* vy, const double* vz, const double* u,
                  const uint8_t* mask, const gzo_params* p, double* grad, double* B,
                  double* grad_raw, double* alpha, double* kappa, gzo_counters* cnt) {
    finder_t fd;
    finder_init(&fd, N, x, y, z, id, p->use_cells, median_cell_len(H, N));
    int64_t nsing = 0, nbig = 0;
#pragma omp parallel reduction(+ : nsing, nbig)
    {
        scratch_t s = {0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < N; ++i) {
            if (mask && !mask[i]) continue;
            const int64_t* list;
            int64_t cntj = gather(&fd, &s, i, H[i], &list);
            double Wi[5], Wj[5], d[3];
            prim(i, m, n, vx, vy, vz, u, p->gamma, Wi);
            double E[6] = {0, 0, 0, 0, 0, 0};
            double S[5][3];
            double fmax[5], fmin[5];
            for (int a = 0; a < 5; ++a) {
                S[a][0] = S[a][1] = S[a][2] = 0.0;
                fmax[a] = fmin[a] = Wi[a];
            }
            const double Hi = H[i];
            /* O6/O7/O8: psi_j(x_i) = W(r_ij, H_i) / n_i over N_i. */
            for (int64_t k = 0; k < cntj; ++k) {
                int64_t j = list[k];
                double r2 = sep(x, y, z, i, j, d);
                if (!(r2 < Hi * Hi)) continue;
                double psi = gzo_W(sqrt(r2), Hi) / n[i];
                E[0] += psi * d[0] * d[0];
                E[1] += psi * d[0] * d[1];
                E[2] += psi * d[0] * d[2];
                E[3] += psi * d[1] * d[1];
                E[4] += psi * d[1] * d[2];
                E[5] += psi * d[2] * d[2];
                prim(j, m, n, vx, vy, vz, u, p->gamma, Wj);
                for (int a = 0; a < 5; ++a) {
                    double df = Wj[a] - Wi[a];
                    S[a][0] += df * d[0] * psi;
                    S[a][1] += df * d[1] * psi;
                    S[a][2] += df * d[2] * psi;
                    if (Wj[a] > fmax[a]) fmax[a] = Wj[a];
                    if (Wj[a] < fmin[a]) fmin[a] = Wj[a];
                }
            }
            /* O7: B = E^-1 by adjugate / determinant. */
            double a = E[0], b = E[1], c = E[2], dd = E[3], e = E[4], ff = E[5];
            double Cxx = dd * ff - e * e, Cxy = c * e - b * ff, Cxz = b * e - c * dd;
            double Cyy = a * ff - c * c, Cyz = b * c - a * e, Czz = a * dd - b * b;
            double det = a * Cxx + b * Cxy + c * Cxz;
            double Bm[6] = {Cxx / det, Cxy / det, Cxz / det, Cyy / det, Cyz / det, Czz / det};
            double nE = sqrt(a * a + dd * dd + ff * ff + 2.0 * (b * b + c * c + e * e));
            double nB = sqrt(Bm[0] * Bm[0] + Bm[3] * Bm[3] + Bm[5] * Bm[5] +
                             2.0 * (Bm[1] * Bm[1] + Bm[2] * Bm[2] + Bm[4] * Bm[4]));
            double kap = nE * nB / 3.0;
            int singular = !(det > 0.0) || !(kap <= 1e8);
            if (singular) {
                nsing++;
                for (int q = 0; q < 6; ++q) Bm[q] = 0.0;
                kap = INFINITY;
            } else if (kap > p->kappa_max) {
                nbig++;
            }
            if (kappa) kappa[i] = kap;
            /* O8: g = B S. */
            double g[5][3];
            for (int q = 0; q < 5; ++q) {
                g[q][0] = Bm[0] * S[q][0] + Bm[1] * S[q][1] + Bm[2] * S[q][2];
                g[q][1] = Bm[1] * S[q][0] + Bm[3] * S[q][1] + Bm[4] * S[q][2];
                g[q][2] = Bm[2] * S[q][0] + Bm[4] * S[q][1] + Bm[5] * S[q][2];
            }
            /* O9: alpha_f = min over j in N_i of alpha_ij, with
             * Delta = g . (s_ij d_ij), s_ij = H_i / (H_i + H_j). */
            double al[5] = {1.0, 1.0, 1.0, 1.0, 1.0};
            for (int64_t k = 0; k < cntj; ++k) {
                int64_t j = list[k];
                double r2 = sep(x, y, z, i, j, d);
                if (!(r2 < Hi * Hi)) continue;
                double sij = Hi / (Hi + H[j]);
                double sd[3] = {sij * d[0], sij * d[1], sij * d[2]};
                for (int q = 0; q < 5; ++q) {
                    double D = (g[q][0] * sd[0] + g[q][1] * sd[1]) + g[q][2] * sd[2];
                    double aij = 1.0;
                    if (D > 0.0) {
                        aij = p->beta * (fmax[q] - Wi[q]) / D;
                        if (aij > 1.0) aij = 1.0;
                    } else if (D < 0.0) {
                        aij = p->beta * (fmin[q] - Wi[q]) / D;
                        if (aij > 1.0) aij = 1.0;
                    }
                    if (aij < al[q]) al[q] = aij;
                }
            }
            for (int q = 0; q < 5; ++q)
                for (int ax = 0; ax < 3; ++ax) {
                    grad[(int64_t)(q * 3 + ax) * N + i] = al[q] * g[q][ax];
                    if (grad_raw) grad_raw[(int64_t)(q * 3 + ax) * N + i] = g[q][ax];
                }
            for (int q = 0; q < 6; ++q) B[(int64_t)q * N + i] = Bm[q];
            if (alpha)
                for (int q = 0; q < 5; ++q) alpha[(int64_t)q * N + i] = al[q];
        }
        scratch_free(&s);
    }
    finder_free(&fd);
    if (cnt) {
        cnt->singular += nsing;
        cnt->kappa_big += nbig;
    }
    return nsing ? 1 : 0;
}

/* ---------------------------------------------------------------- O13 --- */
/* v_sig,ij = c_i + c_j - min(0, (v_j - v_i) . d / r) over flux pairs;
 * dt_i = 2 V_i^(1/3) / max_j v_sig,ij (infinite when i has no pairs);
 * dt = cfl * min_i dt_i. */
int gzo_timestep(int64_t N, const double* x, const double* y, const double* z,
                 const int64_t* id, const double* m, const double* H, const double* n,
                 const double* vx, const double* vy, const double* vz, const double* u,
                 const uint8_t* mask, const gzo_params* p, double* dt_i, double* dt_min) {
    finder_t fd;
    finder_init(&fd, N, x, y, z, id, p->use_cells, median_cell_len(H, N));
    const double Hmax = max_of(H, N);
    double best = INFINITY;
#pragma omp parallel reduction(min : best)
    {
        scratch_t s = {0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < N; ++i) {
            if (mask && !mask[i]) continue;
            const int64_t* list;
            int64_t cntj = gather(&fd, &s, i, Hmax > H[i] ? Hmax : H[i], &list);
            double Wi[5], Wj[5], d[3];
            prim(i, m, n, vx, vy, vz, u, p->gamma, Wi);
            double ci = sqrt(p->gamma * Wi[4] / Wi[0]);
            double vmax = 0.0;
            int any = 0;
            for (int64_t k = 0; k < cntj; ++k) {
                int64_t j = list[k];
                double r2 = sep(x, y, z, i, j, d);
                if (!(r2 < H[i] * H[i] || r2 < H[j] * H[j])) continue;
                prim(j, m, n, vx, vy, vz, u, p->gamma, Wj);
                double cj = sqrt(p->gamma * Wj[4] / Wj[0]);
                double r = sqrt(r2);
                double vd = ((Wj[1] - Wi[1]) * d[0] + (Wj[2] - Wi[2]) * d[1]) +
                            (Wj[3] - Wi[3]) * d[2];
                double w = vd / r;
                double vs = ci + cj - (w < 0.0 ? w : 0.0);
                if (!any || vs > vmax) vmax = vs;
                any = 1;
            }
            double dti = (any && vmax > 0.0) ? 2.0 * cbrt(1.0 / n[i]) / vmax : INFINITY;
            if (dt_i) dt_i[i] = dti;
            if (dti < best) best = dti;
        }
        scratch_free(&s);
    }
    finder_free(&fd);
    *dt_min = p->cfl * best;
    return 0;
}

/* ------------------------------------------------------ O10 - O12 ------- */
/* HLLC with Davis wave speeds S_L = min(u_L - c_L, u_R - c_R),
 * S_R = max(u_L + c_L, u_R + c_R); contact speed
 *   S* = [P_R - P_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R)]
 *        / [rho_L (S_L - u_L) - rho_R (S_R - u_R)]
 * and star pressure P* = P_L + rho_L (S_L - u_L)(S* - u_L). */
void gzo_hllc(double rhoL, double uL, double PL, double rhoR, double uR, double PR,
              double gamma, double* sstar, double* pstar) {
    double cL = sqrt(gamma * PL / rhoL), cR = sqrt(gamma * PR / rhoR);
    double a = uL - cL, b = uR - cR;
    double SL = a < b ? a : b;
    double a2 = uL + cL, b2 = uR + cR;
    double SR = a2 > b2 ? a2 : b2;
    double num = PR - PL + rhoL * uL * (SL - uL) - rhoR * uR * (SR - uR);
    double den = rhoL * (SL - uL) - rhoR * (SR - uR);
    double ss = num / den;
    *sstar = ss;
    *pstar = PL + rhoL * (SL - uL) * (ss - uL);
}

/* MFV: the face moves with vf; in its frame (w = v - vf, u = w . n) the
 * conserved state is U = (rho, rho w, E) with E = P/(g-1) + rho |w|^2 / 2 and
 * the flux along n is F(U) = (rho u, rho u w + P n, u (E + P)).  HLLC takes
 * F_L, F*_L = F_L + S_L (U*_L - U_L), F*_R, F_R on the four sides of the waves
 * S_L, S*, S_R (Davis speeds, S* as in gzo_hllc), with the star states
 * U*_K = rho_K (S_K - u_K)/(S_K - S*) (1, w_K + (S* - u_K) n,
 * E_K/rho_K + (S* - u_K)(S* + P_K/(rho_K (S_K - u_K)))); the face flux is the
 * one at xi = 0.  Back to the lab frame: mass F_rho, momentum F_w + vf F_rho,
 * energy F_E + vf . F_w + |vf|^2 F_rho / 2. */
void gzo_hllc_flux(const double* FL, const double* FR, const double* vf, const double* nh,
                   double gamma, double* Fm, double* Fp, double* FE) {
    const double* S[2] = {FL, FR};
    double rho[2], w[2][3], un[2], P[2], E[2], c[2];
    for (int k = 0; k < 2; ++k) {
        rho[k] = S[k][0];
        P[k] = S[k][4];
        for (int a = 0; a < 3; ++a) w[k][a] = S[k][1 + a] - vf[a];
        un[k] = (w[k][0] * nh[0] + w[k][1] * nh[1]) + w[k][2] * nh[2];
        double w2 = (w[k][0] * w[k][0] + w[k][1] * w[k][1]) + w[k][2] * w[k][2];
        E[k] = P[k] / (gamma - 1.0) + 0.5 * rho[k] * w2;
        c[k] = sqrt(gamma * P[k] / rho[k]);
    }
    double a = un[0] - c[0], b = un[1] - c[1];
    double SL = a < b ? a : b;
    double a2 = un[0] + c[0], b2 = un[1] + c[1];
    double SR = a2 > b2 ? a2 : b2;
    double num = P[1] - P[0] + rho[0] * un[0] * (SL - un[0]) - rho[1] * un[1] * (SR - un[1]);
    double den = rho[0] * (SL - un[0]) - rho[1] * (SR - un[1]);
    double ss = num / den;
    int k;        /* side whose physical flux is used */
    int star;     /* 1: add S_K (U*_K - U_K) */
    if (SL >= 0.0) {
        k = 0;
        star = 0;
    } else if (ss >= 0.0) {
        k = 0;
        star = 1;
    } else if (SR > 0.0) {
        k = 1;
        star = 1;
    } else {
        k = 1;
        star = 0;
    }
    double fr = rho[k] * un[k];
    double fw[3], fe = un[k] * (E[k] + P[k]);
    for (int q = 0; q < 3; ++q) fw[q] = rho[k] * un[k] * w[k][q] + P[k] * nh[q];
    if (star) {
        double SK = k == 0 ? SL : SR;
        double f = rho[k] * (SK - un[k]) / (SK - ss);
        double Us[5], U[5];
        U[0] = rho[k];
        Us[0] = f;
        for (int q = 0; q < 3; ++q) {
            U[1 + q] = rho[k] * w[k][q];
            Us[1 + q] = f * (w[k][q] + (ss - un[k]) * nh[q]);
        }
        U[4] = E[k];
        Us[4] = f * (E[k] / rho[k] + (ss - un[k]) * (ss + P[k] / (rho[k] * (SK - un[k]))));
        fr += SK * (Us[0] - U[0]);
        for (int q = 0; q < 3; ++q) fw[q] += SK * (Us[1 + q] - U[1 + q]);
        fe += SK * (Us[4] - U[4]);
    }
    double vfw = (vf[0] * fw[0] + vf[1] * fw[1]) + vf[2] * fw[2];
    double vf2 = (vf[0] * vf[0] + vf[1] * vf[1]) + vf[2] * vf[2];
    *Fm = fr;
    for (int q = 0; q < 3; ++q) Fp[q] = fw[q] + vf[q] * fr;
    *FE = fe + vfw + 0.5 * vf2 * fr;
}

static inline double clampd(double v, double lo, double hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

/* One face in canonical order (L = lower id).  O10: d = x_R - x_L,
 * A = V_L psi_R(x_L) B_L d + V_R psi_L(x_R) B_R d with V = 1/n and
 * psi_b(x_a) = W(r, H_a) / n_a (zero outside H_a).  O11: s = H_L/(H_L+H_R),
 * v_f = v_L + s (v_R - v_L); W_L = W_L + g_L . (s d), W_R = W_R + g_R . (s_R (-d));
 * Hancock: + (dt/2) (-rho div v, -grad P / rho, -gamma P div v) with the
 * particle's own limited gradients (the face point seen from R is
 * x_R + s_R (x_L - x_R) with s_R = H_R / (H_L + H_R), the same point);
 * clamp each field to
 * [min(f_L, f_R), max(f_L, f_R)]; if rho or P <= 0 on a side use the
 * particle states.  O12: HLLC along n = A/|A| in the face frame; MFM rates
 * to L: dp = -P* A, dE = -P* (S* + v_f . n) |A|.  With riemann = 1 (every
 * face) or 2 (faces where HLLC's P* < 0) the exact solver's star pressure and
 * contact speed replace HLLC's P* and S*.  O15 (scheme = 1): the MFV fluxes. */
int gzo_pair(const double* xL, double HL, double nL, const double* WL, const double* gL,
             const double* BL, const double* xR, double HR, double nR, const double* WR,
             const double* gR, const double* BR, double dt, const gzo_params* p,
             double* A, double* pstar, double* sstar, double* vf, double* dp, double* dE,
             double* dm, int* flags, double* face) {
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = gzo_min_image(xR[a] - xL[a]);
    double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    double r = sqrt(r2);
    double psiRL = r2 < HL * HL ? gzo_W(r, HL) / nL : 0.0; /* psi_R(x_L) */
    double psiLR = r2 < HR * HR ? gzo_W(r, HR) / nR : 0.0; /* psi_L(x_R) */
    double VL = 1.0 / nL, VR = 1.0 / nR;
    double BLd[3] = {BL[0] * d[0] + BL[1] * d[1] + BL[2] * d[2],
                     BL[1] * d[0] + BL[3] * d[1] + BL[4] * d[2],
                     BL[2] * d[0] + BL[4] * d[1] + BL[5] * d[2]};
    double BRd[3] = {BR[0] * d[0] + BR[1] * d[1] + BR[2] * d[2],
                     BR[1] * d[0] + BR[3] * d[1] + BR[4] * d[2],
                     BR[2] * d[0] + BR[4] * d[1] + BR[5] * d[2]};
    for (int a = 0; a < 3; ++a) A[a] = VL * psiRL * BLd[a] + VR * psiLR * BRd[a];
    *flags = 0;
    double Amag = sqrt((A[0] * A[0] + A[1] * A[1]) + A[2] * A[2]);
    dp[0] = dp[1] = dp[2] = 0.0;
    *dE = 0.0;
    *dm = 0.0;
    *pstar = 0.0;
    *sstar = 0.0;
    double s = HL / (HL + HR);
    for (int a = 0; a < 3; ++a) vf[a] = WL[1 + a] + s * (WR[1 + a] - WL[1 + a]);
    if (Amag == 0.0) return 0;
    double nh[3] = {A[0] / Amag, A[1] / Amag, A[2] / Amag};
    /* face point x_f = x_L + s d = x_R + s_R (x_L - x_R), s_R = H_R / (H_L + H_R) */
    double sR = HR / (HL + HR);
    double sdL[3] = {s * d[0], s * d[1], s * d[2]};
    double sdR[3] = {sR * -d[0], sR * -d[1], sR * -d[2]};
    double FL[5], FR[5];
    for (int q = 0; q < 5; ++q) {
        FL[q] = WL[q] + ((gL[q * 3 + 0] * sdL[0] + gL[q * 3 + 1] * sdL[1]) + gL[q * 3 + 2] * sdL[2]);
        FR[q] = WR[q] + ((gR[q * 3 + 0] * sdR[0] + gR[q * 3 + 1] * sdR[1]) + gR[q * 3 + 2] * sdR[2]);
    }
    if (p->hancock) {
        double h = 0.5 * dt;
        double divL = (gL[1 * 3 + 0] + gL[2 * 3 + 1]) + gL[3 * 3 + 2];
        double divR = (gR[1 * 3 + 0] + gR[2 * 3 + 1]) + gR[3 * 3 + 2];
        FL[0] += h * (-WL[0] * divL);
        FR[0] += h * (-WR[0] * divR);
        for (int a = 0; a < 3; ++a) {
            FL[1 + a] += h * (-gL[4 * 3 + a] / WL[0]);
            FR[1 + a] += h * (-gR[4 * 3 + a] / WR[0]);
        }
        FL[4] += h * (-p->gamma * WL[4] * divL);
        FR[4] += h * (-p->gamma * WR[4] * divR);
    }
    if (face)
        for (int q = 0; q < 5; ++q) {
            face[q] = FL[q];
            face[5 + q] = FR[q];
        }
    for (int q = 0; q < 5; ++q) {
        double lo = WL[q] < WR[q] ? WL[q] : WR[q];
        double hi = WL[q] < WR[q] ? WR[q] : WL[q];
        FL[q] = clampd(FL[q], lo, hi);
        FR[q] = clampd(FR[q], lo, hi);
    }
    if (!(FL[0] > 0.0) || !(FL[4] > 0.0) || !(FR[0] > 0.0) || !(FR[4] > 0.0)) {
        for (int q = 0; q < 5; ++q) {
            FL[q] = WL[q];
            FR[q] = WR[q];
        }
        *flags |= 1;
    }
    if (face)
        for (int q = 0; q < 5; ++q) {
            face[10 + q] = FL[q];
            face[15 + q] = FR[q];
        }
    double vfn = (vf[0] * nh[0] + vf[1] * nh[1]) + vf[2] * nh[2];
    double uL = ((FL[1] - vf[0]) * nh[0] + (FL[2] - vf[1]) * nh[1]) + (FL[3] - vf[2]) * nh[2];
    double uR = ((FR[1] - vf[0]) * nh[0] + (FR[2] - vf[1]) * nh[1]) + (FR[3] - vf[2]) * nh[2];
    double ss, ps;
    gzo_hllc(FL[0], uL, FL[4], FR[0], uR, FR[4], p->gamma, &ss, &ps);
    int neg = ps < 0.0;
    if (p->scheme == 0 && (p->riemann == 1 || (p->riemann == 2 && neg))) {
        /* exact star state of the face-frame Riemann problem: P* and the contact
         * speed u* take the places of HLLC's; a vacuum face carries P* = 0 */
        double pe, ue;
        if (gzo_riemann_star(FL[0], uL, FL[4], FR[0], uR, FR[4], p->gamma, &pe, &ue) == 0) {
            ps = pe;
            ss = ue;
            if (p->riemann == 1) neg = 0;
        } else {
            ps = 0.0;
            ss = 0.0;
            neg = 1;
        }
    }
    if (neg) *flags |= 2;
    if (ps < 0.0) ps = 0.0;
    *pstar = ps;
    *sstar = ss;
    if (p->scheme == 1) { /* MFV: full HLLC flux through the face moving with vf */
        double Fm, Fp[3], FE;
        gzo_hllc_flux(FL, FR, vf, nh, p->gamma, &Fm, Fp, &FE);
        *dm = -Fm * Amag;
        for (int a = 0; a < 3; ++a) dp[a] = -Fp[a] * Amag;
        *dE = -FE * Amag;
        return 1;
    }
    for (int a = 0; a < 3; ++a) dp[a] = -ps * A[a];
    *dE = -ps * (ss + vfn) * Amag;
    return 1;
}

static inline void load_side(int64_t j, const double* x, const double* y, const double* z,
                             const double* m, const double* n, const double* vx,
                             const double* vy, const double* vz, const double* u,
                             const double* grad, const double* B, int64_t N, double gamma,
                             double pos[3], double W[5], double g[15], double Bm[6]) {
    pos[0] = x[j];
    pos[1] = y[j];
    pos[2] = z[j];
    prim(j, m, n, vx, vy, vz, u, gamma, W);
    for (int q = 0; q < 15; ++q) g[q] = grad[(int64_t)q * N + j];
    for (int q = 0; q < 6; ++q) Bm[q] = B[(int64_t)q * N + j];
}

int gzo_fluxes(int64_t N, const double* x, const double* y, const double* z,
               const int64_t* id, const double* m, const double* H, const double* n,
               const double* vx, const double* vy, const double* vz, const double* u,
               const double* grad, const double* B, double dt, const uint8_t* mask,
               const gzo_params* p, double* dpdt, double* dEdt, double* dmdt,
               gzo_counters* cnt) {
    finder_t fd;
    finder_init(&fd, N, x, y, z, id, p->use_cells, median_cell_len(H, N));
    const double Hmax = max_of(H, N);
    int64_t nfall = 0, nneg = 0, npairs = 0;
#pragma omp parallel reduction(+ : nfall, nneg, npairs)
    {
        scratch_t s = {0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < N; ++i) {
            if (mask && !mask[i]) continue;
            const int64_t* list;
            int64_t cntj = gather(&fd, &s, i, Hmax > H[i] ? Hmax : H[i], &list);
            double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            double d[3];
            for (int64_t k = 0; k < cntj; ++k) {
                int64_t j = list[k];
                double r2 = sep(x, y, z, i, j, d);
                if (!(r2 < H[i] * H[i] || r2 < H[j] * H[j])) continue;
                npairs++;
                int64_t L = id[i] < id[j] ? i : j;
                int64_t R = id[i] < id[j] ? j : i;
                double pL[3], pR[3], WL[5], WR[5], gL[15], gR[15], BL[6], BR[6];
                load_side(L, x, y, z, m, n, vx, vy, vz, u, grad, B, N, p->gamma, pL, WL, gL, BL);
                load_side(R, x, y, z, m, n, vx, vy, vz, u, grad, B, N, p->gamma, pR, WR, gR, BR);
                double A[3], ps, ss, vf[3], dp[3], dE, dm;
                int fl;
                gzo_pair(pL, H[L], n[L], WL, gL, BL, pR, H[R], n[R], WR, gR, BR, dt, p, A, &ps,
                         &ss, vf, dp, &dE, &dm, &fl, NULL);
                if (fl & 1) nfall++;
                if (fl & 2) nneg++;
                double sg = (i == L) ? 1.0 : -1.0;
                acc[0] += sg * dp[0];
                acc[1] += sg * dp[1];
                acc[2] += sg * dp[2];
                acc[3] += sg * dE;
                acc[4] += sg * dm;
            }
            dpdt[i] = acc[0];
            dpdt[N + i] = acc[1];
            dpdt[2 * N + i] = acc[2];
            dEdt[i] = acc[3];
            if (dmdt) dmdt[i] = acc[4];
        }
        scratch_free(&s);
    }
    finder_free(&fd);
    if (cnt) {
        cnt->fallback += nfall;
        cnt->pstar_neg += nneg;
        cnt->pairs += npairs;
    }
    return 0;
}

/* ---------------------------------------------------------------- O14 --- */
/* p <- p + dt dp/dt, E <- E + dt dE/dt with p = m v and E = m (u + v^2/2);
 * v_new = p / m; x <- wrap(x + dt (v_old + v_new) / 2) where wrap adds 1
 * below 0 and then subtracts 1 at or above 1; u_new = E/m - |v_new|^2/2,
 * floored at u_floor_frac * (lower median of u at step start) when <= 0. */
static int cmp_dbl(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

static double wrap1(double v) {
    if (v < 0.0) v += 1.0;
    if (v >= 1.0) v -= 1.0;
    return v;
}

int gzo_update(int64_t N, double* x, double* y, double* z, double* vx, double* vy,
               double* vz, double* m, double* u, const double* dpdt, const double* dEdt,
               const double* dmdt, double dt, const gzo_params* p, gzo_counters* cnt) {
    /* with dmdt (MFV) m <- m + dt dm/dt and p, E are divided by the new m */
    double umed = 0.0;
    int need_floor = 0;
    for (int64_t i = 0; i < N && !need_floor; ++i) {
        double mn = dmdt ? m[i] + dt * dmdt[i] : m[i];
        double px = m[i] * vx[i] + dt * dpdt[i];
        double py = m[i] * vy[i] + dt * dpdt[N + i];
        double pz = m[i] * vz[i] + dt * dpdt[2 * N + i];
        double v2 = (vx[i] * vx[i] + vy[i] * vy[i]) + vz[i] * vz[i];
        double E = m[i] * (u[i] + 0.5 * v2) + dt * dEdt[i];
        double nx = px / mn, ny = py / mn, nz = pz / mn;
        double un = E / mn - 0.5 * ((nx * nx + ny * ny) + nz * nz);
        if (!(un > 0.0)) need_floor = 1;
    }
    if (need_floor && N > 0) {
        double* tmp = (double*)malloc(sizeof(double) * (size_t)N);
        memcpy(tmp, u, sizeof(double) * (size_t)N);
        qsort(tmp, (size_t)N, sizeof(double), cmp_dbl);
        umed = tmp[(N - 1) / 2];
        free(tmp);
    }
    int64_t nfl = 0, nbad = 0;
    for (int64_t i = 0; i < N; ++i) {
        double mn = dmdt ? m[i] + dt * dmdt[i] : m[i];
        double v2 = (vx[i] * vx[i] + vy[i] * vy[i]) + vz[i] * vz[i];
        double E = m[i] * (u[i] + 0.5 * v2) + dt * dEdt[i];
        double px = m[i] * vx[i] + dt * dpdt[i];
        double py = m[i] * vy[i] + dt * dpdt[N + i];
        double pz = m[i] * vz[i] + dt * dpdt[2 * N + i];
        double nx = px / mn, ny = py / mn, nz = pz / mn;
        x[i] = wrap1(x[i] + dt * (0.5 * (vx[i] + nx)));
        y[i] = wrap1(y[i] + dt * (0.5 * (vy[i] + ny)));
        z[i] = wrap1(z[i] + dt * (0.5 * (vz[i] + nz)));
        double un = E / mn - 0.5 * ((nx * nx + ny * ny) + nz * nz);
        if (!(un > 0.0)) {
            un = p->u_floor_frac * umed;
            nfl++;
        }
        if (!(mn > 0.0)) nbad++;
        vx[i] = nx;
        vy[i] = ny;
        vz[i] = nz;
        u[i] = un;
        if (dmdt) m[i] = mn;
    }
    if (cnt) {
        cnt->ufloor += nfl;
        cnt->nonfinite += nbad;
    }
    return 0;
}

/* ------------------------------------------------------------ step ------ */
int gzo_step(int64_t N, double* x, double* y, double* z, double* vx, double* vy,
             double* vz, double* m, double* u, double* H, const int64_t* id,
             const gzo_params* p, double* dt_inout, double* n_out, double* dpdt,
             double* dEdt, double* dmdt, gzo_counters* cnt) {
    size_t sz = sizeof(double) * (size_t)(N > 0 ? N : 1);
    double* Hn = (double*)malloc(sz);
    double* n = n_out ? n_out : (double*)malloc(sz);
    int32_t* it = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    double* grad = (double*)malloc(sz * 15);
    double* B = (double*)malloc(sz * 6);
    double* dp = dpdt ? dpdt : (double*)malloc(sz * 3);
    double* dE = dEdt ? dEdt : (double*)malloc(sz);
    double* dm = p->scheme == 1 ? (dmdt ? dmdt : (double*)malloc(sz)) : NULL;
    gzo_density(N, x, y, z, id, H, NULL, p, Hn, n, it, NULL, cnt);
    memcpy(H, Hn, sz);
    gzo_gradients(N, x, y, z, id, m, H, n, vx, vy, vz, u, NULL, p, grad, B, NULL, NULL, NULL,
                  cnt);
    double dt = *dt_inout;
    if (!(dt > 0.0)) gzo_timestep(N, x, y, z, id, m, H, n, vx, vy, vz, u, NULL, p, NULL, &dt);
    gzo_fluxes(N, x, y, z, id, m, H, n, vx, vy, vz, u, grad, B, dt, NULL, p, dp, dE, dm, cnt);
    gzo_update(N, x, y, z, vx, vy, vz, m, u, dp, dE, dm, dt, p, cnt);
    *dt_inout = dt;
    free(Hn);
    if (!n_out) free(n);
    free(it);
    free(grad);
    free(B);
    if (!dpdt) free(dp);
    if (!dEdt) free(dE);
    if (dm && !dmdt) free(dm);
    if (dmdt && p->scheme != 1) memset(dmdt, 0, sz);
    return 0;
}

/* ------------------------------------------- hierarchical timesteps ---- */
/* Reading HT (power-of-two timestep bins; the paper names hierarchical
 * adaptive timesteps and gives no formula).  One call advances the box over a
 * sync interval D split into 2^K substeps of D/2^K.  Particle i sits in bin
 * k_i in [0, K] with step dt_i = D/2^k_i; it is active at substep s when
 * s is a multiple of 2^(K - k_i), i.e. when a step of its own starts.
 * Bins: at s = 0 every particle is active and, with its O13 criterion
 * dtc_i = 2 V_i^(1/3)/max v_sig, takes the smallest k with D/2^k <= cfl dtc_i
 * (K at most); D is dt_fixed when given, else
 * min(cfl max_i dtc_i, 2^K cfl min_i dtc_i) (K = 0: the global CFL step).  At
 * later active times a particle may only move to a smaller step (any smaller
 * power of two starts there too); larger steps wait for the next interval.
 * Positions: the caller's x holds each particle's position at the start of
 * its current step (x_a, with velocity v_a then); at substep s every particle
 * is placed at x_a + tau (v_a + v)/2, tau = (s - s_a) D/2^K and v its current
 * velocity, and a step that ends moves x_a to x_a + dt_i (v_a + v)/2 (the
 * trapezoid drift of O14).  Substep s: O4/O5 for the active particles (the
 * others keep H and n of their last active time), O6-O9 and O13 for them
 * (the others keep their gradients and B), re-binning, then every flux pair
 * (O10) with at least one active particle exchanges the face fluxes of
 * O11/O12 over dt_ij = min(dt_i, dt_j) = D/2^max(k_i, k_j) (Hancock with
 * dt_ij/2): each particle accumulates rate * 2^(k_a - k_ij), and its momentum
 * and energy change by dt_a times that sum (exact power-of-two scaling, so
 * the pair's two shares are equal and opposite).  A particle's exchanges
 * happen whenever the smaller-step particle of a pair is active, so every
 * face is integrated over the whole interval exactly once.  u <= 0 after a
 * kick is floored as in O14 with the median of u at the substep start.  Under
 * MFV (O15) the mass share rides along: m += dt_a x (its sum of
 * dm * 2^(k_a - k_ij)), momentum and energy divided by the new mass.  K = 0
 * is gzo_step. */
static int32_t bin_for(double D, double cfl_dtc, int32_t K, int* clamped) {
    for (int32_t k = 0; k <= K; ++k)
        if (ldexp(D, -k) <= cfl_dtc) return k;
    *clamped = 1;
    return K;
}

int gzo_exchange(int64_t N, const double* x, const double* y, const double* z,
                 const int64_t* id, const double* m, const double* H, const double* n,
                 const double* vx, const double* vy, const double* vz, const double* u,
                 const double* grad, const double* B, const int32_t* bin, const uint8_t* active,
                 double D, const gzo_params* p, double* accp, double* accE, double* accm,
                 uint8_t* touched, gzo_counters* cnt) {
    finder_t fd;
    finder_init(&fd, N, x, y, z, id, p->use_cells, median_cell_len(H, N));
    const double Hmax = max_of(H, N);
    int64_t nfall = 0, nneg = 0, npairs = 0;
#pragma omp parallel reduction(+ : nfall, nneg, npairs)
    {
        scratch_t s = {0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < N; ++i) {
            const int64_t* list;
            int64_t cntj = gather(&fd, &s, i, Hmax > H[i] ? Hmax : H[i], &list);
            double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            double d[3];
            int any = 0;
            for (int64_t k = 0; k < cntj; ++k) {
                int64_t j = list[k];
                if (!active[i] && !active[j]) continue;
                double r2 = sep(x, y, z, i, j, d);
                if (!(r2 < H[i] * H[i] || r2 < H[j] * H[j])) continue;
                npairs++;
                any = 1;
                int64_t L = id[i] < id[j] ? i : j;
                int64_t R = id[i] < id[j] ? j : i;
                int32_t kij = bin[i] > bin[j] ? bin[i] : bin[j];
                double dtij = ldexp(D, -kij);
                double pL[3], pR[3], WL[5], WR[5], gL[15], gR[15], BL[6], BR[6];
                load_side(L, x, y, z, m, n, vx, vy, vz, u, grad, B, N, p->gamma, pL, WL, gL, BL);
                load_side(R, x, y, z, m, n, vx, vy, vz, u, grad, B, N, p->gamma, pR, WR, gR, BR);
                double A[3], ps, ss, vf[3], dp[3], dE, dm;
                int fl = 0;
                gzo_pair(pL, H[L], n[L], WL, gL, BL, pR, H[R], n[R], WR, gR, BR, dtij, p, A, &ps,
                         &ss, vf, dp, &dE, &dm, &fl, NULL);
                if (fl & 1) nfall++;
                if (fl & 2) nneg++;
                double sg = ((i == L) ? 1.0 : -1.0) * ldexp(1.0, bin[i] - kij);
                acc[0] += sg * dp[0];
                acc[1] += sg * dp[1];
                acc[2] += sg * dp[2];
                acc[3] += sg * dE;
                acc[4] += sg * dm;
            }
            accp[i] = acc[0];
            accp[N + i] = acc[1];
            accp[2 * N + i] = acc[2];
            accE[i] = acc[3];
            if (accm) accm[i] = acc[4];
            touched[i] = (uint8_t)(any || active[i]);
        }
        scratch_free(&s);
    }
    finder_free(&fd);
    if (cnt) {
        cnt->fallback += nfall;
        cnt->pstar_neg += nneg;
        cnt->pairs += npairs;
    }
    return 0;
}

static double median_u(const double* u, int64_t N) {
    double* tmp = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    memcpy(tmp, u, sizeof(double) * (size_t)N);
    qsort(tmp, (size_t)N, sizeof(double), cmp_dbl);
    double v = tmp[(N - 1) / 2];
    free(tmp);
    return v;
}

int gzo_step_hier(int64_t N, double* x, double* y, double* z, double* vx, double* vy,
                  double* vz, double* m, double* u, double* H, const int64_t* id,
                  const gzo_params* p, int32_t K, double* dt_inout, int32_t* bin_out,
                  int64_t* active_out, gzo_counters* cnt) {
    if (K < 0 || K > 20 || N < 1) return -1;
    const int mfv = p->scheme == 1;
    const size_t sz = sizeof(double) * (size_t)N;
    double* xp = (double*)malloc(sz * 3);
    double *yp = xp + N, *zp = xp + 2 * N;
    double* va = (double*)malloc(sz * 3);
    double* n = (double*)calloc((size_t)N, sizeof(double));
    double* Hn = (double*)malloc(sz);
    double* nn = (double*)malloc(sz);
    double* grad = (double*)calloc((size_t)N * 15, sizeof(double));
    double* B = (double*)calloc((size_t)N * 6, sizeof(double));
    double* dtc = (double*)malloc(sz);
    double* accp = (double*)malloc(sz * 3);
    double* accE = (double*)malloc(sz);
    double* accm = mfv ? (double*)malloc(sz) : NULL;
    int32_t* it = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    int32_t* bin = (int32_t*)calloc((size_t)N, sizeof(int32_t));
    int32_t* sa = (int32_t*)calloc((size_t)N, sizeof(int32_t));
    uint8_t* act = (uint8_t*)malloc((size_t)N);
    uint8_t* tch = (uint8_t*)malloc((size_t)N);
    for (int64_t i = 0; i < N; ++i) {
        va[i] = vx[i];
        va[N + i] = vy[i];
        va[2 * N + i] = vz[i];
    }
    double D = *dt_inout;
    const int32_t S = 1 << K;
    int64_t nact = 0, nfl = 0, nclamp = 0, nbad = 0;
    for (int32_t s = 0; s < S; ++s) {
        int64_t na = 0;
        for (int64_t i = 0; i < N; ++i) {
            act[i] = (uint8_t)(s % (1 << (K - bin[i])) == 0);
            na += act[i];
        }
        nact += na;
        if (na > 0) {
            const double delta = ldexp(D > 0.0 ? D : 0.0, -K);
            for (int64_t i = 0; i < N; ++i) {
                const double tau = delta * (double)(s - sa[i]);
                xp[i] = wrap1(x[i] + tau * (0.5 * (va[i] + vx[i])));
                yp[i] = wrap1(y[i] + tau * (0.5 * (va[N + i] + vy[i])));
                zp[i] = wrap1(z[i] + tau * (0.5 * (va[2 * N + i] + vz[i])));
            }
            gzo_density(N, xp, yp, zp, id, H, act, p, Hn, nn, it, NULL, cnt);
            for (int64_t i = 0; i < N; ++i)
                if (act[i]) {
                    H[i] = Hn[i];
                    n[i] = nn[i];
                }
            gzo_gradients(N, xp, yp, zp, id, m, H, n, vx, vy, vz, u, act, p, grad, B, NULL, NULL,
                          NULL, cnt);
            double dmin_unused;
            gzo_timestep(N, xp, yp, zp, id, m, H, n, vx, vy, vz, u, act, p, dtc, &dmin_unused);
            if (s == 0) {
                if (!(D > 0.0)) {
                    double lo = INFINITY, hi = 0.0;
                    for (int64_t i = 0; i < N; ++i) {
                        if (dtc[i] < lo) lo = dtc[i];
                        if (isfinite(dtc[i]) && dtc[i] > hi) hi = dtc[i];
                    }
                    const double a = p->cfl * hi, b = ldexp(p->cfl * lo, K);
                    D = a < b ? a : b;
                }
                for (int64_t i = 0; i < N; ++i) {
                    int c = 0;
                    bin[i] = bin_for(D, p->cfl * dtc[i], K, &c);
                    nclamp += c;
                }
            } else {
                for (int64_t i = 0; i < N; ++i)
                    if (act[i]) {
                        int c = 0;
                        int32_t k = bin_for(D, p->cfl * dtc[i], K, &c);
                        nclamp += c;
                        if (k > bin[i]) bin[i] = k;
                    }
            }
            double umed = 0.0;
            int have_med = 0;
            gzo_exchange(N, xp, yp, zp, id, m, H, n, vx, vy, vz, u, grad, B, bin, act, D, p, accp,
                         accE, accm, tch, cnt);
            double* u0 = (double*)malloc(sz);
            memcpy(u0, u, sz);
            for (int64_t i = 0; i < N; ++i) {
                if (!tch[i]) continue;
                const double dt = ldexp(D, -bin[i]);
                const double mn = mfv ? m[i] + dt * accm[i] : m[i];
                const double v2 = (vx[i] * vx[i] + vy[i] * vy[i]) + vz[i] * vz[i];
                const double E = m[i] * (u[i] + 0.5 * v2) + dt * accE[i];
                const double nx = (m[i] * vx[i] + dt * accp[i]) / mn;
                const double ny = (m[i] * vy[i] + dt * accp[N + i]) / mn;
                const double nz = (m[i] * vz[i] + dt * accp[2 * N + i]) / mn;
                double un = E / mn - 0.5 * ((nx * nx + ny * ny) + nz * nz);
                if (!(un > 0.0)) {
                    if (!have_med) {
                        umed = median_u(u0, N);
                        have_med = 1;
                    }
                    un = p->u_floor_frac * umed;
                    nfl++;
                }
                if (!(mn > 0.0)) nbad++;
                vx[i] = nx;
                vy[i] = ny;
                vz[i] = nz;
                u[i] = un;
                m[i] = mn;
            }
            free(u0);
        }
        for (int64_t i = 0; i < N; ++i) {
            if ((s + 1) % (1 << (K - bin[i])) != 0) continue;
            const double dt = ldexp(D, -bin[i]);
            x[i] = wrap1(x[i] + dt * (0.5 * (va[i] + vx[i])));
            y[i] = wrap1(y[i] + dt * (0.5 * (va[N + i] + vy[i])));
            z[i] = wrap1(z[i] + dt * (0.5 * (va[2 * N + i] + vz[i])));
            va[i] = vx[i];
            va[N + i] = vy[i];
            va[2 * N + i] = vz[i];
            sa[i] = s + 1;
        }
    }
    *dt_inout = D;
    if (bin_out) memcpy(bin_out, bin, sizeof(int32_t) * (size_t)N);
    if (active_out) *active_out = nact;
    if (cnt) {
        cnt->ufloor += nfl;
        cnt->bin_clamp += nclamp;
        cnt->nonfinite += nbad;
    }
    free(xp);
    free(va);
    free(n);
    free(Hn);
    free(nn);
    free(grad);
    free(B);
    free(dtc);
    free(accp);
    free(accE);
    free(accm);
    free(it);
    free(bin);
    free(sa);
    free(act);
    free(tch);
    return 0;
}

/* ---------------------------------------------- exact Riemann solver ---- */
/* Ideal-gas exact solution (pressure function of each side: shock branch
 * (p - p_K) sqrt(A_K / (p + B_K)) with A_K = 2 / ((g+1) rho_K),
 * B_K = (g-1)/(g+1) p_K; rarefaction branch 2 c_K/(g-1) ((p/p_K)^((g-1)/2g) - 1)),
 * star pressure from f_L(p) + f_R(p) + u_R - u_L = 0 by safeguarded Newton. */
static void pres_fn(double p, double rho, double P, double c, double g, double* f, double* fd) {
    if (p > P) {
        double A = 2.0 / ((g + 1.0) * rho), Bk = (g - 1.0) / (g + 1.0) * P;
        double q = sqrt(A / (p + Bk));
        *f = (p - P) * q;
        *fd = q * (1.0 - 0.5 * (p - P) / (p + Bk));
    } else {
        double e = (g - 1.0) / (2.0 * g);
        *f = 2.0 * c / (g - 1.0) * (pow(p / P, e) - 1.0);
        *fd = 1.0 / (rho * c) * pow(p / P, -(g + 1.0) / (2.0 * g));
    }
}

int gzo_riemann_star(double rhoL, double uL, double PL, double rhoR, double uR, double PR,
                     double g, double* pstar, double* ustar) {
    double cL = sqrt(g * PL / rhoL), cR = sqrt(g * PR / rhoR);
    if (2.0 * (cL + cR) / (g - 1.0) <= uR - uL) return -1; /* vacuum */
    double p = 0.5 * (PL + PR) - 0.125 * (uR - uL) * (rhoL + rhoR) * (cL + cR);
    if (p < 1e-12 * (PL + PR)) p = 1e-12 * (PL + PR);
    double lo = 0.0, hi = 0.0;
    int has_hi = 0;
    for (int it = 0; it < 200; ++it) {
        double fL, dL, fR, dR;
        pres_fn(p, rhoL, PL, cL, g, &fL, &dL);
        pres_fn(p, rhoR, PR, cR, g, &fR, &dR);
        double F = fL + fR + (uR - uL);
        if (F > 0.0) {
            hi = p;
            has_hi = 1;
        } else {
            lo = p;
        }
        double pn = p - F / (dL + dR);
        if (!(pn > lo) || (has_hi && !(pn < hi))) pn = has_hi ? 0.5 * (lo + hi) : 2.0 * p;
        if (fabs(pn - p) <= 1e-15 * (pn + p)) {
            p = pn;
            break;
        }
        p = pn;
    }
    double fL, dL, fR, dR;
    pres_fn(p, rhoL, PL, cL, g, &fL, &dL);
    pres_fn(p, rhoR, PR, cR, g, &fR, &dR);
    *pstar = p;
    *ustar = 0.5 * (uL + uR) + 0.5 * (fR - fL);
    return 0;
}

/* State at xi = x/t in the self-similar solution (interface at xi = 0). */
void gzo_riemann_sample(double rhoL, double uL, double PL, double rhoR, double uR, double PR,
                        double g, double ps, double us, double xi, double* rho, double* u,
                        double* P) {
    double gm = (g - 1.0) / (g + 1.0);
    if (xi <= us) { /* left of contact */
        double c = sqrt(g * PL / rhoL);
        if (ps > PL) {
            double S = uL - c * sqrt((g + 1.0) / (2.0 * g) * ps / PL + (g - 1.0) / (2.0 * g));
            if (xi <= S) {
                *rho = rhoL; *u = uL; *P = PL;
            } else {
                *rho = rhoL * (ps / PL + gm) / (gm * ps / PL + 1.0); *u = us; *P = ps;
            }
        } else {
            double cs = c * pow(ps / PL, (g - 1.0) / (2.0 * g));
            double head = uL - c, tail = us - cs;
            if (xi <= head) {
                *rho = rhoL; *u = uL; *P = PL;
            } else if (xi >= tail) {
                *rho = rhoL * pow(ps / PL, 1.0 / g); *u = us; *P = ps;
            } else {
                double f = 2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * c) * (uL - xi);
                *rho = rhoL * pow(f, 2.0 / (g - 1.0));
                *u = 2.0 / (g + 1.0) * (c + 0.5 * (g - 1.0) * uL + xi);
                *P = PL * pow(f, 2.0 * g / (g - 1.0));
            }
        }
    } else { /* right of contact */
        double c = sqrt(g * PR / rhoR);
        if (ps > PR) {
            double S = uR + c * sqrt((g + 1.0) / (2.0 * g) * ps / PR + (g - 1.0) / (2.0 * g));
            if (xi >= S) {
                *rho = rhoR; *u = uR; *P = PR;
            } else {
                *rho = rhoR * (ps / PR + gm) / (gm * ps / PR + 1.0); *u = us; *P = ps;
            }
        } else {
            double cs = c * pow(ps / PR, (g - 1.0) / (2.0 * g));
            double head = uR + c, tail = us + cs;
            if (xi >= head) {
                *rho = rhoR; *u = uR; *P = PR;
            } else if (xi <= tail) {
                *rho = rhoR * pow(ps / PR, 1.0 / g); *u = us; *P = ps;
            } else {
                double f = 2.0 / (g + 1.0) - (g - 1.0) / ((g + 1.0) * c) * (uR - xi);
                *rho = rhoR * pow(f, 2.0 / (g - 1.0));
                *u = 2.0 / (g + 1.0) * (-c + 0.5 * (g - 1.0) * uR + xi);
                *P = PR * pow(f, 2.0 * g / (g - 1.0));
            }
        }
    }
}

int gzo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void gzo_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
