// Device functions shared by the forward passes and their adjoints.
#pragma once

#include "gz_internal.cuh"

namespace gz {

// Kahan-compensated sum for FP32 neighbour sums; plain sum in FP64.
template <typename T>
struct Acc {
    T s = T(0);
    __device__ __forceinline__ void add(T v) { s += v; }
    __device__ __forceinline__ void merge(const Acc& o) { s += o.s; }
    __device__ __forceinline__ double value() const { return (double)s; }
};
template <>
struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        float y = __fsub_rn(v, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ void merge(const Acc& o) { add(o.fvalue()); }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
    __device__ __forceinline__ float fvalue() const { return __fsub_rn(s, c); }
};

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// Pair-pass division and square roots: the FP32 path uses the hardware
// reciprocal / reciprocal square root (about 2 ulp; deterministic, so both
// particles of a pair still compute identical values); FP64 stays IEEE.
__device__ __forceinline__ float pdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double pdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float psqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double psqrt(double x) { return sqrt(x); }

// Symmetric 3x3 inverse by adjugate; kappa = |E|_F |B|_F / 3.
template <typename A>
__device__ __forceinline__ void invert_sym(const A E[6], A B[6], A& det, A& kap) {
    const A a = E[0], b = E[1], c = E[2], d = E[3], e = E[4], f = E[5];
    const A Cxx = d * f - e * e, Cxy = c * e - b * f, Cxz = b * e - c * d;
    const A Cyy = a * f - c * c, Cyz = b * c - a * e, Czz = a * d - b * b;
    det = a * Cxx + b * Cxy + c * Cxz;
    const A id = A(1) / det;
    B[0] = Cxx * id;
    B[1] = Cxy * id;
    B[2] = Cxz * id;
    B[3] = Cyy * id;
    B[4] = Cyz * id;
    B[5] = Czz * id;
    const A nE = sqrt(a * a + d * d + f * f + A(2) * (b * b + c * c + e * e));
    const A nB = sqrt(B[0] * B[0] + B[3] * B[3] + B[5] * B[5] +
                      A(2) * (B[1] * B[1] + B[2] * B[2] + B[4] * B[4]));
    kap = nE * nB / A(3);
}

// ---------------------------------------------------------- O10-O12
// A flux record is one 128-byte line (FP32) or two (FP64), read with 32-byte
// vector loads (sm_100+ ld.global.v8.f32 / v4.f64): a warp gathering 32
// records from scattered lines then moves whole sectors per L1 wavefront
// instead of half sectors.  Records start on 128-byte boundaries.
__device__ __forceinline__ void load_rec(const float* __restrict__ p, float (&v)[kRecord]) {
#pragma unroll
    for (int k = 0; k < kRecord / 8; ++k)
        asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=f"(v[8 * k]), "=f"(v[8 * k + 1]), "=f"(v[8 * k + 2]), "=f"(v[8 * k + 3]), "=f"(v[8 * k + 4]),
              "=f"(v[8 * k + 5]), "=f"(v[8 * k + 6]), "=f"(v[8 * k + 7])
            : "l"(p + 8 * k));
}
__device__ __forceinline__ void load_rec(const double* __restrict__ p, double (&v)[kRecord]) {
#pragma unroll
    for (int k = 0; k < kRecord / 4; ++k)
        asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
            : "=d"(v[4 * k]), "=d"(v[4 * k + 1]), "=d"(v[4 * k + 2]), "=d"(v[4 * k + 3])
            : "l"(p + 4 * k));
}

// Face state of particle a toward the face at a + s o (o = offset to the
// partner): linear reconstruction with a's limited gradients plus the Hancock
// half step (dt/2) (-rho div v, -grad P / rho, -gamma P div v).
// Hancock half-step increments of a particle's primitives (O11):
// (dt/2)(-rho div v, -grad P / rho, -gamma P div v), each product rounded
// once so that every pass that forms them gets the same bits.
template <typename T>
__device__ __forceinline__ void hancock_inc(const T (&a)[kRecord], T hdt, T gam, bool hancock, T (&inc)[5]) {
    if (!hancock) {
#pragma unroll
        for (int f = 0; f < 5; ++f) inc[f] = T(0);
        return;
    }
    const T div = (a[11 + 3] + a[11 + 7]) + a[11 + 11];
    const T ir = pdiv(T(1), a[6]);
    inc[0] = mul_rn(hdt, -a[6] * div);
    inc[1] = mul_rn(hdt, -a[11 + 12] * ir);
    inc[2] = mul_rn(hdt, -a[11 + 13] * ir);
    inc[3] = mul_rn(hdt, -a[11 + 14] * ir);
    inc[4] = mul_rn(hdt, -gam * a[7] * div);
}

// Face state of a record at offset s (dx, dy, dz) from the particle:
// W + g . (s d) + the Hancock increments.
template <typename T>
__device__ __forceinline__ void face_state(const T (&a)[kRecord], T s, T dx, T dy, T dz, const T (&inc)[5],
                                           T (&F)[5]) {
    const T ox = s * dx, oy = s * dy, oz = s * dz;
    const T W[5] = {a[6], a[8], a[9], a[10], a[7]};
#pragma unroll
    for (int f = 0; f < 5; ++f)
        F[f] = add_rn(W[f] + ((a[11 + 3 * f] * ox + a[12 + 3 * f] * oy) + a[13 + 3 * f] * oz), inc[f]);
}

// n values (a multiple of 32 bytes) from 32-byte-aligned global memory with
// 32-byte vector loads, for per-particle rows read by other particles'
// threads (scattered rows: whole sectors per L1 wavefront).
template <int n>
__device__ __forceinline__ void load_row32(const float* __restrict__ p, float* v) {
    static_assert(n % 8 == 0, "rows of whole 32-byte vectors");
#pragma unroll
    for (int k = 0; k < n / 8; ++k)
        asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=f"(v[8 * k]), "=f"(v[8 * k + 1]), "=f"(v[8 * k + 2]), "=f"(v[8 * k + 3]), "=f"(v[8 * k + 4]),
              "=f"(v[8 * k + 5]), "=f"(v[8 * k + 6]), "=f"(v[8 * k + 7])
            : "l"(p + 8 * k));
}
template <int n>
__device__ __forceinline__ void load_row32(const double* __restrict__ p, double* v) {
    static_assert(n % 4 == 0, "rows of whole 32-byte vectors");
#pragma unroll
    for (int k = 0; k < n / 4; ++k)
        asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
            : "=d"(v[4 * k]), "=d"(v[4 * k + 1]), "=d"(v[4 * k + 2]), "=d"(v[4 * k + 3])
            : "l"(p + 4 * k));
}

// n values (a multiple of 32 bytes) to 32-byte-aligned global memory with
// 32-byte vector stores: a per-particle row written by its thread fills
// whole sectors instead of one 4-byte piece per store.  The rows are read
// by later passes, not by the writing one: not allocated in L1.
template <int n>
__device__ __forceinline__ void store_row32(float* p, const float* v) {
    static_assert(n % 8 == 0, "rows of whole 32-byte vectors");
#pragma unroll
    for (int k = 0; k < n / 8; ++k)
        asm volatile("st.global.L1::no_allocate.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                     :
                     : "l"(p + 8 * k), "f"(v[8 * k]), "f"(v[8 * k + 1]), "f"(v[8 * k + 2]), "f"(v[8 * k + 3]),
                       "f"(v[8 * k + 4]), "f"(v[8 * k + 5]), "f"(v[8 * k + 6]), "f"(v[8 * k + 7])
                     : "memory");
}
template <int n>
__device__ __forceinline__ void store_row32(double* p, const double* v) {
    static_assert(n % 4 == 0, "rows of whole 32-byte vectors");
#pragma unroll
    for (int k = 0; k < n / 4; ++k)
        asm volatile("st.global.L1::no_allocate.v4.f64 [%0], {%1,%2,%3,%4};"
                     :
                     : "l"(p + 4 * k), "d"(v[4 * k]), "d"(v[4 * k + 1]), "d"(v[4 * k + 2]), "d"(v[4 * k + 3])
                     : "memory");
}

// Four values to / from 16-byte-aligned memory.
__device__ __forceinline__ void store4(float* dst, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(dst) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void store4(double* dst, double a, double b, double c, double d) {
    reinterpret_cast<double2*>(dst)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(dst)[1] = make_double2(c, d);
}
__device__ __forceinline__ void load4(const float* src, float (&v)[4]) {
    const float4 w = __ldg(reinterpret_cast<const float4*>(src));
    v[0] = w.x;
    v[1] = w.y;
    v[2] = w.z;
    v[3] = w.w;
}
__device__ __forceinline__ void load4(const double* src, double (&v)[4]) {
    const double2 w0 = __ldg(reinterpret_cast<const double2*>(src));
    const double2 w1 = __ldg(reinterpret_cast<const double2*>(src) + 1);
    v[0] = w0.x;
    v[1] = w0.y;
    v[2] = w1.x;
    v[3] = w1.y;
}

// O15: HLLC flux of mass, momentum and total energy through a face that
// moves with vf (unit normal n from L to R), from the face states FL, FR
// (rho, v, P) and the wave speeds the caller already formed in the face
// frame (u_K = (v_K - vf) . n, S_L, S_R, S*).  In that frame w = v - vf,
// U = (rho, rho w, E) with E = P/(gamma-1) + rho |w|^2/2 and the flux along n
// is F(U) = (rho u, rho u w + P n, u (E + P)).  The flux at the face (xi = 0)
// is F_K or F_K + S_K (U*_K - U_K) for the side K the waves leave it on, with
// the star state U*_K = rho_K (S_K - u_K)/(S_K - S*) (1, w_K + (S* - u_K) n,
// E_K/rho_K + (S* - u_K)(S* + P_K/(rho_K (S_K - u_K)))).  With q = 1/(S_K - S*),
// g = rho_K q, f = g (S_K - u_K) and dS = S* - u_K the jump S_K (U*_K - U_K)
// is S_K dS (g, g w_K + f n, q (E_K + P_K) + f S*), the same quantity without
// the cancellation of U*_K - U_K for weak waves.  Back in the lab frame the
// fluxes are F_m, F_w + vf F_m and F_E + vf . F_w + |vf|^2 F_m / 2.
template <typename T>
__device__ __forceinline__ void mfv_flux(const T (&FL)[5], const T (&FR)[5], T uL, T uR, T SL, T SR,
                                         T ss, T vfx, T vfy, T vfz, T nx, T ny, T nz, T gam, T& Fm,
                                         T (&Fp)[3], T& FE) {
    // side: L when S_L >= 0 or S* >= 0; the star jump unless S_L >= 0 (L) or
    // S_R <= 0 (R); a NaN speed takes R without the jump, like the oracle
    const bool left = SL >= T(0) || ss >= T(0);
    const bool star = left ? !(SL >= T(0)) : SR > T(0);
    const T rho = left ? FL[0] : FR[0];
    const T P = left ? FL[4] : FR[4];
    const T un = left ? uL : uR;
    const T wx = (left ? FL[1] : FR[1]) - vfx;
    const T wy = (left ? FL[2] : FR[2]) - vfy;
    const T wz = (left ? FL[3] : FR[3]) - vfz;
    const T E = pdiv(P, gam - T(1)) + T(0.5) * rho * ((wx * wx + wy * wy) + wz * wz);
    const T ru = rho * un;
    T fr = ru;
    T fx = ru * wx + P * nx, fy = ru * wy + P * ny, fz = ru * wz + P * nz;
    T fe = un * (E + P);
    if (star) {
        const T SK = left ? SL : SR;
        const T q = pdiv(T(1), SK - ss);
        const T g = rho * q, f = g * (SK - un);
        const T k = SK * (ss - un);
        fr += k * g;
        fx += k * (g * wx + f * nx);
        fy += k * (g * wy + f * ny);
        fz += k * (g * wz + f * nz);
        fe += k * (q * (E + P) + f * ss);
    }
    Fm = fr;
    Fp[0] = fx + vfx * fr;
    Fp[1] = fy + vfy * fr;
    Fp[2] = fz + vfz * fr;
    FE = (fe + ((vfx * fx + vfy * fy) + vfz * fz)) + T(0.5) * ((vfx * vfx + vfy * vfy) + vfz * vfz) * fr;
}

// x^y for x > 0: FP32 as 2^(y log2 x) from the hardware base-2 logarithm
// (relative error about 1e-7 (1 + |y log2 x|)); FP64 the library pow.
__device__ __forceinline__ float ppow(float x, float y) { return exp2f(y * __log2f(x)); }
__device__ __forceinline__ double ppow(double x, double y) { return pow(x, y); }

// Exact Riemann problem of the face (option of O12).  Pressure function of one
// side at the trial star pressure p: shock branch (p > P_K)
// (p - P_K) sqrt(A_K/(p + B_K)) with A_K = 2/((gamma+1) rho_K),
// B_K = (gamma-1)/(gamma+1) P_K; rarefaction branch
// 2 c_K/(gamma-1) ((p/P_K)^e - 1), e = (gamma-1)/(2 gamma), whose derivative
// (p/P_K)^(e-1)/(rho_K c_K) is formed from the same power.  f and df/dp.
template <typename T>
__device__ __forceinline__ void pres_side(T p, T rho, T P, T c, T gam, T& f, T& fd) {
    if (p > P) {
        const T A = pdiv(T(2), (gam + T(1)) * rho), Bk = pdiv(gam - T(1), gam + T(1)) * P;
        const T q = psqrt(pdiv(A, p + Bk));
        f = (p - P) * q;
        fd = q * (T(1) - T(0.5) * pdiv(p - P, p + Bk));
    } else {
        const T r = pdiv(p, P);
        const T pe = ppow(r, pdiv(gam - T(1), T(2) * gam));
        f = pdiv(T(2) * c, gam - T(1)) * (pe - T(1));
        fd = pdiv(pe, r * rho * c);
    }
}

// Star pressure and contact speed of the exact solution: the root of
// F(p) = f_L(p) + f_R(p) + u_R - u_L, an increasing concave function.
// Starting point (Toro's adaptive choice): the primitive-variable estimate
// p_PV = (P_L + P_R)/2 - (u_R - u_L)(rho_L + rho_R)(c_L + c_R)/8 when the
// pressures differ by at most 2x and p_PV lies between them; below them the
// two-rarefaction solution [(c_L + c_R - (gamma-1)(u_R - u_L)/2) /
// (c_L P_L^-e + c_R P_R^-e)]^(1/e) (the root itself when both waves are
// rarefactions); above them the two-shock estimate
// (g_L P_L + g_R P_R - (u_R - u_L))/(g_L + g_R), g_K = sqrt(A_K/(p_PV + B_K));
// at least 1e-12 (P_L + P_R).  Newton steps kept inside the bracket the signs
// of F have established (bisection, or doubling while no upper end is known)
// until two iterates agree to 1e-15 (FP64) or 1e-6 (FP32) relative, or F is at
// the rounding level of its terms (FP32: 4e-7 of |f_L| + |f_R| + |u_R - u_L|,
// where a strong rarefaction's F cannot resolve p to 1e-6); at most 200 (FP64)
// or 20 (FP32) steps.  u* = (u_L + u_R)/2 + (f_R - f_L)/2.  Returns false when
// the two fans open a vacuum (2 (c_L + c_R)/(gamma-1) <= u_R - u_L).
template <typename T>
__device__ __forceinline__ bool exact_star(T rL, T uL, T PL, T rR, T uR, T PR, T gam, T& ps, T& us) {
    const T cL = psqrt(pdiv(gam * PL, rL)), cR = psqrt(pdiv(gam * PR, rR));
    const T du = uR - uL;
    if (pdiv(T(2) * (cL + cR), gam - T(1)) <= du) return false;
    const T plo = min(PL, PR), phi = max(PL, PR);
    T p = T(0.5) * (PL + PR) - T(0.125) * du * (rL + rR) * (cL + cR);
    if (!(phi <= T(2) * plo && p >= plo && p <= phi)) {
        if (p < plo) {
            const T e = pdiv(gam - T(1), T(2) * gam);
            const T num = (cL + cR) - T(0.5) * (gam - T(1)) * du;
            const T den = cL * ppow(PL, -e) + cR * ppow(PR, -e);
            p = ppow(pdiv(num, den), pdiv(T(1), e));
        } else {
            const T p0 = max(p, T(0));
            const T gp1 = gam + T(1), gm1 = gam - T(1);
            const T gL = psqrt(pdiv(pdiv(T(2), gp1 * rL), p0 + pdiv(gm1, gp1) * PL));
            const T gR = psqrt(pdiv(pdiv(T(2), gp1 * rR), p0 + pdiv(gm1, gp1) * PR));
            p = pdiv((gL * PL + gR * PR) - du, gL + gR);
        }
    }
    const T pmin = T(1e-12) * (PL + PR);
    if (!(p >= pmin)) p = pmin;
    constexpr bool f32 = sizeof(T) == 4;
    const T tol = f32 ? T(1e-6) : T(1e-15);
    const int cap = f32 ? 20 : 200;
    T lo = T(0), hi = T(0);
    bool has_hi = false;
    for (int it = 0; it < cap; ++it) {
        T fL, dL, fR, dR;
        pres_side(p, rL, PL, cL, gam, fL, dL);
        pres_side(p, rR, PR, cR, gam, fR, dR);
        const T F = (fL + fR) + du;
        if (f32 && fabs(F) <= T(4e-7) * ((fabs(fL) + fabs(fR)) + fabs(du))) break;
        if (F > T(0)) {
            hi = p;
            has_hi = true;
        } else {
            lo = p;
        }
        T pn = p - pdiv(F, dL + dR);
        if (!(pn > lo) || (has_hi && !(pn < hi))) pn = has_hi ? T(0.5) * (lo + hi) : T(2) * p;
        const bool done = fabs(pn - p) <= tol * (pn + p);
        p = pn;
        if (done) break;
    }
    T fL, dL, fR, dR;
    pres_side(p, rL, PL, cL, gam, fL, dL);
    pres_side(p, rR, PR, cR, gam, fR, dR);
    ps = p;
    us = T(0.5) * (uL + uR) + T(0.5) * (fR - fL);
    return true;
}

// Orientation of a pair (sorted indices i, j; ids idi = id of i, sid[]) in
// the forward flux passes: whether i is L.  MFM: the lower sorted index,
// which both particles of the pair know, so no id is gathered.  MFV: the
// lower id.  Either is a fixed order of the pair, so its two particles
// compute the same canonical flux and get bitwise-opposite contributions
// (the adjoint orients by id: its tie rule at the clamp names L).
template <bool kById>
__device__ __forceinline__ bool pair_order(int i, int j, long long idi, const long long* __restrict__ sid) {
    if constexpr (kById)
        return idi < sid[j];
    else
        return i < j;
}

// Contribution of the pair (a, b) to particle a's rates: dp (3), dE and,
// under MFV (O15), dm.  kRiem: the MFM face's star from HLLC (0), the exact
// solver (1), or HLLC with the exact star where HLLC's P* < 0 (2).  Returns
// false when the face area vanishes.  flags: 1 fallback, 2 P* < 0 (or vacuum).
template <typename T, bool kMFV, int kRiem>
__device__ __forceinline__ bool pair_rates(const T (&a)[kRecord], const T (&b)[kRecord], bool aL,
                                           T hdt, T gam, bool hancock, const T (&inca)[5], T (&dp)[3],
                                           T& dE, T& dm, int& fl) {
    const T dx = mi_diff(b[0], a[0], a[0] - T(1));
    const T dy = mi_diff(b[1], a[1], a[1] - T(1));
    const T dz = mi_diff(b[2], a[2], a[2] - T(1));
    const T r2 = sep2(dx, dy, dz);
    const T r = psqrt(r2);
    const T ca = r2 < a[3] * a[3] ? a[5] * kern_w(r * a[4]) : T(0);
    const T cb = r2 < b[3] * b[3] ? b[5] * kern_w(r * b[4]) : T(0);
    const T Bax = (a[26] * dx + a[27] * dy) + a[28] * dz;
    const T Bay = (a[27] * dx + a[29] * dy) + a[30] * dz;
    const T Baz = (a[28] * dx + a[30] * dy) + a[31] * dz;
    const T Bbx = (b[26] * dx + b[27] * dy) + b[28] * dz;
    const T Bby = (b[27] * dx + b[29] * dy) + b[30] * dz;
    const T Bbz = (b[28] * dx + b[30] * dy) + b[31] * dz;
    const T A0 = add_rn(mul_rn(ca, Bax), mul_rn(cb, Bbx));
    const T A1 = add_rn(mul_rn(ca, Bay), mul_rn(cb, Bby));
    const T A2 = add_rn(mul_rn(ca, Baz), mul_rn(cb, Bbz));
    const T Aq = sep2(A0, A1, A2);
    if (!(Aq > T(0))) return false;
    const T Am = psqrt(Aq);
    const T iA = pdiv(T(1), Am);
    const T n0 = A0 * iA, n1 = A1 * iA, n2 = A2 * iA;
    const T Hs = a[3] + b[3];
    const T sa = pdiv(a[3], Hs), sb = pdiv(b[3], Hs);
    T Fa[5], Fb[5];
    T incb[5];
    hancock_inc(b, hdt, gam, hancock, incb);
    face_state(a, sa, dx, dy, dz, inca, Fa);
    face_state(b, sb, -dx, -dy, -dz, incb, Fb);
    const T Wa[5] = {a[6], a[8], a[9], a[10], a[7]};
    const T Wb[5] = {b[6], b[8], b[9], b[10], b[7]};
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        const T lo = min(Wa[f], Wb[f]), hi = max(Wa[f], Wb[f]);
        Fa[f] = min(max(Fa[f], lo), hi);
        Fb[f] = min(max(Fb[f], lo), hi);
    }
    if (!(Fa[0] > T(0) && Fa[4] > T(0) && Fb[0] > T(0) && Fb[4] > T(0))) {
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            Fa[f] = Wa[f];
            Fb[f] = Wb[f];
        }
        fl |= 1;
    }
    // canonical order: L = a when aL (pair_order)
    T FL[5], FR[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        FL[f] = aL ? Fa[f] : Fb[f];
        FR[f] = aL ? Fb[f] : Fa[f];
    }
    const T vLx = aL ? Wa[1] : Wb[1], vLy = aL ? Wa[2] : Wb[2], vLz = aL ? Wa[3] : Wb[3];
    const T vRx = aL ? Wb[1] : Wa[1], vRy = aL ? Wb[2] : Wa[2], vRz = aL ? Wb[3] : Wa[3];
    const T sL = aL ? sa : sb;
    const T nx = aL ? n0 : -n0, ny = aL ? n1 : -n1, nz = aL ? n2 : -n2;
    const T vfx = vLx + sL * (vRx - vLx), vfy = vLy + sL * (vRy - vLy), vfz = vLz + sL * (vRz - vLz);
    const T vfn = (vfx * nx + vfy * ny) + vfz * nz;
    const T uL = ((FL[1] - vfx) * nx + (FL[2] - vfy) * ny) + (FL[3] - vfz) * nz;
    const T uR = ((FR[1] - vfx) * nx + (FR[2] - vfy) * ny) + (FR[3] - vfz) * nz;
    // O12 HLLC with Davis wave speeds
    const T rL = FL[0], PL = FL[4], rR = FR[0], PR = FR[4];
    const T cL = psqrt(pdiv(gam * PL, rL)), cR = psqrt(pdiv(gam * PR, rR));
    const T SL = min(uL - cL, uR - cR), SR = max(uL + cL, uR + cR);
    const T num = ((PR - PL) + rL * uL * (SL - uL)) - rR * uR * (SR - uR);
    const T den = rL * (SL - uL) - rR * (SR - uR);
    const T ss = pdiv(num, den);
    T ps = PL + rL * (SL - uL) * (ss - uL);
    T sm = ss;  // contact speed of the MFM energy rate
    bool neg = ps < T(0);
    if constexpr (!kMFV && kRiem != 0) {
        if (kRiem == 1 || neg) {
            T pe, ue;
            if (exact_star(rL, uL, PL, rR, uR, PR, gam, pe, ue)) {
                ps = pe;
                sm = ue;
                if (kRiem == 1) neg = false;
            } else {
                ps = T(0);
                sm = T(0);
                neg = true;
            }
        }
    }
    if (neg) fl |= 2;
    if (ps < T(0)) ps = T(0);
    if constexpr (kMFV) {
        // both particles of the pair form the same canonical flux bits; L
        // loses what R gains
        T Fm, Fp[3], FE;
        mfv_flux(FL, FR, uL, uR, SL, SR, ss, vfx, vfy, vfz, nx, ny, nz, gam, Fm, Fp, FE);
        const T m = mul_rn(Fm, Am), px = mul_rn(Fp[0], Am), py = mul_rn(Fp[1], Am),
                pz = mul_rn(Fp[2], Am), e = mul_rn(FE, Am);
        dm = aL ? -m : m;
        dp[0] = aL ? -px : px;
        dp[1] = aL ? -py : py;
        dp[2] = aL ? -pz : pz;
        dE = aL ? -e : e;
        return true;
    }
    dm = T(0);
    dp[0] = -mul_rn(ps, A0);
    dp[1] = -mul_rn(ps, A1);
    dp[2] = -mul_rn(ps, A2);
    const T ef = ps * (sm + vfn) * Am;
    dE = aL ? -ef : ef;
    return true;
}

// ----------------------------------------------------------------- O14
__device__ __forceinline__ double wrap1(double v) {
    if (v < 0.0) v += 1.0;
    if (v >= 1.0) v -= 1.0;
    return v;
}

// FP64 state: the literal conserved update, like the oracle, every operation
// rounded explicitly (no contraction), so that each kernel that kicks or
// drifts a particle (the step's update, the hierarchical kick and drift)
// produces the same bits.  Kick: p += dt dp/dt, E += dt dE/dt, v = p/m,
// u = E/m - v^2/2.
__device__ __forceinline__ void kick_one(double m, double& vx, double& vy, double& vz, double& u, double dpx,
                                         double dpy, double dpz, double dE, double dt) {
    const double v2 = __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz));
    const double E = __dadd_rn(__dmul_rn(m, __dadd_rn(u, __dmul_rn(0.5, v2))), __dmul_rn(dt, dE));
    const double nx = __ddiv_rn(__dadd_rn(__dmul_rn(m, vx), __dmul_rn(dt, dpx)), m);
    const double ny = __ddiv_rn(__dadd_rn(__dmul_rn(m, vy), __dmul_rn(dt, dpy)), m);
    const double nz = __ddiv_rn(__dadd_rn(__dmul_rn(m, vz), __dmul_rn(dt, dpz)), m);
    const double n2 = __dadd_rn(__dadd_rn(__dmul_rn(nx, nx), __dmul_rn(ny, ny)), __dmul_rn(nz, nz));
    u = __dsub_rn(__ddiv_rn(E, m), __dmul_rn(0.5, n2));
    vx = nx;
    vy = ny;
    vz = nz;
}
// Trapezoid drift of one coordinate: wrap(x + dt (v_old + v_new)/2).
__device__ __forceinline__ double drift_one(double x, double v_old, double v_new, double dt) {
    return wrap1(__dadd_rn(x, __dmul_rn(dt, __dmul_rn(0.5, __dadd_rn(v_old, v_new)))));
}
__device__ __forceinline__ void update_one(double m, double& x, double& y, double& z, double& vx,
                                           double& vy, double& vz, double& u, double dpx, double dpy,
                                           double dpz, double dE, double dt) {
    const double ox = vx, oy = vy, oz = vz;
    kick_one(m, vx, vy, vz, u, dpx, dpy, dpz, dE, dt);
    x = drift_one(x, ox, vx, dt);
    y = drift_one(y, oy, vy, dt);
    z = drift_one(z, oz, vz, dt);
}
// FP32 state: the same update written with the increments dv = dt (dp/dt)/m
// and du = dt (dE/dt)/m - dv . (v + dv/2), which is E/m - v_new^2/2 - u
// without the cancellation of the literal form; the drift is
// x + dt (v_old + dv/2).  Explicit rounding as above.
__device__ __forceinline__ float wrapf(float v) {
    if (v < 0.f) v += 1.f;
    if (v >= 1.f) v -= 1.f;
    return v;
}
__device__ __forceinline__ void kick_one(float m, float& vx, float& vy, float& vz, float& u, double dpx,
                                         double dpy, double dpz, double dE, double dt, float& dvx,
                                         float& dvy, float& dvz) {
    const float dtf = (float)dt, im = __fdiv_rn(1.f, m);
    dvx = __fmul_rn(__fmul_rn(dtf, (float)dpx), im);
    dvy = __fmul_rn(__fmul_rn(dtf, (float)dpy), im);
    dvz = __fmul_rn(__fmul_rn(dtf, (float)dpz), im);
    const float hx = __fadd_rn(vx, __fmul_rn(0.5f, dvx)), hy = __fadd_rn(vy, __fmul_rn(0.5f, dvy)),
                hz = __fadd_rn(vz, __fmul_rn(0.5f, dvz));
    const float w = __fadd_rn(__fadd_rn(__fmul_rn(dvx, hx), __fmul_rn(dvy, hy)), __fmul_rn(dvz, hz));
    const float du = __fsub_rn(__fmul_rn(__fmul_rn(dtf, (float)dE), im), w);
    u = __fadd_rn(u, du);
    vx = __fadd_rn(vx, dvx);
    vy = __fadd_rn(vy, dvy);
    vz = __fadd_rn(vz, dvz);
}
__device__ __forceinline__ float drift_onef(float x, float v_old, float dv, double dt) {
    return wrapf(__fadd_rn(x, __fmul_rn((float)dt, __fadd_rn(v_old, __fmul_rn(0.5f, dv)))));
}
__device__ __forceinline__ void update_one(float m, float& x, float& y, float& z, float& vx,
                                           float& vy, float& vz, float& u, double dpx, double dpy,
                                           double dpz, double dE, double dt) {
    const float ox = vx, oy = vy, oz = vz;
    float dvx, dvy, dvz;
    kick_one(m, vx, vy, vz, u, dpx, dpy, dpz, dE, dt, dvx, dvy, dvz);
    x = drift_onef(x, ox, dvx, dt);
    y = drift_onef(y, oy, dvy, dt);
    z = drift_onef(z, oz, dvz, dt);
}

// MFV (O15): the mass advances too, m' = m + dt dm/dt, and momentum and
// total energy are divided by m'.  FP64 state: the literal form, like the
// oracle, explicitly rounded like kick_one.
__device__ __forceinline__ void kick_one_mfv(double& m, double& vx, double& vy, double& vz, double& u,
                                             double dpx, double dpy, double dpz, double dE, double dm,
                                             double dt) {
    const double mn = __dadd_rn(m, __dmul_rn(dt, dm));
    const double v2 = __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz));
    const double E = __dadd_rn(__dmul_rn(m, __dadd_rn(u, __dmul_rn(0.5, v2))), __dmul_rn(dt, dE));
    const double nx = __ddiv_rn(__dadd_rn(__dmul_rn(m, vx), __dmul_rn(dt, dpx)), mn);
    const double ny = __ddiv_rn(__dadd_rn(__dmul_rn(m, vy), __dmul_rn(dt, dpy)), mn);
    const double nz = __ddiv_rn(__dadd_rn(__dmul_rn(m, vz), __dmul_rn(dt, dpz)), mn);
    const double n2 = __dadd_rn(__dadd_rn(__dmul_rn(nx, nx), __dmul_rn(ny, ny)), __dmul_rn(nz, nz));
    u = __dsub_rn(__ddiv_rn(E, mn), __dmul_rn(0.5, n2));
    vx = nx;
    vy = ny;
    vz = nz;
    m = mn;
}
__device__ __forceinline__ void update_one_mfv(double& m, double& x, double& y, double& z, double& vx,
                                               double& vy, double& vz, double& u, double dpx, double dpy,
                                               double dpz, double dE, double dm, double dt) {
    const double ox = vx, oy = vy, oz = vz;
    kick_one_mfv(m, vx, vy, vz, u, dpx, dpy, dpz, dE, dm, dt);
    x = drift_one(x, ox, vx, dt);
    y = drift_one(y, oy, vy, dt);
    z = drift_one(z, oz, vz, dt);
}
// FP32 state: with dM = dt dm/dt, m' = m + dM (formed in FP64) and the
// increments dv = (dt dp/dt - dM v)/m' and
// du = (dt dE/dt - dM (u + v^2/2))/m' - dv . (v + dv/2), which equal
// p'/m' - v and E'/m' - v'^2/2 - u without the cancellation of the literal
// form; explicitly rounded like kick_one.
__device__ __forceinline__ void kick_one_mfv(float& m, float& vx, float& vy, float& vz, float& u, double dpx,
                                             double dpy, double dpz, double dE, double dm, double dt,
                                             float& dvx, float& dvy, float& dvz) {
    const float mn = (float)__dadd_rn((double)m, __dmul_rn(dt, dm));
    const float dtf = (float)dt, im = __fdiv_rn(1.f, mn), dM = __fmul_rn(dtf, (float)dm);
    dvx = __fmul_rn(__fsub_rn(__fmul_rn(dtf, (float)dpx), __fmul_rn(dM, vx)), im);
    dvy = __fmul_rn(__fsub_rn(__fmul_rn(dtf, (float)dpy), __fmul_rn(dM, vy)), im);
    dvz = __fmul_rn(__fsub_rn(__fmul_rn(dtf, (float)dpz), __fmul_rn(dM, vz)), im);
    const float hx = __fadd_rn(vx, __fmul_rn(0.5f, dvx)), hy = __fadd_rn(vy, __fmul_rn(0.5f, dvy)),
                hz = __fadd_rn(vz, __fmul_rn(0.5f, dvz));
    const float v2 = __fadd_rn(__fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy)), __fmul_rn(vz, vz));
    const float ek = __fadd_rn(u, __fmul_rn(0.5f, v2));
    const float w = __fadd_rn(__fadd_rn(__fmul_rn(dvx, hx), __fmul_rn(dvy, hy)), __fmul_rn(dvz, hz));
    const float du = __fsub_rn(__fmul_rn(__fsub_rn(__fmul_rn(dtf, (float)dE), __fmul_rn(dM, ek)), im), w);
    u = __fadd_rn(u, du);
    vx = __fadd_rn(vx, dvx);
    vy = __fadd_rn(vy, dvy);
    vz = __fadd_rn(vz, dvz);
    m = mn;
}
__device__ __forceinline__ void update_one_mfv(float& m, float& x, float& y, float& z, float& vx,
                                               float& vy, float& vz, float& u, double dpx, double dpy,
                                               double dpz, double dE, double dm, double dt) {
    const float ox = vx, oy = vy, oz = vz;
    float dvx, dvy, dvz;
    kick_one_mfv(m, vx, vy, vz, u, dpx, dpy, dpz, dE, dm, dt, dvx, dvy, dvz);
    x = drift_onef(x, ox, dvx, dt);
    y = drift_onef(y, oy, dvy, dt);
    z = drift_onef(z, oz, dvz, dt);
}

}  // namespace gz
