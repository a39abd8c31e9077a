// Adjoint (reverse mode) of the MFM step, hand-written pass by pass.
//
// Conventions, identical to the derivative oracle: neighbour sets and the
// flux pair set are frozen at their forward values; dt is a constant; H is
// the root of f(H; x) = 0 and is differentiated implicitly; the u floor is a
// constant; min / max / clamp pass the adjoint to the branch the forward
// took.  Every pass re-evaluates its forward quantities (nothing per pair is
// stored) and accumulates adjoints by gathering: the thread of particle i
// visits i's pairs and adds only the terms that belong to i, so there are no
// atomics and the result is deterministic.
//
// Adjoint record per particle (double, sorted order), kAdj values:
//   0-2 x   3-5 v   6 u   7 m   8 H   9 n   10 rho   11 P   12-26 g (limited)
//   27-32 B (xx xy xz yy yz zz)
#include <algorithm>

#include "gz_device.cuh"
#include "gz_launch.cuh"

namespace gz {

namespace {

inline int blocks(int n, int t) { return (n + t - 1) / t; }

enum : int { AX = 0, AV = 3, AU = 6, AM = 7, AH = 8, AN = 9, ARHO = 10, AP = 11, AG = 12, AB = 27 };

// Derivative of the kernel shape (exact, for both precisions).
template <typename T>
__device__ __forceinline__ T dkern(T q) {
    return kern_dw(q);
}

// Adjoint of particle a's share of the pair (a, b).  wp = dpbar_a - dpbar_b
// and wE = dEbar_a - dEbar_b weight the pair's rate contributions; adj
// receives dJ/d(a's inputs).  Re-evaluates the forward exactly as
// pair_rates does so every branch matches.
template <typename T>
__device__ __forceinline__ void pair_adjoint(const T (&a)[kRecord], const T (&b)[kRecord], bool aL,
                                             T hdt, T gam, bool hancock, T na, const double* wp,
                                             double wE, double* adj) {
    // ---- forward (same operations as pair_rates)
    const T dx = mi_diff(b[0], a[0], a[0] - T(1));
    const T dy = mi_diff(b[1], a[1], a[1] - T(1));
    const T dz = mi_diff(b[2], a[2], a[2] - T(1));
    const T d[3] = {dx, dy, dz};
    const T r2 = sep2(dx, dy, dz);
    const T r = psqrt(r2);
    const bool ina = r2 < a[3] * a[3], inb = r2 < b[3] * b[3];
    const T qa = r * a[4], qb = r * b[4];
    const T wa = kern_w(qa), wb = kern_w(qb);
    const T ca = ina ? a[5] * wa : T(0);
    const T cb = inb ? b[5] * wb : T(0);
    const T* Ba = a + 26;
    const T* Bb = b + 26;
    const T Bda[3] = {(Ba[0] * dx + Ba[1] * dy) + Ba[2] * dz, (Ba[1] * dx + Ba[3] * dy) + Ba[4] * dz,
                      (Ba[2] * dx + Ba[4] * dy) + Ba[5] * dz};
    const T Bdb[3] = {(Bb[0] * dx + Bb[1] * dy) + Bb[2] * dz, (Bb[1] * dx + Bb[3] * dy) + Bb[4] * dz,
                      (Bb[2] * dx + Bb[4] * dy) + Bb[5] * dz};
    T A[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) A[k] = add_rn(mul_rn(ca, Bda[k]), mul_rn(cb, Bdb[k]));
    const T Aq = sep2(A[0], A[1], A[2]);
    if (!(Aq > T(0))) return;
    const T Am = psqrt(Aq);
    const T iA = pdiv(T(1), Am);
    const T nh[3] = {A[0] * iA, A[1] * iA, A[2] * iA};
    const T Hs = a[3] + b[3];
    const T sa = pdiv(a[3], Hs), sb = pdiv(b[3], Hs);
    T Fa[5], Fb[5];
    face_state(a, sa, dx, dy, dz, hdt, gam, hancock, Fa);
    face_state(b, sb, -dx, -dy, -dz, hdt, gam, hancock, Fb);
    const T Wa[5] = {a[6], a[8], a[9], a[10], a[7]};
    const T Wb[5] = {b[6], b[8], b[9], b[10], b[7]};
    // clamp sides: 0 inside, -1 clamped to the lower bound, +1 to the upper
    int ka[5], kb[5];
    T Ca[5], Cb[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        const T lo = min(Wa[f], Wb[f]), hi = max(Wa[f], Wb[f]);
        const T ma = max(Fa[f], lo), mb = max(Fb[f], lo);
        Ca[f] = min(ma, hi);
        Cb[f] = min(mb, hi);
        ka[f] = Fa[f] < lo ? -1 : (ma > hi ? 1 : 0);
        kb[f] = Fb[f] < lo ? -1 : (mb > hi ? 1 : 0);
    }
    const bool fallback = !(Ca[0] > T(0) && Ca[4] > T(0) && Cb[0] > T(0) && Cb[4] > T(0));
    T Ga[5], Gb[5];  // face states after clamp / fallback
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        Ga[f] = fallback ? Wa[f] : Ca[f];
        Gb[f] = fallback ? Wb[f] : Cb[f];
    }
    T FL[5], FR[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        FL[f] = aL ? Ga[f] : Gb[f];
        FR[f] = aL ? Gb[f] : Ga[f];
    }
    const T vL[3] = {aL ? Wa[1] : Wb[1], aL ? Wa[2] : Wb[2], aL ? Wa[3] : Wb[3]};
    const T vR[3] = {aL ? Wb[1] : Wa[1], aL ? Wb[2] : Wa[2], aL ? Wb[3] : Wa[3]};
    const T sL = aL ? sa : sb;
    const T sg = aL ? T(1) : T(-1);
    const T n[3] = {sg * nh[0], sg * nh[1], sg * nh[2]};
    const T vf[3] = {vL[0] + sL * (vR[0] - vL[0]), vL[1] + sL * (vR[1] - vL[1]),
                     vL[2] + sL * (vR[2] - vL[2])};
    const T vfn = (vf[0] * n[0] + vf[1] * n[1]) + vf[2] * n[2];
    const T uL = ((FL[1] - vf[0]) * n[0] + (FL[2] - vf[1]) * n[1]) + (FL[3] - vf[2]) * n[2];
    const T uR = ((FR[1] - vf[0]) * n[0] + (FR[2] - vf[1]) * n[1]) + (FR[3] - vf[2]) * n[2];
    const T rL = FL[0], PL = FL[4], rR = FR[0], PR = FR[4];
    const T cL = psqrt(pdiv(gam * PL, rL)), cR = psqrt(pdiv(gam * PR, rR));
    const T e1 = uL - cL, e2 = uR - cR, e3 = uL + cL, e4 = uR + cR;
    const T SL = min(e1, e2), SR = max(e3, e4);
    const T aLv = SL - uL, aRv = SR - uR;
    const T num = ((PR - PL) + rL * uL * aLv) - rR * uR * aRv;
    const T den = rL * aLv - rR * aRv;
    const T ss = pdiv(num, den);
    const T psr = PL + rL * aLv * (ss - uL);
    const T ps = psr < T(0) ? T(0) : psr;
    // ---- reverse, in double
    const double A_[3] = {A[0], A[1], A[2]};
    const double wpA = (wp[0] * A_[0] + wp[1] * A_[1]) + wp[2] * A_[2];
    // J = -ps (wp . A) - sg wE ps (ss + vfn) |A|
    const double b_ps = -wpA - (double)sg * wE * ((double)ss + vfn) * (double)Am;
    double bA[3] = {-(double)ps * wp[0], -(double)ps * wp[1], -(double)ps * wp[2]};
    double b_ss = -(double)sg * wE * (double)ps * (double)Am;
    const double b_vfn = b_ss;
    const double b_Am = -(double)sg * wE * (double)ps * ((double)ss + vfn);
    // ps = max(psr, 0)
    const double b_psr = psr < T(0) ? 0.0 : b_ps;
    // psr = PL + rL aL (ss - uL)
    double b_PL = b_psr, b_rL = b_psr * aLv * (ss - uL);
    double b_aL = b_psr * (double)rL * (ss - uL);
    b_ss += b_psr * (double)rL * aLv;
    double b_uL = -b_psr * (double)rL * aLv;
    double b_PR = 0.0, b_rR = 0.0, b_uR = 0.0, b_aR = 0.0;
    // ss = num / den
    const double b_num = b_ss / (double)den;
    const double b_den = -b_ss * (double)ss / (double)den;
    b_PR += b_num;
    b_PL -= b_num;
    b_rL += b_num * (double)uL * aLv;
    b_uL += b_num * (double)rL * aLv;
    b_aL += b_num * (double)rL * uL;
    b_rR -= b_num * (double)uR * aRv;
    b_uR -= b_num * (double)rR * aRv;
    b_aR -= b_num * (double)rR * uR;
    b_rL += b_den * aLv;
    b_aL += b_den * rL;
    b_rR -= b_den * aRv;
    b_aR -= b_den * rR;
    // aL = SL - uL, aR = SR - uR
    const double b_SL = b_aL, b_SR = b_aR;
    b_uL -= b_aL;
    b_uR -= b_aR;
    double b_cL = 0.0, b_cR = 0.0;
    if (e1 <= e2) {
        b_uL += b_SL;
        b_cL -= b_SL;
    } else {
        b_uR += b_SL;
        b_cR -= b_SL;
    }
    if (e3 >= e4) {
        b_uL += b_SR;
        b_cL += b_SR;
    } else {
        b_uR += b_SR;
        b_cR += b_SR;
    }
    // c = sqrt(gamma P / rho)
    if (cL > T(0)) {
        b_PL += b_cL * (double)gam / (2.0 * (double)cL * (double)rL);
        b_rL -= b_cL * (double)cL / (2.0 * (double)rL);
    }
    if (cR > T(0)) {
        b_PR += b_cR * (double)gam / (2.0 * (double)cR * (double)rR);
        b_rR -= b_cR * (double)cR / (2.0 * (double)rR);
    }
    double bFL[5] = {b_rL, 0.0, 0.0, 0.0, b_PL};
    double bFR[5] = {b_rR, 0.0, 0.0, 0.0, b_PR};
    double bvf[3], bn[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        bFL[1 + k] = b_uL * n[k];
        bFR[1 + k] = b_uR * n[k];
        bvf[k] = -(b_uL + b_uR) * n[k] + b_vfn * n[k];
        bn[k] = b_uL * ((double)FL[1 + k] - vf[k]) + b_uR * ((double)FR[1 + k] - vf[k]) + b_vfn * vf[k];
    }
    // vf = vL + sL (vR - vL)
    double bvL[3], bvR[3], b_sL = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        bvL[k] = bvf[k] * (1.0 - (double)sL);
        bvR[k] = bvf[k] * (double)sL;
        b_sL += bvf[k] * ((double)vR[k] - vL[k]);
    }
    // back to a / b labels
    double bGa[5], bGb[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        bGa[f] = aL ? bFL[f] : bFR[f];
        bGb[f] = aL ? bFR[f] : bFL[f];
    }
    double bWa[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 3; ++k) bWa[1 + k] += aL ? bvL[k] : bvR[k];
    double b_sa = aL ? b_sL : 0.0, b_sb = aL ? 0.0 : b_sL;
    // normal n = sg A / |A|, and |A| itself
    double bnh[3] = {sg * bn[0], sg * bn[1], sg * bn[2]};
    const double nb_dot = (bnh[0] * nh[0] + bnh[1] * nh[1]) + bnh[2] * nh[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) bA[k] += (bnh[k] - nb_dot * nh[k]) / (double)Am + b_Am * nh[k];
    // fallback and clamps
    double bFa[5], bFb[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        if (fallback) {
            bWa[f] += bGa[f];
            bFa[f] = 0.0;
            bFb[f] = 0.0;
        } else {
            bFa[f] = 0.0;
            bFb[f] = 0.0;
            // a's face value
            if (ka[f] == 0)
                bFa[f] = bGa[f];
            else if (ka[f] < 0)
                bWa[f] += (Wa[f] <= Wb[f]) ? bGa[f] : 0.0;  // lower bound min(Wa, Wb)
            else
                bWa[f] += (Wa[f] >= Wb[f]) ? bGa[f] : 0.0;  // upper bound max(Wa, Wb)
            // b's face value (its bounds can be a's values)
            if (kb[f] == 0)
                bFb[f] = bGb[f];
            else if (kb[f] < 0)
                bWa[f] += (Wa[f] <= Wb[f]) ? bGb[f] : 0.0;
            else
                bWa[f] += (Wa[f] >= Wb[f]) ? bGb[f] : 0.0;
        }
    }
    // face states: F_a = W_a + g_a . (s_a d) + hdt D_a ; F_b = W_b + g_b . (s_b (-d)) + hdt D_b
    double bd[3] = {0.0, 0.0, 0.0};
    double bg[15];
#pragma unroll
    for (int q = 0; q < 15; ++q) bg[q] = 0.0;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        bWa[f] += bFa[f];
        const double g0 = a[11 + 3 * f], g1 = a[12 + 3 * f], g2 = a[13 + 3 * f];
        bg[3 * f] += bFa[f] * sa * dx;
        bg[3 * f + 1] += bFa[f] * sa * dy;
        bg[3 * f + 2] += bFa[f] * sa * dz;
        b_sa += bFa[f] * ((g0 * dx + g1 * dy) + g2 * dz);
        bd[0] += bFa[f] * sa * g0;
        bd[1] += bFa[f] * sa * g1;
        bd[2] += bFa[f] * sa * g2;
        const double h0 = b[11 + 3 * f], h1 = b[12 + 3 * f], h2 = b[13 + 3 * f];
        b_sb -= bFb[f] * ((h0 * dx + h1 * dy) + h2 * dz);
        bd[0] -= bFb[f] * sb * h0;
        bd[1] -= bFb[f] * sb * h1;
        bd[2] -= bFb[f] * sb * h2;
    }
    if (hancock) {
        const double div = ((double)a[11 + 3] + a[11 + 7]) + a[11 + 11];
        const double rho = a[6], P = a[7];
        const double b_div = bFa[0] * hdt * (-rho) + bFa[4] * hdt * (-(double)gam * P);
        bWa[0] += bFa[0] * hdt * (-div);
        for (int k = 0; k < 3; ++k) {
            bWa[0] += bFa[1 + k] * hdt * (double)a[11 + 12 + k] / (rho * rho);
            bg[12 + k] += bFa[1 + k] * hdt * (-1.0 / rho);
        }
        bWa[4] += bFa[4] * hdt * (-(double)gam * div);
        bg[3] += b_div;
        bg[7] += b_div;
        bg[11] += b_div;
    }
    // s_a = Ha / Hs, s_b = Hb / Hs
    const double Hsd = Hs;
    double bHa = b_sa * (double)b[3] / (Hsd * Hsd) - b_sb * (double)b[3] / (Hsd * Hsd);
    // A = ca B_a d + cb B_b d
    const double bca = (bA[0] * Bda[0] + bA[1] * Bda[1]) + bA[2] * Bda[2];
    const double bcb = (bA[0] * Bdb[0] + bA[1] * Bdb[1]) + bA[2] * Bdb[2];
    const double bBda[3] = {(double)ca * bA[0], (double)ca * bA[1], (double)ca * bA[2]};
    const double bBdb[3] = {(double)cb * bA[0], (double)cb * bA[1], (double)cb * bA[2]};
    double bB[6];
    bB[0] = bBda[0] * dx;
    bB[1] = bBda[0] * dy + bBda[1] * dx;
    bB[2] = bBda[0] * dz + bBda[2] * dx;
    bB[3] = bBda[1] * dy;
    bB[4] = bBda[1] * dz + bBda[2] * dy;
    bB[5] = bBda[2] * dz;
    bd[0] += (Ba[0] * bBda[0] + Ba[1] * bBda[1]) + Ba[2] * bBda[2];
    bd[1] += (Ba[1] * bBda[0] + Ba[3] * bBda[1]) + Ba[4] * bBda[2];
    bd[2] += (Ba[2] * bBda[0] + Ba[4] * bBda[1]) + Ba[5] * bBda[2];
    bd[0] += (Bb[0] * bBdb[0] + Bb[1] * bBdb[1]) + Bb[2] * bBdb[2];
    bd[1] += (Bb[1] * bBdb[0] + Bb[3] * bBdb[1]) + Bb[4] * bBdb[2];
    bd[2] += (Bb[2] * bBdb[0] + Bb[4] * bBdb[1]) + Bb[5] * bBdb[2];
    // ca = knorm_a w(r / Ha) inside a's support, cb likewise
    double br = 0.0, bka = 0.0;
    if (ina) {
        bka = bca * wa;
        const double bq = bca * (double)a[5] * dkern(qa);
        br += bq * (double)a[4];
        bHa -= bq * (double)qa / (double)a[3];
    }
    if (inb) br += bcb * (double)b[5] * dkern(qb) * (double)b[4];
    // knorm = 8 / (pi H^3 n^2)
    bHa += bka * (-3.0 * (double)a[5] / (double)a[3]);
    const double bna = bka * (-2.0 * (double)a[5] / (double)na);
    if (r > T(0)) {
        bd[0] += br * dx / (double)r;
        bd[1] += br * dy / (double)r;
        bd[2] += br * dz / (double)r;
    }
    // d = x_b - x_a
    adj[AX] -= bd[0];
    adj[AX + 1] -= bd[1];
    adj[AX + 2] -= bd[2];
    adj[AH] += bHa;
    adj[AN] += bna;
    adj[ARHO] += bWa[0];
    adj[AV] += bWa[1];
    adj[AV + 1] += bWa[2];
    adj[AV + 2] += bWa[3];
    adj[AP] += bWa[4];
#pragma unroll
    for (int q = 0; q < 15; ++q) adj[AG + q] += bg[q];
#pragma unroll
    for (int q = 0; q < 6; ++q) adj[AB + q] += bB[q];
}

// Adjoint of the flux pass: per particle over its pairs (N_i then R_i).
template <typename T>
__global__ void __launch_bounds__(128)
    k_flux_adj(int N, const T* __restrict__ rec, const T* __restrict__ sn, const long long* __restrict__ sid,
               const int* __restrict__ sbox, const unsigned* __restrict__ nbr, const int* __restrict__ ncount,
               const unsigned* __restrict__ rnbr, const int* __restrict__ rcount, KParams p,
               const double* __restrict__ dt_use, const double* __restrict__ wgt, double* __restrict__ adj) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    T a[kRecord];
    load_rec(rec + (size_t)i * kRecord, a);
    const long long idi = sid[i];
    const T hdt = (T)(0.5 * dt_use[sbox[i]]);
    const T gam = (T)p.gamma;
    const bool hancock = p.hancock != 0;
    const T na = sn[i];
    const double wi[4] = {wgt[4 * (size_t)i], wgt[4 * (size_t)i + 1], wgt[4 * (size_t)i + 2],
                          wgt[4 * (size_t)i + 3]};
    double acc[kAdj];
#pragma unroll
    for (int q = 0; q < kAdj; ++q) acc[q] = 0.0;
    for (int list = 0; list < 2; ++list) {
        const unsigned* L = list == 0 ? nbr + (size_t)i * p.cap : rnbr + (size_t)i * p.rcap;
        const int cnt = list == 0 ? min(ncount[i], p.cap) : min(rcount[i], p.rcap);
        for (int k = 0; k < cnt; ++k) {
            const int j = (int)L[k];
            T b[kRecord];
            load_rec(rec + (size_t)j * kRecord, b);
            const double wp[3] = {wi[0] - wgt[4 * (size_t)j], wi[1] - wgt[4 * (size_t)j + 1],
                                  wi[2] - wgt[4 * (size_t)j + 2]};
            const double wE = wi[3] - wgt[4 * (size_t)j + 3];
            pair_adjoint(a, b, idi < sid[j], hdt, gam, hancock, na, wp, wE, acc);
        }
    }
    double* o = adj + (size_t)i * kAdj;
#pragma unroll
    for (int q = 0; q < kAdj; ++q) o[q] += acc[q];
}

// Caller-order adjoint weights of the rates -> sorted [N][4].
__global__ void k_gather_wgt(int N, const unsigned* __restrict__ orig, const double* __restrict__ dpbar,
                             const double* __restrict__ dEbar, double* __restrict__ wgt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned o = orig[i];
    wgt[4 * (size_t)i] = dpbar[o];
    wgt[4 * (size_t)i + 1] = dpbar[(size_t)N + o];
    wgt[4 * (size_t)i + 2] = dpbar[2 * (size_t)N + o];
    wgt[4 * (size_t)i + 3] = dEbar[o];
}

// Sorted adjoint records -> caller-order outputs (any pointer may be null).
__global__ void k_adj_out_flux(int N, const unsigned* __restrict__ orig, const double* __restrict__ adj,
                               double* __restrict__ xbar, double* __restrict__ hbar,
                               double* __restrict__ nbar, double* __restrict__ Wbar,
                               double* __restrict__ gbar, double* __restrict__ Bbar) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned o = orig[i];
    const double* a = adj + (size_t)i * kAdj;
    if (xbar)
        for (int k = 0; k < 3; ++k) xbar[(size_t)k * N + o] = a[AX + k];
    if (hbar) hbar[o] = a[AH];
    if (nbar) nbar[o] = a[AN];
    if (Wbar) {
        Wbar[o] = a[ARHO];
        for (int k = 0; k < 3; ++k) Wbar[(size_t)(1 + k) * N + o] = a[AV + k];
        Wbar[4 * (size_t)N + o] = a[AP];
    }
    if (gbar)
        for (int q = 0; q < 15; ++q) gbar[(size_t)q * N + o] = a[AG + q];
    if (Bbar)
        for (int q = 0; q < 6; ++q) Bbar[(size_t)q * N + o] = a[AB + q];
}

}  // namespace

cudaError_t ensure_adjoint_scratch(Ctx& c) {
    if (c.adj) return cudaSuccess;
    const size_t Nz = (size_t)c.N;
    const size_t bytes = sizeof(double) * Nz * (kAdj + 4 + kSeed) + sizeof(int) * Nz * 10 +
                         (size_t)(c.precision == GZ_FP64 ? 8 : 4) * Nz * kGInfo + 4 * 256;
    char* base = nullptr;
    cudaError_t e = cudaMalloc((void**)&base, bytes);
    if (e != cudaSuccess) return e;
    c.adj_arena = base;
    c.adj = (double*)base;
    base += sizeof(double) * Nz * kAdj;
    c.wgt = (double*)base;
    base += sizeof(double) * Nz * 4;
    c.seeds = (double*)base;
    base += sizeof(double) * Nz * kSeed;
    c.lim = (int*)base;
    base += sizeof(int) * Nz * 10;
    c.ginfo = base;
    return cudaSuccess;
}

template <typename T>
cudaError_t run_flux_adjoint(Ctx& c, const double* dpbar, const double* dEbar) {
    c.launches += 2;
    cudaMemsetAsync(c.adj, 0, sizeof(double) * (size_t)c.N * kAdj, c.stream);
    k_gather_wgt<<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, c.vals, dpbar, dEbar, c.wgt);
    k_flux_adj<T><<<blocks(c.N, 128), 128, 0, c.stream>>>(c.N, (const T*)c.rec, (const T*)c.sn, c.sid,
                                                           c.sbox, c.nbr, c.ncount, c.rnbr, c.rcount,
                                                           kparams(c), c.dt_use, c.wgt, c.adj);
    return cudaGetLastError();
}

cudaError_t run_adj_out_flux(Ctx& c, double* xbar, double* hbar, double* nbar, double* Wbar, double* gbar,
                             double* Bbar) {
    c.launches += 1;
    k_adj_out_flux<<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, c.vals, c.adj, xbar, hbar, nbar, Wbar, gbar,
                                                           Bbar);
    return cudaGetLastError();
}

template cudaError_t run_flux_adjoint<float>(Ctx&, const double*, const double*);
template cudaError_t run_flux_adjoint<double>(Ctx&, const double*, const double*);

}  // namespace gz
