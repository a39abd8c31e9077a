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
// Adjoint record per particle (working precision, sorted order), kAdj values:
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
// pair_rates does so every branch matches.  inv_na = 1/n_a and irho =
// 1/rho_a are the particle's own reciprocals; every division of the reverse
// sweep is a product with a reciprocal (pdiv: hardware reciprocal in FP32).
template <typename T>
__device__ __forceinline__ void pair_adjoint(const T (&a)[kRecord], const T (&b)[kRecord], bool aL,
                                             T hdt, T gam, bool hancock, T inv_na, T irho, const T* wp,
                                             T wE, T* adj) {
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
    T inca[5], incb[5];
    hancock_inc(a, hdt, gam, hancock, inca);
    hancock_inc(b, hdt, gam, hancock, incb);
    face_state(a, sa, dx, dy, dz, inca, Fa);
    face_state(b, sb, -dx, -dy, -dz, incb, Fb);
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
    // ---- reverse, in the working precision
    const T A_[3] = {A[0], A[1], A[2]};
    const T wpA = (wp[0] * A_[0] + wp[1] * A_[1]) + wp[2] * A_[2];
    // J = -ps (wp . A) - sg wE ps (ss + vfn) |A|
    const T b_ps = -wpA - (T)sg * wE * ((T)ss + vfn) * (T)Am;
    T bA[3] = {-(T)ps * wp[0], -(T)ps * wp[1], -(T)ps * wp[2]};
    T b_ss = -(T)sg * wE * (T)ps * (T)Am;
    const T b_vfn = b_ss;
    const T b_Am = -(T)sg * wE * (T)ps * ((T)ss + vfn);
    // ps = max(psr, 0)
    const T b_psr = psr < T(0) ? T(0) : b_ps;
    // psr = PL + rL aL (ss - uL)
    T b_PL = b_psr, b_rL = b_psr * aLv * (ss - uL);
    T b_aL = b_psr * (T)rL * (ss - uL);
    b_ss += b_psr * (T)rL * aLv;
    T b_uL = -b_psr * (T)rL * aLv;
    T b_PR = T(0), b_rR = T(0), b_uR = T(0), b_aR = T(0);
    // ss = num / den
    const T b_num = b_ss * pdiv(T(1), den);
    const T b_den = -b_num * ss;
    b_PR += b_num;
    b_PL -= b_num;
    b_rL += b_num * (T)uL * aLv;
    b_uL += b_num * (T)rL * aLv;
    b_aL += b_num * (T)rL * uL;
    b_rR -= b_num * (T)uR * aRv;
    b_uR -= b_num * (T)rR * aRv;
    b_aR -= b_num * (T)rR * uR;
    b_rL += b_den * aLv;
    b_aL += b_den * rL;
    b_rR -= b_den * aRv;
    b_aR -= b_den * rR;
    // aL = SL - uL, aR = SR - uR
    const T b_SL = b_aL, b_SR = b_aR;
    b_uL -= b_aL;
    b_uR -= b_aR;
    T b_cL = T(0), b_cR = T(0);
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
        const T h = pdiv(T(0.5), rL);
        b_PL += b_cL * gam * pdiv(h, cL);
        b_rL -= b_cL * cL * h;
    }
    if (cR > T(0)) {
        const T h = pdiv(T(0.5), rR);
        b_PR += b_cR * gam * pdiv(h, cR);
        b_rR -= b_cR * cR * h;
    }
    T bFL[5] = {b_rL, T(0), T(0), T(0), b_PL};
    T bFR[5] = {b_rR, T(0), T(0), T(0), b_PR};
    T bvf[3], bn[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        bFL[1 + k] = b_uL * n[k];
        bFR[1 + k] = b_uR * n[k];
        bvf[k] = -(b_uL + b_uR) * n[k] + b_vfn * n[k];
        bn[k] = b_uL * ((T)FL[1 + k] - vf[k]) + b_uR * ((T)FR[1 + k] - vf[k]) + b_vfn * vf[k];
    }
    // vf = vL + sL (vR - vL)
    T bvL[3], bvR[3], b_sL = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        bvL[k] = bvf[k] * (T(1) - (T)sL);
        bvR[k] = bvf[k] * (T)sL;
        b_sL += bvf[k] * ((T)vR[k] - vL[k]);
    }
    // back to a / b labels
    T bGa[5], bGb[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        bGa[f] = aL ? bFL[f] : bFR[f];
        bGb[f] = aL ? bFR[f] : bFL[f];
    }
    T bWa[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 3; ++k) bWa[1 + k] += aL ? bvL[k] : bvR[k];
    T b_sa = aL ? b_sL : T(0), b_sb = aL ? T(0) : b_sL;
    // normal n = sg A / |A|, and |A| itself
    T bnh[3] = {sg * bn[0], sg * bn[1], sg * bn[2]};
    const T nb_dot = (bnh[0] * nh[0] + bnh[1] * nh[1]) + bnh[2] * nh[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) bA[k] += (bnh[k] - nb_dot * nh[k]) * iA + b_Am * nh[k];
    // fallback and clamps; a bound min / max(W_L, W_R) passes its adjoint to
    // L on a tie (the rule the derivative oracle's where() takes), so the two
    // sides of a pair never both claim it
    T bFa[5], bFb[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        bFa[f] = T(0);
        bFb[f] = T(0);
        if (fallback) {
            bWa[f] += bGa[f];
        } else {
            const bool loA = aL ? (Wa[f] <= Wb[f]) : (Wa[f] < Wb[f]);
            const bool hiA = aL ? (Wa[f] >= Wb[f]) : (Wa[f] > Wb[f]);
            // a's face value
            if (ka[f] == 0)
                bFa[f] = bGa[f];
            else
                bWa[f] += ((ka[f] < 0) ? loA : hiA) ? bGa[f] : T(0);
            // b's face value (its bounds can be a's values)
            if (kb[f] == 0)
                bFb[f] = bGb[f];
            else
                bWa[f] += ((kb[f] < 0) ? loA : hiA) ? bGb[f] : T(0);
        }
    }
    // face states: F_a = W_a + g_a . (s_a d) + inc_a ; F_b = W_b + g_b . (s_b (-d)) + inc_b
    T bd[3] = {T(0), T(0), T(0)};
    T bg[15];
#pragma unroll
    for (int q = 0; q < 15; ++q) bg[q] = T(0);
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        bWa[f] += bFa[f];
        const T g0 = a[11 + 3 * f], g1 = a[12 + 3 * f], g2 = a[13 + 3 * f];
        bg[3 * f] += bFa[f] * sa * dx;
        bg[3 * f + 1] += bFa[f] * sa * dy;
        bg[3 * f + 2] += bFa[f] * sa * dz;
        b_sa += bFa[f] * ((g0 * dx + g1 * dy) + g2 * dz);
        bd[0] += bFa[f] * sa * g0;
        bd[1] += bFa[f] * sa * g1;
        bd[2] += bFa[f] * sa * g2;
        const T h0 = b[11 + 3 * f], h1 = b[12 + 3 * f], h2 = b[13 + 3 * f];
        b_sb -= bFb[f] * ((h0 * dx + h1 * dy) + h2 * dz);
        bd[0] -= bFb[f] * sb * h0;
        bd[1] -= bFb[f] * sb * h1;
        bd[2] -= bFb[f] * sb * h2;
    }
    if (hancock) {  // inc_a = (dt/2)(-rho div v, -grad P / rho, -gamma P div v)
        const T div = (a[11 + 3] + a[11 + 7]) + a[11 + 11];
        const T rho = a[6], P = a[7];
        const T b_div = bFa[0] * hdt * (-rho) + bFa[4] * hdt * (-gam * P);
        bWa[0] += bFa[0] * hdt * (-div);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            bWa[0] += bFa[1 + k] * hdt * a[11 + 12 + k] * irho * irho;
            bg[12 + k] -= bFa[1 + k] * hdt * irho;
        }
        bWa[4] += bFa[4] * hdt * (-gam * div);
        bg[3] += b_div;
        bg[7] += b_div;
        bg[11] += b_div;
    }
    // s_a = Ha / Hs, s_b = Hb / Hs
    const T Hsd = Hs;
    T bHa = (b_sa - b_sb) * b[3] * pdiv(T(1), Hsd * Hsd);
    // A = ca B_a d + cb B_b d
    const T bca = (bA[0] * Bda[0] + bA[1] * Bda[1]) + bA[2] * Bda[2];
    const T bcb = (bA[0] * Bdb[0] + bA[1] * Bdb[1]) + bA[2] * Bdb[2];
    const T bBda[3] = {(T)ca * bA[0], (T)ca * bA[1], (T)ca * bA[2]};
    const T bBdb[3] = {(T)cb * bA[0], (T)cb * bA[1], (T)cb * bA[2]};
    T bB[6];
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
    T br = T(0), bka = T(0);
    if (ina) {
        bka = bca * wa;
        const T bq = bca * (T)a[5] * dkern(qa);
        br += bq * (T)a[4];
        bHa -= bq * qa * a[4];
    }
    if (inb) br += bcb * (T)b[5] * dkern(qb) * (T)b[4];
    // knorm = 8 / (pi H^3 n^2)
    bHa += bka * (T(-3) * a[5] * a[4]);
    const T bna = bka * (-T(2) * a[5] * inv_na);
    if (r > T(0)) {
        const T bri = br * pdiv(T(1), r);
        bd[0] += bri * dx;
        bd[1] += bri * dy;
        bd[2] += bri * dz;
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
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 3 : 1)
    k_flux_adj(int N, const T* __restrict__ rec, const T* __restrict__ sn, const long long* __restrict__ sid,
               const int* __restrict__ sbox, const unsigned* __restrict__ nbr, const int* __restrict__ ncount,
               const unsigned* __restrict__ rnbr, const int* __restrict__ rcount, KParams p,
               const double* __restrict__ dt_use, const T* __restrict__ wgt, T* __restrict__ adj) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    T a[kRecord];
    load_rec(rec + (size_t)i * kRecord, a);
    const long long idi = sid[i];
    const T hdt = (T)(0.5 * dt_use[sbox[i]]);
    const T gam = (T)p.gamma;
    const bool hancock = p.hancock != 0;
    const T inv_na = pdiv(T(1), sn[i]), irho = pdiv(T(1), a[6]);
    T wi[4];
    load4(wgt + 4 * (size_t)i, wi);
    T acc[kAdj];
#pragma unroll
    for (int q = 0; q < kAdj; ++q) acc[q] = T(0);
    for (int list = 0; list < 2; ++list) {
        const unsigned* L = list == 0 ? nbr + 4 * (size_t)i : rnbr + 4 * (size_t)i;
        const int cnt = list == 0 ? min(ncount[i], p.cap) : min(rcount[i], p.rcap);
        for (int k = 0; k < cnt; ++k) {
            const int j = (int)L[lcol(k, N)];
            T b[kRecord];
            load_rec(rec + (size_t)j * kRecord, b);
            T wj[4];
            load4(wgt + 4 * (size_t)j, wj);
            const T wp[3] = {wi[0] - wj[0], wi[1] - wj[1], wi[2] - wj[2]};
            const T wE = wi[3] - wj[3];
            pair_adjoint(a, b, idi < sid[j], hdt, gam, hancock, inv_na, irho, wp, wE, acc);
        }
    }
    T* o = adj + (size_t)i * kAdj;
#pragma unroll
    for (int q = 0; q < kAdj; ++q) o[q] += acc[q];
}

// Caller-order adjoint weights of the rates -> sorted [N][4].
template <typename T>
__global__ void k_gather_wgt(int N, const unsigned* __restrict__ orig, const double* __restrict__ dpbar,
                             const double* __restrict__ dEbar, T* __restrict__ wgt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned o = orig[i];
    store4(wgt + 4 * (size_t)i, (T)dpbar[o], (T)dpbar[(size_t)N + o], (T)dpbar[2 * (size_t)N + o], (T)dEbar[o]);
}

// Sorted adjoint records -> caller-order outputs (any pointer may be null).
template <typename T>
__global__ void k_adj_out_flux(int N, const unsigned* __restrict__ orig, const T* __restrict__ adj,
                               double* __restrict__ xbar, double* __restrict__ hbar,
                               double* __restrict__ nbar, double* __restrict__ Wbar,
                               double* __restrict__ gbar, double* __restrict__ Bbar) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned o = orig[i];
    const T* a = adj + (size_t)i * kAdj;
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

// ------------------------------------------------------------- update
// O14 reversed.  v' = v + dt dp/m, x' = x + dt (v + v')/2,
// u' = u + |v|^2/2 + dt dE/m - |v'|^2/2 (a floored u' is a constant).
template <typename T>
__global__ void k_update_adj(int N, Sorted<T> s, const double* __restrict__ dpdt,
                             const double* __restrict__ dEdt, const double* __restrict__ dt_use,
                             gz_particles gend, T* __restrict__ adj, T* __restrict__ wgt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned o = s.orig[i];
    const T dt = (T)dt_use[s.box[i]];
    const T m = s.m[i];
    const T v[3] = {s.vx[i], s.vy[i], s.vz[i]};
    const T dp[3] = {(T)dpdt[i], (T)dpdt[(size_t)N + i], (T)dpdt[2 * (size_t)N + i]};
    const T dE = (T)dEdt[i];
    // forward update in the working precision, for the floor decision
    T X = s.x[i], Y = s.y[i], Z = s.z[i], VX = v[0], VY = v[1], VZ = v[2], U = s.u[i];
    update_one(m, X, Y, Z, VX, VY, VZ, U, dpdt[i], dpdt[(size_t)N + i], dpdt[2 * (size_t)N + i],
               dEdt[i], dt_use[s.box[i]]);
    const bool floored = !(U > T(0));
    const T im = T(1) / m;
    T vn[3];
    for (int k = 0; k < 3; ++k) vn[k] = v[k] + dt * dp[k] * im;
    const T xb[3] = {gend.x ? ((const T*)gend.x)[o] : T(0), gend.y ? ((const T*)gend.y)[o] : T(0),
                     gend.z ? ((const T*)gend.z)[o] : T(0)};
    const T vb[3] = {gend.vx ? ((const T*)gend.vx)[o] : T(0), gend.vy ? ((const T*)gend.vy)[o] : T(0),
                     gend.vz ? ((const T*)gend.vz)[o] : T(0)};
    const T ub = (gend.u && !floored) ? ((const T*)gend.u)[o] : T(0);
    T* a = adj + (size_t)i * kAdj;
    T mb = -ub * dt * dE * im * im;
    T wv[3];
    for (int k = 0; k < 3; ++k) {
        a[AX + k] += xb[k];
        a[AV + k] += vb[k] + dt * xb[k] + ub * (v[k] - vn[k]);
        const T w = vb[k] + T(0.5) * dt * xb[k];
        wv[k] = dt * im * (w - ub * vn[k]);
        mb += -(vn[k] - v[k]) * im * w + ub * vn[k] * (vn[k] - v[k]) * im;
    }
    store4(wgt + 4 * (size_t)i, wv[0], wv[1], wv[2], ub * dt * im);
    a[AU] += ub;
    a[AM] += mb;
}

// ---------------------------------------------------------- gradients
// Seeds of particle i's gradient pass: from the adjoints of its limited
// gradients and of B, through the limiter (active constraint only), g = B S
// and B = E^-1.  Adds i's own terms; stores what i's neighbours gather.
// seeds: [0,15) Sbar, [15,21) Ebar (xx xy xz yy yz zz), then per field f
// at 21 + 5 f: xbar (3) and Hbar of the active neighbour, fbar of the
// extreme particle.
template <typename T>
__global__ void __launch_bounds__(128)
    k_grad_seeds(int N, Sorted<T> s, const T* __restrict__ rec, const T* __restrict__ ginfo,
                 const int* __restrict__ lim, const unsigned* __restrict__ nbr,
                 const int* __restrict__ ncount, KParams p, T* __restrict__ adj,
                 T* __restrict__ seeds, unsigned long long* __restrict__ lbloom) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    T* a = adj + (size_t)i * kAdj;
    T* sd = seeds + (size_t)i * kSeed;
    unsigned long long bloom = 0ull;
    const T* G = ginfo + (size_t)i * kGInfo;
    const T* R = rec + (size_t)i * kRecord;
    const P4<T> me = s.pos[i];
    const T xi = me.x, yi = me.y, zi = me.z, Hi = me.w;
    const T xim1 = xi - T(1), yim1 = yi - T(1), zim1 = zi - T(1);
    const P4<T> pm = s.prim[i];
    const T Wi[5] = {pm.x, pm.y, pm.z, pm.w, s.prim2[i].x};
    const T Bs[6] = {R[26], R[27], R[28], R[29], R[30], R[31]};
    T fbi[5] = {0, 0, 0, 0, 0};
    T xbi[3] = {0, 0, 0};
    T Hbi = T(0.0), nbi = T(0.0);
    T gb[15];
    T Bb[6];
    for (int q = 0; q < 6; ++q) Bb[q] = (T)a[AB + q];
    // the limiter part of the record (28-55) starts at zero: 16-byte stores
    // (rows are 32-byte aligned, 56 values a row)
#pragma unroll
    for (int q = 28; q < kSeed; q += 4) store4(sd + q, T(0), T(0), T(0), T(0));
    const T beta = p.beta;
    for (int f = 0; f < 5; ++f) {
        const T al = G[30 + f];
        const T g[3] = {G[3 * f], G[3 * f + 1], G[3 * f + 2]};
        const T ghb[3] = {(T)a[AG + 3 * f], (T)a[AG + 3 * f + 1], (T)a[AG + 3 * f + 2]};
        for (int k = 0; k < 3; ++k) gb[3 * f + k] = al * ghb[k];
        const T alb = (ghb[0] * g[0] + ghb[1] * g[1]) + ghb[2] * g[2];
        const int j = lim[(size_t)i * 10 + f];
        if (j >= 0 && alb != T(0.0)) {
            const int k = lim[(size_t)i * 10 + 5 + f];
            const T D = G[35 + f];
            const T c1 = alb * beta / D;
            if (k == i) {
                fbi[f] += c1;
            } else {
                sd[28 + 5 * f + 4] = c1;
                bloom |= 1ull << (k & 63);
            }
            fbi[f] -= c1;
            bloom |= 1ull << (j & 63);
            const T Db = -alb * al / D;
            const P4<T> qj = s.pos[j];
            const T dx = mi_diff(qj.x, xi, xim1), dy = mi_diff(qj.y, yi, yim1),
                         dz = mi_diff(qj.z, zi, zim1);
            const T Hj = qj.w, Hs = (T)Hi + Hj;
            const T sij = (T)Hi / Hs;
            const T o[3] = {sij * dx, sij * dy, sij * dz};
            for (int kk = 0; kk < 3; ++kk) gb[3 * f + kk] += Db * o[kk];
            const T ob[3] = {Db * g[0], Db * g[1], Db * g[2]};
            const T sb = (ob[0] * dx + ob[1] * dy) + ob[2] * dz;
            Hbi += sb * Hj / (Hs * Hs);
            sd[28 + 5 * f + 3] = -sb * (T)Hi / (Hs * Hs);
            for (int kk = 0; kk < 3; ++kk) {
                sd[28 + 5 * f + kk] = ob[kk] * sij;
                xbi[kk] -= ob[kk] * sij;
            }
        }
    }
    // g = B S
    const bool singular = Bs[0] == T(0.0) && Bs[1] == T(0.0) && Bs[2] == T(0.0) && Bs[3] == T(0.0) &&
                          Bs[4] == T(0.0) && Bs[5] == T(0.0);
    T Sb[15];
    for (int f = 0; f < 5; ++f) {
        const T S0 = G[15 + 3 * f], S1 = G[16 + 3 * f], S2 = G[17 + 3 * f];
        const T g0 = gb[3 * f], g1 = gb[3 * f + 1], g2 = gb[3 * f + 2];
        Bb[0] += g0 * S0;
        Bb[1] += g0 * S1 + g1 * S0;
        Bb[2] += g0 * S2 + g2 * S0;
        Bb[3] += g1 * S1;
        Bb[4] += g1 * S2 + g2 * S1;
        Bb[5] += g2 * S2;
        Sb[3 * f] = Bs[0] * g0 + Bs[1] * g1 + Bs[2] * g2;
        Sb[3 * f + 1] = Bs[1] * g0 + Bs[3] * g1 + Bs[4] * g2;
        Sb[3 * f + 2] = Bs[2] * g0 + Bs[4] * g1 + Bs[5] * g2;
    }
    // B = E^-1: Ebar = -B Bbar B (full symmetric matrices)
    const T Bm[3][3] = {{Bs[0], Bs[1], Bs[2]}, {Bs[1], Bs[3], Bs[4]}, {Bs[2], Bs[4], Bs[5]}};
    const T Pm[3][3] = {{Bb[0], T(0.5) * Bb[1], T(0.5) * Bb[2]},
                             {T(0.5) * Bb[1], Bb[3], T(0.5) * Bb[4]},
                             {T(0.5) * Bb[2], T(0.5) * Bb[4], Bb[5]}};
    T T1[3][3], Em[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) T1[r][c] = (Pm[r][0] * Bm[0][c] + Pm[r][1] * Bm[1][c]) + Pm[r][2] * Bm[2][c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Em[r][c] = -((Bm[r][0] * T1[0][c] + Bm[r][1] * T1[1][c]) + Bm[r][2] * T1[2][c]);
    T Eb[6] = {Em[0][0], Em[0][1] + Em[1][0], Em[0][2] + Em[2][0], Em[1][1], Em[1][2] + Em[2][1], Em[2][2]};
    if (singular) {
        for (int q = 0; q < 6; ++q) Eb[q] = T(0.0);
        for (int q = 0; q < 15; ++q) Sb[q] = T(0.0);
    }
    // own terms of E = sum psi d d^T and S_f = sum (f_j - f_i) psi d
    const T ni = s.n[i];
    const T iH = T(1) / Hi;
    const T norm = T(8.0 / kPi) * iH * iH * iH / ni;
    // record read by every j with j in N_i (k_grad_gather)
    {  // (16-byte stores)
        const T r0[28] = {Sb[0], Sb[1], Sb[2], Sb[3], Sb[4], Sb[5], Sb[6], Sb[7], Sb[8], Sb[9],
                          Sb[10], Sb[11], Sb[12], Sb[13], Sb[14], Eb[0], Eb[1], Eb[2], Eb[3], Eb[4],
                          Eb[5], norm, Wi[0], Wi[1], Wi[2], Wi[3], Wi[4], T(0)};
#pragma unroll
        for (int q = 0; q < 28; q += 4) store4(sd + q, r0[q], r0[q + 1], r0[q + 2], r0[q + 3]);
    }
    lbloom[i] = bloom;
    T normb = T(0.0);
    const int cnt = min(ncount[i], p.cap);
    const unsigned* L = nbr + 4 * (size_t)i;
    for (int k0 = 0; k0 < cnt; k0 += 4) {  // four neighbours' loads in flight at a time
      const uint4 jj = col4(L, k0, N);
      const unsigned js[4] = {jj.x, jj.y, jj.z, jj.w};
      P4<T> qv[4], pv[4];
      T Pv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
          if (k0 + u < cnt) {
              qv[u] = s.pos[js[u]];
              pv[u] = s.prim[js[u]];
              Pv[u] = s.prim2[js[u]].x;
          }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (k0 + u >= cnt) break;
        const P4<T> qj = qv[u];
        const T dxT = mi_diff(qj.x, xi, xim1), dyT = mi_diff(qj.y, yi, yim1), dzT = mi_diff(qj.z, zi, zim1);
        const T r2 = sep2(dxT, dyT, dzT);
        const T r = psqrt(r2);
        const T q = r * iH;
        const T w = kern_w(q), dw = kern_dw(q);
        const T psi = (T)(norm * kern_w(q));
        const T dx = dxT, dy = dyT, dz = dzT;
        const P4<T> pj = pv[u];
        const T Wj[5] = {pj.x, pj.y, pj.z, pj.w, Pv[u]};
        T psib = ((Eb[0] * dx * dx + Eb[1] * dx * dy) + (Eb[2] * dx * dz + Eb[3] * dy * dy)) +
                      (Eb[4] * dy * dz + Eb[5] * dz * dz);
        T db[3] = {psi * (T(2.0) * Eb[0] * dx + Eb[1] * dy + Eb[2] * dz),
                        psi * (Eb[1] * dx + T(2.0) * Eb[3] * dy + Eb[4] * dz),
                        psi * (Eb[2] * dx + Eb[4] * dy + T(2.0) * Eb[5] * dz)};
        for (int f = 0; f < 5; ++f) {
            const T df = Wj[f] - (T)Wi[f];
            const T t = (Sb[3 * f] * dx + Sb[3 * f + 1] * dy) + Sb[3 * f + 2] * dz;
            fbi[f] -= psi * t;
            psib += df * t;
            db[0] += df * psi * Sb[3 * f];
            db[1] += df * psi * Sb[3 * f + 1];
            db[2] += df * psi * Sb[3 * f + 2];
        }
        normb += psib * w;
        const T qb = psib * (T)norm * dw;
        Hbi -= qb * q * iH;
        if (r > T(0)) {
            const T rb = qb * iH * pdiv(T(1), r);
            db[0] += rb * dx;
            db[1] += rb * dy;
            db[2] += rb * dz;
        }
        xbi[0] -= db[0];
        xbi[1] -= db[1];
        xbi[2] -= db[2];
      }
    }
    Hbi += normb * (-T(3.0) * (T)norm / (T)Hi);
    nbi += normb * (-(T)norm / (T)ni);
    a[AX] += xbi[0];
    a[AX + 1] += xbi[1];
    a[AX + 2] += xbi[2];
    a[AH] += Hbi;
    a[AN] += nbi;
    a[ARHO] += fbi[0];
    a[AV] += fbi[1];
    a[AV + 1] += fbi[2];
    a[AV + 2] += fbi[3];
    a[AP] += fbi[4];
}

// Gradient-pass terms of particle j in the sums of every i with j in N_i
// (all such i are in j's pair lists).  Per candidate i the thread reads i's
// packed position and its 28-value record (S_bar, E_bar, psi norm, W_i) as
// 128-bit loads; the limiter rows are read only when i's bloom mask has the
// bit of j.
template <typename T>
__global__ void __launch_bounds__(128)
    k_grad_gather(int N, Sorted<T> s, const int* __restrict__ lim, const unsigned* __restrict__ nbr,
                  const int* __restrict__ ncount, const unsigned* __restrict__ rnbr,
                  const int* __restrict__ rcount, KParams p, const T* __restrict__ seeds,
                  const unsigned long long* __restrict__ lbloom, T* __restrict__ adj) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const P4<T> mj = s.pos[j];
    const P4<T> pj = s.prim[j];
    const T Wj[5] = {pj.x, pj.y, pj.z, pj.w, s.prim2[j].x};
    const unsigned long long jbit = 1ull << (j & 63);
    T fb[5] = {0, 0, 0, 0, 0}, xb[3] = {0, 0, 0}, Hb = T(0.0);
    for (int list = 0; list < 2; ++list) {
        const unsigned* Lj = list == 0 ? nbr + 4 * (size_t)j : rnbr + 4 * (size_t)j;
        const int cnt = list == 0 ? min(ncount[j], p.cap) : min(rcount[j], p.rcap);
        for (int k0 = 0; k0 < cnt; k0 += 4) {  // four candidates' loads in flight at a time
          const uint4 ii = col4(Lj, k0, N);
          const unsigned is[4] = {ii.x, ii.y, ii.z, ii.w};
          P4<T> mv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
              if (k0 + u < cnt) mv[u] = s.pos[is[u]];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (k0 + u >= cnt) break;
            const int i = (int)is[u];
            const P4<T> mi = mv[u];
            const T Hi = mi.w;
            // offset as seen by i (x_j - x_i), exactly as i's gradient pass computed it
            const T dx = mi_diff(mj.x, mi.x, mi.x - T(1)), dy = mi_diff(mj.y, mi.y, mi.y - T(1)),
                    dz = mi_diff(mj.z, mi.z, mi.z - T(1));
            const T r2 = sep2(dx, dy, dz);
            if (!(r2 < Hi * Hi)) continue;  // j is not in N_i
            const T* R = seeds + (size_t)i * kSeed;
            T sd[32];  // record 0-27 (and 4 limiter values, unused here)
            load_row32<32>(R, sd);
            const T r = psqrt(r2);
            const T iH = T(1) / Hi;
            const T q = r * iH;
            const T norm = sd[21];
            const T psi = (T)(norm * kern_w(q));
            const T dw = kern_dw(q);
            const T* Eb = sd + 15;
            T psib = ((Eb[0] * dx * dx + Eb[1] * dx * dy) + (Eb[2] * dx * dz + Eb[3] * dy * dy)) +
                     (Eb[4] * dy * dz + Eb[5] * dz * dz);
            T db[3] = {psi * (T(2.0) * Eb[0] * dx + Eb[1] * dy + Eb[2] * dz),
                       psi * (Eb[1] * dx + T(2.0) * Eb[3] * dy + Eb[4] * dz),
                       psi * (Eb[2] * dx + Eb[4] * dy + T(2.0) * Eb[5] * dz)};
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                const T df = Wj[f] - sd[22 + f];
                const T t = (sd[3 * f] * dx + sd[3 * f + 1] * dy) + sd[3 * f + 2] * dz;
                fb[f] += psi * t;
                psib += df * t;
                db[0] += df * psi * sd[3 * f];
                db[1] += df * psi * sd[3 * f + 1];
                db[2] += df * psi * sd[3 * f + 2];
            }
            if (r > T(0)) {
                const T rb = psib * norm * dw * iH * pdiv(T(1), r);
                db[0] += rb * dx;
                db[1] += rb * dy;
                db[2] += rb * dz;
            }
            xb[0] += db[0];
            xb[1] += db[1];
            xb[2] += db[2];
            // limiter terms where j is i's active neighbour or extreme particle
            if (__ldg(lbloom + i) & jbit) {
                const int* li = lim + (size_t)i * 10;
                for (int f = 0; f < 5; ++f) {
                    const int ja = li[f];
                    if (ja == j) {
                        xb[0] += R[28 + 5 * f];
                        xb[1] += R[28 + 5 * f + 1];
                        xb[2] += R[28 + 5 * f + 2];
                        Hb += R[28 + 5 * f + 3];
                    }
                    if (ja >= 0 && li[5 + f] == j) fb[f] += R[28 + 5 * f + 4];
                }
            }
          }
        }
    }
    T* a = adj + (size_t)j * kAdj;
    a[AX] += xb[0];
    a[AX + 1] += xb[1];
    a[AX + 2] += xb[2];
    a[AH] += Hb;
    a[ARHO] += fb[0];
    a[AV] += fb[1];
    a[AV + 1] += fb[2];
    a[AV + 2] += fb[3];
    a[AP] += fb[4];
}

// ------------------------------------------------------------ density
// rho = m n, P = (gamma - 1) m n u; n = 8 (1 + sum w) / (pi H^3) with H the
// root of f = (32/3)(1 + sum w) - N_ngb: Hbar_tot = Hbar + nbar dn/dH,
// lambda = -Hbar_tot / f_H, and every r_ij in N_i receives
// (w'(q)/H)(nbar 8/(pi H^3) + lambda 32/3) = kappa_i w'(q_ij).
template <typename T>
__global__ void __launch_bounds__(128)
    k_dens_seeds(int N, Sorted<T> s, const unsigned* __restrict__ nbr, const int* __restrict__ ncount,
                 KParams p, T* __restrict__ adj, T* __restrict__ kap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    T* a = adj + (size_t)i * kAdj;
    const T m = s.m[i], n = s.n[i], u = s.u[i], g1 = T(p.gamma) - T(1.0);
    const T rhob = a[ARHO], Pb = a[AP];
    const T nb = a[AN] + rhob * m + Pb * g1 * m * u;
    a[AM] += rhob * n + Pb * g1 * n * u;
    a[AU] += Pb * g1 * m * n;
    const P4<T> me = s.pos[i];
    const T xi = me.x, yi = me.y, zi = me.z, Hi = me.w;
    const T xim1 = xi - T(1), yim1 = yi - T(1), zim1 = zi - T(1);
    const T iH = T(1) / Hi;
    const int cnt = min(ncount[i], p.cap);
    const unsigned* L = nbr + 4 * (size_t)i;
    // sum over N_i of w'(q) q: the density pass kept its negative (same
    // terms, same order), so no loop over N_i is needed for it here
    const T dsum = -s.sd[i];
    const T H = Hi;
    const T c8 = T(8.0) / (T(kPi) * H * H * H);
    const T dndH = -T(3.0) * n / H - c8 * dsum / H;
    const T fH = -(T(32.0) / T(3.0)) * dsum / H;
    const T Hbt = a[AH] + nb * dndH;
    const T lam = fH != T(0.0) ? -Hbt / fH : T(0.0);
    const T kappa = (nb * c8 + lam * T(32.0) / T(3.0)) / H;
    kap[i] = kappa;
    T xb[3] = {0, 0, 0};
    for (int k0 = 0; k0 < cnt; k0 += 4) {  // four neighbours' loads in flight at a time
        const uint4 jj = col4(L, k0, N);
        const unsigned js[4] = {jj.x, jj.y, jj.z, jj.w};
        P4<T> qv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (k0 + u < cnt) qv[u] = s.pos[js[u]];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (k0 + u >= cnt) break;
            const P4<T> qj = qv[u];
            const T dx = mi_diff(qj.x, xi, xim1), dy = mi_diff(qj.y, yi, yim1), dz = mi_diff(qj.z, zi, zim1);
            const T r = psqrt(sep2(dx, dy, dz));
            if (!(r > T(0))) continue;
            const T c = kappa * (T)kern_dw(r * iH) * pdiv(T(1), r);
            xb[0] -= c * dx;
            xb[1] -= c * dy;
            xb[2] -= c * dz;
        }
    }
    a[AX] += xb[0];
    a[AX + 1] += xb[1];
    a[AX + 2] += xb[2];
}

template <typename T>
__global__ void __launch_bounds__(128)
    k_dens_gather(int N, Sorted<T> s, const unsigned* __restrict__ nbr, const int* __restrict__ ncount,
                  const unsigned* __restrict__ rnbr, const int* __restrict__ rcount, KParams p,
                  const T* __restrict__ kap, T* __restrict__ adj) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const P4<T> mj = s.pos[j];
    T xb[3] = {0, 0, 0};
    for (int list = 0; list < 2; ++list) {
        const unsigned* Lj = list == 0 ? nbr + 4 * (size_t)j : rnbr + 4 * (size_t)j;
        const int cnt = list == 0 ? min(ncount[j], p.cap) : min(rcount[j], p.rcap);
        for (int k0 = 0; k0 < cnt; k0 += 4) {  // four candidates' loads in flight at a time
            const uint4 ii = col4(Lj, k0, N);
            const unsigned is[4] = {ii.x, ii.y, ii.z, ii.w};
            P4<T> mv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (k0 + u < cnt) mv[u] = s.pos[is[u]];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (k0 + u >= cnt) break;
                const int i = (int)is[u];
                const P4<T> mi = mv[u];
                const T dx = mi_diff(mj.x, mi.x, mi.x - T(1)), dy = mi_diff(mj.y, mi.y, mi.y - T(1)),
                        dz = mi_diff(mj.z, mi.z, mi.z - T(1));
                const T r2 = sep2(dx, dy, dz);
                if (!(r2 < mi.w * mi.w)) continue;
                const T r = psqrt(r2);
                if (!(r > T(0))) continue;
                const T c = kap[i] * kern_dw(r * pdiv(T(1), mi.w)) * pdiv(T(1), r);
                xb[0] += c * dx;
                xb[1] += c * dy;
                xb[2] += c * dz;
            }
        }
    }
    T* a = adj + (size_t)j * kAdj;
    a[AX] += xb[0];
    a[AX + 1] += xb[1];
    a[AX + 2] += xb[2];
}

template <typename T>
__global__ void k_adj_out_step(int N, const unsigned* __restrict__ orig, const T* __restrict__ adj,
                               gz_particles gs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned o = orig[i];
    const T* a = adj + (size_t)i * kAdj;
    if (gs.x) ((T*)gs.x)[o] = (T)a[AX];
    if (gs.y) ((T*)gs.y)[o] = (T)a[AX + 1];
    if (gs.z) ((T*)gs.z)[o] = (T)a[AX + 2];
    if (gs.vx) ((T*)gs.vx)[o] = (T)a[AV];
    if (gs.vy) ((T*)gs.vy)[o] = (T)a[AV + 1];
    if (gs.vz) ((T*)gs.vz)[o] = (T)a[AV + 2];
    if (gs.u) ((T*)gs.u)[o] = (T)a[AU];
    if (gs.m) ((T*)gs.m)[o] = (T)a[AM];
}

}  // namespace

template <typename T>
cudaError_t run_step_adjoint(Ctx& c, const gz_particles& gend, gz_particles& gstart) {
    const int N = c.N;
    const KParams kp = kparams(c);
    Sorted<T> s = sorted_view<T>(c);
    c.launches += 8;
    cudaMemsetAsync(c.adj, 0, sizeof(T) * (size_t)N * kAdj, c.stream);
    k_update_adj<T><<<blocks(N, 256), 256, 0, c.stream>>>(N, s, c.dpdt, c.dEdt, c.dt_use, gend, (T*)c.adj, (T*)c.wgt);
    k_flux_adj<T><<<blocks(N, 128), 128, 0, c.stream>>>(N, (const T*)c.rec, (const T*)c.sn, c.sid, c.sbox,
                                                         c.nbr, c.ncount, c.rnbr, c.rcount, kp, c.dt_use,
                                                         (const T*)c.wgt, (T*)c.adj);
    k_grad_seeds<T><<<blocks(N, 128), 128, 0, c.stream>>>(N, s, (const T*)c.rec, (const T*)c.ginfo, c.lim,
                                                           c.nbr, c.ncount, kp, (T*)c.adj, (T*)c.seeds,
                                                           c.lbloom);
    k_grad_gather<T><<<blocks(N, 128), 128, 0, c.stream>>>(N, s, c.lim, c.nbr, c.ncount, c.rnbr, c.rcount,
                                                            kp, (const T*)c.seeds, c.lbloom, (T*)c.adj);
    k_dens_seeds<T><<<blocks(N, 128), 128, 0, c.stream>>>(N, s, c.nbr, c.ncount, kp, (T*)c.adj, (T*)c.wgt);
    k_dens_gather<T><<<blocks(N, 128), 128, 0, c.stream>>>(N, s, c.nbr, c.ncount, c.rnbr, c.rcount, kp,
                                                            (const T*)c.wgt, (T*)c.adj);
    k_adj_out_step<T><<<blocks(N, 256), 256, 0, c.stream>>>(N, c.vals, (const T*)c.adj, gstart);
    return cudaGetLastError();
}
template cudaError_t run_step_adjoint<float>(Ctx&, const gz_particles&, gz_particles&);
template cudaError_t run_step_adjoint<double>(Ctx&, const gz_particles&, gz_particles&);

cudaError_t ensure_adjoint_scratch(Ctx& c) {
    if (c.adj) return cudaSuccess;
    const size_t Nz = (size_t)c.capacity;  // (a subdomain context's N changes)
    const size_t tsz = c.precision == GZ_FP64 ? 8 : 4;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };  // 256-byte aligned slices
    const size_t sz[6] = {up(sizeof(double) * Nz * kAdj), up(sizeof(double) * Nz * 4), up(tsz * Nz * kSeed),
                          up(sizeof(unsigned long long) * Nz), up(sizeof(int) * Nz * 10),
                          up(tsz * Nz * kGInfo)};
    size_t bytes = 0;
    for (size_t b : sz) bytes += b;
    char* base = nullptr;
    cudaError_t e = cudaMalloc((void**)&base, bytes);
    if (e != cudaSuccess) return e;
    c.adj_arena = base;
    c.adj = base;
    base += sz[0];
    c.wgt = base;
    base += sz[1];
    c.seeds = base;
    base += sz[2];
    c.lbloom = (unsigned long long*)base;
    base += sz[3];
    c.lim = (int*)base;
    base += sz[4];
    c.ginfo = base;
    return cudaSuccess;
}

template <typename T>
cudaError_t run_flux_adjoint(Ctx& c, const double* dpbar, const double* dEbar) {
    c.launches += 2;
    cudaMemsetAsync(c.adj, 0, sizeof(T) * (size_t)c.N * kAdj, c.stream);
    k_gather_wgt<T><<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, c.vals, dpbar, dEbar, (T*)c.wgt);
    k_flux_adj<T><<<blocks(c.N, 128), 128, 0, c.stream>>>(c.N, (const T*)c.rec, (const T*)c.sn, c.sid,
                                                           c.sbox, c.nbr, c.ncount, c.rnbr, c.rcount,
                                                           kparams(c), c.dt_use, (const T*)c.wgt, (T*)c.adj);
    return cudaGetLastError();
}

cudaError_t run_adj_out_flux(Ctx& c, double* xbar, double* hbar, double* nbar, double* Wbar, double* gbar,
                             double* Bbar) {
    c.launches += 1;
    if (c.precision == GZ_FP64)
        k_adj_out_flux<double><<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, c.vals, (const double*)c.adj, xbar,
                                                                       hbar, nbar, Wbar, gbar, Bbar);
    else
        k_adj_out_flux<float><<<blocks(c.N, 256), 256, 0, c.stream>>>(c.N, c.vals, (const float*)c.adj, xbar,
                                                                      hbar, nbar, Wbar, gbar, Bbar);
    return cudaGetLastError();
}

template cudaError_t run_flux_adjoint<float>(Ctx&, const double*, const double*);
template cudaError_t run_flux_adjoint<double>(Ctx&, const double*, const double*);

}  // namespace gz
