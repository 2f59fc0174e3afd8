// vg_matern.cuh -- Matern correlation with general smoothness on the device.
//
// CUDA has no modified Bessel function of the second kind (the paper's Sec. 5 names this
// as the reason its software cannot offer the Matern family with arbitrary smoothness).
// Here M_nu(x) = 2^(1-nu)/Gamma(nu) x^nu K_nu(x) and the two derivatives the likelihood
// needs are evaluated in two layers:
//
//  1. matern_sums_warp / matern_finish_warp (table builder): K_nu, K_(nu-1) and dK_nu/dnu
//     from the integral
//        K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
//     (and its nu-derivative int exp(-x cosh t) t sinh(nu t) dt), trapezoid rule in t,
//     the nodes shared by the 32 lanes of a warp.  The integrands are even and entire in t
//     and decay double-exponentially, so the trapezoid sum converges geometrically in 1/h.
//     Scales are kept in log space.
//  2. A per-pass coefficient table.  Within one pass theta is fixed, so the three functions
//        F0(s) = sigma2 M_nu(sqrt s),
//        F1(s) = (sigma2 / rho) (-x dM/dx),  -x dM/dx = 2^(1-nu)/Gamma(nu) x^(nu+1) K_(nu-1)(x)
//                = rho dM/drho, so F1 = dC/drho,
//        F2(s) = sigma2 dM/dnu = dC/dnu,
//     of s = x^2 = |h|^2 / rho^2 are tabulated once per pass as polynomials of degree D on
//     dyadic sub-intervals: octave [2^e, 2^(e+1)) split into J equal parts.  The octave and
//     part come from the exponent and leading mantissa bits of s (integer work), the local
//     variable w = mantissa - centre is exact, and each function is a D-step Horner chain.
//     Working in s avoids a square root per entry.  The only singularity of F(s) is at
//     s = 0 (terms s^nu and s^nu log s), so on a part [a, a (1 + 1/J)] the Chebyshev
//     interpolant converges like (4J + 2)^-D; with J = 4 and D = 12 that is < 1e-16
//     relative to M(0) = 1.  Below 2^E0 the small-argument expansion (matern_small) is
//     used; at and above 2^E1 the functions are below 1e-20 for every nu <= 20 and are
//     returned as 0.
#pragma once
#include "vg_common.cuh"

namespace vg {

// table geometry (MT_*) is defined in vg_common.cuh

// F0, F1, F2 below the table (0 < s < 2^E0, so u = s/4 < 2^-32) from the small-argument
// expansion.  For non-integer nu the series of I_(-nu) and I_nu give
//   M_nu(x) = Gamma(1-nu) sum_k u^k / (k! Gamma(k+1-nu))
//             - Gamma(1-nu) u^nu sum_k u^k / (k! Gamma(k+1+nu)),
// and for u < 2^-32 every term other than 1, A1 u, C u^nu and, for nu < 1,
// C u^(nu+1)/(1+nu) is below 3e-18, where A1 = 1/(1-nu) and C = -Gamma(1-nu)/Gamma(1+nu).
// A1 and C have poles at nu = 1 whose sum stays finite, so for |nu - 1| < 0.01 the pair is
// evaluated as
//   A1 u + C u^nu = u [(g - 1)/delta + g expm1(delta l)/delta],
//   delta = nu - 1, l = log u, g = Gamma(1-delta)/Gamma(2+delta),
// which tends to u (log u + 2 gamma_E - 1) at nu = 1 (the expansion of x K_1(x)).  At
// nu = 2 the u^nu term and the u^2 term have canceling poles too; both are O(u^2 log u)
// together, and the u^nu term is dropped for nu >= 1.99 (it is below u^1.99 |C| there).
// F1 = -2u dM/du and F2 = dM/dnu follow term by term.  psi = digamma(nu).
static __device__ __noinline__ void matern_small(double nu, double s, double psi, double& F0, double& F1,
                                    double& F2) {
    const double u = 0.25 * s;
    const double l = log(u);
    const double EULER = 0.57721566490153286061;
    const double PI = 3.14159265358979323846;
    const double dl = nu - 1.0;
    if (fabs(dl) < 0.01) {
        const double lgg = lgamma(1.0 - dl) - lgamma(2.0 + dl);
        const double g = exp(lgg);
        const double gp = g * (-dev_digamma(1.0 - dl) - dev_digamma(2.0 + dl));  // dg/ddelta
        const double c1 = 2.0 * EULER - 1.0;   // g'(0): limit of (g - 1)/delta
        const double c2 = 0.5 * (c1 * c1 + 1.0);  // g''(0)/2: limit of d/ddelta (g - 1)/delta
        const double G1 = fabs(dl) < 1e-6 ? c1 + c2 * dl : expm1(lgg) / dl;
        const double G1p = fabs(dl) < 1e-3 ? c2 : (gp * dl - (g - 1.0)) / (dl * dl);
        const double z = dl * l;
        double E, Ep;  // expm1(delta l)/delta and its delta-derivative
        if (fabs(z) < 1e-3) {
            E = l * (1.0 + z * (0.5 + z * (1.0 / 6.0 + z * (1.0 / 24.0))));
            Ep = l * l * (0.5 + z * (1.0 / 3.0 + z * 0.125));
        } else {
            const double em = expm1(z);
            E = em / dl;
            Ep = (z * (em + 1.0) - em) / (dl * dl);
        }
        F0 = 1.0 + u * (G1 + g * E);
        F1 = -2.0 * u * (G1 + g * (E + exp(z)));
        F2 = u * (G1p + gp * E + g * Ep);
        return;
    }
    const double A1 = 1.0 / (1.0 - nu);
    F0 = 1.0 + A1 * u;
    F1 = -2.0 * A1 * u;
    F2 = A1 * A1 * u;
    if (nu < 1.99) {
        const double C = -tgamma(1.0 - nu) / tgamma(1.0 + nu);
        // d log|C| / dnu = -psi(1-nu) - psi(1+nu), with psi(1-nu) = psi(nu) + pi cot(pi nu)
        const double D = -2.0 * psi - 1.0 / nu - PI / tan(PI * nu);
        const double t = C * exp(nu * l);  // C u^nu
        F0 += t;
        F1 -= 2.0 * nu * t;
        F2 += t * (D + l);
        if (nu < 1.0) {
            const double t1 = t * u / (1.0 + nu);  // C u^(nu+1) / (1+nu)
            F0 += t1;
            F1 -= 2.0 * (1.0 + nu) * t1;
            F2 += t1 * (D + l - 1.0 / (1.0 + nu));
        }
    }
}

// Locates s in the table.  Returns the interval index and the local variable w, or
// -1 when s < 2^E0 (direct formula, includes s == 0), or -2 when s >= 2^E1 (zero).
// w = mantissa - centre, the centre 1 + (2j+1)/(2J) of interval j, is a multiple of 2^-52
// of magnitude at most 1/(2J): an integer W of at most 50 bits in units of 2^-52 (from the
// bits, no FP64 instruction).  It is returned as an exact unevaluated sum of two FP32
// numbers, split by rounding at 2^25: wh = round(W / 2^25) 2^-27 and
// wl = (W - round(W / 2^25) 2^25) 2^-52, each part at most 2^24 in units and so exact.
__device__ __forceinline__ int mtab_locate(double s, float& wh, float& wl) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(s);
    const int e = (int)((bits >> 52) & 0x7ffull) - 1023;
    if (e < MT_E0) return -1;
    if (e >= MT_E1) return -2;
    const unsigned long long j = (bits >> (52 - MT_LOGJ)) & (unsigned long long)(MT_J - 1);
    const long long W = (long long)(bits & 0x000fffffffffffffull) -
                        (long long)((2ull * j + 1ull) << (52 - MT_LOGJ - 1));
    const long long Wh = (W + (1ll << 24)) >> 25;
    wh = __int2float_rn((int)Wh) * 0x1p-27f;
    wl = __int2float_rn((int)(W - (Wh << 25))) * 0x1p-52f;
    return (e - MT_E0) * MT_J + (int)j;
}

// Degree-12 polynomial in w, |w| <= 1/8, evaluated in three precisions (the table layout
// per function: c0 in FP64; c1..c7 as (hi, lo) FP32 pairs; c8..c12 in FP32):
//   * the tail w^8..w^12 (summing to below ~1e-9 on every interval) in FP32;
//   * P = c1 + w (c2 + ...) in double-float arithmetic (a value is an unevaluated FP32
//     pair, ~48 significant bits; the two-product uses the FMA's exact remainder, the sum
//     Knuth's two-sum), with w = wh + wl exact (mtab_locate);
//   * q = w P in double-float: wh ph exactly as its rounded product and the FMA's
//     remainder, plus the cross terms wh pl and wl ph (wl pl is below 2^-52 of |q|);
//   * c0 + q_hi + q_lo in FP64: two additions.
// q enters the result with |q| <= |c1|/8 + ..., and its double-float rounding (~2^-48 of
// |q|) lands at ~2^-50 of |c1|: a few units of the last place of the covariance scale
// sigma2, below what the likelihood resolves even at a nugget of 0.001.  FP32 runs at 64x
// the FP64 rate on this GPU, so the chain costs 2 FP64 additions instead of 9 FP64
// operations.  The error-free steps use explicitly rounded intrinsics so that no
// multiply-add is fused.
__device__ __forceinline__ double horner_split(const double* c, float wh, float wl) {
    const float* t = reinterpret_cast<const float*>(c + MT_NHEAD);
    float ph = t[4];
    ph = fmaf(ph, wh, t[3]);
    ph = fmaf(ph, wh, t[2]);
    ph = fmaf(ph, wh, t[1]);
    ph = fmaf(ph, wh, t[0]);
    float pl = 0.0f;
    const float2* mid = reinterpret_cast<const float2*>(c + 1);
#pragma unroll
    for (int k = MT_NHEAD - 2; k >= 0; --k) {      // c7 .. c1
        const float2 ck = mid[k];
        const float hi = __fmul_rn(ph, wh);
        float lo = fmaf(ph, wh, -hi);               // exact remainder of ph wh
        lo = fmaf(ph, wl, lo);
        lo = fmaf(pl, wh, lo);
        const float sm = __fadd_rn(hi, ck.x);
        const float z = __fsub_rn(sm, hi);
        float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(sm, z)), __fsub_rn(ck.x, z));
        er = __fadd_rn(er, __fadd_rn(lo, ck.y));
        ph = __fadd_rn(sm, er);
        pl = __fsub_rn(er, __fsub_rn(ph, sm));
    }
    const float qh = __fmul_rn(wh, ph);
    float ql = fmaf(wh, ph, -qh);                   // exact remainder of wh ph
    ql = fmaf(wh, pl, ql);
    ql = fmaf(wl, ph, ql);
    return (c[0] + f32_to_f64_bits(qh)) + f32_to_f64_bits(ql);
}

// Locates s in the table like mtab_locate, but returns the local variable only as the
// FP32 pair (wf, wl): integer and FP32 work, no FP64 instruction.
__device__ __forceinline__ int mtab_locate_pair(double s, float& wf, float& wl) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(s);
    const int e = (int)((bits >> 52) & 0x7ffull) - 1023;
    if (e < MT_E0) return -1;
    if (e >= MT_E1) return -2;
    const unsigned long long j = (bits >> (52 - MT_LOGJ)) & (unsigned long long)(MT_J - 1);
    const float mantf = __uint_as_float(0x3f800000u | (unsigned)((bits >> 29) & 0x7fffffull));
    const float cenf = __uint_as_float(0x3f800000u | (unsigned)((2ull * j + 1ull) << (23 - MT_LOGJ - 1)));
    wf = mantf - cenf;
    wl = __uint2float_rn((unsigned)(bits & 0x1fffffffull)) * 0x1p-52f;
    return (e - MT_E0) * MT_J + (int)j;
}

// Degree-12 polynomial entirely in double-float FP32 arithmetic (the derivative tables'
// layout: c0..c7 as (hi, lo) FP32 pairs, c8..c12 in FP32); the result is the pair's sum in
// FP64, one FP64 addition.  Relative accuracy about 2^-46: enough for the derivative
// matrices, which enter the gradient and information linearly (an error of 2^-44 relative
// in every derivative entry moves the gradient by ~1e-11 of its scale even at a nugget of
// 0.001), whereas the covariance itself is amplified by the block's conditioning and keeps
// its FP64 head (horner_split).
__device__ __forceinline__ float2 horner_df_pair(const double* c, float wh, float wl) {
    const float* t = reinterpret_cast<const float*>(c + MT_NHEAD);
    float ph = t[4];
    ph = fmaf(ph, wh, t[3]);
    ph = fmaf(ph, wh, t[2]);
    ph = fmaf(ph, wh, t[1]);
    ph = fmaf(ph, wh, t[0]);
    float pl = 0.0f;
    const float2* mid = reinterpret_cast<const float2*>(c);
#pragma unroll
    for (int k = MT_NHEAD - 1; k >= 0; --k) {      // c7 .. c0
        const float2 ck = mid[k];
        const float hi = __fmul_rn(ph, wh);
        float lo = fmaf(ph, wh, -hi);               // exact remainder of ph wh
        lo = fmaf(ph, wl, lo);
        lo = fmaf(pl, wh, lo);
        const float sm = __fadd_rn(hi, ck.x);
        const float z = __fsub_rn(sm, hi);
        float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(sm, z)), __fsub_rn(ck.x, z));
        er = __fadd_rn(er, __fadd_rn(lo, ck.y));
        ph = __fadd_rn(sm, er);
        pl = __fsub_rn(er, __fsub_rn(ph, sm));
    }
    return make_float2(ph, pl);
}
__device__ __forceinline__ double horner_df(const double* c, float wh, float wl) {
    const float2 r = horner_df_pair(c, wh, wl);
    return f32_to_f64_bits(r.x) + f32_to_f64_bits(r.y);
}

// The derivative pair F1, F2 at s given as a double-float value sh + sl (FP32 numbers,
// |sl| <= ulp(sh)): the interval comes from the bits of sh, and the local variable
// w = (mantissa(sh) - centre) + sl 2^-e is the exact FP32 difference plus the scaled low
// part; no FP64 instruction except the two final additions of horner_df.  Arguments below
// the table take the FP64 expansion at sh + sl.
__device__ __forceinline__ void matern_F12_df(const double* tab, float sh, float sl, double nu,
                                              double psi, double sc1, double sc2, double& F1,
                                              double& F2) {
    const unsigned bits = __float_as_uint(sh);
    const int e = (int)((bits >> 23) & 0xffu) - 127;
    if (e >= MT_E0 && e < MT_E1) {
        const unsigned j = (bits >> (23 - MT_LOGJ)) & (unsigned)(MT_J - 1);
        const float mant = __uint_as_float((bits & 0x007fffffu) | 0x3f800000u);
        const float cen = __uint_as_float(0x3f800000u | ((2u * j + 1u) << (23 - MT_LOGJ - 1)));
        const float wf = mant - cen;                                  // exact
        const float wl = __fmul_rn(sl, __uint_as_float((unsigned)(127 - e) << 23));  // sl 2^-e
        const double* cf = tab + ((e - MT_E0) * MT_J + (int)j) * MT_PER_INT;
        F1 = horner_df(cf + MT_FSTRIDE, wf, wl);
        F2 = horner_df(cf + 2 * MT_FSTRIDE, wf, wl);
    } else if (e >= MT_E1 || !(sh > 0.0f)) {
        F1 = 0.0;
        F2 = 0.0;
    } else {
        double f0;
        matern_small(nu, f32_to_f64_bits(sh) + f32_to_f64_bits(sl), psi, f0, F1, F2);
        F1 *= sc1;
        F2 *= sc2;
    }
}

// The table holds the covariance and its derivatives, not M itself: F0 = sigma2 M,
// F1 = sigma2 dM/drho = sigma2 (rho dM/drho) / rho, F2 = sigma2 dM/dnu (the builder folds
// the scales in).  Below the table the expansion's values are scaled here (sc0 = sigma2,
// sc1 = sigma2 / rho, sc2 = sigma2); above it all three are 0.
__device__ __forceinline__ double matern_F0(const double* tab, double s, double nu, double psi,
                                            double sc0) {
    float wh, wl;
    int it = mtab_locate(s, wh, wl);
    if (it >= 0) return horner_split(tab + it * MT_PER_INT, wh, wl);
    if (it == -2) return 0.0;
    if (!(s > 0.0)) return sc0;
    double f0, f1, f2;
    matern_small(nu, s, psi, f0, f1, f2);
    return sc0 * f0;
}
__device__ __forceinline__ void matern_F12(const double* tab, double s, double nu, double psi,
                                           double sc1, double sc2, double& F1, double& F2) {
    float wf, wl;
    int it = mtab_locate_pair(s, wf, wl);
    if (it >= 0) {
        const double* cf = tab + it * MT_PER_INT;
        F1 = horner_df(cf + MT_FSTRIDE, wf, wl);
        F2 = horner_df(cf + 2 * MT_FSTRIDE, wf, wl);
    } else if (it == -2 || !(s > 0.0)) {
        F1 = 0.0;
        F2 = 0.0;
    } else {
        double f0;
        matern_small(nu, s, psi, f0, F1, F2);
        F1 *= sc1;
        F2 *= sc2;
    }
}

// The exponential families from a table of the same layout, built in closed form by the
// same builder: F0 = sigma2 e^-x, F1 = sigma2 x e^-x (rho dC/drho of the isotropic
// exponential), F2 = sigma2 e^-x / x (the pair weight C / D of the space-time and the
// per-coordinate ranges families), all at s = x^2 in scaled coordinates.  F0 keeps the
// FP64 head (horner_split); the weights are double-float (horner_df), like the Matern
// derivatives.  Below the table the functions are evaluated directly (F2 = 0 for
// coincident points, where every range derivative vanishes); above it they are 0.
__device__ __forceinline__ double exp_F0(const double* tab, double s, double sig2) {
    float wh, wl;
    const int it = mtab_locate(s, wh, wl);
    if (it >= 0) return horner_split(tab + it * MT_PER_INT, wh, wl);
    if (it == -2) return 0.0;
    return sig2 * exp(-sqrt(s));
}
__device__ __forceinline__ double exp_F12(const double* tab, double s, double sig2, int f) {
    float wf, wl;
    const int it = mtab_locate_pair(s, wf, wl);
    if (it >= 0) return horner_df(tab + it * MT_PER_INT + f * MT_FSTRIDE, wf, wl);
    if (it == -2 || !(s > 0.0)) return 0.0;
    const double x = sqrt(s), e = sig2 * exp(-x);
    return f == 1 ? x * e : e / x;
}
// exp_F12 as an unevaluated double-float pair (hi + lo is the value, about 2^-46
// relative), for callers that go on in double-float arithmetic: no FP64 instruction inside
// the table; outside it the FP64 value, split.
__device__ __forceinline__ float2 exp_F12_pair(const double* tab, double s, double sig2, int f) {
    float wf, wl;
    const int it = mtab_locate_pair(s, wf, wl);
    if (it >= 0) return horner_df_pair(tab + it * MT_PER_INT + f * MT_FSTRIDE, wf, wl);
    const double v = exp_F12(tab, s, sig2, f);
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}

// F0, F1, F2 at x > 0 by the trapezoid rule (h = 0.1; see the header), for the table
// builder, in two steps.  matern_sums_warp: the three trapezoid sums with the envelope
// exponent mu t - x cosh t (mu = max(nu, |nu-1|) bounds all three integrands) and its
// maximum Phi factored out; lane l sums the nodes t = (l + 32 i) h, then the partial sums
// are combined in a fixed order.  Along a lane's nodes e^t, e^-t and the four exponentials
// e^(c t) of the cosh(nu t), cosh((nu-1) t) and t sinh(nu t) factors are geometric in i
// (ratio e^(32 c h)), so they are advanced by one multiplication each and only the
// envelope's exponential is evaluated per node (a lane takes at most ~7 nodes, so the
// products add a few units of the last place).  matern_finish_warp: the scaling
// 2^(1-nu) x^nu / Gamma(nu) and the nu-derivative's digamma term (psi = digamma(nu),
// lgnu = lgamma(nu)).
__device__ inline void matern_sums_warp(double nu, double x, double& S0, double& S1,
                                        double& S2, double& Phi) {
    const double h = 0.1;
    const int lane = threadIdx.x & 31;
    const double mu = fmax(nu, fabs(nu - 1.0));
    const double ts = asinh(mu / x);
    Phi = mu * ts - x * cosh(ts);
    const double nu1 = fabs(nu - 1.0);
    const double t0 = lane * h, H = 32.0 * h;
    double ep = exp(t0), em = exp(-t0);
    double a = exp((nu - mu) * t0), b = exp(-(nu + mu) * t0);
    double c = exp((nu1 - mu) * t0), dd = exp(-(nu1 + mu) * t0);
    const double rp = exp(H), rm = exp(-H);
    const double ra = exp((nu - mu) * H), rb = exp(-(nu + mu) * H);
    const double rc = exp((nu1 - mu) * H), rd = exp(-(nu1 + mu) * H);
    S0 = 0.0;
    S1 = 0.0;
    S2 = 0.0;
    double t = t0;
    for (int k = lane; k < 20000; k += 32) {
        const double ph = mu * t - x * (0.5 * (ep + em)) - Phi;
        const double E = exp(ph) * (k == 0 ? 0.5 : 1.0);
        S0 += E * 0.5 * (a + b);
        S1 += E * 0.5 * (c + dd);
        S2 += E * 0.5 * t * (a - b);
        if (t > ts && ph < -50.0) break;  // the integrand decreases from here on
        t += H;
        ep *= rp;
        em *= rm;
        a *= ra;
        b *= rb;
        c *= rc;
        dd *= rd;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        S0 += __shfl_xor_sync(0xffffffffu, S0, o);
        S1 += __shfl_xor_sync(0xffffffffu, S1, o);
        S2 += __shfl_xor_sync(0xffffffffu, S2, o);
    }
}
__device__ inline void matern_finish_warp(double nu, double x, double psi, double lgnu,
                                          double S0, double S1, double S2, double Phi,
                                          double& F0, double& F1, double& F2) {
    const double h = 0.1;
    const double LN2 = 0.6931471805599453;
    double lx = log(x);
    double logA = (1.0 - nu) * LN2 - lgnu + nu * lx + Phi + log(h);
    double A = exp(logA);
    F0 = A * S0;
    F1 = A * x * S1;
    F2 = F0 * (-LN2 - psi + lx) + A * S2;
}

// FP32 table (mixed path): same intervals, 13 FP32 coefficients per function, located
// from the FP32 bits of s.
__device__ __forceinline__ int mtab_locate_f(float s, float& w) {
    const unsigned bits = __float_as_uint(s);
    const int e = (int)((bits >> 23) & 0xffu) - 127;
    if (e < MT_E0) return -1;
    if (e >= MT_E1) return -2;
    const unsigned j = (bits >> (23 - MT_LOGJ)) & (unsigned)(MT_J - 1);
    const float mant = __uint_as_float((bits & 0x007fffffu) | 0x3f800000u);
    const float cen = __uint_as_float(0x3f800000u | ((2u * j + 1u) << (23 - MT_LOGJ - 1)));
    w = mant - cen;
    return (e - MT_E0) * MT_J + (int)j;
}
__device__ __forceinline__ float horner13f(const float* c, float w) {
    float p = c[12];
#pragma unroll
    for (int k = 11; k >= 0; --k) p = fmaf(p, w, c[k]);
    return p;
}
__device__ __forceinline__ float matern_F0f(const float* tab, float s, double nu, double psi,
                                            double sc0) {
    float w;
    int it = mtab_locate_f(s, w);
    if (it >= 0) return horner13f(tab + it * MT_PER_INT_F, w);
    if (it == -2) return 0.0f;
    if (!(s > 0.0f)) return (float)sc0;
    double f0, f1, f2;
    matern_small(nu, (double)s, psi, f0, f1, f2);
    return (float)(sc0 * f0);
}
__device__ __forceinline__ void matern_F12f(const float* tab, float s, double nu, double psi,
                                            double sc1, double sc2, float& F1, float& F2) {
    float w;
    int it = mtab_locate_f(s, w);
    if (it >= 0) {
        const float* cf = tab + it * MT_PER_INT_F;
        F1 = horner13f(cf + MT_NC, w);
        F2 = horner13f(cf + 2 * MT_NC, w);
    } else if (it == -2 || !(s > 0.0f)) {
        F1 = 0.0f;
        F2 = 0.0f;
    } else {
        double f0, f1, f2;
        matern_small(nu, (double)s, psi, f0, f1, f2);
        F1 = (float)(sc1 * f1);
        F2 = (float)(sc2 * f2);
    }
}

}  // namespace vg
