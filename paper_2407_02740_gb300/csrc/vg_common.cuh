// vg_common.cuh -- device helpers shared by the Vecchia kernels (CUDA library side).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace vg {

// status codes written by kernels (same numbering as vec_status in include/vecchia.h)
enum : int { ST_OK = 0, ST_ARG = 1, ST_NOT_PD = 2, ST_NONFINITE = 3 };

// COV_ANISO: the exponential with one range per coordinate (Sec. 4.3, Eq. 6 with
// rho_1..rho_d), theta = (sigma2, rho_1, ..., rho_d, tau2).
enum : int { COV_EXP = 0, COV_MATERN = 1, COV_ST = 2, COV_ANISO = 3 };

constexpr int KMAX = 81;   // largest conditioning block (m <= 80)
// Grouped conditioning forms the terms of up to GCH members of a group together (each
// pair of the block evaluated once for all of them, that many times the items between
// barriers); the planner takes fewer where the larger slot does not fit, and a caller may
// ask for up to GCH_MAX.
constexpr int GCH = 4;
constexpr int GCH_MAX = 8;
constexpr int PMAX = 8;    // largest number of regression columns
constexpr int DMAX = 3;    // largest location dimension of the isotropic families
constexpr int DMAX_ANISO = 20;          // largest dimension with one range per coordinate
constexpr int QMAX = DMAX_ANISO + 2;    // largest number of covariance parameters

// Geometry of the per-pass coefficient table (see vg_matern.cuh).  Each function on each
// interval is a degree-12 polynomial in w stored in 11 double slots: the covariance F0 as
// w^0 in FP64 and w^1..w^7 as (hi, lo) FP32 pairs, the derivatives F1, F2 as w^0..w^7 in
// pairs; then w^8..w^12 in FP32 (padded to 6 floats).
constexpr int MT_E0 = -30;   // table covers s in [2^-30, 2^13)
constexpr int MT_E1 = 13;
constexpr int MT_LOGJ = 2;
constexpr int MT_J = 1 << MT_LOGJ;
constexpr int MT_D = 12;     // polynomial degree
constexpr int MT_NC = MT_D + 1;
constexpr int MT_NHEAD = 8;  // slots before the FP32 tail
constexpr int MT_FSTRIDE = MT_NHEAD + 3;       // double slots per function
constexpr int MT_NINT = (MT_E1 - MT_E0) * MT_J;
constexpr int MT_PER_INT = 3 * MT_FSTRIDE;     // F0, F1, F2 per interval
constexpr int MT_DOUBLES = MT_NINT * MT_PER_INT;
// FP32 copy for the mixed path: 13 FP32 coefficients per function and interval
constexpr int MT_PER_INT_F = 3 * MT_NC;
constexpr int MT_FLOATS = MT_NINT * MT_PER_INT_F;

// Families whose pass reads a per-pass coefficient table: the Matern family always (its
// FP64 table, and an FP32 copy for the mixed path), the exponential families on the FP64
// path (prec 0), whose covariance and pair weights come from the same kind of table
// instead of a square root, an exponential and a division per pair.
__host__ __device__ constexpr bool uses_table(int cov, int prec) {
    return cov == COV_MATERN || prec == 0;
}

// number of covariance parameters (d: location dimension, used by COV_ANISO only)
__host__ __device__ constexpr int nparms(int cov, int d = 0) {
    return cov == COV_EXP ? 3 : (cov == COV_ANISO ? d + 2 : 4);
}
// number of covariance parameters whose derivative matrix needs a per-pair evaluation
// (sigma2 and tau2 are handled in closed form)
__host__ __device__ constexpr int npair_derivs(int cov, int d = 0) {
    return cov == COV_EXP ? 1 : (cov == COV_ANISO ? d : 2);
}

// theta inside the family's domain: every parameter positive and finite, the Matern
// smoothness in [0.05, 20].
__host__ __device__ inline bool theta_ok(int cov, int d, const double* th) {
    const int q = nparms(cov, d);
    for (int j = 0; j < q; ++j)
        if (!(th[j] > 0.0 && th[j] <= 1.7976931348623157e308)) return false;   // finite
    if (cov == COV_MATERN && !(th[2] >= 0.05 && th[2] <= 20.0)) return false;
    return true;
}

// Per-observation record (the Algorithm 1 sums) in packed symmetric storage.
//   [logdet, ySy, XSX (p(p+1)/2), ySX (p),
//    for each derivative parameter j in 0..Q-1 (theta index j+1):
//       dlogdet_j, dySy_j, dySX_j (p), dXSX_j (p(p+1)/2),
//    info_jl for 0 <= j <= l < Q]
// The sigma2 entries are not accumulated: with the relative nugget, dSigma/dsigma2 =
// Sigma/sigma2, so every sigma2 term follows from the totals (see the profile kernel).
struct RecLayout {
    int p, Q, P2, per_j, base_j, base_info, nstat;
    __host__ __device__ void init(int p_, int Q_) {
        p = p_; Q = Q_; P2 = p * (p + 1) / 2;   // Q <= QMAX - 1, p <= PMAX
        per_j = 2 + p + P2;
        base_j = 2 + P2 + p;
        base_info = base_j + Q * per_j;
        nstat = base_info + Q * (Q + 1) / 2;
    }
};

// largest record (p = PMAX, Q = QMAX - 1)
constexpr int REC_MAX = 2 + PMAX * (PMAX + 1) / 2 + PMAX +
                        (QMAX - 1) * (2 + PMAX + PMAX * (PMAX + 1) / 2) + (QMAX - 1) * QMAX / 2;

// FP32 -> FP64 from the bits (integer work only): exact for normal numbers; zero and
// subnormals (below 1.2e-38, far below every scale the kernels use) give 0.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ex = (u >> 23) & 0xffu;
    if (ex == 0u) return 0.0;
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(ex + 896u) << 52) |
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)b);
}

// 1/sqrt(v), v > 0, for the Cholesky pivots.  The FP32 seed rsqrtf(v) (v's mantissa
// truncated to 23 bits, built from the bits like the conversions, so no FP64 <-> FP32
// conversion instruction is issued) has a relative error e < 2^-21; one third-order step
//   r = 1 - v y^2,  y <- y (1 + r/2 + 3 r^2 / 8)
// (the series of (1 - r)^(-1/2) to second order) leaves 5/16 |r|^3 ~ 2.5 e^3 < 2^-61, so the
// result carries FP64 accuracy: r is formed by one FMA from the rounded v y, and the
// correction is a small multiple of y.  Five FP64 operations.  v outside the FP32 normal
// range takes the FP64 library routine.
__device__ __forceinline__ double rsqrt_newton(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ffull) - 1023;
    if (ex < -126 || ex > 127) return rsqrt(v);
    const float vf = __uint_as_float(((unsigned)(ex + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffull));
    const double y = f32_to_f64_bits(rsqrtf(vf));
    const double r = fma(-v * y, y, 1.0);
    return fma(y * r, fma(r, 0.375, 0.5), y);
}

// 1/v, v > 0, for the LDL^T pivots, in two FP64 operations.  With v = M 2^ex (M in
// [1, 2)):
//   * y0 = the approximate FP32 reciprocal of M's first 24 bits (relative error < 2^-21);
//   * e = 1 - M y0 in FP32, from M split into its first 24 bits and the rest (each
//     product through an FMA), so y0 (1 + e) is within ~2^-42 of 1/M;
//   * that value as a fixed-point integer in units of 2^-53 (y0 exactly, plus y0 e
//     rounded to units of 2^-45), normalised into an FP64 number with 2^-ex folded into
//     its exponent: integer work only;
//   * one FP64 Newton step, e2 = 1 - v y1, y = y1 + y1 e2, squares that error (below
//     2^-80 before the last rounding).
// v outside [2^-125, 2^126) takes an FP64 division.
__device__ __forceinline__ double rcp_newton(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ffull) - 1023;
    if (ex < -125 || ex > 125) return 1.0 / v;
    const float mh = __uint_as_float(0x3f800000u | (unsigned)((b >> 29) & 0x7fffffull));
    const float ml = __uint2float_rn((unsigned)(b & 0x1fffffffull)) * 0x1p-52f;
    float y0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(mh));
    float e = fmaf(-mh, y0, 1.0f);
    e = fmaf(-ml, y0, e);
    const float dlt = __fmul_rn(y0, e);
    const unsigned uy = __float_as_uint(y0);
    const int sh = (int)((uy >> 23) & 0xffu) - 127 + 30;     // y0 in [1/2, 1]: 29 or 30
    if (sh < 0 || sh > 40) return 1.0 / v;
    const long long q0 = (long long)(0x800000u | (uy & 0x7fffffu)) << sh;
    const long long q1 = q0 + ((long long)__float2int_rn(dlt * 0x1p45f) << 8);
    const int top = 63 - __clzll(q1);                        // 51 .. 53
    const unsigned long long mant = top >= 52 ? (unsigned long long)q1 >> (top - 52)
                                              : (unsigned long long)q1 << (52 - top);
    const long long bits = ((long long)(1023 + top - 53 - ex) << 52) |
                           (long long)(mant & 0x000fffffffffffffull);
    const double y1 = __longlong_as_double(bits);
    return fma(y1, fma(-v, y1, 1.0), y1);
}

// digamma(x), x > 0: shift upward with psi(x) = psi(x+1) - 1/x until x >= 12, then the
// asymptotic expansion psi(z) = ln z - 1/(2z) - sum_k B_2k / (2k z^2k).  Outside the
// domain (x <= 0, NaN or infinite) the result is NaN; the shift loop then never starts,
// so it runs at most 12 times for every input.
__device__ inline double dev_digamma(double x) {
    if (!(x > 0.0) || !(x <= 1.7976931348623157e308)) return __longlong_as_double(0x7ff8000000000000ll);
    double acc = 0.0;
    while (x < 12.0) { acc -= 1.0 / x; x += 1.0; }
    double iz = 1.0 / x, z2 = iz * iz;
    double s = z2 * (1.0 / 12.0 - z2 * (1.0 / 120.0 - z2 * (1.0 / 252.0 - z2 * (1.0 / 240.0
               - z2 * (1.0 / 132.0 - z2 * (691.0 / 32760.0))))));
    return acc + log(x) - 0.5 * iz - s;
}

// Arguments of the pass kernel (K1).
struct PassArgs {
    const double* __restrict__ locs;
    const double* __restrict__ y;
    const double* __restrict__ X;
    const int32_t* __restrict__ NN;
    const double* __restrict__ covparms;
    const double* __restrict__ mtab;   // Matern table (global), or nullptr
    const float* __restrict__ mtabf;   // FP32 Matern table for the mixed path, or nullptr
    double* __restrict__ partials;     // [gridDim.x][nstat]
    int* status;                       // [0] status code
    long long* bad;                    // first failing observation
    long long n;
    int d, p, m;
    int nstat, nv;
    int slot_stride;                   // doubles per slot
    int acc_per_lane;                  // ceil(nstat / L)
    int tab_in_smem;                   // copy the Matern table into shared memory
    // grouped conditioning (the grouped kernels only): block b is blk_idx[blk_off[b] ..
    // blk_off[b + 1]), its conditioning set then its nmemb[b] members
    const long long* blk_off;
    const int32_t* blk_idx;
    const int32_t* nmemb;
    const int32_t* gorder;             // unit u is group gorder[u] (nullptr: group u)
    long long ngroups;                 // units of this launch
    long long ngroups_all;             // groups in blk_off / nmemb
    int gchunk = 1;                    // members whose terms are formed together
    int* unit_counter = nullptr;       // grouped: next unit for a slot (zero at launch), or
                                       // nullptr for a fixed stride; one record per unit
};

// Arguments of the batched pass kernel: many datasets (common d, p, covariance family),
// concatenated; each has its own n, m and theta.  Work is a list of tiles, each a range of
// observations of one dataset; each tile's sums become one record.
// Where dataset b of a batch lives: offsets (in rows of locs and X, entries of y and of
// the flat NNarray) and its n and m.  Datasets may share rows (fields observed at the
// same locations share locs, X and NNarray).
struct DatasetDesc {
    long long loc, x, y, nn;
    int n, m;
};

struct BatchArgs {
    PassArgs base;                      // locs/y/X/NN base pointers; m = largest m; sizes
    const DatasetDesc* __restrict__ desc;   // nbatch
    const double* __restrict__ covparms_b;  // nbatch x q
    const double* __restrict__ tabs;        // nbatch x MT_DOUBLES (Matern)
    const float* __restrict__ tabsf;        // nbatch x MT_FLOATS (Matern, mixed)
    const int4* __restrict__ tiles;         // (dataset, first, end, unused)
    const int* __restrict__ tile_ids;       // this launch's tiles (indices into tiles), or
                                            // nullptr for tiles 0 .. ntiles - 1
    int ntiles;                             // tiles of this launch
    int* tile_counter;
    int* status_b;                      // nbatch
    long long* bad_b;                   // nbatch
    const int* active_b;                // nbatch flags (datasets to evaluate), or nullptr = all
    double* factor;                     // nullptr, or the factor rows (see vecchia_point)
};

// Device-side error reporting: the first error code wins; the smallest failing
// observation index is kept.
__device__ __forceinline__ void report(int* status, long long* bad, int code, long long i) {
    atomicCAS(status, 0, code);
    if (i >= 0) atomicMin(bad, i);
}

}  // namespace vg
