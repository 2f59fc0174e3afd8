// vg_pass.cuh -- K1: the fused per-observation Vecchia pass, FP64 or mixed precision.
//
// Algorithm 1 of the paper, one observation at a time per "group" of L lanes of a warp
// (L = 1, 2, 4, 8, 16 or 32 lanes per observation, chosen per block size).  The
// conditioning block of an observation lives in a shared-memory slot owned by its group;
// every step is done by the L lanes together:
//
//   gather      NNarray row -> block indices (neighbours reversed, observation last),
//               coordinates relative to the observation and divided by their range,
//               y and X rows                                        (Algorithm 1: the
//               substitution of the neighbours, covariance, factor, solves, sums)
//   assembly    strict lower triangle of the covariance, FP64 diagonal sigma2 (1 + tau2)
//   factor      right-looking LDL^T (Sigma = U D U^T, U unit lower); y and X ride along as
//               extra rows of a bordered matrix, so the same sweep produces
//               z = D^-1 U^-1 (y, X); FP64 blocks make every update of a step one item
//               and spread the items evenly over the lanes, FP32 blocks give each lane
//               whole rows (their cost is instructions, not FP64 slots).  The Cholesky factor of Algorithm 1 is
//               L = U D^1/2: L^-1 y = D^1/2 z, log det = sum log d_c, and its last row of
//               the inverse is b = d_K^-1/2 u with u the last row of U^-1
//   terms       logdet_i = log d_K, ell = d_K^1/2 z_y[K], x = d_K^1/2 z_X[K]
//   derivative  u (back substitution, no divisions), h_j = dSigma_j u^T with each pair
//               (a, c) evaluated once (a conflict-free round-robin pair schedule lets the
//               lanes scatter into h without atomics), f_j = U^-1 h_j, then the dot
//               products that give dlogdet, dySy, dySX, dXSX and the information (the
//               derivative terms Algorithm 1 leaves out, written out from
//               dL = L Phi(L^-1 dSigma L^-T) and rescaled from L to U and D)
//   accumulate  per-observation values into per-lane FP64 running sums (shared memory),
//               then a fixed-order block reduction into one partial record per block.
//
// The steps are device functions (assemble_block, ldl_augmented, conditional_terms,
// finish_terms, ...) shared by three bodies: vecchia_point (one observation),
// vecchia_group (grouped conditioning: one factorisation per group, then
// conditional_terms for each member on the leading block ending at its row) and
// vecchia_point_aniso (one range per coordinate: the d + 1 derivative vectors live in the
// slot and their work is split into lane items).
//
// T is the working type of the block.  T = double is the FP64 path.  T = float is the
// mixed path: the covariance entries, the trailing updates of the factorisation, the
// solves and the derivative vectors are FP32; the pivots (the diagonal of the
// factorisation, accumulated in FP64 from the exact products of FP32 values), the
// per-observation dot products and values, every sum over observations, the profile step
// and the Fisher step are FP64.
//
// FP64 on this GPU issues one warp instruction per 64 cycles per SM sub-partition whatever
// the number of active lanes, so the mapping keeps all lanes busy: updates, pairs and dot
// products are items spread evenly over the L lanes of a group, the pivots are FP64
// reciprocals from an FP32 seed and one third-order correction (rcp_newton, three FP64
// operations), and the derivative solves need no divisions.
#pragma once
#include "vg_common.cuh"
#include "vg_matern.cuh"

namespace vg {

// Per-type arithmetic used by the pass.  to64 widens a block value to FP64 (exactly; from
// the bits for FP32, so that no conversion instruction is issued), fromd narrows an FP64
// value to the working type (round to nearest, from the bits for FP32).
template <typename T>
struct Num;
template <>
struct Num<double> {
    static __device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ double to64(double x) { return x; }
    static __device__ __forceinline__ double fromd(double x) { return x; }
};
template <>
struct Num<float> {
    static __device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    static __device__ __forceinline__ double to64(float x) { return f32_to_f64_bits(x); }
    static __device__ __forceinline__ float fromd(double x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(x);
        const int ex = (int)((b >> 52) & 0x7ffull) - 1023;
        if (ex < -126 || ex > 127) return (float)x;
        unsigned u = ((unsigned)(b >> 32) & 0x80000000u) | ((unsigned)(ex + 127) << 23) |
                     (unsigned)((b >> 29) & 0x7fffffull);
        u += (unsigned)((b >> 28) & 1ull);       // round half up; a carry moves the exponent
        return __uint_as_float(u);
    }
};

// Matern lookups in the working type: FP64 table (split Horner) or FP32 table.
template <typename T>
struct MaternT;
template <>
struct MaternT<double> {
    using Tab = double;
    static __device__ __forceinline__ double F0(const double* tab, double s, double nu, double psi,
                                                double sc0) {
        return matern_F0(tab, s, nu, psi, sc0);
    }
    static __device__ __forceinline__ void F12(const double* tab, double s, double nu, double psi,
                                               double sc1, double sc2, double& F1, double& F2) {
        matern_F12(tab, s, nu, psi, sc1, sc2, F1, F2);
    }
};
template <>
struct MaternT<float> {
    using Tab = float;
    static __device__ __forceinline__ float F0(const float* tab, float s, double nu, double psi,
                                               double sc0) {
        return matern_F0f(tab, s, nu, psi, sc0);
    }
    static __device__ __forceinline__ void F12(const float* tab, float s, double nu, double psi,
                                               double sc1, double sc2, float& F1, float& F2) {
        matern_F12f(tab, s, nu, psi, sc1, sc2, F1, F2);
    }
};

// Layout of one slot.  Working-type arrays first (offsets in T elements), then FP64 arrays
// (offsets in doubles from Dbyte).  K = m + 1, Q = derivative vectors.
//   A     packed strict lower triangle (row r at r (r - 1) / 2, entries c < r; the
//         diagonal lives in dg); after
//         the derivative solves the same bytes hold Gs (Q x K FP64), except in the grouped
//         kernels, whose factor serves every member of the group: there Gs has its own
//         region after V
//   Y     (1 + p) x K augmented rows: y and the columns of X, then z = D^-1 U^-1 (y, X)
//   loc   d x K coordinates relative to the observation, divided by their ranges
//   u     K: the unscaled pivot column during the factorisation, then u = last row of U^-1;
//         then (sized for it) the FP64 per-observation values V.  Grouped kernels: gchunk
//         rows of U^-1, one per member whose terms are formed together
//   G     Q x K: h_j = dSigma_j u^T, then f_j = U^-1 h_j (grouped: gchunk such blocks)
//   D1    exponential families (all but the Matern): per-pair weights reused by the
//         derivative step
//   (lf)  Matern, FP64 block: once the covariance is assembled, loc is rewritten in place
//         as double-float pairs (hi, lo FP32), from which the derivative step forms squared
//         distances without FP64 work
//   dg    K FP64: diagonal of the factorisation, then the pivots d_c
//   dinv  K FP64: 1 / d_c
//   lp    2 FP64: the group's running product of pivot mantissas and sum of exponents, so
//         that log det needs one logarithm per group and tile, not one per observation
struct SlotLayout {
    int K, A, Y, loc, u, G, D1, nT, Dbyte, dg, dinv, lp, Gs, bytes;
    __host__ __device__ void init(int m, int d, int p, int cov, int nv, int tsize,
                                  bool grouped = false, int gchunk = 1) {
        K = m + 1;
        const int Q = npair_derivs(cov, d) + 1;
        int asz = K * (K - 1) / 2;
        const int gs = (Q * K * 8 + tsize - 1) / tsize;
        if (!grouped && gs > asz) asz = gs;
        const int ch = grouped ? gchunk : 1;   // members whose terms are formed together
        A = 0;
        Y = A + asz;
        loc = Y + (1 + p) * K;
        u = loc + d * K;
        if (tsize == 4) u += (u & 1);          // 8-byte aligned: V is FP64
        int usz = (nv * 8 + tsize - 1) / tsize;
        if (usz < ch * K) usz = ch * K;
        G = u + usz;
        D1 = G + ch * Q * K;
        nT = D1 + (cov == COV_MATERN ? 0 : K * (K - 1) / 2);
        Dbyte = ((nT * tsize + 7) / 8) * 8;
        dg = 0;
        dinv = K;
        lp = 2 * K;
        Gs = grouped ? 2 * K + 2 : -1;         // -1: over A
        bytes = Dbyte + (2 * K + 2 + (grouped ? Q * K : 0)) * 8;
        bytes = ((bytes / 8) | 1) * 8;  // odd number of 8-byte words: slots spread over banks
    }
};

// Synchronises the lanes of a group and orders their shared-memory accesses.  Also
// issued for one-lane groups: it is then a memory barrier between the phases.
template <int L>
__device__ __forceinline__ void gsync(unsigned mask) {
    __syncwarp(mask);
}

// sums over the L lanes of a group (xor partners stay inside the group)
template <int L, typename U>
__device__ __forceinline__ U gsum(U v, unsigned mask) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// Pair k of round r of the round-robin (circle) schedule on Nv = Kp or Kp+1 vertices.
// Within a round all pairs are vertex-disjoint.  Returns false for pairs with the dummy
// vertex (odd Kp).  The pair is returned with a > c.
__device__ __forceinline__ bool circle_pair(int Kp, int Nv, int r, int k, int& a, int& c) {
    int u, v;
    if (k == 0) { u = Nv - 1; v = r; }
    else {
        u = r + k; if (u >= Nv - 1) u -= Nv - 1;
        v = r - k; if (v < 0) v += Nv - 1;
    }
    if (u >= Kp || v >= Kp) return false;
    a = u > v ? u : v;
    c = u > v ? v : u;
    return true;
}

// Everything the per-observation body needs: the group's lanes and shared-memory slot,
// the data of the dataset being processed, and per-pass constants derived from theta.
template <typename T, typename Tab>
struct PassEnv {
    // group
    int gl;
    unsigned gmask;
    // slot (shared memory)
    T *A, *Yg, *loc, *u, *G, *D1;
    float2* locf;         // Matern, FP64 block: the coordinates as double-float pairs
    double *Gs, *dg, *dinv, *V, *lp;
    int Kmax;             // slot stride: largest block size of the launch
    // dataset
    const double* locs;
    const double* y;
    const double* X;
    const int32_t* NN;
    int d, p, m;          // m: NNarray row width - 1 of this dataset
    int* status;
    long long* bad;
    // theta-derived
    double nu, m_psi, sig2, inv_r1, inv_r2, diag64;
    T sig2T, inv_r1T, inv_r2T;
    const double* inv_rk;  // COV_ANISO: 1 / rho_k, k < d (shared memory)
    const T* inv_rkT;
    const Tab* tab;
    // record formulas and per-lane sums
    const uint64_t* sidx;
    double* acc;
    int nstat, vb0, vstep, vmm;
    // factor mode: when set, the body stops after b = last row of L^-1 and writes it here
    // (row i at factor + i (m+1), in NNarray order: entry 0 for the observation, entry c for
    // neighbour NNarray[i][c], 0 for padding)
    double* factor;
    // grouped conditioning (see PassArgs)
    const long long* blk_off;
    const int32_t* blk_idx;
    const int32_t* nmemb;
    long long n;
    int gchunk;           // members whose terms are formed together
};

// Record formulas: entry t of the per-observation record is V[u1] V[v1] + V[u2] V[v2],
// the four indices packed as 16-bit fields.
__host__ __device__ constexpr uint64_t rec_pack(int a, int b, int c, int e) {
    return (uint64_t)a | ((uint64_t)b << 16) | ((uint64_t)c << 32) | ((uint64_t)e << 48);
}

// Writes the record formulas for p regression columns and Q derivative parameters.
//   V[0] = 1, V[1] = 0, V[2] = 0 (logdet_i goes through the group's pivot product),
//   V[3] = ell, V[4..4+p) = x,
//   V[vb_j + 0] = md_j, +1 = dell_j, +2.. = dx_j (p), +2+p = -md_j/2,
//   then mm_jl = m_j . m_l for j <= l (from vmm on).
__device__ inline void build_record_index(uint64_t* sidx, int p, int Q, int vb0, int vstep,
                                          int vmm) {
    int t = 0;
    sidx[t++] = rec_pack(2, 0, 1, 1);                                   // logdet
    sidx[t++] = rec_pack(3, 3, 1, 1);                                   // ySy
    for (int a = 0; a < p; ++a)
        for (int b = a; b < p; ++b) sidx[t++] = rec_pack(4 + a, 4 + b, 1, 1);   // XSX
    for (int a = 0; a < p; ++a) sidx[t++] = rec_pack(3, 4 + a, 1, 1);           // ySX
    for (int j = 0; j < Q; ++j) {
        const int vb = vb0 + j * vstep;
        sidx[t++] = rec_pack(vb, 0, 1, 1);                              // dlogdet_j
        sidx[t++] = rec_pack(3, vb + 1, vb + 1, 3);                     // dySy_j = 2 ell dell_j
        for (int a = 0; a < p; ++a) sidx[t++] = rec_pack(vb + 1, 4 + a, 3, vb + 2 + a);  // dySX
        for (int a = 0; a < p; ++a)
            for (int b = a; b < p; ++b)
                sidx[t++] = rec_pack(vb + 2 + a, 4 + b, 4 + a, vb + 2 + b);          // dXSX
    }
    int mm = vmm;
    for (int j = 0; j < Q; ++j)
        for (int l = j; l < Q; ++l)
            sidx[t++] = rec_pack(mm++, 0, vb0 + j * vstep, vb0 + l * vstep + 2 + p);  // info
}

// LDL^T factorisation of the packed block A (Kp x Kp, diagonal in dg) with the naug rows of
// Yg (stride Kmax) riding along as extra rows of a bordered matrix, right-looking, one
// column per step.  Step c: pivot d_c = dg[c] and its reciprocal (every lane, FP64); the
// column below the pivot is scaled (l_rc = a_rc / d_c, the unscaled a_rc kept in tmp; for
// the augmented rows the scaled entry is z_c); then every entry of the trailing triangle
// and of the augmented rows right of c, a_rk -= l_rc a_kc, is one item, and the items are
// spread evenly over the group's lanes (at most one item per lane of imbalance per step).
// On return the strict lower triangle of A holds U (unit lower, Sigma = U D U^T), dg the
// pivots d_c, dinv their reciprocals and Yg rows z = D^-1 U^-1 (y, X).  The pivots and the
// diagonal updates are FP64 for both working types: with T = float every product of two
// FP32 values is exact in FP64, so the pivots carry no FP32 rounding of their own.
// Returns false when a pivot is not positive and finite.
template <int L, typename T>
__device__ __forceinline__ bool ldl_augmented(T* A, T* Yg, double* dg, double* dinv, T* tmp, int Kp,
                                              int naug, int Kmax, int gl, unsigned gmask) {
    using N = Num<T>;
    constexpr bool F64 = sizeof(T) == 8;
    for (int c = 0; c < Kp; ++c) {
        const double dc = dg[c];
        // d_c positive and finite, tested on the bits (an FP64 comparison would take the
        // FP64 unit): as a signed 64-bit integer a positive finite double lies strictly
        // between 0 and the bits of +infinity; zero, negatives and NaN fall outside
        const long long dcb = __double_as_longlong(dc);
        if (dcb <= 0 || dcb >= 0x7ff0000000000000LL) return false;
        // the reciprocal scales the FP32 column with FP32 accuracy on the mixed path (an FP32
        // reciprocal of the FP64 pivot; only the last pivot's reciprocal is taken again in
        // FP64, where the values need it)
        double ic;
        T icT;
        if constexpr (F64) {
            ic = rcp_newton(dc);
            icT = ic;
        } else {
            float r;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(N::fromd(dc)));
            icT = r;
            ic = N::to64(r);
        }
        if (((c - gl) & (L - 1)) == 0) dinv[c] = ic;
        const int nr = Kp - 1 - c;
        for (int e = gl; e < nr + naug; e += L) {
            if (e < nr) {
                const int r = c + 1 + e;
                T* Ar = A + r * (r - 1) / 2;
                const T t = Ar[c];
                tmp[r] = t;
                Ar[c] = t * icT;
            } else {
                T* z = Yg + (e - nr) * Kmax + c;
                *z = *z * icT;
            }
        }
        gsync<L>(gmask);
        // FP32 blocks: the FP64 diagonal updates form their own loop (one FP64 instruction
        // per L rows); FP64 blocks: they are items of the triangle like the rest
        if constexpr (!F64)
            for (int r = c + 1 + gl; r < Kp; r += L)
                dg[r] = fma(-N::to64(A[r * (r - 1) / 2 + c]), N::to64(tmp[r]), dg[r]);
        if constexpr (!F64) {
            // FP32 blocks: whole rows of the strict lower triangle per lane (rows c + 2 ..,
            // in a zigzag over the lanes so that long and short rows pair up), then the
            // augmented rows entry by entry.  A row costs one load of its pivot-column
            // entry and, per update, the loads of the entry and of tmp[k] (the same k in
            // every lane at once); the item bookkeeping of the FP64 blocks (which keeps
            // every lane's FP64 slots busy) would cost more integer instructions than the
            // FP32 update itself.
            const int nrt = nr - 1;
            for (int b0 = 0; b0 < nrt; b0 += 2 * L) {
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int jr = h2 == 0 ? b0 + gl : b0 + 2 * L - 1 - gl;
                    if (jr >= nrt) continue;
                    const int r = c + 2 + jr;
                    T* Ar = A + r * (r - 1) / 2;
                    const T l = Ar[c];
                    for (int k = c + 1; k < r; ++k) Ar[k] = N::fma_(-l, tmp[k], Ar[k]);
                }
            }
            for (int k = c + 1 + gl; k < Kp; k += L) {
                const T tk = tmp[k];
                for (int a = 0; a < naug; ++a) {
                    T* z = Yg + a * Kmax;
                    z[k] = N::fma_(-z[c], tk, z[k]);
                }
            }
        } else {
            // FP64 blocks: every update of the trailing triangle (diagonal included) and of
            // the augmented rows is one item; the items are spread evenly over the lanes
            const int nrt = nr;                             // rows of the item triangle
            const int ntri = nrt > 0 ? nrt * (nrt + 1) / 2 : 0;
            int e = gl;
            if (e < ntri) {
                int rr = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
                while (rr * (rr + 1) / 2 > e) --rr;
                while ((rr + 1) * (rr + 2) / 2 <= e) ++rr;
                int kk = e - rr * (rr + 1) / 2;
                for (; e < ntri; e += L) {
                    const int r = c + 1 + rr;
                    T* Ar = A + r * (r - 1) / 2;
                    const T l = Ar[c];
                    const int k = c + 1 + kk;
                    if (k == r) {
                        dg[r] = fma(-N::to64(l), N::to64(tmp[r]), dg[r]);
                    } else {
                        Ar[k] = N::fma_(-l, tmp[k], Ar[k]);
                    }
                    kk += L;
                    while (kk > rr) { kk -= rr + 1; ++rr; }
                }
            }
            if (naug > 0 && nr > 0) {
                const int e2 = e - ntri;
                int a = e2 / nr, kk = e2 - a * nr;
                while (a < naug) {
                    T* z = Yg + a * Kmax;
                    const int k = c + 1 + kk;
                    z[k] = N::fma_(-z[c], tmp[k], z[k]);
                    kk += L;
                    while (kk >= nr) { kk -= nr; ++a; }
                }
            }
        }
        gsync<L>(gmask);
    }
    return true;
}

// u = last row of U^-1 (U^T u^T = e_last, U unit lower in A): u[last] = 1 and, from the
// bottom row up, u[a] -= U[r][a] u[r] for a < r once u[r] is final.  No divisions.
template <int L, typename T>
__device__ __forceinline__ void last_row_of_Uinv(const T* A, T* u, int Kp, int gl, unsigned gmask) {
    using N = Num<T>;
    const int last = Kp - 1;
    for (int a = gl; a < Kp; a += L) u[a] = (a == last) ? (T)1 : (T)0;
    gsync<L>(gmask);
    for (int r = last; r >= 1; --r) {
        const T ur = u[r];
        const T* Ur = A + r * (r - 1) / 2;
        for (int a = gl; a < r; a += L) u[a] = N::fma_(-Ur[a], ur, u[a]);
        gsync<L>(gmask);
    }
}

// Adds the per-observation record (formulas in sidx over the value vector V) to the
// lane's FP64 running sums: lane gl owns entries gl, gl + L, ...
template <int L>
__device__ __forceinline__ void accumulate_record(const uint64_t* sidx, const double* V,
                                                  double* acc, int nstat, int gl,
                                                  unsigned gmask) {
    for (int t = gl, k = 0; t < nstat; t += L, ++k) {
        const uint64_t w = sidx[t];
        const double v1 = V[w & 0xffffu] * V[(w >> 16) & 0xffffu];
        acc[k] += fma(V[(w >> 32) & 0xffffu], V[w >> 48], v1);
    }
    gsync<L>(gmask);
}

// Covariance of the block in the slot (coordinates in loc, relative and scaled): the packed
// strict lower triangle of A and the FP64 diagonal dg (sigma2 (1 + tau2)); for the
// exponential families also the pair weights D1 that the derivative step reuses.
template <int COV, int L, typename T, typename Tab>
__device__ __forceinline__ void assemble_block(const PassEnv<T, Tab>& E, int Kp) {
    using N = Num<T>;
    using MT = MaternT<T>;
    const int gl = E.gl;
    const unsigned gmask = E.gmask;
    const int d = E.d, Kmax = E.Kmax;
    T* A = E.A; T* loc = E.loc; T* D1 = E.D1;
    const T sig2T = E.sig2T;
    const double m_psi = E.m_psi;
    const Tab* tab = E.tab;
    // the diagonal (FP64), then the strict lower triangle: pair e is (a, c) with
    // a (a - 1) / 2 <= e < a (a + 1) / 2, so every round of the loop is all off-diagonal
    for (int a = gl; a < Kp; a += L) E.dg[a] = E.diag64;
    const int ntri = Kp * (Kp - 1) / 2;
    for (int e = gl; e < ntri; e += L) {
        int a = (int)((sqrtf(8.0f * (float)e + 1.0f) + 1.0f) * 0.5f);
        while (a * (a - 1) / 2 > e) --a;
        while (a * (a + 1) / 2 <= e) ++a;
        const int c = e - a * (a - 1) / 2;
        const int ea = a * (a - 1) / 2 + c;           // packed position of (a, c)
        T C;
        if (COV == COV_EXP) {
            T s = (T)0;
            for (int k = 0; k < d; ++k) {
                T t = loc[k * Kmax + a] - loc[k * Kmax + c];
                s = N::fma_(t, t, s);
            }
            if constexpr (sizeof(T) == 8) {              // the per-pass table
                C = exp_F0(tab, s, E.sig2);
                D1[a * (a - 1) / 2 + c] = exp_F12(tab, s, E.sig2, 1);   // rho dC/drho
            } else {
                T x = N::sqrt_(s);
                T ex = sig2T * N::exp_(-x);
                C = ex;
                D1[a * (a - 1) / 2 + c] = ex * x;          // rho dC/drho
            }
        } else if (COV == COV_ST) {
            T t0 = loc[a] - loc[c];
            T t1 = loc[Kmax + a] - loc[Kmax + c];
            T t2 = loc[2 * Kmax + a] - loc[2 * Kmax + c];
            T uu = N::fma_(t0, t0, N::fma_(t1, t1, t2 * t2));
            if constexpr (sizeof(T) == 8) {              // the per-pass table
                C = exp_F0(tab, uu, E.sig2);
                D1[a * (a - 1) / 2 + c] = exp_F12(tab, uu, E.sig2, 2);  // C / D
            } else {
                T D = N::sqrt_(uu);
                T ex = sig2T * N::exp_(-D);
                C = ex;
                D1[a * (a - 1) / 2 + c] = D > (T)0 ? ex / D : (T)0;
            }
        } else {  // Matern
            T s = (T)0;
            for (int k = 0; k < d; ++k) {
                T t = loc[k * Kmax + a] - loc[k * Kmax + c];
                s = N::fma_(t, t, s);
            }
            C = MT::F0(tab, s, E.nu, m_psi, E.sig2);   // the table holds sigma2 M
        }
        A[ea] = C;
    }
    gsync<L>(gmask);
    if constexpr (COV == COV_MATERN && sizeof(T) == 8) {
        // the coordinates as double-float pairs, in place, for the derivative step
        for (int a = gl; a < Kp; a += L)
            for (int k = 0; k < d; ++k) {
                const double v = loc[k * Kmax + a];
                const float hi = Num<float>::fromd(v);
                E.locf[k * Kmax + a] = make_float2(hi, Num<float>::fromd(v - f32_to_f64_bits(hi)));
            }
        gsync<L>(gmask);
    }
}

// log d over many pivots with one logarithm: lp[0] holds a product of mantissas in [1, 2)
// (renormalised from the bits after each multiplication), the bytes of lp[1] a 64-bit
// integer sum of the binary exponents taken out; log of the whole product is
// log(lp[0]) + lp[1] log 2 (log_fold).  One FP64 multiplication per pivot instead of a
// logarithm, and the exponent sum is integer work.  A zeroed lp[1] is an exponent sum of 0.
__device__ __forceinline__ void log_pivot(double* lp, double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const long long ev = (long long)((b >> 52) & 0x7ffull) - 1023;
    const double mv = __longlong_as_double((long long)((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
    const unsigned long long pb = (unsigned long long)__double_as_longlong(lp[0] * mv);
    const long long ep = (long long)((pb >> 52) & 0x7ffull) - 1023;
    lp[0] = __longlong_as_double((long long)((pb & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
    long long* es = reinterpret_cast<long long*>(lp + 1);
    *es += ev + ep;
}
__device__ __forceinline__ double log_fold(double* lp) {
    long long* es = reinterpret_cast<long long*>(lp + 1);
    const double r = log(lp[0]) + (double)*es * 0.69314718055994530942;
    lp[0] = 1.0;
    *es = 0;
    return r;
}

// The derivative solves and the per-observation values on the leading Kp x Kp block, once
// G holds h_j = dSigma_j u^T for the Q derivative vectors (u = last row of U^-1):
//   f_j = U^-1 h_j      unit forward substitution, column by column; the items (j, a > c)
//                       of a column are spread over the lanes
//   Gs_j = f_j / d      FP64, in the bytes of A (no longer needed)
//   values              with b = d_K^-1/2 u the last row of L^-1 (L = U D^1/2) and
//                       m_j = L^-1 dSigma_j b^T = d_K^-1/2 D^-1/2 f_j:
//                         logdet_i = log d_K,  ell = d_K^1/2 z_y[K],  x = d_K^1/2 z_X[K],
//                         md_j = m_j[K] = f_j[K] / d_K,
//                         dell_j = -m_j . hat(L^-1 y) = -d_K^-1/2 f_j . hat(z_y),
//                         dx_j = -d_K^-1/2 f_j . hat(z_X),
//                         m_j . m_l = d_K^-1 f_j . Gs_l,
//                       each dot product one item (FP64 accumulation for both working
//                       types), hat() halving the last entry
// then the record is added to the lane's sums.
// finish_values: the steps after the solves, for the derivative vectors f_j at G + j Kmax
// (f_j = U^-1 h_j already formed).
template <int L, typename T, typename Tab>
__device__ __forceinline__ void finish_values(const PassEnv<T, Tab>& E, const T* G, int Kp, int Q) {
    using N = Num<T>;
    const int gl = E.gl;
    const unsigned gmask = E.gmask;
    const int p = E.p, Kmax = E.Kmax;
    const T* Yg = E.Yg;
    double* V = E.V;
    const int last = Kp - 1;
    // ---------------- Gs = f / d (FP64, over A) ----------------
    double* Gs = E.Gs;
    {
        int j = gl / Kp, a = gl - j * Kp;
        const int jstep = L / Kp, astep = L - jstep * Kp;
        while (j < Q) {
            Gs[j * Kmax + a] = N::to64(G[j * Kmax + a]) * E.dinv[a];
            j += jstep;
            a += astep;
            if (a >= Kp) { a -= Kp; ++j; }
        }
    }
    gsync<L>(gmask);
    // ---------------- per-observation values ----------------
    const double dK = E.dg[last];
    const double idK = sizeof(T) == 8 ? E.dinv[last] : rcp_newton(dK);
    const double rs = rsqrt_newton(dK);
    const double sq = dK * rs;
    const int vb0 = E.vb0, vstep = E.vstep, vmm = E.vmm;
    if (gl == 0) {
        V[0] = 1.0;
        V[1] = 0.0;
        V[2] = 0.0;                 // log d_K goes into the group's product (log_pivot)
        log_pivot(E.lp, dK);
        V[3] = N::to64(Yg[last]) * sq;
        for (int t = 0; t < p; ++t) V[4 + t] = N::to64(Yg[(1 + t) * Kmax + last]) * sq;
    }
    for (int j = gl; j < Q; j += L) {
        const double md = N::to64(G[j * Kmax + last]) * idK;
        V[vb0 + j * vstep] = md;
        V[vb0 + j * vstep + 2 + p] = -0.5 * md;
    }
    const int P1 = 1 + p;
    const int nz = Q * P1, nitems = nz + Q * (Q + 1) / 2;
    // Partial sum of item it over the rows a0, a0 + astep, ...: the nz items f_j . z_t over
    // the rows before the last (the halved last term is added by fin), the others
    // f_j . Gs_l over all Kp rows.
    auto part = [&](int it, int a0, int astep) -> double {
        const T* g;
        const T* zt = nullptr;
        const double* h = nullptr;
        int len;
        if (it < nz) {
            const int j = it / P1, t = it - j * P1;
            g = G + j * Kmax;
            zt = Yg + t * Kmax;
            len = last;
        } else {
            int r = it - nz, j = 0;
            while (r >= Q - j) { r -= Q - j; ++j; }
            g = G + j * Kmax;
            h = Gs + (j + r) * Kmax;
            len = Kp;
        }
        double s0 = 0.0, s1 = 0.0;
        int a = a0;
        if (zt) {
            for (; a + astep < len; a += 2 * astep) {
                s0 = fma(N::to64(g[a]), N::to64(zt[a]), s0);
                s1 = fma(N::to64(g[a + astep]), N::to64(zt[a + astep]), s1);
            }
            if (a < len) s0 = fma(N::to64(g[a]), N::to64(zt[a]), s0);
        } else {
            for (; a + astep < len; a += 2 * astep) {
                s0 = fma(N::to64(g[a]), h[a], s0);
                s1 = fma(N::to64(g[a + astep]), h[a + astep], s1);
            }
            if (a < len) s0 = fma(N::to64(g[a]), h[a], s0);
        }
        return s0 + s1;
    };
    auto fin = [&](int it, double sm) {
        if (it < nz) {
            const int j = it / P1, t = it - j * P1;
            sm = fma(0.5 * N::to64(G[j * Kmax + last]), N::to64(Yg[t * Kmax + last]), sm);  // hat()
            V[vb0 + j * vstep + 1 + t] = -sm * rs;
        } else {
            V[vmm + (it - nz)] = sm * idK;
        }
    };
    // Whole rounds of L items take one item per lane.  The rest, fewer than L items, are
    // split: each gets sub lanes (L / rest rounded down to a power of two) that take every
    // sub-th row and add their partial sums by shuffles, so that the last round does not
    // cost a whole item's length for a few busy lanes.
    const int full = nitems - nitems % L;
    for (int it = gl; it < full; it += L) fin(it, part(it, 0, 1));
    if (full < nitems) {
        const int rest = nitems - full;
        const int sub = 1 << (31 - __clz(L / rest));
        const int it = full + gl / sub, a0 = gl & (sub - 1);
        double sm = it < nitems ? part(it, a0, sub) : 0.0;
        for (int o = sub / 2; o > 0; o >>= 1) sm += __shfl_xor_sync(gmask, sm, o);
        if (it < nitems && a0 == 0) fin(it, sm);
    }
    gsync<L>(gmask);
    accumulate_record<L>(E.sidx, V, E.acc, E.nstat, gl, gmask);
}

template <int L, typename T, typename Tab>
__device__ __forceinline__ void finish_terms(const PassEnv<T, Tab>& E, int Kp, int Q) {
    using N = Num<T>;
    const int gl = E.gl;
    const unsigned gmask = E.gmask;
    const int Kmax = E.Kmax;
    const T* A = E.A; T* G = E.G;
    const int last = Kp - 1;
    // ---------------- f_j = U^-1 h_j (unit lower, in place) ----------------
    // FP64 blocks: the items (j, a > c) of a column spread evenly over the lanes; FP32
    // blocks: rows a per lane, all Q vectors of a row together (one load of U[a][c], no
    // item bookkeeping)
    for (int c = 0; c < last; ++c) {
        if constexpr (sizeof(T) == 4) {
            for (int a = c + 1 + gl; a < Kp; a += L) {
                const T l = A[a * (a - 1) / 2 + c];
                for (int j = 0; j < Q; ++j)
                    G[j * Kmax + a] = N::fma_(-l, G[j * Kmax + c], G[j * Kmax + a]);
            }
        } else {
            const int nr = last - c;
            int j = gl / nr, off = gl - j * nr;
            const int jstep = L / nr, ostep = L - jstep * nr;
            while (j < Q) {
                const int a = c + 1 + off;
                G[j * Kmax + a] = N::fma_(-A[a * (a - 1) / 2 + c], G[j * Kmax + c], G[j * Kmax + a]);
                j += jstep;
                off += ostep;
                if (off >= nr) { off -= nr; ++j; }
            }
        }
        gsync<L>(gmask);
    }
    finish_values<L, T, Tab>(E, G, Kp, Q);
}

// The pair-derivative entries dSigma_j[a][c], j < NG, of the block in the slot (a > c):
// from the pair weights D1 kept by the assembly (exponential families), or from the
// coordinates and the per-pass table (Matern; on the FP64 path the squared distance in
// double-float arithmetic from the pairs in locf, about 2^-46 relative, enough for
// derivative entries, so that the only FP64 work left per pair is the two table values).
template <int COV, typename T, typename Tab>
__device__ __forceinline__ void pair_derivs(const PassEnv<T, Tab>& E, int a, int c, T* dv) {
    using N = Num<T>;
    using MT = MaternT<T>;
    constexpr int NG = npair_derivs(COV);
    const int d = E.d, Kmax = E.Kmax;
    const T* loc = E.loc; const T* D1 = E.D1;
    const T inv_r1T = E.inv_r1T, inv_r2T = E.inv_r2T;
    const double inv_r1 = E.inv_r1, m_psi = E.m_psi;
    const Tab* tab = E.tab;
    if (COV == COV_EXP) {
        dv[0] = D1[a * (a - 1) / 2 + c] * inv_r1T;
    } else if (COV == COV_ST) {
        T t0 = loc[a] - loc[c];
        T t1 = loc[Kmax + a] - loc[Kmax + c];
        T t2 = loc[2 * Kmax + a] - loc[2 * Kmax + c];
        T w = D1[a * (a - 1) / 2 + c];
        dv[0] = w * N::fma_(t0, t0, t1 * t1) * inv_r1T;
        if (NG > 1) dv[NG - 1] = w * t2 * t2 * inv_r2T;
    } else if constexpr (sizeof(T) == 8) {
        float sh = 0.0f, sl = 0.0f;
        for (int kk = 0; kk < d; ++kk) {
            const float2 pa = E.locf[kk * Kmax + a], pc = E.locf[kk * Kmax + c];
            const float th = __fsub_rn(pa.x, pc.x);          // two-sum of the highs
            const float bb = __fsub_rn(th, pa.x);
            float te = __fadd_rn(__fsub_rn(pa.x, __fsub_rn(th, bb)), __fsub_rn(-pc.x, bb));
            te = __fadd_rn(te, __fsub_rn(pa.y, pc.y));       // plus the lows
            const float t1 = __fadd_rn(th, te);
            const float tl = __fsub_rn(te, __fsub_rn(t1, th));
            const float pp = __fmul_rn(t1, t1);              // t^2 = t1^2 + 2 t1 tl
            float pe = fmaf(t1, t1, -pp);
            pe = fmaf(2.0f * t1, tl, pe);
            const float ss = __fadd_rn(sh, pp);              // (sh, sl) += (pp, pe)
            const float b2 = __fsub_rn(ss, sh);
            float er = __fadd_rn(__fsub_rn(sh, __fsub_rn(ss, b2)), __fsub_rn(pp, b2));
            er = __fadd_rn(er, __fadd_rn(sl, pe));
            sh = __fadd_rn(ss, er);
            sl = __fsub_rn(er, __fsub_rn(sh, ss));
        }
        double F1, F2;
        matern_F12_df(tab, sh, sl, E.nu, m_psi, E.sig2 * inv_r1, E.sig2, F1, F2);
        dv[0] = F1;                      // dC/drho and dC/dnu from the table
        if (NG > 1) dv[NG - 1] = F2;
    } else {
        T s = (T)0;
        for (int kk = 0; kk < d; ++kk) {
            T t = loc[kk * Kmax + a] - loc[kk * Kmax + c];
            s = N::fma_(t, t, s);
        }
        T F1, F2;
        MT::F12(tab, s, E.nu, m_psi, E.sig2 * inv_r1, E.sig2, F1, F2);
        dv[0] = F1;                      // dC/drho and dC/dnu from the table
        if (NG > 1) dv[NG - 1] = F2;
    }
}

// One conditional on the leading Kp x Kp block of the factor in the slot (its last row,
// Kp - 1, is the observation; the rows above are what it conditions on): u = last row of
// U^-1, h_j = dSigma_j u^T with each pair (a, c) evaluated once (a conflict-free round-robin
// pair schedule lets the lanes scatter into h without atomics), then finish_terms.
// i is the observation (factor rows).
template <int COV, int L, typename T, typename Tab>
__device__ __forceinline__ void conditional_terms(const PassEnv<T, Tab>& E, int Kp, long long i) {
    using N = Num<T>;
    constexpr int NG = npair_derivs(COV);
    constexpr int Q = NG + 1;
    const int gl = E.gl;
    const unsigned gmask = E.gmask;
    const int m = E.m, Kmax = E.Kmax;
    T* u = E.u; T* G = E.G;
    const T sig2T = E.sig2T;

    last_row_of_Uinv<L, T>(E.A, u, Kp, gl, gmask);
    if (E.factor) {
        // b = last row of L^-1 = d_K^-1/2 u, in NNarray order
        const double rs = rsqrt_newton(E.dg[Kp - 1]);
        double* fr = E.factor + i * (long long)(m + 1);
        for (int c = gl; c <= m; c += L) fr[c] = (c < Kp) ? N::to64(u[Kp - 1 - c]) * rs : 0.0;
        gsync<L>(gmask);
        return;
    }

    // ---------------- h_j = dSigma_j u^T ----------------
    // h for the pair-derivative parameters starts at 0; the nugget one is sigma2 u.
    for (int a = gl; a < Kp; a += L) {
#pragma unroll
        for (int j = 0; j < NG; ++j) G[j * Kmax + a] = (T)0;
        G[NG * Kmax + a] = sig2T * u[a];
    }
    gsync<L>(gmask);
    {
        const int Nv = (Kp & 1) ? Kp + 1 : Kp;
        const int npr = Nv / 2;
        for (int r = 0; r < Nv - 1; ++r) {
            for (int k = gl; k < npr; k += L) {
                int a, c;
                if (!circle_pair(Kp, Nv, r, k, a, c)) continue;
                T dv[NG];
                pair_derivs<COV, T, Tab>(E, a, c, dv);
                const T ua = u[a], uc = u[c];
#pragma unroll
                for (int j = 0; j < NG; ++j) {
                    G[j * Kmax + a] = N::fma_(dv[j], uc, G[j * Kmax + a]);
                    G[j * Kmax + c] = N::fma_(dv[j], ua, G[j * Kmax + c]);
                }
            }
            gsync<L>(gmask);
        }
    }
    finish_terms<L, T, Tab>(E, Kp, Q);
}

// Grouped conditioning: the terms of members r0 .. r0 + cnt - 1 (cnt <= gchunk) of the
// factored block in the slot.  Member r's terms are the single-observation terms on the
// leading (r + 1) block: u_r = row r of U^-1 (the leading block's U^-1 is the leading block
// of U^-1), h_j = dSigma_j u_r^T on rows <= r, f_j = U^-1 h_j, then the values.  Formed
// together, each pair (a, c) of the chunk's block (Kc = r0 + cnt rows) is evaluated once
// for all its members, and every step carries up to cnt members' items between the same
// barriers:
//   W   row k = u_{r0+k} (zero past its own row), by back substitution from row Kc - 1 up:
//       row t updates the members whose row t is final (r0 + k >= t)
//   H   G + k Q Kmax holds member k's h_j; pair (a, c) adds to the members with
//       r0 + k >= a (both rows inside the member's block)
//   F   unit forward substitution of all members' vectors, column by column (rows past a
//       member's own are carried along and never read)
// then Gs, the values and the record of each member in turn (finish_values; V reuses W).
template <int COV, int L, typename T, typename Tab>
__device__ __forceinline__ void group_chunk_terms(const PassEnv<T, Tab>& E, int r0, int cnt) {
    using N = Num<T>;
    constexpr int NG = npair_derivs(COV);
    constexpr int Q = NG + 1;
    const int gl = E.gl;
    const unsigned gmask = E.gmask;
    const int Kmax = E.Kmax;
    const T* A = E.A;
    T* W = E.u;
    T* G = E.G;
    const int Kc = r0 + cnt;
    // ---------------- W: rows r0 .. Kc - 1 of U^-1 ----------------
    {
        int k = gl / Kc, a = gl - k * Kc;
        const int ks = L / Kc, as = L - ks * Kc;
        while (k < cnt) {
            W[k * Kmax + a] = (a == r0 + k) ? (T)1 : (T)0;
            k += ks;
            a += as;
            if (a >= Kc) { a -= Kc; ++k; }
        }
    }
    gsync<L>(gmask);
    for (int t = Kc - 1; t >= 1; --t) {
        const int k0 = t > r0 ? t - r0 : 0;
        const T* Ut = A + t * (t - 1) / 2;
        int k = gl / t, a = gl - k * t;
        k += k0;
        const int ks = L / t, as = L - ks * t;
        while (k < cnt) {
            W[k * Kmax + a] = N::fma_(-Ut[a], W[k * Kmax + t], W[k * Kmax + a]);
            k += ks;
            a += as;
            if (a >= t) { a -= t; ++k; }
        }
        gsync<L>(gmask);
    }
    // ---------------- H: h_j = dSigma_j u^T per member ----------------
    {
        int k = gl / Kc, a = gl - k * Kc;
        const int ks = L / Kc, as = L - ks * Kc;
        while (k < cnt) {
            T* Gk = G + k * Q * Kmax;
#pragma unroll
            for (int j = 0; j < NG; ++j) Gk[j * Kmax + a] = (T)0;
            Gk[NG * Kmax + a] = E.sig2T * W[k * Kmax + a];
            k += ks;
            a += as;
            if (a >= Kc) { a -= Kc; ++k; }
        }
    }
    gsync<L>(gmask);
    {
        const int Nv = (Kc & 1) ? Kc + 1 : Kc;
        const int npr = Nv / 2;
        for (int r = 0; r < Nv - 1; ++r) {
            for (int q = gl; q < npr; q += L) {
                int a, c;
                if (!circle_pair(Kc, Nv, r, q, a, c)) continue;
                T dv[NG];
                pair_derivs<COV, T, Tab>(E, a, c, dv);
                for (int k = a > r0 ? a - r0 : 0; k < cnt; ++k) {
                    T* Gk = G + k * Q * Kmax;
                    const T wa = W[k * Kmax + a], wc = W[k * Kmax + c];
#pragma unroll
                    for (int j = 0; j < NG; ++j) {
                        Gk[j * Kmax + a] = N::fma_(dv[j], wc, Gk[j * Kmax + a]);
                        Gk[j * Kmax + c] = N::fma_(dv[j], wa, Gk[j * Kmax + c]);
                    }
                }
            }
            gsync<L>(gmask);
        }
    }
    // ---------------- F: f_j = U^-1 h_j per member (unit lower, in place) ----------------
    for (int c = 0; c < Kc - 1; ++c) {
        const int k0 = c >= r0 ? c - r0 + 1 : 0;      // members with rows past c
        const int nr = Kc - 1 - c;
        const int nkj = (cnt - k0) * Q;
        T* Gc = G + k0 * Q * Kmax;
        if constexpr (sizeof(T) == 4) {          // FP32: rows per lane (see finish_terms)
            for (int a = c + 1 + gl; a < Kc; a += L) {
                const T l = A[a * (a - 1) / 2 + c];
                for (int kj = 0; kj < nkj; ++kj) {
                    T* g = Gc + kj * Kmax;
                    g[a] = N::fma_(-l, g[c], g[a]);
                }
            }
        } else {
            int kj = gl / nr, off = gl - kj * nr;
            const int ks = L / nr, os = L - ks * nr;
            while (kj < nkj) {
                T* g = Gc + kj * Kmax;
                const int a = c + 1 + off;
                g[a] = N::fma_(-A[a * (a - 1) / 2 + c], g[c], g[a]);
                kj += ks;
                off += os;
                if (off >= nr) { off -= nr; ++kj; }
            }
        }
        gsync<L>(gmask);
    }
    for (int k = 0; k < cnt; ++k) finish_values<L, T, Tab>(E, G + k * Q * Kmax, r0 + k + 1, Q);
}

// Algorithm 1 for observation i of the dataset in E (all L lanes of the group call it).
template <int COV, int L, typename T, typename Tab>
__device__ __forceinline__ void vecchia_point(const PassEnv<T, Tab>& E, long long i) {
    const int gl = E.gl;
    const unsigned gmask = E.gmask;
    const int d = E.d, p = E.p, m = E.m, Kmax = E.Kmax;
    T* Yg = E.Yg; T* loc = E.loc;
    const double inv_r1 = E.inv_r1, inv_r2 = E.inv_r2;
    // ---------------- gather ----------------
    const int32_t* row = E.NN + i * (long long)(m + 1);
    int cnt = 0, badrow = 0;
    for (int c = gl; c <= m; c += L) {
        int v = row[c];
        if (c == 0) badrow |= (v != (int)i);
        else if (v >= 0) {
            cnt++;
            badrow |= (v >= i) | (c >= 2 && row[c - 1] < 0);
        } else if (v != -1) badrow = 1;
    }
    cnt = gsum<L>(cnt, gmask);
    badrow = gsum<L>(badrow, gmask);
    if (badrow) {
        if (gl == 0) report(E.status, E.bad, ST_ARG, i);
        return;
    }
    const int Kp = cnt + 1;
    const double* li = E.locs + i * (long long)d;
    for (int a = gl; a < Kp; a += L) {
        int j = row[Kp - 1 - a];
        // coordinates relative to the observation, divided by their range parameter
        // (FP64 difference, then rounded to T): squared distances come out scaled
        for (int k = 0; k < d; ++k)
            loc[k * Kmax + a] = (T)((E.locs[(long long)j * d + k] - li[k]) *
                                    ((COV == COV_ST && k == 2) ? inv_r2 : inv_r1));
        Yg[a] = (T)E.y[j];
        for (int t = 0; t < p; ++t) Yg[(1 + t) * Kmax + a] = (T)E.X[(long long)j * p + t];
    }
    gsync<L>(gmask);

    assemble_block<COV, L, T, Tab>(E, Kp);

    // ---------------- LDL^T + forward solves of y and X ----------------
    if (!ldl_augmented<L, T>(E.A, Yg, E.dg, E.dinv, E.u, Kp, 1 + p, Kmax, gl, gmask)) {
        if (gl == 0) report(E.status, E.bad, ST_NOT_PD, i);
        gsync<L>(gmask);
        return;
    }

    conditional_terms<COV, L, T, Tab>(E, Kp, i);
}

// Grouped conditioning: block g holds a conditioning set U (ascending observation indices)
// followed by its members, consecutive observations s .. e - 1 that all come after U.  The
// group's contribution is that of the joint conditional p(y_B | y_U), which factors into
// one conditional per member on U and the earlier members: after one factorisation of the
// whole block, member row r is the last row of the leading (r + 1) x (r + 1) block (the
// leading part of U, D and z is the factorisation of the leading block), so each member's
// terms are the single-observation terms on that leading block.
template <int COV, int L, typename T, typename Tab>
__device__ __forceinline__ void vecchia_group(const PassEnv<T, Tab>& E, long long g) {
    const int gl = E.gl;
    const unsigned gmask = E.gmask;
    const int d = E.d, p = E.p, Kmax = E.Kmax;
    T* Yg = E.Yg; T* loc = E.loc;
    const long long o0 = E.blk_off[g], len = E.blk_off[g + 1] - o0;
    const int32_t* blk = E.blk_idx + o0;
    const int nm = E.nmemb[g];
    // a valid block: 1 <= members <= length <= Kmax, indices in [0, n), the conditioning
    // set ascending and before the first member, the members consecutive
    int bad = !(len >= 1 && len <= Kmax && nm >= 1 && nm <= len);
    if (!bad) {
        const int nu = (int)len - nm;
        for (int a = gl; a < (int)len; a += L) {
            const int v = blk[a];
            bad |= (v < 0) | ((long long)v >= E.n);
            if (a >= 1) {
                const int u = blk[a - 1];
                bad |= (a > nu) ? (v != u + 1) : (u >= v);
            }
        }
    }
    bad = gsum<L>(bad, gmask);
    if (bad) {
        if (gl == 0) report(E.status, E.bad, ST_ARG, g);
        return;
    }
    const int Kp = (int)len;
    // coordinates relative to the last member, divided by their range parameter
    const double* ref = E.locs + (long long)blk[Kp - 1] * d;
    for (int a = gl; a < Kp; a += L) {
        const int j = blk[a];
        for (int k = 0; k < d; ++k)
            loc[k * Kmax + a] = (T)((E.locs[(long long)j * d + k] - ref[k]) *
                                    ((COV == COV_ST && k == 2) ? E.inv_r2 : E.inv_r1));
        Yg[a] = (T)E.y[j];
        for (int t = 0; t < p; ++t) Yg[(1 + t) * Kmax + a] = (T)E.X[(long long)j * p + t];
    }
    gsync<L>(gmask);
    assemble_block<COV, L, T, Tab>(E, Kp);
    if (!ldl_augmented<L, T>(E.A, Yg, E.dg, E.dinv, E.u, Kp, 1 + p, Kmax, gl, gmask)) {
        if (gl == 0) report(E.status, E.bad, ST_NOT_PD, blk[Kp - nm]);
        gsync<L>(gmask);
        return;
    }
    const int ch = E.gchunk;
    for (int r0 = Kp - nm; r0 < Kp; r0 += ch)
        group_chunk_terms<COV, L, T, Tab>(E, r0, Kp - r0 < ch ? Kp - r0 : ch);
}

// Algorithm 1 for the exponential with one range per coordinate (COV_ANISO): Q = d + 1
// derivative vectors (d ranges, then the nugget), too many for per-lane registers, so
// every per-parameter quantity lives in the slot and the work on it is split into items
// spread over the group's lanes:
//   covariance  C = sigma2 e^-D, D = |h / rho| (coordinates stored divided by their
//               ranges), and w = C / D kept per pair
//   h_k         = dSigma_k u^T with dC/drho_k = w u_k^2 / rho_k (u = scaled difference),
//               pairs once in the round-robin schedule, the 1/rho_k applied afterwards
//   then the derivative solves and values of finish_terms.
template <int L, typename T, typename Tab>
__device__ __forceinline__ void vecchia_point_aniso(const PassEnv<T, Tab>& E, long long i) {
    using N = Num<T>;
    const int gl = E.gl;
    const unsigned gmask = E.gmask;
    const int d = E.d, p = E.p, m = E.m, Kmax = E.Kmax;
    const int NG = d, Q = d + 1;
    T* A = E.A; T* Yg = E.Yg; T* loc = E.loc; T* u = E.u; T* G = E.G; T* D1 = E.D1;
    // ---------------- gather ----------------
    const int32_t* row = E.NN + i * (long long)(m + 1);
    int cnt = 0, badrow = 0;
    for (int c = gl; c <= m; c += L) {
        const int v = row[c];
        if (c == 0) badrow |= (v != (int)i);
        else if (v >= 0) {
            cnt++;
            badrow |= (v >= i) | (c >= 2 && row[c - 1] < 0);
        } else if (v != -1) badrow = 1;
    }
    cnt = gsum<L>(cnt, gmask);
    badrow = gsum<L>(badrow, gmask);
    if (badrow) {
        if (gl == 0) report(E.status, E.bad, ST_ARG, i);
        return;
    }
    const int Kp = cnt + 1;
    const double* li = E.locs + i * (long long)d;
    for (int a = gl; a < Kp; a += L) {
        const int j = row[Kp - 1 - a];
        for (int k = 0; k < d; ++k)
            loc[k * Kmax + a] = (T)((E.locs[(long long)j * d + k] - li[k]) * E.inv_rk[k]);
        Yg[a] = (T)E.y[j];
        for (int t = 0; t < p; ++t) Yg[(1 + t) * Kmax + a] = (T)E.X[(long long)j * p + t];
    }
    gsync<L>(gmask);

    // ---------------- covariance assembly ----------------
    for (int a = gl; a < Kp; a += L) E.dg[a] = E.diag64;
    const int ntri = Kp * (Kp - 1) / 2;
    for (int e = gl; e < ntri; e += L) {
        int a = (int)((sqrtf(8.0f * (float)e + 1.0f) + 1.0f) * 0.5f);
        while (a * (a - 1) / 2 > e) --a;
        while (a * (a + 1) / 2 <= e) ++a;
        const int c = e - a * (a - 1) / 2;
        const int ea = a * (a - 1) / 2 + c;
        T s0 = (T)0, s1 = (T)0;
        int k = 0;
        for (; k + 1 < d; k += 2) {
            const T t0 = loc[k * Kmax + a] - loc[k * Kmax + c];
            const T t1 = loc[(k + 1) * Kmax + a] - loc[(k + 1) * Kmax + c];
            s0 = N::fma_(t0, t0, s0);
            s1 = N::fma_(t1, t1, s1);
        }
        if (k < d) {
            const T t0 = loc[k * Kmax + a] - loc[k * Kmax + c];
            s0 = N::fma_(t0, t0, s0);
        }
        if constexpr (sizeof(T) == 8) {                  // the per-pass table
            A[ea] = exp_F0(E.tab, s0 + s1, E.sig2);
            // C / D as a double-float pair (the derivative step works in double-float)
            reinterpret_cast<float2*>(D1)[ea] = exp_F12_pair(E.tab, s0 + s1, E.sig2, 2);
        } else {
            const T Dd = N::sqrt_(s0 + s1);
            const T C = E.sig2T * N::exp_(-Dd);
            D1[a * (a - 1) / 2 + c] = Dd > (T)0 ? C / Dd : (T)0;
            A[ea] = C;
        }
    }
    gsync<L>(gmask);

    // ---------------- LDL^T + forward solves, u ----------------
    if (!ldl_augmented<L, T>(A, Yg, E.dg, E.dinv, u, Kp, 1 + p, Kmax, gl, gmask)) {
        if (gl == 0) report(E.status, E.bad, ST_NOT_PD, i);
        gsync<L>(gmask);
        return;
    }
    last_row_of_Uinv<L, T>(A, u, Kp, gl, gmask);
    if (E.factor) {
        const double rs = rsqrt_newton(E.dg[Kp - 1]);
        double* fr = E.factor + i * (long long)(m + 1);
        for (int c = gl; c <= m; c += L) fr[c] = (c < Kp) ? N::to64(u[Kp - 1 - c]) * rs : 0.0;
        gsync<L>(gmask);
        return;
    }

    // ---------------- h_k = dSigma_k u^T ----------------
    for (int a = gl; a < Kp; a += L) {
        for (int k = 0; k < NG; ++k) G[k * Kmax + a] = (T)0;
        G[NG * Kmax + a] = E.sig2T * u[a];
        if constexpr (sizeof(T) == 8)     // the coordinates as double-float pairs, in place
            for (int k = 0; k < d; ++k) {
                const double v = loc[k * Kmax + a];
                const float hi = Num<float>::fromd(v);
                E.locf[k * Kmax + a] = make_float2(hi, Num<float>::fromd(v - f32_to_f64_bits(hi)));
            }
    }
    gsync<L>(gmask);
    {
        // Each round's items are (pair, coordinate): d per pair, spread over all the lanes
        // (the pairs of a round are vertex-disjoint, so no two items write one entry).  On
        // the FP64 path the entry w t_k^2 is formed in double-float arithmetic (t_k from the
        // coordinate pairs, w from the assembly's pair weights; about 2^-46 relative, enough
        // for derivative entries) and enters the FP64 scatter through one addition.
        const int Nv = (Kp & 1) ? Kp + 1 : Kp;
        const int npr = Nv / 2;
        for (int r = 0; r < Nv - 1; ++r) {
            int k2 = gl / NG, k = gl - k2 * NG;
            const int k2s = L / NG, ks = L - k2s * NG;
            for (; k2 < npr; ) {
                int a, c;
                if (circle_pair(Kp, Nv, r, k2, a, c)) {
                    T v;
                    if constexpr (sizeof(T) == 8) {
                        const float2 w = reinterpret_cast<const float2*>(D1)[a * (a - 1) / 2 + c];
                        const float2 pa = E.locf[k * Kmax + a], pc = E.locf[k * Kmax + c];
                        const float th = __fsub_rn(pa.x, pc.x);          // two-sum of the highs
                        const float bb = __fsub_rn(th, pa.x);
                        float te = __fadd_rn(__fsub_rn(pa.x, __fsub_rn(th, bb)), __fsub_rn(-pc.x, bb));
                        te = __fadd_rn(te, __fsub_rn(pa.y, pc.y));       // plus the lows
                        const float t1 = __fadd_rn(th, te);
                        const float tl = __fsub_rn(te, __fsub_rn(t1, th));
                        const float pp = __fmul_rn(t1, t1);              // t^2 = t1^2 + 2 t1 tl
                        float pe = fmaf(t1, t1, -pp);
                        pe = fmaf(2.0f * t1, tl, pe);
                        const float vh = __fmul_rn(w.x, pp);             // w t^2
                        float vl = fmaf(w.x, pp, -vh);
                        vl = fmaf(w.x, pe, vl);
                        vl = fmaf(w.y, pp, vl);
                        v = f32_to_f64_bits(vh) + f32_to_f64_bits(vl);
                    } else {
                        const T w = D1[a * (a - 1) / 2 + c];
                        const T t = loc[k * Kmax + a] - loc[k * Kmax + c];
                        v = (w * t) * t;
                    }
                    G[k * Kmax + a] = N::fma_(v, u[c], G[k * Kmax + a]);
                    G[k * Kmax + c] = N::fma_(v, u[a], G[k * Kmax + c]);
                }
                k2 += k2s;
                k += ks;
                if (k >= NG) { k -= NG; ++k2; }
            }
            gsync<L>(gmask);
        }
    }
    // dC/drho_k = w u_k^2 / rho_k
    for (int a = gl; a < Kp; a += L)
        for (int k = 0; k < NG; ++k) G[k * Kmax + a] *= E.inv_rkT[k];
    gsync<L>(gmask);

    finish_terms<L, T, Tab>(E, Kp, Q);
}

// The FP32 (mixed) instantiations are latency-bound: ask for three resident blocks of 256
// threads (at most 85 registers a thread; they need 80, with no meaningful spill) so that
// registers no longer cap the resident warps at 16 per SM.  The FP64 ones ask for two
// blocks of 256 threads (at most 128 registers), which lets four blocks of 128 threads or
// five of 96 share an SM when their shared memory allows.
constexpr int pass_min_blocks(int tsize) { return tsize == 4 ? 3 : 2; }

// GROUPED: the units are the blocks of grouped conditioning (PassArgs.blk_*), not single
// observations; m + 1 is then the largest block.
template <int COV, int L, typename T, bool GROUPED = false>
__global__ void __launch_bounds__(256, pass_min_blocks(sizeof(T))) k_pass(PassArgs args) {
    extern __shared__ __align__(16) double smem[];
    using MT = MaternT<T>;
    using Tab = typename MT::Tab;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int gl = lane & (L - 1);
    const int grp = tid / L;
    const int ngrp = blockDim.x / L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (lane & ~(L - 1)));
    const int d = args.d, p = args.p, m = args.m;
    const int Kmax = m + 1;
    const int Q = npair_derivs(COV, d) + 1;

    // ---- shared-memory carve-up: [Matern table | inverse ranges][stat index table][acc]
    //      [slots][int slots]
    double* sp = smem;
    const Tab* tab = sizeof(T) == 8 ? reinterpret_cast<const Tab*>(args.mtab)
                                    : reinterpret_cast<const Tab*>(args.mtabf);
    if (uses_table(COV, sizeof(T) == 8 ? 0 : 1) && args.tab_in_smem) {
        const int nwords = sizeof(T) == 8 ? MT_DOUBLES : (MT_FLOATS + 1) / 2;
        const double* src = sizeof(T) == 8 ? args.mtab : reinterpret_cast<const double*>(args.mtabf);
        for (int t = tid; t < nwords; t += blockDim.x) sp[t] = src[t];
        tab = reinterpret_cast<const Tab*>(sp);
        sp += nwords;
    }
    double* inv_rk = sp;                                   // COV_ANISO: 1 / rho_k, then in T
    T* inv_rkT = reinterpret_cast<T*>(sp + DMAX_ANISO);
    if (COV == COV_ANISO) sp += 2 * DMAX_ANISO;
    uint64_t* sidx = reinterpret_cast<uint64_t*>(sp);
    sp += args.nstat;
    double* acc = sp + (size_t)tid * args.acc_per_lane;
    double* accbase = sp;
    sp += (size_t)blockDim.x * args.acc_per_lane;
    SlotLayout SL;
    SL.init(m, d, p, COV, args.nv, (int)sizeof(T), GROUPED, args.gchunk);
    char* slotc = reinterpret_cast<char*>(sp) + (size_t)grp * args.slot_stride;
    T* slot = reinterpret_cast<T*>(slotc);
    double* slotd = reinterpret_cast<double*>(slotc + SL.Dbyte);

    // ---- per-observation value vector V (see build_record_index)
    const int vb0 = 4 + p, vstep = 3 + p, vmm = vb0 + Q * vstep;
    if (tid == 0) build_record_index(sidx, p, Q, vb0, vstep, vmm);
    for (int k = 0; k < args.acc_per_lane; ++k) acc[k] = 0.0;

    // ---- covariance parameters
    const double* th = args.covparms;
    const double sig2 = th[0];
    const double tau2 = th[nparms(COV, d) - 1];
    const bool ok = theta_ok(COV, d, th);
    if (!ok) {
        if (blockIdx.x == 0 && tid == 0) report(args.status, args.bad, ST_ARG, -1);
    }
    if (COV == COV_ANISO && ok)
        for (int k = tid; k < d; k += blockDim.x) {
            inv_rk[k] = 1.0 / th[1 + k];
            inv_rkT[k] = (T)inv_rk[k];
        }
    const T sig2T = (T)sig2;
    // EXP: rho = th[1]; MATERN: rho = th[1], nu = th[2]; ST: rho_s = th[1], rho_t = th[2]
    const double inv_r1 = 1.0 / th[1];
    const double inv_r2 = (COV == COV_ST) ? 1.0 / th[2] : 1.0;
    const T inv_r1T = (T)inv_r1, inv_r2T = (T)inv_r2;
    double m_psi = 0.0;
    if (COV == COV_MATERN && ok) m_psi = dev_digamma(th[2]);
    __syncthreads();

    const long long n = args.n;
    const long long gstride = (long long)gridDim.x * ngrp;
    PassEnv<T, Tab> E;
    E.gl = gl; E.gmask = gmask;
    E.A = slot + SL.A; E.Yg = slot + SL.Y; E.loc = slot + SL.loc; E.u = slot + SL.u;
    E.G = slot + SL.G; E.D1 = slot + SL.D1; E.locf = reinterpret_cast<float2*>(slot + SL.loc);
    E.Gs = SL.Gs < 0 ? reinterpret_cast<double*>(slotc) : slotd + SL.Gs;
    E.dg = slotd + SL.dg; E.dinv = slotd + SL.dinv; E.lp = slotd + SL.lp;
    E.V = reinterpret_cast<double*>(slot + SL.u);
    E.Kmax = Kmax;
    E.locs = args.locs; E.y = args.y; E.X = args.X; E.NN = args.NN;
    E.d = d; E.p = p; E.m = m; E.status = args.status; E.bad = args.bad;
    E.nu = (COV == COV_MATERN) ? th[2] : 0.0; E.m_psi = m_psi; E.sig2 = sig2;
    E.inv_r1 = inv_r1; E.inv_r2 = inv_r2;
    E.sig2T = sig2T; E.diag64 = sig2 * (1.0 + tau2); E.inv_r1T = inv_r1T; E.inv_r2T = inv_r2T;
    E.inv_rk = inv_rk; E.inv_rkT = inv_rkT;
    E.tab = tab; E.sidx = sidx; E.acc = acc; E.nstat = args.nstat;
    E.vb0 = vb0; E.vstep = vstep; E.vmm = vmm; E.factor = nullptr;
    E.blk_off = args.blk_off; E.blk_idx = args.blk_idx; E.nmemb = args.nmemb; E.n = n;
    E.gchunk = args.gchunk;
    if (gl == 0) { E.lp[0] = 1.0; *reinterpret_cast<long long*>(E.lp + 1) = 0; }
    if constexpr (GROUPED) {
        // Units (groups) are taken by each slot from a counter (dynamic: the groups' costs
        // vary with their block sizes, and launches of several classes may share the GPU),
        // or in a fixed stride without one.  Each unit writes its own record (the lanes'
        // sums, log det folded in), so the result does not depend on which slot ran it.
        const int lead = lane & ~(L - 1);
        long long u = (long long)blockIdx.x * ngrp + grp;
        if (args.unit_counter) {
            int v = 0;
            if (gl == 0) v = atomicAdd(args.unit_counter, 1);
            u = __shfl_sync(gmask, v, lead);
        }
        while (ok && u < args.ngroups) {
            const long long g = args.gorder ? (long long)args.gorder[u] : u;
            if (g < 0 || g >= args.ngroups_all) {
                if (gl == 0) report(args.status, args.bad, ST_ARG, u);
            } else {
                vecchia_group<COV, L, T, Tab>(E, g);
            }
            if (gl == 0) acc[0] += log_fold(E.lp);
            for (int t = gl, k = 0; t < args.nstat; t += L, ++k) {
                args.partials[(size_t)u * args.nstat + t] = acc[k];
                acc[k] = 0.0;
            }
            if (args.unit_counter) {
                int v = 0;
                if (gl == 0) v = atomicAdd(args.unit_counter, 1);
                u = __shfl_sync(gmask, v, lead);
            } else {
                u += gstride;
            }
        }
        return;
    } else {
        for (long long i = (long long)blockIdx.x * ngrp + grp; ok && i < n; i += gstride) {
            if constexpr (COV == COV_ANISO) vecchia_point_aniso<L, T, Tab>(E, i);
            else vecchia_point<COV, L, T, Tab>(E, i);
        }
    }
    // log det of the group's pivots into the record's first entry (owned by lane 0)
    if (gl == 0) acc[0] += log_fold(E.lp);

    // ---------------- block reduction (fixed order) ----------------
    __syncthreads();
    for (int t = tid; t < args.nstat; t += blockDim.x) {
        const int lr = t % L, k = t / L;
        double s = 0.0;
        for (int g = 0; g < ngrp; ++g) s += accbase[(size_t)(g * L + lr) * args.acc_per_lane + k];
        args.partials[(size_t)blockIdx.x * args.nstat + t] = s;
    }
}

// Batched pass: CTAs take tiles from an atomic counter; for each tile they stage the
// dataset's Matern table and theta-derived constants, run Algorithm 1 on the tile's
// observations and reduce the tile's sums into its own record (so the result does not
// depend on which CTA ran which tile).
template <int COV, int L, typename T>
__global__ void __launch_bounds__(256, pass_min_blocks(sizeof(T))) k_pass_batch(BatchArgs bargs) {
    extern __shared__ __align__(16) double smem[];
    using MT = MaternT<T>;
    using Tab = typename MT::Tab;
    const PassArgs& args = bargs.base;
    __shared__ int s_tile;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int gl = lane & (L - 1);
    const int grp = tid / L;
    const int ngrp = blockDim.x / L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (lane & ~(L - 1)));
    const int d = args.d, p = args.p;
    const int Kmax = args.m + 1;
    const int q = nparms(COV, d);
    const int Q = npair_derivs(COV, d) + 1;

    double* sp = smem;
    Tab* stab = reinterpret_cast<Tab*>(sp);
    const int tab_words = (uses_table(COV, sizeof(T) == 8 ? 0 : 1) && args.tab_in_smem)
                              ? (sizeof(T) == 8 ? MT_DOUBLES : (MT_FLOATS + 1) / 2) : 0;
    sp += tab_words;
    double* inv_rk = sp;                                   // COV_ANISO: 1 / rho_k, then in T
    T* inv_rkT = reinterpret_cast<T*>(sp + DMAX_ANISO);
    if (COV == COV_ANISO) sp += 2 * DMAX_ANISO;
    uint64_t* sidx = reinterpret_cast<uint64_t*>(sp);
    sp += args.nstat;
    double* acc = sp + (size_t)tid * args.acc_per_lane;
    double* accbase = sp;
    sp += (size_t)blockDim.x * args.acc_per_lane;
    SlotLayout SL;
    SL.init(args.m, d, p, COV, args.nv, (int)sizeof(T));
    char* slotc = reinterpret_cast<char*>(sp) + (size_t)grp * args.slot_stride;
    T* slot = reinterpret_cast<T*>(slotc);

    const int vb0 = 4 + p, vstep = 3 + p, vmm = vb0 + Q * vstep;
    if (tid == 0) build_record_index(sidx, p, Q, vb0, vstep, vmm);

    PassEnv<T, Tab> E;
    E.gl = gl; E.gmask = gmask;
    double* slotd = reinterpret_cast<double*>(slotc + SL.Dbyte);
    E.A = slot + SL.A; E.Yg = slot + SL.Y; E.loc = slot + SL.loc; E.u = slot + SL.u;
    E.G = slot + SL.G; E.D1 = slot + SL.D1; E.locf = reinterpret_cast<float2*>(slot + SL.loc);
    E.Gs = SL.Gs < 0 ? reinterpret_cast<double*>(slotc) : slotd + SL.Gs;
    E.dg = slotd + SL.dg; E.dinv = slotd + SL.dinv; E.lp = slotd + SL.lp;
    E.V = reinterpret_cast<double*>(slot + SL.u);
    E.Kmax = Kmax;
    E.d = d; E.p = p; E.sidx = sidx; E.acc = acc; E.nstat = args.nstat;
    E.vb0 = vb0; E.vstep = vstep; E.vmm = vmm;
    E.inv_rk = inv_rk; E.inv_rkT = inv_rkT;

    int cur_b = -1;
    bool ok = false;
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(bargs.tile_counter, 1);
        __syncthreads();
        if (s_tile >= bargs.ntiles) break;
        const int t = bargs.tile_ids ? bargs.tile_ids[s_tile] : s_tile;   // record index
        const int4 tile = bargs.tiles[t];
        const int b = tile.x;
        if (b != cur_b) {
            cur_b = b;
            const double* th = bargs.covparms_b + (size_t)b * q;
            const double sig2 = th[0], tau2 = th[q - 1];
            ok = theta_ok(COV, d, th);
            // the previous tile's lanes are past the barrier at the top of the loop
            if (COV == COV_ANISO && ok)
                for (int k = tid; k < d; k += blockDim.x) {
                    inv_rk[k] = 1.0 / th[1 + k];
                    inv_rkT[k] = (T)inv_rk[k];
                }
            E.inv_r1 = 1.0 / th[1];
            E.inv_r2 = (COV == COV_ST) ? 1.0 / th[2] : 1.0;
            E.sig2T = (T)sig2;
            E.diag64 = sig2 * (1.0 + tau2);
            E.inv_r1T = (T)E.inv_r1;
            E.inv_r2T = (T)E.inv_r2;
            E.nu = (COV == COV_MATERN) ? th[2] : 0.0;
            E.m_psi = (COV == COV_MATERN && ok) ? dev_digamma(th[2]) : 0.0;
            E.sig2 = sig2;
            const DatasetDesc D = bargs.desc[b];
            E.locs = args.locs + D.loc * d;
            E.y = args.y + D.y;
            E.X = args.X + D.x * p;
            E.NN = args.NN + D.nn;
            E.m = D.m;
            E.factor = bargs.factor ? bargs.factor + D.y * (long long)(D.m + 1) : nullptr;
            E.status = bargs.status_b + b;
            E.bad = bargs.bad_b + b;
            if (uses_table(COV, sizeof(T) == 8 ? 0 : 1)) {
                const Tab* gt = sizeof(T) == 8
                    ? reinterpret_cast<const Tab*>(bargs.tabs + (size_t)b * MT_DOUBLES)
                    : reinterpret_cast<const Tab*>(bargs.tabsf + (size_t)b * MT_FLOATS);
                if (tab_words) {
                    const double* src = reinterpret_cast<const double*>(gt);
                    double* dst = reinterpret_cast<double*>(stab);
                    for (int k = tid; k < tab_words; k += blockDim.x) dst[k] = src[k];
                    E.tab = stab;
                } else {
                    E.tab = gt;
                }
            } else {
                E.tab = nullptr;
            }
            if (!ok && tid == 0) report(E.status, E.bad, ST_ARG, -1);
        }
        for (int k = 0; k < args.acc_per_lane; ++k) acc[k] = 0.0;
        if (gl == 0) { E.lp[0] = 1.0; *reinterpret_cast<long long*>(E.lp + 1) = 0; }
        __syncthreads();
        const bool active = bargs.active_b == nullptr || bargs.active_b[b] != 0;
        if (ok && active)
            for (long long i = tile.y + grp; i < tile.z; i += ngrp) {
                if constexpr (COV == COV_ANISO) vecchia_point_aniso<L, T, Tab>(E, i);
                else vecchia_point<COV, L, T, Tab>(E, i);
            }
        if (gl == 0) acc[0] += log_fold(E.lp);
        __syncthreads();
        for (int u = tid; u < args.nstat; u += blockDim.x) {
            const int lr = u % L, k = u / L;
            double s = 0.0;
            for (int g = 0; g < ngrp; ++g) s += accbase[(size_t)(g * L + lr) * args.acc_per_lane + k];
            args.partials[(size_t)t * args.nstat + u] = s;
        }
        __syncthreads();
    }
}

}  // namespace vg
