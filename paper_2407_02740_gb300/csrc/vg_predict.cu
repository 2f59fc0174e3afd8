// vg_predict.cu -- Vecchia prediction (kriging with a neighbour set) on the device.
//
// For a target location s* with covariates x* and its m nearest observations N (rows of
// an m-column neighbour array, nearest first, -1 padded), the Gaussian process gives
//   E[y* | y_N] = x*' beta + k' Sigma_NN^-1 (y_N - X_N beta),
//   Var[y* | y_N] = c** - k' Sigma_NN^-1 k,
// with Sigma_NN the neighbours' covariance (nugget on its diagonal), k the covariances of
// s* with them and c** = sigma2 for the latent field or sigma2 (1 + tau2) for a new
// observation.  One group of L lanes per target builds the block of the neighbours
// (reversed) and the target last, with one extra row holding the residuals r = y - X beta
// (0 for the target), and runs the same left-looking Cholesky sweep as the likelihood
// pass: then the last pivot L_KK is the conditional standard deviation and the last entry
// of L^-1 r is -(k' Sigma_NN^-1 r_N) / L_KK, so mean = x*' beta - L_KK (L^-1 r)_K and
// variance = L_KK^2.  FP64 throughout.
#include <climits>

#include "vg_internal.h"
#include "vg_matern.cuh"
#include "vg_pass.cuh"

namespace vg {

struct PredArgs {
    const double* locs;      // n x d observations
    const double* y;         // n
    const double* X;         // n x p
    const double* beta;      // p
    const double* qlocs;     // nq x d targets
    const double* qX;        // nq x p
    const int32_t* NN;       // nq x m
    const double* covparms;  // q
    const double* tab;       // Matern table (sigma2 M, ...)
    double* mean;            // nq
    double* var;             // nq
    int* status;
    long long* bad;
    long long n, nq;
    int d, p, m, latent;
    int slot_doubles;        // per group: A, r, inv, loc (Kmax = m + 1)
};

template <int COV, int L>
__global__ void __launch_bounds__(128) k_predict(PredArgs a) {
    extern __shared__ __align__(16) double smem[];
    using N = Num<double>;
    const int tid = threadIdx.x, lane = tid & 31;
    const int gl = lane & (L - 1), grp = tid / L, ngrp = blockDim.x / L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (lane & ~(L - 1)));
    const int Kmax = a.m + 1, d = a.d, p = a.p;
    double* A = smem + (size_t)grp * a.slot_doubles;
    double* R = A + Kmax * (Kmax + 1) / 2;
    double* invd = R + Kmax;
    double* loc = invd + Kmax;
    const double* th = a.covparms;
    const int q = nparms(COV, d);
    const double sig2 = th[0], tau2 = th[q - 1];
    if (!theta_ok(COV, d, th)) {   // the same for every thread of the grid
        if (blockIdx.x == 0 && tid == 0) report(a.status, a.bad, ST_ARG, -1);
        return;
    }
    __shared__ double s_invr[DMAX_ANISO];   // COV_ANISO: 1 / rho_k
    if (COV == COV_ANISO) {
        for (int k = tid; k < d; k += blockDim.x) s_invr[k] = 1.0 / th[1 + k];
        __syncthreads();
    }
    const double inv_r1 = 1.0 / th[1];
    const double inv_r2 = (COV == COV_ST) ? 1.0 / th[2] : 1.0;
    const double diag_obs = sig2 * (1.0 + tau2);
    const double diag_tgt = a.latent ? sig2 : diag_obs;
    const double nu = (COV == COV_MATERN) ? th[2] : 0.0;
    const double psi = (COV == COV_MATERN) ? dev_digamma(nu) : 0.0;
    const long long gstride = (long long)gridDim.x * ngrp;
    for (long long i = (long long)blockIdx.x * ngrp + grp; i < a.nq; i += gstride) {
        // ---- neighbours: a valid prefix of the row, indices in [0, n)
        const int32_t* row = a.NN + i * (long long)a.m;
        int cnt = 0, badrow = 0;
        for (int c = gl; c < a.m; c += L) {
            const int v = row[c];
            if (v >= 0) {
                cnt++;
                badrow |= (v >= a.n) | (c >= 1 && row[c - 1] < 0);
            } else if (v != -1) {
                badrow = 1;
            }
        }
        cnt = gsum<L>(cnt, gmask);
        badrow = gsum<L>(badrow, gmask);
        if (badrow) {
            if (gl == 0) report(a.status, a.bad, ST_ARG, i);
            continue;
        }
        const int Kp = cnt + 1, last = cnt;
        const double* qi = a.qlocs + i * (long long)d;
        for (int b = gl; b < Kp; b += L) {
            if (b < cnt) {
                const int j = row[cnt - 1 - b];
                for (int k = 0; k < d; ++k)
                    loc[k * Kmax + b] = (a.locs[(long long)j * d + k] - qi[k]) *
                                        (COV == COV_ANISO ? s_invr[k]
                                                          : ((COV == COV_ST && k == 2) ? inv_r2 : inv_r1));
                double r = a.y[j];
                for (int t = 0; t < p; ++t) r = fma(-a.X[(long long)j * p + t], a.beta[t], r);
                R[b] = r;
            } else {
                for (int k = 0; k < d; ++k) loc[k * Kmax + b] = 0.0;
                R[b] = 0.0;
            }
        }
        gsync<L>(gmask);
        // ---- covariance (packed lower triangle)
        const int ntri = Kp * (Kp + 1) / 2;
        for (int e = gl; e < ntri; e += L) {
            int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
            while (r * (r + 1) / 2 > e) --r;
            while ((r + 1) * (r + 2) / 2 <= e) ++r;
            const int c = e - r * (r + 1) / 2;
            double C;
            if (r == c) {
                C = (r == last) ? diag_tgt : diag_obs;
            } else if (COV == COV_EXP || COV == COV_ANISO) {
                double s = 0.0;
                for (int k = 0; k < d; ++k) {
                    const double t = loc[k * Kmax + r] - loc[k * Kmax + c];
                    s = fma(t, t, s);
                }
                C = sig2 * exp(-sqrt(s));
            } else if (COV == COV_ST) {
                const double t0 = loc[r] - loc[c], t1 = loc[Kmax + r] - loc[Kmax + c];
                const double t2 = loc[2 * Kmax + r] - loc[2 * Kmax + c];
                C = sig2 * exp(-sqrt(fma(t0, t0, fma(t1, t1, t2 * t2))));
            } else {
                double s = 0.0;
                for (int k = 0; k < d; ++k) {
                    const double t = loc[k * Kmax + r] - loc[k * Kmax + c];
                    s = fma(t, t, s);
                }
                C = matern_F0(a.tab, s, nu, psi, sig2);   // the table holds sigma2 M
            }
            A[e] = C;
        }
        gsync<L>(gmask);
        // ---- Cholesky; the residual row rides along (row index Kp)
        const int Rn = Kp + 1;
        bool pd = true;
        for (int c = 0; c < Kp; ++c) {
            const double* Lc = A + c * (c + 1) / 2;
            const int r0 = c + ((gl - c) & (L - 1));
            for (int r = r0; r < Rn; r += L) {
                double* Rr = r < Kp ? A + r * (r + 1) / 2 : R;
                double v0 = Rr[c], v1 = 0.0;
                int s = 0;
                for (; s + 1 < c; s += 2) {
                    v0 = fma(-Rr[s], Lc[s], v0);
                    v1 = fma(-Rr[s + 1], Lc[s + 1], v1);
                }
                if (s < c) v0 = fma(-Rr[s], Lc[s], v0);
                Rr[c] = v0 + v1;
            }
            gsync<L>(gmask);
            const double vc = Lc[c];
            if (!(vc > 0.0) || !isfinite(vc)) { pd = false; break; }
            const double ic = rsqrt_newton(vc);
            if (r0 == c) invd[c] = ic;
            for (int r = (r0 == c ? r0 + L : r0); r < Rn; r += L) {
                double* Rr = r < Kp ? A + r * (r + 1) / 2 : R;
                Rr[c] *= ic;
            }
            gsync<L>(gmask);
        }
        if (!pd) {
            if (gl == 0) report(a.status, a.bad, ST_NOT_PD, i);
            gsync<L>(gmask);
            continue;
        }
        if (gl == 0) {
            const double sd = 1.0 / invd[last];
            double xb = 0.0;
            for (int t = 0; t < p; ++t) xb = fma(a.qX[i * (long long)p + t], a.beta[t], xb);
            a.mean[i] = xb - R[last] * sd;
            a.var[i] = sd * sd;
        }
        gsync<L>(gmask);
    }
}

static const void* predict_kernel(int cov, int L) {
#define VG_PRED(C, LL) \
    if (cov == C && L == LL) return reinterpret_cast<const void*>(&k_predict<C, LL>);
    VG_PRED(COV_EXP, 4) VG_PRED(COV_EXP, 8) VG_PRED(COV_EXP, 16) VG_PRED(COV_EXP, 32)
    VG_PRED(COV_MATERN, 4) VG_PRED(COV_MATERN, 8) VG_PRED(COV_MATERN, 16) VG_PRED(COV_MATERN, 32)
    VG_PRED(COV_ST, 4) VG_PRED(COV_ST, 8) VG_PRED(COV_ST, 16) VG_PRED(COV_ST, 32)
    VG_PRED(COV_ANISO, 4) VG_PRED(COV_ANISO, 8) VG_PRED(COV_ANISO, 16) VG_PRED(COV_ANISO, 32)
#undef VG_PRED
    return nullptr;
}

cudaError_t launch_predict(int cov, const double* locs, const double* y, const double* X,
                           const double* beta, long long n, const double* qlocs,
                           const double* qX, const int32_t* NN, long long nq, int d, int p,
                           int m, const double* covparms, const double* tab, int latent,
                           int nsm, double* mean, double* var, int* status, long long* bad,
                           cudaStream_t st) {
    // lanes per target: more lanes (fewer targets per block) as the blocks grow, so that
    // 128 threads' slots fit in shared memory (m = 80: 4 slots of 29 KB)
    const int L = m < 16 ? 4 : (m <= 40 ? 8 : (m <= 60 ? 16 : 32));
    const int K = m + 1;
    PredArgs a;
    a.locs = locs; a.y = y; a.X = X; a.beta = beta; a.qlocs = qlocs; a.qX = qX; a.NN = NN;
    a.covparms = covparms; a.tab = tab; a.mean = mean; a.var = var; a.status = status;
    a.bad = bad; a.n = n; a.nq = nq; a.d = d; a.p = p; a.m = m; a.latent = latent;
    a.slot_doubles = K * (K + 1) / 2 + 2 * K + d * K;
    if (a.slot_doubles % 2 == 0) a.slot_doubles += 1;   // odd stride: groups spread over banks
    const int threads = 128;
    const size_t smem = (size_t)(threads / L) * a.slot_doubles * sizeof(double);
    const void* fn = predict_kernel(cov, L);
    if (!fn) return cudaErrorInvalidValue;
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    // the dynamic limit leaves room for the kernel's static shared memory
    const int dyn_max = optin - (int)fa.sharedSizeBytes;
    if ((int)smem > dyn_max) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidValue;
    void* params[] = {&a};
    return cudaLaunchKernel(fn, dim3(nsm * per_sm), dim3(threads), params, smem, st);
}

}  // namespace vg
