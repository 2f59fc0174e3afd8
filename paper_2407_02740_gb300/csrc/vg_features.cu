// vg_features.cu -- binned empirical semivariogram features of many fields at shared
// locations (the input of the learned starting point for Fisher scoring; the paper has no
// counterpart).
//
// For field f with observations y (n values) at locs, the pairs are
//   (i)  every (i, NNarray[i][c]) with c >= 1 and NNarray[i][c] >= 0, and
//   (ii) P pairs (i, j) = (floor(r1 n / 2^32), floor(r2 n / 2^32)) from caller-supplied
//        32-bit words (r1, r2), the same words for every field.
// A pair's lag h = |s_i - s_j| falls in bin k when e_k <= h^2 < e_(k+1) for the caller's
// ascending squared edges e_0..e_nbins (h^2 summed coordinate by coordinate in FP64 with
// no fused multiply-add, so any FP64 implementation takes the same bin decision); pairs
// outside [e_0, e_nbins) are ignored.  Bin k's value is the mean of (y_i - y_j)^2 / 2 over
// its pairs, divided by the population variance of y; an empty bin takes the value of the
// nearest non-empty bin (the lower one on a tie); all bins empty gives NaN.
//
// Kernels (deterministic: no floating-point atomics):
//   k_field_moments  one block per field: mean, then variance (two passes, fixed-order
//                    block reductions)
//   k_vario          grid (slices, fields): each thread accumulates its pairs into private
//                    bins in shared memory (sum FP64, count), then a fixed-order reduction
//                    over the block's threads writes one partial per slice
//   k_vario_finish   one thread per field: slices summed in order, fill rule, FP32 output
#include <climits>
#include <cmath>
#include <cstdint>

#include "vg_internal.h"

namespace vg {

constexpr int VG_THREADS = 128;

__global__ void __launch_bounds__(256) k_field_moments(const double* __restrict__ Y, int n,
                                                       double* __restrict__ mean,
                                                       double* __restrict__ var) {
    __shared__ double red[256];
    const int f = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
    const double* y = Y + (size_t)f * n;
    double s = 0.0;
    for (int i = tid; i < n; i += T) s += y[i];
    red[tid] = s;
    __syncthreads();
    for (int o = T / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    const double mu = red[0] / n;
    __syncthreads();
    double s2 = 0.0;
    for (int i = tid; i < n; i += T) {
        const double t = y[i] - mu;
        s2 = fma(t, t, s2);
    }
    red[tid] = s2;
    __syncthreads();
    for (int o = T / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    if (tid == 0) {
        mean[f] = mu;
        var[f] = red[0] / n;
    }
}

__global__ void __launch_bounds__(VG_THREADS) k_vario(
    const double* __restrict__ locs, int d, const int32_t* __restrict__ NN, int n, int m,
    const double* __restrict__ Y, const uint32_t* __restrict__ R, long long P,
    const double* __restrict__ edges2, int nbins, int slices, double* __restrict__ psum,
    long long* __restrict__ pcnt) {
    extern __shared__ __align__(16) double sm[];
    const int T = VG_THREADS;
    double* sE = sm;                                    // nbins + 1 squared edges
    double* sS = sE + (nbins + 1);                      // nbins x T private sums
    unsigned* sC = reinterpret_cast<unsigned*>(sS + (size_t)nbins * T);  // nbins x T counts
    const int f = blockIdx.y, sl = blockIdx.x, tid = threadIdx.x;
    for (int k = tid; k <= nbins; k += T) sE[k] = edges2[k];
    for (int k = 0; k < nbins; ++k) {
        sS[k * T + tid] = 0.0;
        sC[k * T + tid] = 0u;
    }
    __syncthreads();
    const long long nnp = (long long)n * m;
    const long long W = nnp + P;
    const long long per = (W + slices - 1) / slices;
    const long long t0 = (long long)sl * per;
    const long long t1 = t0 + per < W ? t0 + per : W;
    const double* y = Y + (size_t)f * n;
    const double lo_e = sE[0], hi_e = sE[nbins];
    for (long long t = t0 + tid; t < t1; t += T) {
        int i, j;
        if (t < nnp) {
            i = (int)(t / m);
            const int c = 1 + (int)(t - (long long)i * m);
            j = NN[(size_t)i * (m + 1) + c];
            if (j < 0) continue;
        } else {
            const long long r = t - nnp;
            i = (int)(((unsigned long long)R[2 * r] * (unsigned long long)n) >> 32);
            j = (int)(((unsigned long long)R[2 * r + 1] * (unsigned long long)n) >> 32);
        }
        const double* a = locs + (size_t)i * d;
        const double* b = locs + (size_t)j * d;
        double h2 = 0.0;
        for (int k = 0; k < d; ++k) {
            const double dk = __dsub_rn(a[k], b[k]);
            h2 = (k == 0) ? __dmul_rn(dk, dk) : __dadd_rn(h2, __dmul_rn(dk, dk));
        }
        if (!(h2 >= lo_e) || !(h2 < hi_e)) continue;
        int lo = 0, hi = nbins;  // sE[lo] <= h2 < sE[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sE[mid] <= h2) lo = mid; else hi = mid;
        }
        const double dy = __dsub_rn(y[i], y[j]);
        sS[lo * T + tid] += __dmul_rn(0.5, __dmul_rn(dy, dy));
        sC[lo * T + tid] += 1u;
    }
    __syncthreads();
    for (int k = tid; k < nbins; k += T) {
        double s = 0.0;
        long long c = 0;
        for (int u = 0; u < T; ++u) {
            s += sS[k * T + u];
            c += sC[k * T + u];
        }
        const size_t o = ((size_t)f * slices + sl) * nbins + k;
        psum[o] = s;
        pcnt[o] = c;
    }
}

__global__ void k_vario_finish(const double* __restrict__ psum, const long long* __restrict__ pcnt,
                               int slices, int nbins, const double* __restrict__ var,
                               int nfields, float* __restrict__ feat, double* bin_sum,
                               long long* bin_count) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfields) return;
    double S[VG_MAX_BINS];
    long long C[VG_MAX_BINS];
    for (int k = 0; k < nbins; ++k) {
        double s = 0.0;
        long long c = 0;
        for (int sl = 0; sl < slices; ++sl) {
            const size_t o = ((size_t)f * slices + sl) * nbins + k;
            s += psum[o];
            c += pcnt[o];
        }
        S[k] = s;
        C[k] = c;
        if (bin_sum) bin_sum[(size_t)f * nbins + k] = s;
        if (bin_count) bin_count[(size_t)f * nbins + k] = c;
    }
    const double v = var[f];
    for (int k = 0; k < nbins; ++k) {
        int src = -1;
        if (C[k] > 0) {
            src = k;
        } else {
            for (int dist = 1; dist < nbins && src < 0; ++dist) {
                if (k - dist >= 0 && C[k - dist] > 0) src = k - dist;
                else if (k + dist < nbins && C[k + dist] > 0) src = k + dist;
            }
        }
        const double g = src < 0 ? __longlong_as_double(0x7ff8000000000000ll)
                                 : S[src] / (double)C[src] / v;
        feat[(size_t)f * nbins + k] = (float)g;
    }
}

size_t vario_smem_bytes(int nbins) {
    return (size_t)(nbins + 1) * sizeof(double) + (size_t)nbins * VG_THREADS * (sizeof(double) + sizeof(unsigned));
}

cudaError_t launch_field_moments(const double* Y, int n, int nfields, double* mean, double* var,
                                 cudaStream_t st) {
    k_field_moments<<<nfields, 256, 0, st>>>(Y, n, mean, var);
    return cudaGetLastError();
}

cudaError_t launch_vario(const double* locs, int d, const int32_t* NN, int n, int m, const double* Y,
                         int nfields, const uint32_t* R, long long P, const double* edges2,
                         int nbins, int slices, double* psum, long long* pcnt, cudaStream_t st) {
    const size_t smem = vario_smem_bytes(nbins);
    cudaError_t e = cudaFuncSetAttribute(k_vario, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_vario<<<dim3(slices, nfields), VG_THREADS, smem, st>>>(locs, d, NN, n, m, Y, R, P, edges2,
                                                            nbins, slices, psum, pcnt);
    return cudaGetLastError();
}

cudaError_t launch_vario_finish(const double* psum, const long long* pcnt, int slices, int nbins,
                                const double* var, int nfields, float* feat, double* bin_sum,
                                long long* bin_count, cudaStream_t st) {
    k_vario_finish<<<(nfields + 127) / 128, 128, 0, st>>>(psum, pcnt, slices, nbins, var, nfields,
                                                          feat, bin_sum, bin_count);
    return cudaGetLastError();
}

}  // namespace vg
