// vg_mlp.cu -- the small multilayer perceptron of the learned starting point for Fisher
// scoring (the paper has no counterpart): 32 semivariogram features -> 128 -> 128 -> 4
// standardised log-parameter targets, ReLU after the two hidden layers, FP32.
//
// Parameters, one flat FP32 array (row-major, out x in):
//   W1 [128][32], b1 [128], W2 [128][128], b2 [128], W3 [4][128], b3 [4]   (21252 values)
// Standardisation, one flat FP32 array: x_mean[32], x_std[32], t_mean[4], t_std[4].  The
// network sees (x - x_mean) / x_std; its raw outputs o are standardised targets, so a
// prediction is o * t_std + t_mean and training compares o with (t - t_mean) / t_std.
//
// Kernels:
//   k_mlp_fwdbwd   one block of 128 threads per 32 samples (rows of X and T, or the rows an
//                  index array lists: a minibatch); all weights staged in shared
//                  memory (W1 transposed, W2 in both orientations, so that every access
//                  is conflict-free), activations kept in shared memory; writes the
//                  predictions, or the block's loss and gradient partial sums
//   k_mlp_update   sums the block partials in a fixed order (deterministic), then either
//                  writes the gradient or takes one Adam step
//   k_col_moments  column means and standard deviations of a sample matrix (FP64 sums)
// Loss: mean over samples and the 4 outputs of the squared error.
#include <cmath>
#include <cstdint>

#include "vg_internal.h"

namespace vg {

constexpr int MI = 32, MH = 128, MO = 4, MS = 32;  // inputs, hidden, outputs, samples/block
constexpr int MHP = MH + 1;  // row stride of the transposed copies (conflict-free transpose)
constexpr int OW1 = 0, OB1 = OW1 + MH * MI, OW2 = OB1 + MH, OB2 = OW2 + MH * MH,
              OW3 = OB2 + MH, OB3 = OW3 + MO * MH, NPAR = OB3 + MO;
static_assert(NPAR == 21252, "parameter count");

size_t mlp_smem_bytes() {
    return sizeof(float) * ((size_t)MI * MHP + MH + (size_t)MH * MH + (size_t)MH * MHP + MH +
                            MO * MH + MO  // weights
                            + MS * MI + 4 * MS * MH + 2 * MS * MO + 2 * MI + 2 * MO);
}

// mode 0: predictions out[s][o] = o * t_std + t_mean; mode 1: loss and gradient partials.
__global__ void __launch_bounds__(MH) k_mlp_fwdbwd(const float* __restrict__ P,
                                                   const float* __restrict__ norm,
                                                   const float* __restrict__ X,
                                                   const float* __restrict__ T,
                                                   const int* __restrict__ index, int B, int mode,
                                                   float* __restrict__ out,
                                                   float* __restrict__ gpart,
                                                   float* __restrict__ lpart) {
    extern __shared__ __align__(16) float sm[];
    float* W1T = sm;                  // [k][j] = W1[j][k], row stride MHP
    float* b1 = W1T + MI * MHP;
    float* W2 = b1 + MH;              // [j][k]
    float* W2T = W2 + MH * MH;        // [k][j] = W2[j][k], row stride MHP
    float* b2 = W2T + MH * MHP;
    float* W3 = b2 + MH;              // [o][k]
    float* b3 = W3 + MO * MH;
    float* xs = b3 + MO;              // [s][k] standardised inputs
    float* h1 = xs + MS * MI;         // [s][j]
    float* h2 = h1 + MS * MH;
    float* d2 = h2 + MS * MH;         // dL/d(pre-activation of layer 2) [s][j]
    float* d1 = d2 + MS * MH;         // layer 1 [s][j]
    float* ov = d1 + MS * MH;         // outputs [s][o]
    float* dv = ov + MS * MO;         // dL/do [s][o]
    float* nx = dv + MS * MO;         // x_mean, x_std, t_mean, t_std
    const int tid = threadIdx.x;
    const int s0 = blockIdx.x * MS;
    const int ns = (B - s0) < MS ? (B - s0) : MS;

    for (int e = tid; e < MH * MI; e += MH) {
        const int j = e / MI, k = e % MI;
        W1T[k * MHP + j] = P[OW1 + e];
    }
    for (int e = tid; e < MH * MH; e += MH) {
        const float w = P[OW2 + e];
        W2[e] = w;
        W2T[(e % MH) * MHP + e / MH] = w;
    }
    for (int e = tid; e < MO * MH; e += MH) W3[e] = P[OW3 + e];
    b1[tid] = P[OB1 + tid];
    b2[tid] = P[OB2 + tid];
    if (tid < MO) b3[tid] = P[OB3 + tid];
    if (tid < 2 * MI + 2 * MO) nx[tid] = norm[tid];
    __syncthreads();
    for (int e = tid; e < MS * MI; e += MH) {
        const int s = e / MI, k = e % MI;
        const size_t row = s < ns ? (size_t)(index ? index[s0 + s] : s0 + s) : 0;
        xs[e] = s < ns ? (X[row * MI + k] - nx[k]) / nx[MI + k] : 0.0f;
    }
    __syncthreads();
    // layer 1 and 2: thread j owns hidden unit j
    const int j = tid;
    for (int s = 0; s < MS; ++s) {
        float a = b1[j];
#pragma unroll 8
        for (int k = 0; k < MI; ++k) a = fmaf(W1T[k * MHP + j], xs[s * MI + k], a);
        h1[s * MH + j] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    for (int s = 0; s < MS; ++s) {
        float a = b2[j];
#pragma unroll 8
        for (int k = 0; k < MH; ++k) a = fmaf(W2T[k * MHP + j], h1[s * MH + k], a);
        h2[s * MH + j] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    // outputs: thread t -> (sample t / 4, output t % 4)
    {
        const int s = tid / MO, o = tid % MO;
        float a = b3[o];
#pragma unroll 8
        for (int k = 0; k < MH; ++k) a = fmaf(W3[o * MH + k], h2[s * MH + k], a);
        ov[s * MO + o] = a;
        if (mode == 0) {
            if (s < ns) out[(size_t)(s0 + s) * MO + o] = a * nx[2 * MI + MO + o] + nx[2 * MI + o];
        } else {
            float r = 0.0f;
            if (s < ns) {
                const size_t row = (size_t)(index ? index[s0 + s] : s0 + s);
                const float t = (T[row * MO + o] - nx[2 * MI + o]) / nx[2 * MI + MO + o];
                r = a - t;
            }
            dv[s * MO + o] = 2.0f * r / (float)(B * MO);
            // block loss partial: fixed-order warp and block sums of r^2 / (B * MO)
            float l = r * r / (float)(B * MO);
#pragma unroll
            for (int w = 16; w > 0; w >>= 1) l += __shfl_xor_sync(0xffffffffu, l, w);
            if ((tid & 31) == 0) d1[tid >> 5] = l;   // d1 is free until the backward pass
        }
    }
    if (mode == 0) return;
    __syncthreads();
    if (tid == 0) lpart[blockIdx.x] = (d1[0] + d1[1]) + (d1[2] + d1[3]);
    __syncthreads();
    // backward: layer 2 pre-activation gradient
    for (int s = 0; s < MS; ++s) {
        float a = 0.0f;
#pragma unroll
        for (int o = 0; o < MO; ++o) a = fmaf(W3[o * MH + j], dv[s * MO + o], a);
        d2[s * MH + j] = h2[s * MH + j] > 0.0f ? a : 0.0f;
    }
    __syncthreads();
    // layer 1: d1[s][k] = [h1 > 0] sum_j W2[j][k] d2[s][j]; thread k = tid
    for (int s = 0; s < MS; ++s) {
        float a = 0.0f;
#pragma unroll 8
        for (int jj = 0; jj < MH; ++jj) a = fmaf(W2[jj * MH + j], d2[s * MH + jj], a);
        d1[s * MH + j] = h1[s * MH + j] > 0.0f ? a : 0.0f;
    }
    __syncthreads();
    float* g = gpart + (size_t)blockIdx.x * NPAR;
    // W3, b3: thread k
    for (int o = 0; o < MO; ++o) {
        float a = 0.0f;
        for (int s = 0; s < MS; ++s) a = fmaf(dv[s * MO + o], h2[s * MH + j], a);
        g[OW3 + o * MH + j] = a;
    }
    if (tid < MO) {
        float a = 0.0f;
        for (int s = 0; s < MS; ++s) a += dv[s * MO + tid];
        g[OB3 + tid] = a;
    }
    // W2[r][k] = sum_s d2[s][r] h1[s][k]: thread k, rows r in turn (coalesced rows)
    for (int r = 0; r < MH; ++r) {
        float a = 0.0f;
#pragma unroll 8
        for (int s = 0; s < MS; ++s) a = fmaf(d2[s * MH + r], h1[s * MH + j], a);
        g[OW2 + r * MH + j] = a;
    }
    {
        float a = 0.0f, c = 0.0f;
        for (int s = 0; s < MS; ++s) {
            a += d2[s * MH + j];
            c += d1[s * MH + j];
        }
        g[OB2 + j] = a;
        g[OB1 + j] = c;
    }
    // W1[r][k] = sum_s d1[s][r] xs[s][k]: entries e = tid + 128 t
    for (int e = tid; e < MH * MI; e += MH) {
        const int r = e / MI, k = e % MI;
        float a = 0.0f;
#pragma unroll 8
        for (int s = 0; s < MS; ++s) a = fmaf(d1[s * MH + r], xs[s * MI + k], a);
        g[OW1 + e] = a;
    }
}

// Sums the block partials in order.  grad != nullptr: write the gradient and the loss.
// Otherwise one Adam step (step = 1, 2, ... for the bias corrections) on P, m, v.
__global__ void k_mlp_update(const float* __restrict__ gpart, const float* __restrict__ lpart,
                             int nblk, float* P, float* m, float* v, int step, float lr,
                             float beta1, float beta2, float eps, float* grad, float* loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && loss) {
        float l = 0.0f;
        for (int b = 0; b < nblk; ++b) l += lpart[b];
        *loss = l;
    }
    if (p >= NPAR) return;
    float g = 0.0f;
    for (int b = 0; b < nblk; ++b) g += gpart[(size_t)b * NPAR + p];
    if (grad) {
        grad[p] = g;
        return;
    }
    const float mm = beta1 * m[p] + (1.0f - beta1) * g;
    const float vv = beta2 * v[p] + (1.0f - beta2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float mh = mm / (1.0f - powf(beta1, (float)step));
    const float vh = vv / (1.0f - powf(beta2, (float)step));
    P[p] -= lr * mh / (sqrtf(vh) + eps);
}

// Column means and standard deviations (population) of X (rows x cols), FP64 sums in
// row order; a column with zero spread gets std 1.  One thread per column.
__global__ void k_col_moments(const float* __restrict__ X, int rows, int cols, float* mean,
                              float* sd) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s += X[(size_t)r * cols + c];
    const double mu = s / rows;
    double s2 = 0.0;
    for (int r = 0; r < rows; ++r) {
        const double t = X[(size_t)r * cols + c] - mu;
        s2 += t * t;
    }
    const double v = s2 / rows;
    mean[c] = (float)mu;
    sd[c] = v > 0.0 ? (float)sqrt(v) : 1.0f;
}

cudaError_t launch_mlp_fwdbwd(const float* P, const float* norm, const float* X, const float* T,
                              const int* index, int B, int mode, float* out, float* gpart,
                              float* lpart, cudaStream_t st) {
    const size_t smem = mlp_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_fwdbwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_mlp_fwdbwd<<<(B + MS - 1) / MS, MH, smem, st>>>(P, norm, X, T, index, B, mode, out, gpart,
                                                      lpart);
    return cudaGetLastError();
}

cudaError_t launch_mlp_update(const float* gpart, const float* lpart, int nblk, float* P, float* m,
                              float* v, int step, float lr, float beta1, float beta2, float eps,
                              float* grad, float* loss, cudaStream_t st) {
    k_mlp_update<<<(NPAR + 255) / 256, 256, 0, st>>>(gpart, lpart, nblk, P, m, v, step, lr, beta1,
                                                      beta2, eps, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_col_moments(const float* X, int rows, int cols, float* mean, float* sd,
                               cudaStream_t st) {
    k_col_moments<<<(cols + 31) / 32, 32, 0, st>>>(X, rows, cols, mean, sd);
    return cudaGetLastError();
}

// theta0 of the isotropic Matern family from the network's predictions of
// (log(sigma2 / var y), log rho, log nu, log tau2); nu is clamped to [0.05, 20] like the fit.
__global__ void k_theta_from_pred(const float* __restrict__ pred, const double* __restrict__ var,
                                  int nfields, double* __restrict__ theta) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfields) return;
    const float* p = pred + (size_t)f * MO;
    double* t = theta + (size_t)f * 4;
    t[0] = var[f] * exp((double)p[0]);
    t[1] = exp((double)p[1]);
    t[2] = fmin(20.0, fmax(0.05, exp((double)p[2])));
    t[3] = exp((double)p[3]);
}

// Per field: the learned start unless it is not finite, its pass failed, or its loglik is
// below the default start's (a failed default pass counts as -inf).
__global__ void k_choose_start(const double* __restrict__ theta0, const double* __restrict__ dflt,
                               const double* __restrict__ out0, const long long* __restrict__ st0,
                               const double* __restrict__ out1, const long long* __restrict__ st1,
                               int nfields, int q, int nout, double* __restrict__ start,
                               int* __restrict__ used) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfields) return;
    bool ok = st0[2 * (size_t)f] == 0 && isfinite(out0[(size_t)f * nout]);
    for (int j = 0; j < q; ++j) ok = ok && isfinite(theta0[(size_t)f * q + j]);
    const bool dok = st1[2 * (size_t)f] == 0 && isfinite(out1[(size_t)f * nout]);
    if (ok && dok) ok = !(out0[(size_t)f * nout] < out1[(size_t)f * nout]);
    for (int j = 0; j < q; ++j)
        start[(size_t)f * q + j] = ok ? theta0[(size_t)f * q + j] : dflt[(size_t)f * q + j];
    used[f] = ok ? 1 : 0;
}

// Training targets from fitted parameters: t_j = log theta_j (log(sigma2 / var y) for
// j = 0), clamped to [log lo_j, log hi_j], FP32.
struct TargetRange {
    double lo[4], hi[4];
};
__global__ void k_targets_from_theta(const double* __restrict__ theta, const double* __restrict__ var,
                                     int nfields, TargetRange R, float* __restrict__ T) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfields) return;
    const double* th = theta + (size_t)f * 4;
    for (int j = 0; j < 4; ++j) {
        double t = log(th[j]);
        if (j == 0) t -= log(var[f]);
        t = fmin(log(R.hi[j]), fmax(log(R.lo[j]), t));
        T[(size_t)f * MO + j] = (float)t;
    }
}

cudaError_t launch_targets_from_theta(const double* theta, const double* var, int nfields,
                                      const double* lo, const double* hi, float* T, cudaStream_t st) {
    TargetRange R;
    for (int j = 0; j < 4; ++j) { R.lo[j] = lo[j]; R.hi[j] = hi[j]; }
    k_targets_from_theta<<<(nfields + 127) / 128, 128, 0, st>>>(theta, var, nfields, R, T);
    return cudaGetLastError();
}

cudaError_t launch_theta_from_pred(const float* pred, const double* var, int nfields, double* theta,
                                   cudaStream_t st) {
    k_theta_from_pred<<<(nfields + 127) / 128, 128, 0, st>>>(pred, var, nfields, theta);
    return cudaGetLastError();
}

cudaError_t launch_choose_start(const double* theta0, const double* dflt, const double* out0,
                                const long long* st0, const double* out1, const long long* st1,
                                int nfields, int q, int nout, double* start, int* used,
                                cudaStream_t st) {
    k_choose_start<<<(nfields + 127) / 128, 128, 0, st>>>(theta0, dflt, out0, st0, out1, st1,
                                                          nfields, q, nout, start, used);
    return cudaGetLastError();
}

int mlp_nparams() { return NPAR; }
int mlp_block_samples() { return MS; }

}  // namespace vg
