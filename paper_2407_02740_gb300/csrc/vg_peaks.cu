// vg_peaks.cu -- measured throughputs of this GPU for the roofline of the pass kernels:
// FP64 and FP32 FMA chains (the ALU peaks the pass is bound by) and the cost of one
// covariance evaluation as the pass does it (exponential: square root, exponential and
// division; Matern: the table's value and its two derivatives).
#include <algorithm>

#include "vg_internal.h"
#include "vg_matern.cuh"

namespace vg {

constexpr int kChains = 8;     // independent FMA chains per thread (hides the FMA latency)
constexpr int kUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T* sink, int iters, T a, T b) {
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) acc[c] = acc[c] * a + b;
        }
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == (T)-12345) sink[0] = s;   // keeps the chains live; never true in practice
}

// FP64 on the tensor cores: independent chains of the m8n8k4 double-precision matrix
// multiply-add (an 8 x 4 by 4 x 8 product added into 8 x 8: 512 flops per warp
// instruction), the FP64 tensor operation this GPU offers.  Measured so that the choice of
// the FP64 ALU for the pass's contractions rests on a number.
__global__ void __launch_bounds__(256) k_dmma_chain(double* sink, int iters, double a, double b) {
    double c0[kChains], c1[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        c0[c] = (double)(threadIdx.x + c);
        c1[c] = (double)(threadIdx.x - c);
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                             : "+d"(c0[c]), "+d"(c1[c])
                             : "d"(a), "d"(b));
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += c0[c] + c1[c];
    if (s == -12345.0) sink[0] = s;
}

// One pair evaluation per iteration and thread, at squared distances spread over the
// range the pass meets (s from ~1e-4 to ~40 in units of the range).
__global__ void __launch_bounds__(256) k_exp_eval(double* sink, int iters) {
    double s = 1e-4 * (1.0 + threadIdx.x), acc = 0.0;
    for (int it = 0; it < iters; ++it) {
        const double D = sqrt(s);
        const double C = 1.3 * exp(-D);
        acc += C / D;                  // the value and the derivative weight, as in the pass
        s = s * 1.0009765625 + 1e-7;
        if (s > 40.0) s = 1e-4;
    }
    if (acc == -12345.0) sink[0] = acc;
}

__global__ void __launch_bounds__(256) k_matern_eval(const double* __restrict__ tab, double nu,
                                                     double psi, double* sink, int iters) {
    double s = 1e-4 * (1.0 + threadIdx.x), acc = 0.0;
    for (int it = 0; it < iters; ++it) {
        const double C = matern_F0(tab, s, nu, psi, 1.3);
        double F1, F2;
        matern_F12(tab, s, nu, psi, 1.3 / 0.05, 1.3, F1, F2);
        acc += C + F1 + F2;
        s = s * 1.0009765625 + 1e-7;
        if (s > 40.0) s = 1e-4;
    }
    if (acc == -12345.0) sink[0] = acc;
}

}  // namespace vg

namespace {

// Times launch() with CUDA events on st (one untimed launch first); milliseconds.
template <typename F>
cudaError_t time_launch(cudaStream_t st, F launch, float* ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace

namespace vg {

// out = {FP64 GFLOP/s, FP32 GFLOP/s, exponential pairs/s, Matern pairs/s,
//        FP64 tensor-core GFLOP/s}
cudaError_t measure_peaks(int nsm, cudaStream_t st, double* out) {
    double* sink = nullptr;
    double* tab = nullptr;
    double* theta = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&sink), sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&tab), sizeof(double) * mtab_doubles());
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&theta), sizeof(double) * 4);
    const double th[4] = {1.3, 0.05, 1.5, 0.05};
    if (e == cudaSuccess) e = cudaMemcpyAsync(theta, th, sizeof(th), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_mtab_build(COV_MATERN, theta, tab, nullptr, st);
    // two blocks of 256 threads per SM: 16 warps, 4 per sub-partition
    const dim3 grid(2 * nsm), block(256);
    const double threads = (double)grid.x * block.x;
    float ms = 0.f;
    const int it64 = 2000, it32 = 64000, itev = 4000;
    if (e == cudaSuccess)
        e = time_launch(st, [&] { k_fma_chain<double><<<grid, block, 0, st>>>(sink, it64, 1.0000001, 1e-9); }, &ms);
    if (e == cudaSuccess) out[0] = 2.0 * threads * it64 * kUnroll * kChains / (ms * 1e-3) / 1e9;
    if (e == cudaSuccess)
        e = time_launch(st, [&] {
            k_fma_chain<float><<<grid, block, 0, st>>>(reinterpret_cast<float*>(sink), it32, 1.0000001f, 1e-9f);
        }, &ms);
    if (e == cudaSuccess) out[1] = 2.0 * threads * it32 * kUnroll * kChains / (ms * 1e-3) / 1e9;
    if (e == cudaSuccess) e = time_launch(st, [&] { k_exp_eval<<<grid, block, 0, st>>>(sink, itev); }, &ms);
    if (e == cudaSuccess) out[2] = threads * itev / (ms * 1e-3);
    // digamma(1.5) = 2 - 2 log 2 - Euler's constant
    const double psi = 2.0 - 2.0 * 0.69314718055994530942 - 0.57721566490153286061;
    if (e == cudaSuccess)
        e = time_launch(st, [&] { k_matern_eval<<<grid, block, 0, st>>>(tab, 1.5, psi, sink, itev); }, &ms);
    if (e == cudaSuccess) out[3] = threads * itev / (ms * 1e-3);
    const int itmm = 500;
    if (e == cudaSuccess)
        e = time_launch(st, [&] { k_dmma_chain<<<grid, block, 0, st>>>(sink, itmm, 1e-3, 1e-3); }, &ms);
    if (e == cudaSuccess) out[4] = 512.0 * (threads / 32.0) * itmm * kUnroll * kChains / (ms * 1e-3) / 1e9;
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    cudaFree(sink);
    cudaFree(tab);
    cudaFree(theta);
    return e;
}

}  // namespace vg
