// vg_capi.cu -- the extern "C" boundary of the Vecchia library (declared in
// include/vecchia.h): handles, argument validation, scratch management and launch order.
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/vecchia.h"
#include "vg_internal.h"
#include "vg_common.cuh"

namespace {

thread_local std::string g_last_error;

vec_status fail(vec_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
vec_status fail(vec_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

vec_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(VEC_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(VEC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int old = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&old) != cudaSuccess) old = -1;
        ok = (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard() {
        if (old >= 0) cudaSetDevice(old);
    }
};

template <typename T>
cudaError_t grow(T** p, size_t* cap, size_t need) {
    if (*cap >= need && *p) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t want = need < 64 ? 64 : need;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), want * sizeof(T));
    if (e == cudaSuccess) *cap = want;
    return e;
}

}  // namespace

void vg::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

struct vec_handle_s {
    int device = 0;
    int nsm = 0;
    int lanes = 0;    // 0 = automatic
    int threads = 0;  // 0 = automatic
    cudaStream_t stream = nullptr;
    // tracing
    int timing = 0;
    int traced = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // pass scratch
    double* partials = nullptr;
    size_t partials_cap = 0;
    double* mtab = nullptr;
    int* status = nullptr;
    long long* bad = nullptr;
    // staging for the host-memory entry point
    double* h_locs = nullptr; size_t c_locs = 0;
    double* h_y = nullptr; size_t c_y = 0;
    double* h_X = nullptr; size_t c_X = 0;
    int32_t* h_NN = nullptr; size_t c_NN = 0;
    double* h_cov = nullptr; size_t c_cov = 0;
    double* h_out = nullptr; size_t c_out = 0;
    long long* h_st = nullptr; size_t c_st = 0;
};

extern "C" {

const char* vecchia_last_error(void) { return g_last_error.c_str(); }

int vecchia_nparms(vec_covfun covfun) {
    switch (covfun) {
    case VEC_EXP_ISO: return 3;
    case VEC_MATERN_ISO: return 4;
    case VEC_EXP_SPACETIME: return 4;
    default: return -1;
    }
}

int vecchia_max_m(void) { return vg::KMAX - 1; }

vec_status vecchia_set_timing(vec_handle h, int enable) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_set_timing: NULL handle");
    if (enable && !h->ev[0]) {
        DeviceGuard g(h->device);
        for (int k = 0; k < 4; ++k) {
            cudaError_t e = cudaEventCreate(&h->ev[k]);
            if (e != cudaSuccess) return cuda_fail(e, "vecchia_set_timing: cudaEventCreate");
        }
    }
    h->timing = enable ? 1 : 0;
    return VEC_OK;
}

vec_status vecchia_last_timing(vec_handle h, float* ms_setup, float* ms_pass, float* ms_profile) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_last_timing: NULL handle");
    if (!h->traced) return fail(VEC_ERR_ARG, "vecchia_last_timing: no traced pass yet");
    DeviceGuard g(h->device);
    cudaError_t e = cudaEventSynchronize(h->ev[3]);
    float t[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventElapsedTime(&t[k], h->ev[k], h->ev[k + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_last_timing");
    if (ms_setup) *ms_setup = t[0];
    if (ms_pass) *ms_pass = t[1];
    if (ms_profile) *ms_profile = t[2];
    return VEC_OK;
}

int vecchia_kernels_per_pass(vec_covfun covfun) {
    if (vecchia_nparms(covfun) < 0) return -1;
    return covfun == VEC_MATERN_ISO ? 4 : 3;
}

vec_status vecchia_set_lanes(vec_handle h, int lanes) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_set_lanes: NULL handle");
    if (!(lanes == 0 || lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8 || lanes == 16 ||
          lanes == 32))
        return fail(VEC_ERR_ARG, "lanes must be 0, 1, 2, 4, 8, 16 or 32 (got %d)", lanes);
    h->lanes = lanes;
    return VEC_OK;
}

vec_status vecchia_set_block_threads(vec_handle h, int threads) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_set_block_threads: NULL handle");
    if (!(threads == 0 || threads == 32 || threads == 64 || threads == 128 || threads == 256))
        return fail(VEC_ERR_ARG, "threads must be 0, 32, 64, 128 or 256 (got %d)", threads);
    h->threads = threads;
    return VEC_OK;
}

vec_status vecchia_create(vec_handle* out, int device) {
    if (!out) return fail(VEC_ERR_ARG, "vecchia_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_create: cudaGetDeviceCount");
    if (device < 0 || device >= ndev)
        return fail(VEC_ERR_ARG, "vecchia_create: device %d out of range (%d devices)", device, ndev);
    DeviceGuard g(device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "vecchia_create: cannot select device %d", device);
    vec_handle h = new (std::nothrow) vec_handle_s();
    if (!h) return fail(VEC_ERR_NOMEM, "vecchia_create: host allocation failed");
    h->device = device;
    e = cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&h->mtab),
                                         sizeof(double) * vg::mtab_doubles());
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&h->status), sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&h->bad), sizeof(long long) * 2);
    if (e != cudaSuccess) {
        vecchia_destroy(h);
        return cuda_fail(e, "vecchia_create");
    }
    *out = h;
    return VEC_OK;
}

vec_status vecchia_destroy(vec_handle h) {
    if (!h) return VEC_OK;
    DeviceGuard g(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaFree(h->partials);
    cudaFree(h->mtab);
    cudaFree(h->status);
    cudaFree(h->bad);
    cudaFree(h->h_locs);
    cudaFree(h->h_y);
    cudaFree(h->h_X);
    cudaFree(h->h_NN);
    cudaFree(h->h_cov);
    cudaFree(h->h_out);
    cudaFree(h->h_st);
    for (int k = 0; k < 4; ++k)
        if (h->ev[k]) cudaEventDestroy(h->ev[k]);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return VEC_OK;
}

}  // extern "C"

namespace {

vec_status check_args(const void* locs, const void* y, const void* X, const void* NN,
                      int64_t n, int d, int p, int m, const void* covparms, vec_covfun covfun,
                      vec_precision prec) {
    if (!locs || !y || !X || !NN || !covparms)
        return fail(VEC_ERR_ARG, "a required pointer is NULL");
    if (n < 1 || n > (int64_t)INT_MAX) return fail(VEC_ERR_ARG, "n = %lld out of range", (long long)n);
    if (vecchia_nparms(covfun) < 0) return fail(VEC_ERR_ARG, "unknown covariance function %d", (int)covfun);
    if (d < 1 || d > vg::DMAX) return fail(VEC_ERR_ARG, "d = %d out of range [1, 3]", d);
    if (covfun == VEC_EXP_SPACETIME && d != 3)
        return fail(VEC_ERR_ARG, "the space-time covariance needs d = 3 (lon, lat, time)");
    if (p < 1 || p > vg::PMAX) return fail(VEC_ERR_ARG, "p = %d out of range [1, %d]", p, vg::PMAX);
    if (m < 0 || m > vg::KMAX - 1)
        return fail(VEC_ERR_UNSUPPORTED, "m = %d out of range [0, %d]", m, vg::KMAX - 1);
    if (prec != VEC_FP64 && prec != VEC_MIXED) return fail(VEC_ERR_ARG, "unknown precision %d", (int)prec);
    if (prec == VEC_MIXED) return fail(VEC_ERR_UNSUPPORTED, "mixed precision is not available in this build");
    return VEC_OK;
}

// Enqueues the full pass on `st`.  Device pointers only.
vec_status enqueue_pass(vec_handle h, const double* locs, const double* y, const double* X,
                        const int32_t* NN, int64_t n, int d, int p, int m,
                        const double* covparms, vec_covfun covfun, cudaStream_t st,
                        double* out, long long* dev_status) {
    const int cov = (int)covfun;
    vg::PassPlan plan;
    int pr = vg::plan_pass(cov, m, d, p, h->nsm, h->lanes, h->threads, &plan);
    if (pr == -1) return fail(VEC_ERR_UNSUPPORTED, "no kernel mapping fits m = %d, p = %d", m, p);
    if (pr != 0) return cuda_fail(cudaGetLastError(), "planning the pass kernel");
    cudaError_t e = grow(&h->partials, &h->partials_cap, (size_t)plan.grid * plan.nstat);
    if (e != cudaSuccess) return cuda_fail(e, "allocating partial sums");
    const bool tr = h->timing != 0;
    if (tr) cudaEventRecord(h->ev[0], st);
    e = vg::launch_init_status(h->status, h->bad, st);
    if (e == cudaSuccess && cov == vg::COV_MATERN) e = vg::launch_mtab_build(covparms, h->mtab, st);
    if (e != cudaSuccess) return cuda_fail(e, "launching the setup kernels");
    vg::PassArgs a;
    a.locs = locs; a.y = y; a.X = X; a.NN = NN; a.covparms = covparms;
    a.mtab = h->mtab; a.partials = h->partials; a.status = h->status; a.bad = h->bad;
    a.n = n; a.d = d; a.p = p; a.m = m;
    a.nstat = plan.nstat; a.nv = plan.nv; a.slot_stride = plan.slot_stride;
    a.acc_per_lane = plan.acc_per_lane; a.tab_in_smem = plan.tab_smem;
    if (tr) cudaEventRecord(h->ev[1], st);
    e = vg::launch_pass(cov, plan, a, st);
    if (e != cudaSuccess) return cuda_fail(e, "launching the pass kernel");
    if (tr) cudaEventRecord(h->ev[2], st);
    e = vg::launch_profile(h->partials, plan.grid, plan.nstat, p, cov, n, covparms, h->status,
                           h->bad, out, dev_status, st);
    if (e != cudaSuccess) return cuda_fail(e, "launching the profile kernel");
    if (tr) {
        cudaEventRecord(h->ev[3], st);
        h->traced = 1;
    }
    return VEC_OK;
}

}  // namespace

extern "C" {

vec_status vecchia_loglik_grad_info(vec_handle h, const double* locs, const double* y,
                                    const double* X, const int32_t* NNarray, int64_t n, int d,
                                    int p, int m, const double* covparms, vec_covfun covfun,
                                    vec_precision prec, void* stream, double* out,
                                    int64_t* dev_status) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_loglik_grad_info: NULL handle");
    vec_status s = check_args(locs, y, X, NNarray, n, d, p, m, covparms, covfun, prec);
    if (s != VEC_OK) return s;
    if (!out || !dev_status) return fail(VEC_ERR_ARG, "out and dev_status are required");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    return enqueue_pass(h, locs, y, X, NNarray, n, d, p, m, covparms, covfun,
                        reinterpret_cast<cudaStream_t>(stream), out,
                        reinterpret_cast<long long*>(dev_status));
}

vec_status vecchia_loglik_grad_info_host(vec_handle h, const double* locs, const double* y,
                                         const double* X, const int32_t* NNarray, int64_t n,
                                         int d, int p, int m, const double* covparms,
                                         vec_covfun covfun, vec_precision prec,
                                         double* loglik, double* grad, double* info,
                                         double* betahat, int64_t* bad_index) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_loglik_grad_info_host: NULL handle");
    vec_status s = check_args(locs, y, X, NNarray, n, d, p, m, covparms, covfun, prec);
    if (s != VEC_OK) return s;
    if (!loglik || !grad || !info || !betahat) return fail(VEC_ERR_ARG, "an output pointer is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    const int q = vecchia_nparms(covfun);
    const size_t nout = 1 + q + (size_t)q * q + p;
    cudaError_t e = grow(&h->h_locs, &h->c_locs, (size_t)n * d);
    if (e == cudaSuccess) e = grow(&h->h_y, &h->c_y, (size_t)n);
    if (e == cudaSuccess) e = grow(&h->h_X, &h->c_X, (size_t)n * p);
    if (e == cudaSuccess) e = grow(&h->h_NN, &h->c_NN, (size_t)n * (m + 1));
    if (e == cudaSuccess) e = grow(&h->h_cov, &h->c_cov, (size_t)q);
    if (e == cudaSuccess) e = grow(&h->h_out, &h->c_out, nout);
    if (e == cudaSuccess) e = grow(&h->h_st, &h->c_st, (size_t)2);
    if (e != cudaSuccess) return cuda_fail(e, "allocating staging buffers");
    cudaStream_t st = h->stream;
    e = cudaMemcpyAsync(h->h_locs, locs, sizeof(double) * n * d, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_y, y, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_X, X, sizeof(double) * n * p, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->h_NN, NNarray, sizeof(int32_t) * n * (m + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_cov, covparms, sizeof(double) * q, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "copying inputs to the device");
    s = enqueue_pass(h, h->h_locs, h->h_y, h->h_X, h->h_NN, n, d, p, m, h->h_cov, covfun, st,
                     h->h_out, h->h_st);
    if (s != VEC_OK) return s;
    double res[1 + 4 + 16 + vg::PMAX];
    long long dst[2];
    e = cudaMemcpyAsync(res, h->h_out, sizeof(double) * nout, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, h->h_st, sizeof(long long) * 2, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "running the pass");
    *loglik = res[0];
    for (int j = 0; j < q; ++j) grad[j] = res[1 + j];
    for (int t = 0; t < q * q; ++t) info[t] = res[1 + q + t];
    for (int a = 0; a < p; ++a) betahat[a] = res[1 + q + q * q + a];
    if (bad_index) *bad_index = dst[1];
    if (dst[0] != 0) {
        static const char* names[] = {"ok", "bad argument or NNarray row", "block not positive definite",
                                      "non-finite result"};
        int code = (int)dst[0];
        return fail((vec_status)code, "pass failed: %s (first observation %lld)",
                    (code >= 0 && code < 4) ? names[code] : "?", (long long)dst[1]);
    }
    return VEC_OK;
}

vec_status vecchia_covariance_pairs(vec_handle h, vec_covfun covfun, const double* covparms,
                                    int d, int64_t npairs, const double* la, const double* lb,
                                    const int32_t* same, double* C, double* dC, void* stream) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_covariance_pairs: NULL handle");
    if (vecchia_nparms(covfun) < 0) return fail(VEC_ERR_ARG, "unknown covariance function");
    if (d < 1 || d > vg::DMAX || (covfun == VEC_EXP_SPACETIME && d != 3))
        return fail(VEC_ERR_ARG, "bad d = %d", d);
    if (npairs < 0) return fail(VEC_ERR_ARG, "npairs < 0");
    if (npairs > 0 && (!covparms || !la || !lb || !same || !C || !dC))
        return fail(VEC_ERR_ARG, "a required pointer is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (covfun == VEC_MATERN_ISO) e = vg::launch_mtab_build(covparms, h->mtab, st);
    if (e == cudaSuccess)
        e = vg::launch_cov_pairs((int)covfun, covparms, h->mtab, d, npairs, la, lb, same, C, dC, st);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_covariance_pairs");
    return VEC_OK;
}

}  // extern "C"
