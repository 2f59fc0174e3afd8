// vg_capi.cu -- the extern "C" boundary of the Vecchia library (declared in
// include/vecchia.h): handles, argument validation, scratch management and launch order.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <vector>

#include "../../include/vecchia.h"
#include "vg_internal.h"
#include "vg_common.cuh"
#include "vg_fit.h"

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

constexpr int kFitKey = 24;  // words of the single-fit graph cache key

struct TuneEntry {
    int cov, m, d, p, prec, log2n, lanes, threads;
    float ms;
    int tab;  // Matern table placement of the mapping: 1 shared memory, 0 global, -1 planner's
};

// Device buffers of a batched pass: the work list (tiles of observations), per-dataset
// offsets and m, status words, per-tile partial records and per-dataset Matern tables.
struct BatchScratch {
    int4* tiles = nullptr; size_t c_tiles = 0;
    int* tile_off = nullptr; size_t c_tile_off = 0;
    vg::DatasetDesc* desc = nullptr; size_t c_desc = 0;
    int* status = nullptr; size_t c_status = 0;
    long long* bad = nullptr; size_t c_bad = 0;
    int* counter = nullptr; size_t c_counter = 0;
    int* tile_ids = nullptr; size_t c_tile_ids = 0;
    double* partials = nullptr; size_t c_part = 0;
    double* tabs = nullptr; size_t c_tabs = 0;
    float* tabsf = nullptr; size_t c_tabsf = 0;
    void release() {
        cudaFree(tiles); cudaFree(tile_off); cudaFree(desc);
        cudaFree(status); cudaFree(bad); cudaFree(counter); cudaFree(tile_ids); cudaFree(partials);
        cudaFree(tabs); cudaFree(tabsf);
        *this = BatchScratch();
    }
};

struct vec_handle_s {
    int device = 0;
    int nsm = 0;
    int lanes = 0;    // 0 = automatic
    int threads = 0;  // 0 = automatic
    int tab_mode = -1;  // forced Matern table placement (-1 = planner's or autotuned choice)
    int gchunk = 0;     // grouped: members formed together (0 = planner's choice)
    cudaStream_t stream = nullptr;
    // tracing
    int timing = 0;
    int traced = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // Fisher-scoring driver
    vg::FitState* fs = nullptr;
    double* fit_out = nullptr;
    long long* fit_st = nullptr;
    double* fit_start = nullptr;
    cudaGraph_t fit_graph[2] = {nullptr, nullptr};
    cudaGraphExec_t fit_exec[2] = {nullptr, nullptr};
    unsigned long long fit_key[2][kFitKey] = {{0}, {0}};
    int fit_lru = 0;
    // autotuned mappings
    std::vector<TuneEntry> tune;
    // batched pass scratch
    BatchScratch bs;
    // batched fit state
    vg::FitState* bf_fs = nullptr; size_t c_bf_fs = 0;
    double* bf_theta = nullptr; size_t c_bf_theta = 0;
    int* bf_active = nullptr; size_t c_bf_active = 0;
    int* bf_any = nullptr; size_t c_bf_any = 0;
    double* bf_out = nullptr; size_t c_bf_out = 0;
    long long* bf_st = nullptr; size_t c_bf_st = 0;
    // simulation factor rows
    double* sim_factor = nullptr; size_t c_sim_factor = 0;
    // semivariogram scratch
    double* vg_mean = nullptr; size_t c_vg_mean = 0;
    double* vg_var = nullptr; size_t c_vg_var = 0;
    double* vg_psum = nullptr; size_t c_vg_psum = 0;
    long long* vg_pcnt = nullptr; size_t c_vg_pcnt = 0;
    // MLP and learned start scratch
    float* mlp_gpart = nullptr; size_t c_mlp_gpart = 0;
    float* mlp_lpart = nullptr; size_t c_mlp_lpart = 0;
    float* ws_feat = nullptr; size_t c_ws_feat = 0;
    float* ws_pred = nullptr; size_t c_ws_pred = 0;
    double* ws_theta0 = nullptr; size_t c_ws_theta0 = 0;
    double* ws_out = nullptr; size_t c_ws_out = 0;
    long long* ws_st = nullptr; size_t c_ws_st = 0;
    // ordered-neighbour search scratch
    char* nn_scratch = nullptr; size_t c_nn_scratch = 0;
    // maxmin ordering scratch
    char* mm_scratch = nullptr; size_t c_mm_scratch = 0;
    // grouped pass: unit counters of the class launches, and the side streams and events
    // that let the classes share the GPU (created on first use)
    int* gcount = nullptr; size_t c_gcount = 0;
    cudaStream_t gside[2] = {nullptr, nullptr};
    cudaEvent_t gev[3] = {nullptr, nullptr, nullptr};
    double* mm_bbox = nullptr; size_t c_mm_bbox = 0;
    int* mm_err = nullptr; size_t c_mm_err = 0;
    // pass scratch
    double* partials = nullptr;
    size_t partials_cap = 0;
    double* mtab = nullptr;
    float* mtabf = nullptr;
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

int vecchia_nparms_d(vec_covfun covfun, int d) {
    switch (covfun) {
    case VEC_EXP_ISO: return (d >= 1 && d <= vg::DMAX) ? 3 : -1;
    case VEC_MATERN_ISO: return (d >= 1 && d <= vg::DMAX) ? 4 : -1;
    case VEC_EXP_SPACETIME: return d == 3 ? 4 : -1;
    case VEC_EXP_ANISO: return (d >= 1 && d <= vg::DMAX_ANISO) ? d + 2 : -1;
    default: return -1;
    }
}

int vecchia_nparms(vec_covfun covfun) {
    switch (covfun) {
    case VEC_EXP_ISO: return 3;
    case VEC_MATERN_ISO: return 4;
    case VEC_EXP_SPACETIME: return 4;
    default: return -1;   // unknown, or a count that depends on d (VEC_EXP_ANISO)
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
    if (vecchia_nparms_d(covfun, covfun == VEC_EXP_SPACETIME ? 3 : 1) < 0) return -1;
    return 5;   // status reset, table, pass, record sums, profile (FP64: every family's table)
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
    if (!(threads == 0 || threads == 32 || threads == 64 || threads == 96 || threads == 128 ||
          threads == 192 || threads == 256))
        return fail(VEC_ERR_ARG, "threads must be 0, 32, 64, 96, 128, 192 or 256 (got %d)", threads);
    h->threads = threads;
    return VEC_OK;
}

vec_status vecchia_set_group_chunk(vec_handle h, int chunk) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_set_group_chunk: NULL handle");
    if (chunk < 0 || chunk > vg::GCH_MAX)
        return fail(VEC_ERR_ARG, "chunk must be 0..%d (got %d)", vg::GCH_MAX, chunk);
    h->gchunk = chunk;
    return VEC_OK;
}

vec_status vecchia_set_matern_table(vec_handle h, int placement) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_set_matern_table: NULL handle");
    if (placement < -1 || placement > 1)
        return fail(VEC_ERR_ARG, "placement must be -1, 0 or 1 (got %d)", placement);
    h->tab_mode = placement;
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
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&h->mtabf),
                                         sizeof(float) * vg::mtab_floats());
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
    cudaFree(h->gcount);
    for (int k = 0; k < 2; ++k)
        if (h->gside[k]) cudaStreamDestroy(h->gside[k]);
    for (int k = 0; k < 3; ++k)
        if (h->gev[k]) cudaEventDestroy(h->gev[k]);
    cudaFree(h->mm_scratch);
    cudaFree(h->mm_bbox);
    cudaFree(h->mm_err);
    cudaFree(h->mtab);
    cudaFree(h->mtabf);
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
    for (int k = 0; k < 2; ++k) {
        if (h->fit_exec[k]) cudaGraphExecDestroy(h->fit_exec[k]);
        if (h->fit_graph[k]) cudaGraphDestroy(h->fit_graph[k]);
    }
    cudaFree(h->fs);
    cudaFree(h->fit_out);
    cudaFree(h->fit_st);
    cudaFree(h->fit_start);
    h->bs.release();
    cudaFree(h->bf_fs); cudaFree(h->bf_theta); cudaFree(h->bf_active); cudaFree(h->bf_any);
    cudaFree(h->bf_out); cudaFree(h->bf_st); cudaFree(h->sim_factor);
    cudaFree(h->vg_mean); cudaFree(h->vg_var); cudaFree(h->vg_psum); cudaFree(h->vg_pcnt);
    cudaFree(h->mlp_gpart); cudaFree(h->mlp_lpart); cudaFree(h->ws_feat); cudaFree(h->ws_pred);
    cudaFree(h->ws_theta0); cudaFree(h->ws_out); cudaFree(h->ws_st); cudaFree(h->nn_scratch);
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
    if (vecchia_nparms_d(covfun, d) < 0)
        return fail(VEC_ERR_ARG, "covariance function %d does not take d = %d (isotropic: 1..3, "
                    "space-time: 3, one range per coordinate: 1..%d)", (int)covfun, d, vg::DMAX_ANISO);
    if (p < 1 || p > vg::PMAX) return fail(VEC_ERR_ARG, "p = %d out of range [1, %d]", p, vg::PMAX);
    if (m < 0 || m > vg::KMAX - 1)
        return fail(VEC_ERR_UNSUPPORTED, "m = %d out of range [0, %d]", m, vg::KMAX - 1);
    if (prec != VEC_FP64 && prec != VEC_MIXED) return fail(VEC_ERR_ARG, "unknown precision %d", (int)prec);
    return VEC_OK;
}

// Chooses the kernel mapping and makes sure the partial-sum scratch is large enough
// (the only allocation a pass may need; done before any graph capture).
int ilog2(int64_t n) {
    int k = 0;
    while ((1ll << (k + 1)) <= n) ++k;
    return k;
}

// Block records are summed this many at a time by k_reduce_records before the profile
// step (fixed order, so the result does not depend on the grid).
constexpr int kRecChunk = 64;

vec_status prepare_pass(vec_handle h, int cov, int m, int d, int p, vg::PassPlan* plan,
                        int64_t n = 0, int prec = 0) {
    int L = h->lanes, thr = h->threads, tab = -1;
    if (L == 0 && thr == 0 && n > 0) {
        const int lg = ilog2(n);
        for (const TuneEntry& t : h->tune)
            if (t.cov == cov && t.m == m && t.d == d && t.p == p && t.prec == prec && t.log2n == lg) {
                L = t.lanes;
                thr = t.threads;
                tab = t.tab;
            }
    }
    if (h->tab_mode >= 0) tab = h->tab_mode;
    int pr = vg::plan_pass(cov, m, d, p, h->nsm, L, thr, plan, prec, false, tab);
    if (pr == -1)  // a stale record or a placement that does not fit: plan afresh
        pr = vg::plan_pass(cov, m, d, p, h->nsm, h->lanes, h->threads, plan, prec);
    if (pr == -1) return fail(VEC_ERR_UNSUPPORTED, "no kernel mapping fits m = %d, p = %d", m, p);
    if (pr != 0) return cuda_fail(cudaGetLastError(), "planning the pass kernel");
    // the blocks' records, then their sums kRecChunk at a time
    const size_t nsum = ((size_t)plan->grid + kRecChunk - 1) / kRecChunk;
    cudaError_t e = grow(&h->partials, &h->partials_cap, ((size_t)plan->grid + nsum) * plan->nstat);
    if (e != cudaSuccess) return cuda_fail(e, "allocating partial sums");
    return VEC_OK;
}

// Enqueues the full pass on `st`.  Device pointers only.
vec_status enqueue_pass(vec_handle h, const double* locs, const double* y, const double* X,
                        const int32_t* NN, int64_t n, int d, int p, int m,
                        const double* covparms, vec_covfun covfun, cudaStream_t st,
                        double* out, long long* dev_status, int prec) {
    const int cov = (int)covfun;
    vg::PassPlan plan;
    vec_status ps = prepare_pass(h, cov, m, d, p, &plan, n, prec);
    if (ps != VEC_OK) return ps;
    cudaError_t e;
    const bool tr = h->timing != 0;
    if (tr) cudaEventRecord(h->ev[0], st);
    e = vg::launch_init_status(h->status, h->bad, st);
    if (e == cudaSuccess && vg::uses_table(cov, prec))
        e = vg::launch_mtab_build(cov, covparms, h->mtab, prec ? h->mtabf : nullptr, st);
    if (e != cudaSuccess) return cuda_fail(e, "launching the setup kernels");
    vg::PassArgs a;
    a.locs = locs; a.y = y; a.X = X; a.NN = NN; a.covparms = covparms;
    a.mtab = h->mtab; a.mtabf = h->mtabf; a.partials = h->partials; a.status = h->status;
    a.bad = h->bad;
    a.n = n; a.d = d; a.p = p; a.m = m;
    a.nstat = plan.nstat; a.nv = plan.nv; a.slot_stride = plan.slot_stride;
    a.acc_per_lane = plan.acc_per_lane; a.tab_in_smem = plan.tab_smem;
    if (tr) cudaEventRecord(h->ev[1], st);
    e = vg::launch_pass(cov, plan, a, st);
    if (e != cudaSuccess) return cuda_fail(e, "launching the pass kernel");
    if (tr) cudaEventRecord(h->ev[2], st);
    // the block records summed kRecChunk at a time (in order, by many blocks), then the
    // profile step over those sums
    double* sums = h->partials + (size_t)plan.grid * plan.nstat;
    const int nsum = (plan.grid + kRecChunk - 1) / kRecChunk;
    e = vg::launch_reduce_records(h->partials, plan.grid, plan.nstat, kRecChunk, sums, st);
    if (e == cudaSuccess)
        e = vg::launch_profile(sums, nsum, plan.nstat, p, vg::nparms(cov, d), n, covparms,
                               h->status, h->bad, out, dev_status, st);
    if (e != cudaSuccess) return cuda_fail(e, "launching the profile kernels");
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
                        reinterpret_cast<long long*>(dev_status), (int)prec);
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
    const int q = vecchia_nparms_d(covfun, d);
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
                     h->h_out, h->h_st, (int)prec);
    if (s != VEC_OK) return s;
    double res[1 + vg::QMAX + vg::QMAX * vg::QMAX + vg::PMAX];
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

vec_status vecchia_fit(vec_handle h, const double* locs, const double* y, const double* X,
                       const int32_t* NNarray, int64_t n, int d, int p, int m, vec_covfun covfun,
                       const double* start, const vec_fit_opts* opts, void* stream,
                       double* theta_out, double* betahat, double* loglik, double* grad,
                       double* info, vec_fit_info* fit_info) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_fit: NULL handle");
    vec_fit_opts o = {1e-4, 40, 10, 1, (int)VEC_FP64};
    if (opts) o = *opts;
    // VEC_FIT_MIXED_ONLY (fit option only): every pass in mixed precision, no FP64 phase
    const bool mixed_only = (o.prec == VEC_FIT_MIXED_ONLY);
    vec_status s = check_args(locs, y, X, NNarray, n, d, p, m, start, covfun,
                              mixed_only ? VEC_MIXED : (vec_precision)o.prec);
    if (s != VEC_OK) return s;
    if (!theta_out || !betahat || !loglik || !grad || !info)
        return fail(VEC_ERR_ARG, "vecchia_fit: an output pointer is NULL");
    if (!(o.tol >= 0.0) || o.maxit < 0 || o.maxit > 100000 || o.max_halvings < 0 || o.max_halvings > 60)
        return fail(VEC_ERR_ARG, "vecchia_fit: bad options (tol %g, maxit %d, max_halvings %d)", o.tol,
                    o.maxit, o.max_halvings);
    const int q = vecchia_nparms_d(covfun, d);
    for (int j = 0; j < q; ++j)
        if (!(start[j] > 0.0) || !std::isfinite(start[j]))
            return fail(VEC_ERR_ARG, "vecchia_fit: start[%d] = %g is not a positive number", j, start[j]);
    if (covfun == VEC_MATERN_ISO && !(start[2] >= 0.05 && start[2] <= 20.0))
        return fail(VEC_ERR_ARG, "vecchia_fit: start smoothness %g outside [0.05, 20]", start[2]);
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    const int cov = (int)covfun;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (!h->fs) e = cudaMalloc(reinterpret_cast<void**>(&h->fs), sizeof(vg::FitState));
    if (e == cudaSuccess && !h->fit_out)
        e = cudaMalloc(reinterpret_cast<void**>(&h->fit_out),
                       sizeof(double) * (1 + vg::QMAX + vg::QMAX * vg::QMAX + vg::PMAX));
    if (e == cudaSuccess && !h->fit_st) e = cudaMalloc(reinterpret_cast<void**>(&h->fit_st), sizeof(long long) * 2);
    if (e == cudaSuccess && !h->fit_start) e = cudaMalloc(reinterpret_cast<void**>(&h->fit_start), sizeof(double) * vg::QMAX);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_fit: allocating the fit state");
    const double* theta_trial = h->fs->theta_trial;  // device address of the member
    // a hard bound on the number of passes, so the device loop always ends
    const int max_evals = (o.maxit + 2) * (o.max_halvings + 2);
    e = cudaMemcpyAsync(h->fit_start, start, sizeof(double) * q, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_fit: initialising");
    const int saved_timing = h->timing;
    h->timing = 0;
    // phases: a mixed-precision fit first (when asked), then FP64 from where it stopped
    const int nphase = (o.prec == (int)VEC_MIXED) ? 2 : 1;
    int total_iters = 0, total_evals = 0;
    for (int phase = 0; phase < nphase; ++phase) {
        const int prec = (mixed_only || (nphase == 2 && phase == 0)) ? 1 : 0;
        const double* phase_start = (phase == 0) ? h->fit_start : h->fs->theta_cur;
        vg::PassPlan pplan;
        s = prepare_pass(h, cov, m, d, p, &pplan, n, prec);
        if (s != VEC_OK) { h->timing = saved_timing; return s; }
        e = vg::launch_fit_init(h->fs, phase_start, q, st);
        if (e != cudaSuccess) { h->timing = saved_timing; return cuda_fail(e, "vecchia_fit: initialising"); }
        if (o.use_graph) {
            // everything the captured kernels read: inputs, sizes, options, the mapping and
            // the handle's scratch buffers (a later call may have reallocated them)
            unsigned long long key[kFitKey] = {
                (unsigned long long)(uintptr_t)locs, (unsigned long long)(uintptr_t)y,
                (unsigned long long)(uintptr_t)X, (unsigned long long)(uintptr_t)NNarray,
                (unsigned long long)n, (unsigned long long)d, (unsigned long long)p,
                (unsigned long long)m, (unsigned long long)cov, (unsigned long long)prec,
                (unsigned long long)o.maxit, (unsigned long long)o.max_halvings, 0ull,
                (unsigned long long)pplan.L, (unsigned long long)pplan.threads,
                (unsigned long long)pplan.grid, (unsigned long long)(uintptr_t)h->partials,
                (unsigned long long)(uintptr_t)h->mtab, (unsigned long long)(uintptr_t)h->mtabf,
                (unsigned long long)(uintptr_t)h->status, (unsigned long long)(uintptr_t)h->bad,
                (unsigned long long)(uintptr_t)h->fs, (unsigned long long)(uintptr_t)h->fit_out,
                (unsigned long long)(uintptr_t)h->fit_st};
            std::memcpy(&key[12], &o.tol, sizeof(double));
            int slot = -1;
            for (int k = 0; k < 2; ++k)
                if (h->fit_exec[k] && std::memcmp(key, h->fit_key[k], sizeof(key)) == 0) slot = k;
            if (slot < 0) {
                slot = h->fit_lru;
                h->fit_lru ^= 1;
                if (h->fit_exec[slot]) { cudaGraphExecDestroy(h->fit_exec[slot]); h->fit_exec[slot] = nullptr; }
                if (h->fit_graph[slot]) { cudaGraphDestroy(h->fit_graph[slot]); h->fit_graph[slot] = nullptr; }
                cudaGraph_t graph = nullptr;
                cudaGraphConditionalHandle cond;
                cudaGraphNode_t node;
                e = cudaGraphCreate(&graph, 0);
                if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
                cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
                cp.conditional.handle = cond;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
                if (e != cudaSuccess) {
                    if (graph) cudaGraphDestroy(graph);
                    h->timing = saved_timing;
                    return cuda_fail(e, "vecchia_fit: building the iteration graph");
                }
                cudaGraph_t body = cp.conditional.phGraph_out[0];
                e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed);
                vec_status ps = VEC_OK;
                if (e == cudaSuccess) {
                    ps = enqueue_pass(h, locs, y, X, NNarray, n, d, p, m, theta_trial, covfun, h->stream,
                                      h->fit_out, h->fit_st, prec);
                    cudaError_t e2 = vg::launch_fit_step(h->fs, h->fit_out, h->fit_st, q, p, cov, o.tol,
                                                         o.maxit, o.max_halvings, cond, 1, h->stream);
                    cudaGraph_t captured = nullptr;
                    e = cudaStreamEndCapture(h->stream, &captured);
                    if (e == cudaSuccess) e = e2;
                }
                if (e == cudaSuccess && ps == VEC_OK) e = cudaGraphInstantiate(&h->fit_exec[slot], graph, 0);
                if (e != cudaSuccess || ps != VEC_OK) {
                    cudaGraphDestroy(graph);
                    h->fit_exec[slot] = nullptr;
                    h->timing = saved_timing;
                    if (ps != VEC_OK) return ps;
                    return cuda_fail(e, "vecchia_fit: capturing the iteration graph");
                }
                h->fit_graph[slot] = graph;
                std::memcpy(h->fit_key[slot], key, sizeof(key));
            }
            e = cudaGraphLaunch(h->fit_exec[slot], st);
            if (e != cudaSuccess) {
                h->timing = saved_timing;
                return cuda_fail(e, "vecchia_fit: launching the iteration graph");
            }
        } else {
            for (int ev = 0; ev < max_evals; ++ev) {
                s = enqueue_pass(h, locs, y, X, NNarray, n, d, p, m, theta_trial, covfun, st,
                                 h->fit_out, h->fit_st, prec);
                if (s != VEC_OK) { h->timing = saved_timing; return s; }
                cudaGraphConditionalHandle none = 0;
                e = vg::launch_fit_step(h->fs, h->fit_out, h->fit_st, q, p, cov, o.tol, o.maxit,
                                        o.max_halvings, none, 0, st);
                int done = 0;
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(&done, &h->fs->done, sizeof(int), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) { h->timing = saved_timing; return cuda_fail(e, "vecchia_fit: iterating"); }
                if (done) break;
            }
        }
        if (nphase == 2 && phase == 0) {
            vg::FitState f0;
            e = cudaMemcpyAsync(&f0, h->fs, sizeof(f0), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { h->timing = saved_timing; return cuda_fail(e, "vecchia_fit: reading phase 1"); }
            total_iters += f0.iters;
            total_evals += f0.evals;
            if (f0.status == vg::FIT_START_FAILED) break;  // the FP64 phase starts from the same point
        }
    }
    h->timing = saved_timing;
    vg::FitState fs;
    e = cudaMemcpyAsync(&fs, h->fs, sizeof(fs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_fit: reading the result");
    for (int j = 0; j < q; ++j) { theta_out[j] = fs.theta_cur[j]; grad[j] = fs.grad[j]; }
    for (int t = 0; t < q * q; ++t) info[t] = fs.info[t];
    for (int a = 0; a < p; ++a) betahat[a] = fs.beta[a];
    *loglik = fs.loglik;
    if (fit_info) {
        fit_info->status = fs.done ? fs.status : vg::FIT_MAXIT;
        fit_info->iters = total_iters + fs.iters;
        fit_info->evals = total_evals + fs.evals;
        fit_info->pass_status = fs.pass_status;
    }
    return VEC_OK;
}

vec_status vecchia_autotune(vec_handle h, const double* locs, const double* y, const double* X,
                            const int32_t* NNarray, int64_t n, int d, int p, int m,
                            const double* covparms, vec_covfun covfun, vec_precision prec,
                            void* stream, int reps, int* lanes_out, int* threads_out,
                            float* ms_out) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_autotune: NULL handle");
    vec_status s = check_args(locs, y, X, NNarray, n, d, p, m, covparms, covfun, prec);
    if (s != VEC_OK) return s;
    if (reps < 1) reps = 1;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int cov = (int)covfun;
    const int q = vecchia_nparms_d(covfun, d);
    double* out = nullptr;
    long long* dst = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&out), sizeof(double) * (1 + q + q * q + p));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&dst), sizeof(long long) * 2);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int saved_L = h->lanes, saved_T = h->threads, saved_timing = h->timing;
    const int saved_tab = h->tab_mode;
    h->timing = 0;
    int bestL = 0, bestT = 0;
    float best = 1e30f;
    static const int thr_list[] = {256, 192, 128, 96, 64};
    int bestTab = -1;
    const int ntab = vg::uses_table(cov, (int)prec) ? 2 : 1;
    for (int ti = 0; ti < 5 && e == cudaSuccess; ++ti) {
        for (int L = 1; L <= 32 && e == cudaSuccess; L *= 2)
        for (int tb = 0; tb < ntab && e == cudaSuccess; ++tb) {
            const int tab = vg::uses_table(cov, (int)prec) ? 1 - tb : -1;  // shared memory first
            if (L > thr_list[ti]) continue;
            vg::PassPlan plan;
            if (vg::plan_pass(cov, m, d, p, h->nsm, L, thr_list[ti], &plan, (int)prec, false, tab) != 0)
                continue;
            if (plan.L != L || plan.threads != thr_list[ti]) continue;
            h->lanes = L;
            h->threads = thr_list[ti];
            h->tab_mode = tab;
            s = enqueue_pass(h, locs, y, X, NNarray, n, d, p, m, covparms, covfun, st, out, dst,
                             (int)prec);
            if (s != VEC_OK) break;
            float tmin = 1e30f;
            for (int r = 0; r < reps && e == cudaSuccess; ++r) {
                e = cudaEventRecord(e0, st);
                s = enqueue_pass(h, locs, y, X, NNarray, n, d, p, m, covparms, covfun, st, out, dst,
                                 (int)prec);
                if (s != VEC_OK) break;
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (ms < tmin) tmin = ms;
            }
            if (s != VEC_OK) break;
            if (tmin < best) { best = tmin; bestL = L; bestT = thr_list[ti]; bestTab = tab; }
        }
        if (s != VEC_OK) break;
    }
    h->lanes = saved_L;
    h->threads = saved_T;
    h->tab_mode = saved_tab;
    h->timing = saved_timing;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(dst);
    if (s != VEC_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_autotune");
    if (bestL == 0) return fail(VEC_ERR_UNSUPPORTED, "vecchia_autotune: no mapping fits");
    TuneEntry t = {cov, m, d, p, (int)prec, ilog2(n), bestL, bestT, best, bestTab};
    bool replaced = false;
    for (TuneEntry& u : h->tune)
        if (u.cov == t.cov && u.m == t.m && u.d == t.d && u.p == t.p && u.prec == t.prec &&
            u.log2n == t.log2n) { u = t; replaced = true; }
    if (!replaced) h->tune.push_back(t);
    if (lanes_out) *lanes_out = bestL;
    if (threads_out) *threads_out = bestT;
    if (ms_out) *ms_out = best;
    return VEC_OK;
}

vec_status vecchia_autotune_save(vec_handle h, const char* path) {
    if (!h || !path) return fail(VEC_ERR_ARG, "vecchia_autotune_save: NULL argument");
    FILE* f = std::fopen(path, "w");
    if (!f) return fail(VEC_ERR_ARG, "vecchia_autotune_save: cannot open %s", path);
    std::fprintf(f, "[\n");
    for (size_t i = 0; i < h->tune.size(); ++i) {
        const TuneEntry& t = h->tune[i];
        std::fprintf(f, "  {\"covfun\": %d, \"m\": %d, \"d\": %d, \"p\": %d, \"prec\": %d, "
                        "\"log2n\": %d, \"lanes\": %d, \"threads\": %d, \"ms\": %.6f, "
                        "\"tab\": %d}%s\n",
                     t.cov, t.m, t.d, t.p, t.prec, t.log2n, t.lanes, t.threads, t.ms, t.tab,
                     i + 1 < h->tune.size() ? "," : "");
    }
    std::fprintf(f, "]\n");
    std::fclose(f);
    return VEC_OK;
}

vec_status vecchia_autotune_load(vec_handle h, const char* path) {
    if (!h || !path) return fail(VEC_ERR_ARG, "vecchia_autotune_load: NULL argument");
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(VEC_ERR_ARG, "vecchia_autotune_load: cannot open %s", path);
    std::string txt;
    char buf[4096];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, k);
    std::fclose(f);
    // one record per {...}; every key must be present
    size_t pos = 0;
    int loaded = 0;
    while ((pos = txt.find('{', pos)) != std::string::npos) {
        size_t end = txt.find('}', pos);
        if (end == std::string::npos) break;
        std::string rec = txt.substr(pos, end - pos);
        auto get = [&](const char* key, double* v) {
            std::string pat = std::string("\"") + key + "\"";
            size_t at = rec.find(pat);
            if (at == std::string::npos) return false;
            at = rec.find(':', at);
            if (at == std::string::npos) return false;
            return std::sscanf(rec.c_str() + at + 1, "%lf", v) == 1;
        };
        double v[9];
        const char* keys[9] = {"covfun", "m", "d", "p", "prec", "log2n", "lanes", "threads", "ms"};
        bool ok = true;
        for (int i = 0; i < 9 && ok; ++i) ok = get(keys[i], &v[i]);
        if (!ok) return fail(VEC_ERR_ARG, "vecchia_autotune_load: malformed record in %s", path);
        double tabv = -1.0;  // optional key
        if (!get("tab", &tabv)) tabv = -1.0;
        TuneEntry t = {(int)v[0], (int)v[1], (int)v[2], (int)v[3], (int)v[4], (int)v[5], (int)v[6],
                       (int)v[7], (float)v[8], (int)tabv};
        bool replaced = false;
        for (TuneEntry& u : h->tune)
            if (u.cov == t.cov && u.m == t.m && u.d == t.d && u.p == t.p && u.prec == t.prec &&
                u.log2n == t.log2n) { u = t; replaced = true; }
        if (!replaced) h->tune.push_back(t);
        ++loaded;
        pos = end + 1;
    }
    (void)loaded;
    return VEC_OK;
}

}  // extern "C"

namespace {

// Host-side description of a batch and the uploads shared by the batched pass and fit.
// Datasets are split into up to three classes by block size K = m + 1 (K <= 16, K <= 32,
// larger), each launched with its own kernel mapping and slots sized for its largest m: a
// K = 11 block on the lanes chosen for K = 41 leaves most of them idle.  Tiles stay in
// dataset order (records per tile, reduced per dataset); each class launch takes its
// tiles from its own index list and counter.
constexpr int kBatchClasses = 3;

static int batch_class_of(int m) { return m + 1 <= 16 ? 0 : (m + 1 <= 32 ? 1 : 2); }

struct BatchPlan {
    int nbatch, mmax, ntiles;
    long long ntot;
    vg::PassPlan plan;                   // the class with the most observations (reported)
    int nclass;                          // classes with datasets
    vg::PassPlan cplan[kBatchClasses];
    int cmmax[kBatchClasses];
    int cbeg[kBatchClasses + 1];         // class c's tiles: tile_ids[cbeg[c] .. cbeg[c + 1])
    std::vector<int4> tiles;
    std::vector<int> tile_off;
    std::vector<int> tile_ids;
    std::vector<vg::DatasetDesc> desc;
};

// Mapping of one class: forced, else autotuned for (cov, class mmax, d, p, prec, class
// observations), else planned.  Returns a vec_status.
static vec_status plan_batch_class(vec_handle h, int cov, int mmax, long long ntot, int d, int p,
                                   int prec, vg::PassPlan* plan) {
    int L = h->lanes, thr = h->threads, tab = -1;
    if (L == 0 && thr == 0) {
        const int lg = ilog2(ntot);
        for (const TuneEntry& t : h->tune)
            if (t.cov == cov && t.m == mmax && t.d == d && t.p == p && t.prec == prec + 2 &&
                t.log2n == lg) { L = t.lanes; thr = t.threads; tab = t.tab; }
    }
    if (h->tab_mode >= 0) tab = h->tab_mode;
    int pr = vg::plan_pass(cov, mmax, d, p, h->nsm, L, thr, plan, prec, true, tab);
    if (pr == -1) pr = vg::plan_pass(cov, mmax, d, p, h->nsm, h->lanes, h->threads, plan, prec, true);
    if (pr == -1) return fail(VEC_ERR_UNSUPPORTED, "no kernel mapping fits m = %d, p = %d", mmax, p);
    if (pr != 0) return cuda_fail(cudaGetLastError(), "planning the batched pass");
    return VEC_OK;
}

// Plans and uploads a batch described dataset by dataset (B->desc filled by the caller).
vec_status prepare_batch_desc(vec_handle h, BatchScratch& S, int d, int p, vec_covfun covfun,
                              int prec, cudaStream_t st, BatchPlan* B) {
    const int nbatch = (int)B->desc.size();
    if (nbatch < 1) return fail(VEC_ERR_ARG, "nbatch = %d", nbatch);
    B->nbatch = nbatch;
    B->mmax = 0;
    B->ntot = 0;
    long long cn[kBatchClasses] = {0, 0, 0};
    for (int c = 0; c < kBatchClasses; ++c) B->cmmax[c] = -1;
    for (int b = 0; b < nbatch; ++b) {
        const vg::DatasetDesc& D = B->desc[b];
        if (D.n < 1) return fail(VEC_ERR_ARG, "dataset %d has n = %d", b, D.n);
        if (D.m < 0 || D.m > vg::KMAX - 1)
            return fail(VEC_ERR_UNSUPPORTED, "dataset %d: m = %d out of range", b, D.m);
        if (D.m > B->mmax) B->mmax = D.m;
        B->ntot += D.n;
        const int c = batch_class_of(D.m);
        cn[c] += D.n;
        if (D.m > B->cmmax[c]) B->cmmax[c] = D.m;
    }
    const int cov = (int)covfun;
    B->nclass = 0;
    int main_c = -1;
    for (int c = 0; c < kBatchClasses; ++c) {
        if (cn[c] == 0) continue;
        ++B->nclass;
        vec_status s = plan_batch_class(h, cov, B->cmmax[c], cn[c], d, p, prec, &B->cplan[c]);
        if (s != VEC_OK) return s;
        if (main_c < 0 || cn[c] > cn[main_c]) main_c = c;
    }
    B->plan = B->cplan[main_c];
    // tiles in dataset order; a class's tiles hold up to 32 observations per group of its
    // mapping, fewer where that would leave fewer than about four tiles per block of its
    // launch (the last tiles of a launch set its tail); then the index lists
    long long csize[kBatchClasses];
    for (int c = 0; c < kBatchClasses; ++c) {
        if (cn[c] == 0) continue;
        const vg::PassPlan& P = B->cplan[c];
        const long long ngrp = P.threads / P.L;
        const long long per = (cn[c] + 4LL * P.grid - 1) / (4LL * P.grid);
        long long t = per > ngrp ? per : ngrp;
        t = t > 64 ? t : 64;
        csize[c] = t < ngrp * 32 ? t : ngrp * 32;
    }
    B->tiles.clear();
    B->tile_off.assign(nbatch + 1, 0);
    for (int b = 0; b < nbatch; ++b) {
        const long long tsize = csize[batch_class_of(B->desc[b].m)];
        const long long nb = B->desc[b].n;
        for (long long s0 = 0; s0 < nb; s0 += tsize) {
            long long e0 = s0 + tsize < nb ? s0 + tsize : nb;
            B->tiles.push_back(make_int4(b, (int)s0, (int)e0, 0));
        }
        B->tile_off[b + 1] = (int)B->tiles.size();
    }
    B->ntiles = (int)B->tiles.size();
    B->tile_ids.clear();
    for (int c = 0; c < kBatchClasses; ++c) {
        B->cbeg[c] = (int)B->tile_ids.size();
        if (B->nclass > 1)
            for (int b = 0; b < nbatch; ++b)
                if (batch_class_of(B->desc[b].m) == c)
                    for (int t = B->tile_off[b]; t < B->tile_off[b + 1]; ++t) B->tile_ids.push_back(t);
    }
    B->cbeg[kBatchClasses] = (int)B->tile_ids.size();
    cudaError_t e = grow(&S.tiles, &S.c_tiles, (size_t)B->ntiles);
    if (e == cudaSuccess) e = grow(&S.tile_off, &S.c_tile_off, (size_t)nbatch + 1);
    if (e == cudaSuccess) e = grow(&S.desc, &S.c_desc, (size_t)nbatch);
    if (e == cudaSuccess) e = grow(&S.status, &S.c_status, (size_t)nbatch);
    if (e == cudaSuccess) e = grow(&S.bad, &S.c_bad, (size_t)nbatch);
    if (e == cudaSuccess) e = grow(&S.counter, &S.c_counter, (size_t)kBatchClasses);
    if (e == cudaSuccess && !B->tile_ids.empty())
        e = grow(&S.tile_ids, &S.c_tile_ids, B->tile_ids.size());
    if (e == cudaSuccess) e = grow(&S.partials, &S.c_part, (size_t)B->ntiles * B->plan.nstat);
    if (e == cudaSuccess && vg::uses_table(cov, prec))
        e = grow(&S.tabs, &S.c_tabs, (size_t)nbatch * vg::mtab_doubles());
    if (e == cudaSuccess && cov == vg::COV_MATERN && prec)
        e = grow(&S.tabsf, &S.c_tabsf, (size_t)nbatch * vg::mtab_floats());
    if (e != cudaSuccess) return cuda_fail(e, "allocating batch scratch");
    e = cudaMemcpyAsync(S.tiles, B->tiles.data(), sizeof(int4) * B->ntiles, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S.tile_off, B->tile_off.data(), sizeof(int) * (nbatch + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S.desc, B->desc.data(), sizeof(vg::DatasetDesc) * nbatch, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !B->tile_ids.empty())
        e = cudaMemcpyAsync(S.tile_ids, B->tile_ids.data(), sizeof(int) * B->tile_ids.size(),
                            cudaMemcpyHostToDevice, st);
    // the host vectors are released when B goes out of scope: make the copies complete
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "uploading the batch description");
    return VEC_OK;
}

// Dataset descriptions of concatenated datasets: dataset b owns rows [off[b], off[b+1])
// and the next n_b (m_b+1) NNarray entries.
vec_status batch_descs(int nbatch, const int64_t* point_offsets, const int* m,
                       std::vector<vg::DatasetDesc>* desc) {
    desc->assign(nbatch, vg::DatasetDesc());
    long long nn = 0;
    for (int b = 0; b < nbatch; ++b) {
        const long long nb = point_offsets[b + 1] - point_offsets[b];
        if (nb < 1) return fail(VEC_ERR_ARG, "dataset %d has n = %lld", b, nb);
        vg::DatasetDesc& D = (*desc)[b];
        D.loc = D.x = D.y = point_offsets[b];
        D.nn = nn;
        D.n = (int)nb;
        D.m = m[b];
        nn += nb * (long long)(m[b] + 1);
    }
    return VEC_OK;
}

// Concatenated datasets (batch_descs), planned and uploaded.
vec_status prepare_batch(vec_handle h, BatchScratch& S, int nbatch, const int64_t* point_offsets,
                         const int* m, int d, int p, vec_covfun covfun, int prec, cudaStream_t st,
                         BatchPlan* B) {
    if (nbatch < 1) return fail(VEC_ERR_ARG, "nbatch = %d", nbatch);
    if (!point_offsets || !m) return fail(VEC_ERR_ARG, "point_offsets and m are required");
    if (point_offsets[0] != 0) return fail(VEC_ERR_ARG, "point_offsets[0] must be 0");
    if (point_offsets[nbatch] > (int64_t)INT_MAX) return fail(VEC_ERR_ARG, "too many observations");
    vec_status s = batch_descs(nbatch, point_offsets, m, &B->desc);
    if (s != VEC_OK) return s;
    return prepare_batch_desc(h, S, d, p, covfun, prec, st, B);
}

// Fields at shared locations: every field uses locs, X and NNarray from row 0; field b's
// observations are y[b n, (b+1) n).
vec_status prepare_fields(vec_handle h, BatchScratch& S, int nfields, int64_t n, int m, int d,
                          int p, vec_covfun covfun, int prec, cudaStream_t st, BatchPlan* B) {
    if (nfields < 1) return fail(VEC_ERR_ARG, "nfields = %d", nfields);
    if (n < 1 || n > (int64_t)INT_MAX) return fail(VEC_ERR_ARG, "n = %lld out of range", (long long)n);
    if ((long long)nfields * n > (long long)INT_MAX * 64)
        return fail(VEC_ERR_ARG, "nfields x n too large");
    B->desc.assign(nfields, vg::DatasetDesc());
    for (int b = 0; b < nfields; ++b) {
        vg::DatasetDesc& D = B->desc[b];
        D.loc = D.x = D.nn = 0;
        D.y = (long long)b * n;
        D.n = (int)n;
        D.m = m;
    }
    return prepare_batch_desc(h, S, d, p, covfun, prec, st, B);
}

// Enqueues one batched pass (device pointers): kernel launches only, no allocation, copy
// or host synchronisation, so it may be captured into a CUDA graph.
vec_status enqueue_batch(const BatchScratch& S, const BatchPlan& B, const double* locs,
                         const double* y, const double* X, const int32_t* NN, int d, int p,
                         const double* covparms, vec_covfun covfun, int prec, cudaStream_t st,
                         double* out, long long* dev_status, const int* active,
                         double* factor = nullptr) {
    const int cov = (int)covfun;
    const int q = vecchia_nparms_d(covfun, d);
    cudaError_t e = vg::launch_init_batch(S.status, S.bad, B.nbatch, S.counter, kBatchClasses, st);
    if (e == cudaSuccess && vg::uses_table(cov, prec))
        e = vg::launch_mtab_build_batch(cov, covparms, B.nbatch, q, S.tabs, prec ? S.tabsf : nullptr,
                                        active, st);
    if (e != cudaSuccess) return cuda_fail(e, "launching the batch setup kernels");
    for (int c = 0; c < kBatchClasses && e == cudaSuccess; ++c) {
        const int one = B.nclass == 1;
        if (B.cmmax[c] < 0) continue;
        const vg::PassPlan& P = B.cplan[c];
        vg::BatchArgs a;
        a.base.locs = locs; a.base.y = y; a.base.X = X; a.base.NN = NN; a.base.covparms = nullptr;
        a.base.mtab = nullptr; a.base.mtabf = nullptr; a.base.partials = S.partials;
        a.base.status = nullptr; a.base.bad = nullptr;
        a.base.n = B.ntot; a.base.d = d; a.base.p = p; a.base.m = B.cmmax[c];
        a.base.nstat = P.nstat; a.base.nv = P.nv; a.base.slot_stride = P.slot_stride;
        a.base.acc_per_lane = P.acc_per_lane; a.base.tab_in_smem = P.tab_smem;
        a.desc = S.desc; a.covparms_b = covparms; a.factor = factor;
        a.tabs = S.tabs; a.tabsf = S.tabsf; a.tiles = S.tiles;
        a.tile_ids = one ? nullptr : S.tile_ids + B.cbeg[c];
        a.ntiles = one ? B.ntiles : B.cbeg[c + 1] - B.cbeg[c];
        a.tile_counter = S.counter + c; a.status_b = S.status; a.bad_b = S.bad; a.active_b = active;
        e = vg::launch_pass_batch(cov, P, a, st);
    }
    if (e == cudaSuccess && factor)  // factor rows only: report the per-dataset status
        e = vg::launch_batch_status(S.status, S.bad, B.nbatch, dev_status, st);
    else if (e == cudaSuccess)
        e = vg::launch_profile_batch(S.partials, S.tile_off, B.nbatch, B.plan.nstat, p, q,
                                     S.desc, covparms, S.status, S.bad, out, dev_status, st);
    if (e != cudaSuccess) return cuda_fail(e, "launching the batched pass");
    return VEC_OK;
}

}  // namespace

extern "C" {

static vec_status check_batch_args(const char* who, vec_handle h, int nbatch, const double* locs,
                                   const double* y, const double* X, const int32_t* NNarray,
                                   const int64_t* point_offsets, const int* m, int d, int p,
                                   vec_covfun covfun, int prec) {
    if (!h) return fail(VEC_ERR_ARG, "%s: NULL handle", who);
    if (!locs || !y || !X || !NNarray || !point_offsets || !m)
        return fail(VEC_ERR_ARG, "%s: a required pointer is NULL", who);
    if (nbatch < 1) return fail(VEC_ERR_ARG, "%s: nbatch = %d", who, nbatch);
    if (vecchia_nparms_d(covfun, d) < 0)
        return fail(VEC_ERR_ARG, "%s: covariance function %d does not take d = %d", who, (int)covfun, d);
    if (p < 1 || p > vg::PMAX) return fail(VEC_ERR_ARG, "%s: p = %d out of range", who, p);
    if (prec != VEC_FP64 && prec != VEC_MIXED) return fail(VEC_ERR_ARG, "%s: unknown precision", who);
    return VEC_OK;
}

vec_status vecchia_batch_loglik_grad_info(vec_handle h, int nbatch, const double* locs,
                                          const double* y, const double* X, const int32_t* NNarray,
                                          const int64_t* point_offsets, const int* m, int d, int p,
                                          const double* covparms, vec_covfun covfun,
                                          vec_precision prec, void* stream, double* out,
                                          int64_t* dev_status) {
    vec_status s = check_batch_args("vecchia_batch_loglik_grad_info", h, nbatch, locs, y, X, NNarray,
                                    point_offsets, m, d, p, covfun, (int)prec);
    if (s != VEC_OK) return s;
    if (!covparms || !out || !dev_status) return fail(VEC_ERR_ARG, "a required pointer is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    BatchPlan B;
    s = prepare_batch(h, h->bs, nbatch, point_offsets, m, d, p, covfun, (int)prec, st, &B);
    if (s != VEC_OK) return s;
    return enqueue_batch(h->bs, B, locs, y, X, NNarray, d, p, covparms, covfun, (int)prec, st, out,
                         reinterpret_cast<long long*>(dev_status), nullptr);
}

}  // extern "C"

struct vec_batch_plan_s {
    int device = 0;
    int nbatch = 0, d = 0, p = 0, prec = 0;
    vec_covfun covfun = VEC_EXP_ISO;
    BatchPlan B;
    BatchScratch S;
};

extern "C" {

vec_status vecchia_batch_plan_create(vec_handle h, int nbatch, const int64_t* point_offsets,
                                     const int* m, int d, int p, vec_covfun covfun,
                                     vec_precision prec, vec_batch_plan* plan_out) {
    if (!plan_out) return fail(VEC_ERR_ARG, "vecchia_batch_plan_create: plan_out is NULL");
    *plan_out = nullptr;
    if (!h) return fail(VEC_ERR_ARG, "vecchia_batch_plan_create: NULL handle");
    if (!point_offsets || !m) return fail(VEC_ERR_ARG, "vecchia_batch_plan_create: point_offsets and m are required");
    if (vecchia_nparms_d(covfun, d) < 0)
        return fail(VEC_ERR_ARG, "covariance function %d does not take d = %d", (int)covfun, d);
    if (p < 1 || p > vg::PMAX) return fail(VEC_ERR_ARG, "p = %d out of range", p);
    if (prec != VEC_FP64 && prec != VEC_MIXED) return fail(VEC_ERR_ARG, "unknown precision");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    vec_batch_plan_s* P = new (std::nothrow) vec_batch_plan_s;
    if (!P) return fail(VEC_ERR_NOMEM, "vecchia_batch_plan_create: out of host memory");
    P->device = h->device;
    P->nbatch = nbatch;
    P->d = d;
    P->p = p;
    P->prec = (int)prec;
    P->covfun = covfun;
    vec_status s = prepare_batch(h, P->S, nbatch, point_offsets, m, d, p, covfun, (int)prec,
                                 h->stream, &P->B);
    if (s != VEC_OK) {
        P->S.release();
        delete P;
        return s;
    }
    *plan_out = P;
    return VEC_OK;
}

vec_status vecchia_batch_plan_run(vec_batch_plan plan, const double* locs, const double* y,
                                  const double* X, const int32_t* NNarray, const double* covparms,
                                  void* stream, double* out, int64_t* dev_status) {
    if (!plan) return fail(VEC_ERR_ARG, "vecchia_batch_plan_run: NULL plan");
    if (!locs || !y || !X || !NNarray || !covparms || !out || !dev_status)
        return fail(VEC_ERR_ARG, "vecchia_batch_plan_run: a required pointer is NULL");
    DeviceGuard g(plan->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", plan->device);
    return enqueue_batch(plan->S, plan->B, locs, y, X, NNarray, plan->d, plan->p, covparms,
                         plan->covfun, plan->prec, reinterpret_cast<cudaStream_t>(stream), out,
                         reinterpret_cast<long long*>(dev_status), nullptr);
}

vec_status vecchia_batch_plan_mapping(vec_batch_plan plan, int* lanes, int* threads, int* ntiles) {
    if (!plan) return fail(VEC_ERR_ARG, "vecchia_batch_plan_mapping: NULL plan");
    if (lanes) *lanes = plan->B.plan.L;
    if (threads) *threads = plan->B.plan.threads;
    if (ntiles) *ntiles = plan->B.ntiles;
    return VEC_OK;
}

vec_status vecchia_batch_plan_class(vec_batch_plan plan, int c, int* mmax, int* lanes, int* threads,
                                    int* ntiles) {
    if (!plan) return fail(VEC_ERR_ARG, "vecchia_batch_plan_class: NULL plan");
    if (c < 0 || c >= kBatchClasses) return fail(VEC_ERR_ARG, "vecchia_batch_plan_class: class %d", c);
    const BatchPlan& B = plan->B;
    const bool has = B.cmmax[c] >= 0;
    if (mmax) *mmax = has ? B.cmmax[c] : -1;
    if (lanes) *lanes = has ? B.cplan[c].L : 0;
    if (threads) *threads = has ? B.cplan[c].threads : 0;
    if (ntiles) *ntiles = !has ? 0 : (B.nclass == 1 ? B.ntiles : B.cbeg[c + 1] - B.cbeg[c]);
    return VEC_OK;
}

vec_status vecchia_batch_plan_destroy(vec_batch_plan plan) {
    if (!plan) return VEC_OK;
    DeviceGuard g(plan->device);
    plan->S.release();
    delete plan;
    return VEC_OK;
}

}  // extern "C"

// Batched Fisher scoring over the batch that prep(prec, &plan) describes (see
// vecchia_batch_fit).  Arguments are checked by the callers.
static vec_status batch_fit_impl(vec_handle h, int nbatch,
                                 const std::function<vec_status(int, BatchPlan*)>& prep,
                                 const double* locs, const double* y, const double* X,
                                 const int32_t* NNarray, int d, int p, vec_covfun covfun,
                                 const double* start, const vec_fit_opts& o, void* stream,
                                 double* theta_out, double* out, vec_fit_info* fit_info) {
    vec_status s = VEC_OK;
    if (!start || !theta_out || !out) return fail(VEC_ERR_ARG, "batched fit: a required pointer is NULL");
    if (!(o.tol >= 0.0) || o.maxit < 0 || o.maxit > 100000 || o.max_halvings < 0 || o.max_halvings > 60)
        return fail(VEC_ERR_ARG, "batched fit: bad options (tol %g, maxit %d, max_halvings %d)",
                    o.tol, o.maxit, o.max_halvings);
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    const int cov = (int)covfun;
    const int q = vecchia_nparms_d(covfun, d);
    const int nout = 1 + q + q * q + p;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = grow(&h->bf_fs, &h->c_bf_fs, (size_t)nbatch);
    if (e == cudaSuccess) e = grow(&h->bf_theta, &h->c_bf_theta, (size_t)nbatch * q);
    if (e == cudaSuccess) e = grow(&h->bf_active, &h->c_bf_active, (size_t)nbatch);
    if (e == cudaSuccess) e = grow(&h->bf_any, &h->c_bf_any, (size_t)1);
    if (e == cudaSuccess) e = grow(&h->bf_out, &h->c_bf_out, (size_t)nbatch * nout);
    if (e == cudaSuccess) e = grow(&h->bf_st, &h->c_bf_st, (size_t)nbatch * 2);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_batch_fit: allocating the fit state");
    const int max_evals = (o.maxit + 2) * (o.max_halvings + 2);
    const bool mixed_only = (o.prec == VEC_FIT_MIXED_ONLY);
    const int nphase = (o.prec == (int)VEC_MIXED) ? 2 : 1;
    std::vector<vg::FitState> fsh((size_t)nbatch);
    std::vector<int> iters0((size_t)nbatch, 0), evals0((size_t)nbatch, 0);
    const int saved_timing = h->timing;
    h->timing = 0;
    for (int phase = 0; phase < nphase; ++phase) {
        const int prec = (mixed_only || (nphase == 2 && phase == 0)) ? 1 : 0;
        BatchPlan B;
        s = prep(prec, &B);
        if (s != VEC_OK) break;
        e = vg::launch_fit_init_batch(h->bf_fs, start, phase > 0 ? 1 : 0, q, nbatch, h->bf_theta,
                                      h->bf_active, st);
        if (e != cudaSuccess) { s = cuda_fail(e, "vecchia_batch_fit: initialising"); break; }
        if (o.use_graph) {
            // WHILE node around (batched pass, batched step); built for this call only,
            // since it captures the handle's batch buffers as they are now
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            cudaGraphConditionalHandle cond;
            cudaGraphNode_t node;
            e = cudaGraphCreate(&graph, 0);
            if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
            cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
            cp.conditional.handle = cond;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
            vec_status ps = VEC_OK;
            if (e == cudaSuccess) {
                e = cudaStreamBeginCaptureToGraph(h->stream, cp.conditional.phGraph_out[0], nullptr,
                                                  nullptr, 0, cudaStreamCaptureModeRelaxed);
                if (e == cudaSuccess) {
                    ps = enqueue_batch(h->bs, B, locs, y, X, NNarray, d, p, h->bf_theta, covfun, prec,
                                       h->stream, h->bf_out, h->bf_st, h->bf_active);
                    cudaError_t e2 = vg::launch_fit_step_batch(
                        h->bf_fs, h->bf_out, h->bf_st, q, p, cov, o.tol, o.maxit, o.max_halvings,
                        nbatch, h->bf_theta, h->bf_active, h->bf_any, cond, 1, h->stream);
                    cudaGraph_t captured = nullptr;
                    e = cudaStreamEndCapture(h->stream, &captured);
                    if (e == cudaSuccess) e = e2;
                }
            }
            if (e == cudaSuccess && ps == VEC_OK) e = cudaGraphInstantiate(&exec, graph, 0);
            if (e == cudaSuccess && ps == VEC_OK) e = cudaGraphLaunch(exec, st);
            if (e == cudaSuccess && ps == VEC_OK) e = cudaStreamSynchronize(st);
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            if (ps != VEC_OK) { s = ps; break; }
            if (e != cudaSuccess) { s = cuda_fail(e, "vecchia_batch_fit: running the iteration graph"); break; }
        } else {
            for (int ev = 0; ev < max_evals; ++ev) {
                s = enqueue_batch(h->bs, B, locs, y, X, NNarray, d, p, h->bf_theta, covfun, prec, st,
                                  h->bf_out, h->bf_st, h->bf_active);
                if (s != VEC_OK) break;
                cudaGraphConditionalHandle none = 0;
                e = vg::launch_fit_step_batch(h->bf_fs, h->bf_out, h->bf_st, q, p, cov, o.tol, o.maxit,
                                              o.max_halvings, nbatch, h->bf_theta, h->bf_active,
                                              h->bf_any, none, 0, st);
                int any = 0;
                if (e == cudaSuccess) e = cudaMemcpyAsync(&any, h->bf_any, sizeof(int), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) { s = cuda_fail(e, "vecchia_batch_fit: iterating"); break; }
                if (!any) break;
            }
            if (s != VEC_OK) break;
        }
        if (nphase == 2 && phase == 0) {
            e = cudaMemcpyAsync(fsh.data(), h->bf_fs, sizeof(vg::FitState) * nbatch, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { s = cuda_fail(e, "vecchia_batch_fit: reading phase 1"); break; }
            for (int b = 0; b < nbatch; ++b) { iters0[b] = fsh[b].iters; evals0[b] = fsh[b].evals; }
        }
    }
    h->timing = saved_timing;
    if (s != VEC_OK) return s;
    e = vg::launch_fit_export_batch(h->bf_fs, nbatch, q, p, theta_out, out, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(fsh.data(), h->bf_fs, sizeof(vg::FitState) * nbatch, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_batch_fit: reading the result");
    if (fit_info)
        for (int b = 0; b < nbatch; ++b) {
            fit_info[b].status = fsh[b].done ? fsh[b].status : vg::FIT_MAXIT;
            fit_info[b].iters = iters0[b] + fsh[b].iters;
            fit_info[b].evals = evals0[b] + fsh[b].evals;
            fit_info[b].pass_status = fsh[b].pass_status;
        }
    return VEC_OK;
}

extern "C" {

vec_status vecchia_batch_fit(vec_handle h, int nbatch, const double* locs, const double* y,
                             const double* X, const int32_t* NNarray, const int64_t* point_offsets,
                             const int* m, int d, int p, vec_covfun covfun, const double* start,
                             const vec_fit_opts* opts, void* stream, double* theta_out, double* out,
                             vec_fit_info* fit_info) {
    vec_fit_opts o = {1e-4, 40, 10, 1, (int)VEC_FP64};
    if (opts) o = *opts;
    vec_status s = check_batch_args("vecchia_batch_fit", h, nbatch, locs, y, X, NNarray,
                                    point_offsets, m, d, p, covfun,
                                    o.prec == VEC_FIT_MIXED_ONLY ? (int)VEC_MIXED : o.prec);
    if (s != VEC_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    auto prep = [&](int prec, BatchPlan* B) {
        return prepare_batch(h, h->bs, nbatch, point_offsets, m, d, p, covfun, prec, st, B);
    };
    return batch_fit_impl(h, nbatch, prep, locs, y, X, NNarray, d, p, covfun, start, o, stream,
                          theta_out, out, fit_info);
}

vec_status vecchia_batch_autotune(vec_handle h, int nbatch, const double* locs, const double* y,
                                  const double* X, const int32_t* NNarray,
                                  const int64_t* point_offsets, const int* m, int d, int p,
                                  const double* covparms, vec_covfun covfun, vec_precision prec,
                                  void* stream, int reps, int* lanes_out, int* threads_out,
                                  float* ms_out) {
    vec_status s = check_batch_args("vecchia_batch_autotune", h, nbatch, locs, y, X, NNarray,
                                    point_offsets, m, d, p, covfun, (int)prec);
    if (s != VEC_OK) return s;
    if (!covparms) return fail(VEC_ERR_ARG, "vecchia_batch_autotune: covparms is NULL");
    if (reps < 1) reps = 1;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int cov = (int)covfun;
    const int q = vecchia_nparms_d(covfun, d);
    double* out = nullptr;
    long long* dst = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&out), sizeof(double) * nbatch * (1 + q + q * q + p));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&dst), sizeof(long long) * 2 * nbatch);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int saved_L = h->lanes, saved_T = h->threads, saved_tab = h->tab_mode;
    // each class of datasets (by block size, as the batch plan splits them) is tuned on its
    // own datasets, and recorded under its largest m and its observation count
    std::vector<vg::DatasetDesc> all;
    if (e == cudaSuccess) s = batch_descs(nbatch, point_offsets, m, &all);
    int repL = 0, repT = 0;
    long long repN = -1;
    float total = 0.f;
    static const int thr_list[] = {256, 192, 128, 96, 64};
    const int ntab = vg::uses_table(cov, (int)prec) ? 2 : 1;
    for (int c = 0; c < kBatchClasses && e == cudaSuccess && s == VEC_OK; ++c) {
        std::vector<vg::DatasetDesc> sub;
        int mmax = 0;
        long long ntot = 0;
        for (const vg::DatasetDesc& D : all)
            if (batch_class_of(D.m) == c) {
                sub.push_back(D);
                mmax = D.m > mmax ? D.m : mmax;
                ntot += D.n;
            }
        if (sub.empty()) continue;
        int bestL = 0, bestT = 0, bestTab = -1;
        float best = 1e30f;
        for (int ti = 0; ti < 5 && e == cudaSuccess && s == VEC_OK; ++ti) {
            for (int L = 1; L <= 32 && e == cudaSuccess && s == VEC_OK; L *= 2)
            for (int tb = 0; tb < ntab && e == cudaSuccess; ++tb) {
                const int tab = vg::uses_table(cov, (int)prec) ? 1 - tb : -1;
                if (L > thr_list[ti]) continue;
                vg::PassPlan plan;
                if (vg::plan_pass(cov, mmax, d, p, h->nsm, L, thr_list[ti], &plan, (int)prec, true, tab) != 0)
                    continue;
                if (plan.L != L || plan.threads != thr_list[ti]) continue;
                h->lanes = L;
                h->threads = thr_list[ti];
                h->tab_mode = tab;
                BatchPlan B;
                B.desc = sub;
                s = prepare_batch_desc(h, h->bs, d, p, covfun, (int)prec, st, &B);
                if (s != VEC_OK) break;
                s = enqueue_batch(h->bs, B, locs, y, X, NNarray, d, p, covparms, covfun, (int)prec, st,
                                  out, dst, nullptr);
                if (s != VEC_OK) break;
                float tmin = 1e30f;
                for (int r = 0; r < reps && e == cudaSuccess; ++r) {
                    e = cudaEventRecord(e0, st);
                    s = enqueue_batch(h->bs, B, locs, y, X, NNarray, d, p, covparms, covfun, (int)prec,
                                      st, out, dst, nullptr);
                    if (s != VEC_OK) break;
                    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float ms = 0.f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < tmin) tmin = ms;
                }
                if (s != VEC_OK) break;
                if (tmin < best) { best = tmin; bestL = L; bestT = thr_list[ti]; bestTab = tab; }
            }
        }
        if (s != VEC_OK || e != cudaSuccess) break;
        if (bestL == 0) { s = fail(VEC_ERR_UNSUPPORTED, "vecchia_batch_autotune: no mapping fits"); break; }
        // batched records are kept apart from single-dataset ones: prec + 2
        TuneEntry t = {cov, mmax, d, p, (int)prec + 2, ilog2(ntot), bestL, bestT, best, bestTab};
        bool replaced = false;
        for (TuneEntry& u : h->tune)
            if (u.cov == t.cov && u.m == t.m && u.d == t.d && u.p == t.p && u.prec == t.prec &&
                u.log2n == t.log2n) { u = t; replaced = true; }
        if (!replaced) h->tune.push_back(t);
        total += best;
        if (ntot > repN) { repN = ntot; repL = bestL; repT = bestT; }
    }
    h->lanes = saved_L;
    h->threads = saved_T;
    h->tab_mode = saved_tab;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(dst);
    if (s != VEC_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_batch_autotune");
    if (lanes_out) *lanes_out = repL;
    if (threads_out) *threads_out = repT;
    if (ms_out) *ms_out = total;
    return VEC_OK;
}

static vec_status check_fields_args(const char* who, vec_handle h, int nfields, const double* locs,
                                    const double* X, const int32_t* NNarray, int64_t n, int d,
                                    int p, int m, const double* Y, vec_covfun covfun, int prec) {
    if (!h) return fail(VEC_ERR_ARG, "%s: NULL handle", who);
    if (!locs || !X || !NNarray || !Y) return fail(VEC_ERR_ARG, "%s: a required pointer is NULL", who);
    if (nfields < 1) return fail(VEC_ERR_ARG, "%s: nfields = %d", who, nfields);
    if (n < 1 || n > (int64_t)INT_MAX) return fail(VEC_ERR_ARG, "%s: n = %lld", who, (long long)n);
    if (m < 0 || m > vg::KMAX - 1) return fail(VEC_ERR_UNSUPPORTED, "%s: m = %d out of range", who, m);
    if (vecchia_nparms_d(covfun, d) < 0)
        return fail(VEC_ERR_ARG, "%s: covariance function %d does not take d = %d", who, (int)covfun, d);
    if (p < 1 || p > vg::PMAX) return fail(VEC_ERR_ARG, "%s: p = %d out of range", who, p);
    if (prec != VEC_FP64 && prec != VEC_MIXED) return fail(VEC_ERR_ARG, "%s: unknown precision", who);
    return VEC_OK;
}

vec_status vecchia_fields_loglik_grad_info(vec_handle h, int nfields, const double* locs,
                                           const double* X, const int32_t* NNarray, int64_t n,
                                           int d, int p, int m, const double* Y,
                                           const double* covparms, vec_covfun covfun,
                                           vec_precision prec, void* stream, double* out,
                                           int64_t* dev_status) {
    vec_status s = check_fields_args("vecchia_fields_loglik_grad_info", h, nfields, locs, X, NNarray,
                                     n, d, p, m, Y, covfun, (int)prec);
    if (s != VEC_OK) return s;
    if (!covparms || !out || !dev_status) return fail(VEC_ERR_ARG, "a required pointer is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    BatchPlan B;
    s = prepare_fields(h, h->bs, nfields, n, m, d, p, covfun, (int)prec, st, &B);
    if (s != VEC_OK) return s;
    return enqueue_batch(h->bs, B, locs, Y, X, NNarray, d, p, covparms, covfun, (int)prec, st, out,
                         reinterpret_cast<long long*>(dev_status), nullptr);
}

vec_status vecchia_fields_fit(vec_handle h, int nfields, const double* locs, const double* X,
                              const int32_t* NNarray, int64_t n, int d, int p, int m,
                              const double* Y, vec_covfun covfun, const double* start,
                              const vec_fit_opts* opts, void* stream, double* theta_out,
                              double* out, vec_fit_info* fit_info) {
    vec_fit_opts o = {1e-4, 40, 10, 1, (int)VEC_FP64};
    if (opts) o = *opts;
    vec_status s = check_fields_args("vecchia_fields_fit", h, nfields, locs, X, NNarray, n, d, p, m,
                                     Y, covfun, o.prec == VEC_FIT_MIXED_ONLY ? (int)VEC_MIXED : o.prec);
    if (s != VEC_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    auto prep = [&](int prec, BatchPlan* B) {
        return prepare_fields(h, h->bs, nfields, n, m, d, p, covfun, prec, st, B);
    };
    return batch_fit_impl(h, nfields, prep, locs, Y, X, NNarray, d, p, covfun, start, o, stream,
                          theta_out, out, fit_info);
}

vec_status vecchia_fields_simulate(vec_handle h, int nfields, const double* locs,
                                   const int32_t* NNarray, int64_t n, int d, int m,
                                   const double* covparms, vec_covfun covfun, const double* z,
                                   void* stream, double* y, int64_t* dev_status) {
    // X is not read in factor mode beyond a gather of one column: locs serves as that column
    vec_status s = check_fields_args("vecchia_fields_simulate", h, nfields, locs, locs, NNarray, n,
                                     d, 1, m, z, covfun, 0);
    if (s != VEC_OK) return s;
    if (!covparms || !y || !dev_status) return fail(VEC_ERR_ARG, "a required pointer is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int q = vecchia_nparms_d(covfun, d);
    const size_t row = (size_t)n * (m + 1);
    // factor rows of a chunk of fields at a time, at most ~1 GiB of scratch
    const size_t chunk = std::max<size_t>(1, std::min<size_t>((size_t)nfields, ((size_t)1 << 27) / row));
    cudaError_t e = grow(&h->sim_factor, &h->c_sim_factor, chunk * row);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_fields_simulate: allocating factor rows");
    for (size_t f0 = 0; f0 < (size_t)nfields; f0 += chunk) {
        const int nf = (int)std::min(chunk, (size_t)nfields - f0);
        BatchPlan B;
        s = prepare_fields(h, h->bs, nf, n, m, d, 1, covfun, 0, st, &B);
        if (s != VEC_OK) return s;
        s = enqueue_batch(h->bs, B, locs, z + f0 * n, locs, NNarray, d, 1, covparms + f0 * q, covfun,
                          0, st, nullptr, reinterpret_cast<long long*>(dev_status) + 2 * f0, nullptr,
                          h->sim_factor);
        if (s != VEC_OK) return s;
        e = vg::launch_sim_recur(h->sim_factor, NNarray, (int)n, m, nf, z + f0 * n, y + f0 * n, st);
        if (e != cudaSuccess) return cuda_fail(e, "vecchia_fields_simulate: launching the recurrence");
    }
    return VEC_OK;
}

vec_status vecchia_fields_variogram(vec_handle h, int nfields, const double* locs,
                                    const int32_t* NNarray, int64_t n, int d, int m,
                                    const double* Y, const uint32_t* rand_pairs, int64_t npairs,
                                    const double* edges2, int nbins, void* stream, float* features,
                                    double* bin_sum, int64_t* bin_count) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_fields_variogram: NULL handle");
    if (!locs || !NNarray || !Y || !edges2 || !features || (npairs > 0 && !rand_pairs))
        return fail(VEC_ERR_ARG, "vecchia_fields_variogram: a required pointer is NULL");
    if (nfields < 1 || n < 2 || n > (int64_t)INT_MAX || d < 1 || d > vg::DMAX || m < 0 ||
        m > vg::KMAX - 1 || npairs < 0 || nbins < 1 || nbins > vg::VG_MAX_BINS)
        return fail(VEC_ERR_ARG, "vecchia_fields_variogram: bad sizes (nfields %d, n %lld, d %d, m %d, "
                    "npairs %lld, nbins %d)", nfields, (long long)n, d, m, (long long)npairs, nbins);
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // slices per field: enough blocks to fill the GPU, at least 8192 pairs per block
    const long long W = n * (long long)m + npairs;
    long long slices = (4LL * h->nsm * 4 + nfields - 1) / nfields;
    const long long cap = W / 8192 > 1 ? W / 8192 : 1;
    if (slices > cap) slices = cap;
    if (slices < 1) slices = 1;
    const size_t np = (size_t)nfields * slices * nbins;
    cudaError_t e = grow(&h->vg_mean, &h->c_vg_mean, (size_t)nfields);
    if (e == cudaSuccess) e = grow(&h->vg_var, &h->c_vg_var, (size_t)nfields);
    if (e == cudaSuccess) e = grow(&h->vg_psum, &h->c_vg_psum, np);
    if (e == cudaSuccess) e = grow(&h->vg_pcnt, &h->c_vg_pcnt, np);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_fields_variogram: allocating scratch");
    e = vg::launch_field_moments(Y, (int)n, nfields, h->vg_mean, h->vg_var, st);
    if (e == cudaSuccess)
        e = vg::launch_vario(locs, d, NNarray, (int)n, m, Y, nfields, rand_pairs, (long long)npairs,
                             edges2, nbins, (int)slices, h->vg_psum, h->vg_pcnt, st);
    if (e == cudaSuccess)
        e = vg::launch_vario_finish(h->vg_psum, h->vg_pcnt, (int)slices, nbins, h->vg_var, nfields,
                                    features, bin_sum, reinterpret_cast<long long*>(bin_count), st);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_fields_variogram: launching");
    return VEC_OK;
}

vec_status vecchia_fields_moments(vec_handle h, int nfields, int64_t n, const double* Y,
                                  void* stream, double* mean, double* var) {
    if (!h || !Y || !mean || !var || nfields < 1 || n < 1 || n > (int64_t)INT_MAX)
        return fail(VEC_ERR_ARG, "vecchia_fields_moments: bad argument");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaError_t e = vg::launch_field_moments(Y, (int)n, nfields, mean, var,
                                             reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_fields_moments");
    return VEC_OK;
}

vec_status vecchia_mlp_targets(vec_handle h, int nfields, const double* theta, const double* var,
                               const double* lo, const double* hi, void* stream, float* targets) {
    if (!h || !theta || !var || !lo || !hi || !targets || nfields < 1)
        return fail(VEC_ERR_ARG, "vecchia_mlp_targets: bad argument");
    for (int j = 0; j < 4; ++j)
        if (!(lo[j] > 0.0 && hi[j] >= lo[j] && std::isfinite(hi[j])))
            return fail(VEC_ERR_ARG, "vecchia_mlp_targets: range %d is not 0 < lo <= hi < inf", j);
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaError_t e = vg::launch_targets_from_theta(theta, var, nfields, lo, hi, targets,
                                                  reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_mlp_targets");
    return VEC_OK;
}

vec_status vecchia_mlp_theta(vec_handle h, int nfields, const float* pred, const double* var,
                             void* stream, double* theta) {
    if (!h || !pred || !var || !theta || nfields < 1)
        return fail(VEC_ERR_ARG, "vecchia_mlp_theta: bad argument");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaError_t e = vg::launch_theta_from_pred(pred, var, nfields, theta,
                                               reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_mlp_theta");
    return VEC_OK;
}

vec_status vecchia_mlp_forward(vec_handle h, const float* params, const float* norm,
                               const float* X, int nsamples, void* stream, float* out) {
    if (!h || !params || !norm || !X || !out) return fail(VEC_ERR_ARG, "vecchia_mlp_forward: NULL argument");
    if (nsamples < 1) return fail(VEC_ERR_ARG, "vecchia_mlp_forward: nsamples = %d", nsamples);
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaError_t e = vg::launch_mlp_fwdbwd(params, norm, X, nullptr, nullptr, nsamples, 0, out,
                                          nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_mlp_forward");
    return VEC_OK;
}

// Loss and gradient (grad != nullptr) or one Adam step.
static vec_status mlp_train(vec_handle h, float* params, float* adam_m, float* adam_v, int step,
                            float lr, const float* norm, const float* X, const float* T,
                            const int32_t* index, int nsamples, void* stream, float* grad,
                            float* loss) {
    if (nsamples < 1) return fail(VEC_ERR_ARG, "MLP: nsamples = %d", nsamples);
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int nblk = (nsamples + vg::mlp_block_samples() - 1) / vg::mlp_block_samples();
    cudaError_t e = grow(&h->mlp_gpart, &h->c_mlp_gpart, (size_t)nblk * vg::mlp_nparams());
    if (e == cudaSuccess) e = grow(&h->mlp_lpart, &h->c_mlp_lpart, (size_t)nblk);
    if (e != cudaSuccess) return cuda_fail(e, "MLP: allocating gradient partials");
    e = vg::launch_mlp_fwdbwd(params, norm, X, T, index, nsamples, 1, nullptr, h->mlp_gpart,
                              h->mlp_lpart, st);
    if (e == cudaSuccess)
        e = vg::launch_mlp_update(h->mlp_gpart, h->mlp_lpart, nblk, params, adam_m, adam_v, step, lr,
                                  0.9f, 0.999f, 1e-8f, grad, loss, st);
    if (e != cudaSuccess) return cuda_fail(e, "MLP: launching");
    return VEC_OK;
}

vec_status vecchia_mlp_grad(vec_handle h, const float* params, const float* norm, const float* X,
                            const float* T, const int32_t* index, int nsamples, void* stream,
                            float* grad, float* loss) {
    if (!h || !params || !norm || !X || !T || !grad || !loss)
        return fail(VEC_ERR_ARG, "vecchia_mlp_grad: NULL argument");
    return mlp_train(h, const_cast<float*>(params), nullptr, nullptr, 0, 0.0f, norm, X, T, index,
                     nsamples, stream, grad, loss);
}

vec_status vecchia_mlp_adam_step(vec_handle h, float* params, float* adam_m, float* adam_v,
                                 int step, float lr, const float* norm, const float* X,
                                 const float* T, const int32_t* index, int nsamples, void* stream,
                                 float* loss) {
    if (!h || !params || !adam_m || !adam_v || !norm || !X || !T)
        return fail(VEC_ERR_ARG, "vecchia_mlp_adam_step: NULL argument");
    if (step < 1 || !(lr > 0.0f)) return fail(VEC_ERR_ARG, "vecchia_mlp_adam_step: step %d, lr %g", step, lr);
    return mlp_train(h, params, adam_m, adam_v, step, lr, norm, X, T, index, nsamples, stream,
                     nullptr, loss);
}

vec_status vecchia_mlp_column_moments(vec_handle h, const float* X, int rows, int cols,
                                      void* stream, float* mean, float* sd) {
    if (!h || !X || !mean || !sd || rows < 1 || cols < 1)
        return fail(VEC_ERR_ARG, "vecchia_mlp_column_moments: bad argument");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaError_t e = vg::launch_col_moments(X, rows, cols, mean, sd, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_mlp_column_moments");
    return VEC_OK;
}

vec_status vecchia_fields_warm_start(vec_handle h, const float* params, const float* norm,
                                     int nfields, const double* locs, const double* X,
                                     const int32_t* NNarray, int64_t n, int d, int p, int m,
                                     const double* Y, const uint32_t* rand_pairs, int64_t npairs,
                                     const double* edges2, const double* default_start,
                                     vec_precision prec, void* stream, double* start,
                                     int* used_learned, float* features) {
    if (!h || !params || !norm || !default_start || !start || !used_learned)
        return fail(VEC_ERR_ARG, "vecchia_fields_warm_start: NULL argument");
    vec_status s = check_fields_args("vecchia_fields_warm_start", h, nfields, locs, X, NNarray, n, d,
                                     p, m, Y, VEC_MATERN_ISO, (int)prec);
    if (s != VEC_OK) return s;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int q = 4, nout = 1 + q + q * q + p, nbins = 32;
    cudaError_t e = grow(&h->ws_feat, &h->c_ws_feat, (size_t)nfields * nbins);
    if (e == cudaSuccess) e = grow(&h->ws_pred, &h->c_ws_pred, (size_t)nfields * 4);
    if (e == cudaSuccess) e = grow(&h->ws_theta0, &h->c_ws_theta0, (size_t)nfields * q);
    if (e == cudaSuccess) e = grow(&h->ws_out, &h->c_ws_out, (size_t)2 * nfields * nout);
    if (e == cudaSuccess) e = grow(&h->ws_st, &h->c_ws_st, (size_t)4 * nfields);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_fields_warm_start: allocating scratch");
    float* feat = features ? features : h->ws_feat;
    s = vecchia_fields_variogram(h, nfields, locs, NNarray, n, d, m, Y, rand_pairs, npairs, edges2,
                                 nbins, stream, feat, nullptr, nullptr);
    if (s != VEC_OK) return s;
    s = vecchia_mlp_forward(h, params, norm, feat, nfields, stream, h->ws_pred);
    if (s != VEC_OK) return s;
    e = vg::launch_theta_from_pred(h->ws_pred, h->vg_var, nfields, h->ws_theta0, st);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_fields_warm_start: predicted parameters");
    BatchPlan B;
    s = prepare_fields(h, h->bs, nfields, n, m, d, p, VEC_MATERN_ISO, (int)prec, st, &B);
    if (s != VEC_OK) return s;
    double* out0 = h->ws_out;
    double* out1 = h->ws_out + (size_t)nfields * nout;
    long long* st0 = h->ws_st;
    long long* st1 = h->ws_st + 2 * (size_t)nfields;
    s = enqueue_batch(h->bs, B, locs, Y, X, NNarray, d, p, h->ws_theta0, VEC_MATERN_ISO, (int)prec,
                      st, out0, st0, nullptr);
    if (s == VEC_OK)
        s = enqueue_batch(h->bs, B, locs, Y, X, NNarray, d, p, default_start, VEC_MATERN_ISO,
                          (int)prec, st, out1, st1, nullptr);
    if (s != VEC_OK) return s;
    e = vg::launch_choose_start(h->ws_theta0, default_start, out0, st0, out1, st1, nfields, q, nout,
                                start, used_learned, st);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_fields_warm_start: choosing starts");
    return VEC_OK;
}

vec_status vecchia_ordered_nn(vec_handle h, const double* locs, int64_t n, int d, int m,
                              void* stream, int32_t* NNarray) {
    if (!h || !locs || !NNarray) return fail(VEC_ERR_ARG, "vecchia_ordered_nn: NULL argument");
    if (n < 1 || n > (int64_t)INT_MAX || d < 1 || d > vg::DMAX || m < 0 || m > vg::KMAX - 1)
        return fail(VEC_ERR_ARG, "vecchia_ordered_nn: bad sizes (n %lld, d %d, m %d)", (long long)n, d, m);
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    // about two observations per cell of a G x G grid over the first two coordinates
    const double cells = std::max(1.0, (double)n / 2.0);
    const int G = d > 1 ? std::max(1, (int)std::sqrt(cells)) : (int)std::min<double>(cells, 1 << 30);
    cudaError_t e = grow(&h->nn_scratch, &h->c_nn_scratch, vg::ordered_nn_scratch_bytes(n, d, G));
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_ordered_nn: allocating scratch");
    e = vg::launch_ordered_nn(locs, n, d, m, G, h->nn_scratch, NNarray,
                              reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_ordered_nn: launching");
    return VEC_OK;
}

vec_status vecchia_maxmin_order(vec_handle h, const double* locs, int64_t n, int d, void* stream,
                                int64_t* order) {
    if (!h || !locs || !order) return fail(VEC_ERR_ARG, "vecchia_maxmin_order: NULL argument");
    if (n < 1 || n > (int64_t)INT_MAX || d < 1 || d > vg::DMAX)
        return fail(VEC_ERR_ARG, "vecchia_maxmin_order: bad sizes (n %lld, d %d)", (long long)n, d);
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int nblk = vg::maxmin_blocks(h->nsm);
    if (nblk < 1) return cuda_fail(cudaGetLastError(), "vecchia_maxmin_order: occupancy of the step kernel");
    cudaError_t e = grow(&h->mm_bbox, &h->c_mm_bbox, (size_t)nblk * 6);
    if (e == cudaSuccess) e = grow(&h->mm_err, &h->c_mm_err, (size_t)1);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_maxmin_order: allocating scratch");
    std::vector<double> part((size_t)nblk * 6);
    e = vg::launch_maxmin_bbox(locs, n, d, nblk, h->mm_bbox, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(part.data(), h->mm_bbox, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_maxmin_order: bounding box");
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) {
        lo[k] = part[k];
        hi[k] = part[3 + k];
        for (int b = 1; b < nblk; ++b) {
            lo[k] = std::min(lo[k], part[(size_t)b * 6 + k]);
            hi[k] = std::max(hi[k], part[(size_t)b * 6 + 3 + k]);
        }
        if (!std::isfinite(lo[k]) || !std::isfinite(hi[k]))
            return fail(VEC_ERR_ARG, "vecchia_maxmin_order: coordinate %d is not finite", k);
    }
    double hcell;
    int nc[3];
    long long ncell;
    vg::maxmin_grid(n, d, lo, hi, &hcell, nc, &ncell);
    const size_t need = vg::maxmin_scratch_bytes(n, nblk, ncell);
    e = grow(&h->mm_scratch, &h->c_mm_scratch, need);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_maxmin_order: allocating scratch");
    e = vg::launch_maxmin(locs, n, d, lo, nblk, hcell, nc, ncell, h->mm_scratch, h->c_mm_scratch,
                          reinterpret_cast<long long*>(order), h->mm_err, st);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, h->mm_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_maxmin_order: launching");
    if (err == 1) return fail(VEC_ERR_TIMEOUT, "vecchia_maxmin_order: a grid barrier waited too long");
    if (err != 0) return fail(VEC_ERR_CUDA, "vecchia_maxmin_order: the ordering did not complete (%d)", err);
    return VEC_OK;
}

vec_status vecchia_nearest(vec_handle h, const double* locs_ref, int64_t nref,
                           const double* locs_query, int64_t nquery, int d, int m, void* stream,
                           int32_t* NNarray) {
    if (!h || !locs_ref || !locs_query || !NNarray)
        return fail(VEC_ERR_ARG, "vecchia_nearest: NULL argument");
    if (nref < 1 || nref > (int64_t)INT_MAX || nquery < 1 || d < 1 || d > vg::DMAX || m < 1 ||
        m > vg::KMAX - 1)
        return fail(VEC_ERR_ARG, "vecchia_nearest: bad sizes (nref %lld, nquery %lld, d %d, m %d)",
                    (long long)nref, (long long)nquery, d, m);
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    const double cells = std::max(1.0, (double)nref / 2.0);
    const int G = d > 1 ? std::max(1, (int)std::sqrt(cells)) : (int)std::min<double>(cells, 1 << 30);
    cudaError_t e = grow(&h->nn_scratch, &h->c_nn_scratch, vg::ordered_nn_scratch_bytes(nref, d, G));
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_nearest: allocating scratch");
    e = vg::launch_ordered_nn(locs_ref, nref, d, m, G, h->nn_scratch, NNarray,
                              reinterpret_cast<cudaStream_t>(stream), locs_query, nquery);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_nearest: launching");
    return VEC_OK;
}

vec_status vecchia_predict(vec_handle h, const double* locs, const double* y, const double* X,
                           int64_t n, const double* beta, const double* locs_pred,
                           const double* X_pred, const int32_t* NN_pred, int64_t npred, int d,
                           int p, int m, const double* covparms, vec_covfun covfun, int latent,
                           void* stream, double* mean, double* var, int64_t* dev_status) {
    if (!h || !locs || !y || !X || !beta || !locs_pred || !X_pred || !covparms || !mean || !var ||
        !dev_status || (m > 0 && !NN_pred))
        return fail(VEC_ERR_ARG, "vecchia_predict: NULL argument");
    if (vecchia_nparms_d(covfun, d) < 0)
        return fail(VEC_ERR_ARG, "covariance function %d does not take d = %d", (int)covfun, d);
    if (n < 1 || npred < 1 ||
        p < 1 || p > vg::PMAX || m < 0 || m > vg::KMAX - 1 || npred > (int64_t)INT_MAX * 16)
        return fail(VEC_ERR_ARG, "vecchia_predict: bad sizes (n %lld, npred %lld, d %d, p %d, m %d)",
                    (long long)n, (long long)npred, d, p, m);
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = vg::launch_init_status(h->status, h->bad, st);
    if (e == cudaSuccess && covfun == VEC_MATERN_ISO) e = vg::launch_mtab_build(vg::COV_MATERN, covparms, h->mtab, nullptr, st);
    if (e == cudaSuccess)
        e = vg::launch_predict((int)covfun, locs, y, X, beta, n, locs_pred, X_pred, NN_pred, npred,
                               d, p, m, covparms, h->mtab, latent ? 1 : 0, h->nsm, mean, var,
                               h->status, h->bad, st);
    if (e == cudaSuccess)
        e = vg::launch_batch_status(h->status, h->bad, 1, reinterpret_cast<long long*>(dev_status), st);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_predict: launching");
    return VEC_OK;
}

vec_status vecchia_group_blocks(const int32_t* NNarray, int64_t n, int m, const int64_t* group_off,
                                int64_t ngroups, int64_t* block_off, int32_t* block_idx,
                                int32_t* nmemb, int* kmax) {
    if (!NNarray || !group_off || !block_off || !kmax || (block_idx && !nmemb) ||
        (!block_idx && nmemb))
        return fail(VEC_ERR_ARG, "vecchia_group_blocks: NULL argument");
    if (n < 1 || n > (int64_t)INT_MAX || m < 0 || ngroups < 1 || ngroups > n)
        return fail(VEC_ERR_ARG, "vecchia_group_blocks: bad sizes (n %lld, m %d, ngroups %lld)",
                    (long long)n, m, (long long)ngroups);
    if (group_off[0] != 0 || group_off[ngroups] != n)
        return fail(VEC_ERR_ARG, "vecchia_group_blocks: groups must cover 0 .. n-1");
    const int64_t W = (int64_t)m + 1;
    std::vector<int32_t> u;
    int64_t off = 0;
    int kx = 0;
    block_off[0] = 0;
    for (int64_t b = 0; b < ngroups; ++b) {
        const int64_t s = group_off[b], e = group_off[b + 1];
        if (e <= s) return fail(VEC_ERR_ARG, "vecchia_group_blocks: group %lld is empty", (long long)b);
        u.clear();
        for (int64_t i = s; i < e; ++i) {
            const int32_t* row = NNarray + i * W;
            if (row[0] != (int32_t)i)
                return fail(VEC_ERR_ARG, "vecchia_group_blocks: NNarray row %lld does not start with %lld",
                            (long long)i, (long long)i);
            bool pad = false;   // a valid row: neighbours, then only -1 padding
            for (int c = 1; c <= m; ++c) {
                const int32_t v = row[c];
                if (v < 0) {
                    if (v != -1)
                        return fail(VEC_ERR_ARG, "vecchia_group_blocks: NNarray row %lld lists %d",
                                    (long long)i, v);
                    pad = true;
                    continue;
                }
                if (pad || (int64_t)v >= i)
                    return fail(VEC_ERR_ARG, "vecchia_group_blocks: NNarray row %lld lists %d", (long long)i, v);
                if ((int64_t)v < s) u.push_back(v);   // neighbours from s on are members
            }
        }
        std::sort(u.begin(), u.end());
        u.erase(std::unique(u.begin(), u.end()), u.end());
        const int64_t len = (int64_t)u.size() + (e - s);
        if (block_idx) {
            for (size_t k = 0; k < u.size(); ++k) block_idx[off + (int64_t)k] = u[k];
            for (int64_t i = s; i < e; ++i) block_idx[off + (int64_t)u.size() + (i - s)] = (int32_t)i;
            nmemb[b] = (int32_t)(e - s);
        }
        off += len;
        block_off[b + 1] = off;
        if (len > kx) kx = (int)std::min<int64_t>(len, INT_MAX);
    }
    *kmax = kx;
    return VEC_OK;
}

vec_status vecchia_group_classes(const int64_t* block_off, int64_t ngroups, int nclass,
                                 int32_t* gorder, int64_t* class_off, int* class_kmax) {
    if (!block_off || !gorder || !class_off || !class_kmax)
        return fail(VEC_ERR_ARG, "vecchia_group_classes: NULL argument");
    if (ngroups < 1 || ngroups > (int64_t)INT_MAX || nclass < 1 || nclass > 16)
        return fail(VEC_ERR_ARG, "vecchia_group_classes: ngroups %lld, nclass %d", (long long)ngroups, nclass);
    // histogram of block sizes (1 .. KMAX; larger blocks share the top bin)
    const int V = vg::KMAX + 1;
    std::vector<int64_t> cnt(V + 1, 0);
    std::vector<int> len((size_t)ngroups);
    for (int64_t b = 0; b < ngroups; ++b) {
        const int64_t l = block_off[b + 1] - block_off[b];
        if (l < 1) return fail(VEC_ERR_ARG, "vecchia_group_classes: block %lld is empty", (long long)b);
        len[(size_t)b] = (int)std::min<int64_t>(l, V);
        cnt[(size_t)len[(size_t)b]]++;
    }
    // classes = ranges of sizes; cost of a class = its groups x (its largest size)^2 (the
    // slot size, so the inverse occupancy); minimise the total over at most nclass classes
    std::vector<int> sizes;
    for (int v = 1; v <= V; ++v)
        if (cnt[(size_t)v]) sizes.push_back(v);
    const int S = (int)sizes.size();
    std::vector<int64_t> pre(S + 1, 0);
    for (int k = 0; k < S; ++k) pre[k + 1] = pre[k] + cnt[(size_t)sizes[k]];
    const int C = std::min(nclass, S);
    const double INF = 1e300;
    std::vector<double> best((size_t)(C + 1) * (S + 1), INF);
    std::vector<int> from((size_t)(C + 1) * (S + 1), -1);
    auto at = [&](int c, int k) -> size_t { return (size_t)c * (S + 1) + k; };
    best[at(0, 0)] = 0.0;
    for (int c = 1; c <= C; ++c)
        for (int k = 1; k <= S; ++k)
            for (int j = c - 1; j < k; ++j) {
                if (best[at(c - 1, j)] >= INF) continue;
                const double kk = (double)sizes[k - 1];
                const double v = best[at(c - 1, j)] + (double)(pre[k] - pre[j]) * kk * kk;
                if (v < best[at(c, k)]) { best[at(c, k)] = v; from[at(c, k)] = j; }
            }
    int cb = 1;
    for (int c = 1; c <= C; ++c)
        if (best[at(c, S)] < best[at(cb, S)]) cb = c;
    std::vector<int> upper;   // largest size of each class, ascending
    for (int c = cb, k = S; c > 0; --c) {
        upper.push_back(sizes[k - 1]);
        k = from[at(c, k)];
    }
    std::reverse(upper.begin(), upper.end());
    // groups ordered by class; within a class the larger blocks first (slots take groups in
    // this order, so the last groups handed out are the quickest), then by index
    class_off[0] = 0;
    int64_t pos = 0;
    for (size_t c = 0; c < upper.size(); ++c) {
        const int lo = c == 0 ? 0 : upper[c - 1];
        for (int v = upper[c]; v > lo; --v)
            for (int64_t b = 0; b < ngroups; ++b)
                if (len[(size_t)b] == v) gorder[pos++] = (int32_t)b;
        class_off[c + 1] = pos;
        class_kmax[c] = upper[c];
    }
    for (int c = (int)upper.size(); c < nclass; ++c) {
        class_off[c + 1] = pos;
        class_kmax[c] = 0;
    }
    return VEC_OK;
}

vec_status vecchia_grouped_loglik_grad_info(vec_handle h, const double* locs, const double* y,
                                            const double* X, int64_t n, int d, int p, int64_t ngroups,
                                            const int64_t* block_off, const int32_t* block_idx,
                                            const int32_t* nmemb, const int32_t* gorder, int nclass,
                                            const int64_t* class_off, const int* class_kmax,
                                            const double* covparms, vec_covfun covfun,
                                            vec_precision prec, void* stream, double* out,
                                            int64_t* dev_status) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_grouped_loglik_grad_info: NULL handle");
    if (!locs || !y || !X || !block_off || !block_idx || !nmemb || !covparms || !out ||
        !dev_status || !class_off || !class_kmax)
        return fail(VEC_ERR_ARG, "vecchia_grouped_loglik_grad_info: a required pointer is NULL");
    if (n < 1 || n > (int64_t)INT_MAX || ngroups < 1 || ngroups > n)
        return fail(VEC_ERR_ARG, "n = %lld, ngroups = %lld out of range", (long long)n, (long long)ngroups);
    if (nclass < 1 || nclass > 16 || (!gorder && nclass != 1) || class_off[0] != 0 ||
        class_off[nclass] != ngroups)
        return fail(VEC_ERR_ARG, "bad group classes (nclass %d)", nclass);
    for (int c = 0; c < nclass; ++c) {
        if (class_off[c + 1] < class_off[c]) return fail(VEC_ERR_ARG, "class_off is not ascending");
        if (class_off[c + 1] > class_off[c] && (class_kmax[c] < 1 || class_kmax[c] > vg::KMAX))
            return fail(VEC_ERR_UNSUPPORTED, "largest block %d of class %d outside [1, %d]",
                        class_kmax[c], c, vg::KMAX);
    }
    if (covfun != VEC_EXP_ISO && covfun != VEC_MATERN_ISO && covfun != VEC_EXP_SPACETIME)
        return fail(VEC_ERR_UNSUPPORTED, "grouped conditioning: isotropic and space-time families only");
    const int q = vecchia_nparms_d(covfun, d);
    if (q < 0) return fail(VEC_ERR_ARG, "covariance function %d does not take d = %d", (int)covfun, d);
    if (p < 1 || p > vg::PMAX) return fail(VEC_ERR_ARG, "p = %d out of range [1, %d]", p, vg::PMAX);
    if (prec != VEC_FP64 && prec != VEC_MIXED) return fail(VEC_ERR_ARG, "unknown precision %d", (int)prec);
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    const int cov = (int)covfun;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // one launch per class, each sized by the class's largest block, taking its groups from
    // its own counter and writing one record per group; the launches run side by side on
    // the caller's stream and two side streams (a class's last groups then overlap the
    // next class's work); one profile step over all the records, in group order
    vg::PassPlan plans[16];
    int nstat = 0;
    for (int c = 0; c < nclass; ++c) {
        if (class_off[c + 1] == class_off[c]) continue;
        int pr = vg::plan_pass(cov, class_kmax[c] - 1, d, p, h->nsm, h->lanes, h->threads, &plans[c],
                               (int)prec, false, h->tab_mode, true, h->gchunk);
        if (pr == -1) return fail(VEC_ERR_UNSUPPORTED, "no kernel mapping fits blocks of %d", class_kmax[c]);
        if (pr != 0) return cuda_fail(cudaGetLastError(), "planning the grouped pass kernel");
        nstat = plans[c].nstat;
    }
    // group records, then their sums 64 at a time (the profile step adds those)
    const int rchunk = kRecChunk;
    const int nsum = (int)((ngroups + rchunk - 1) / rchunk);
    cudaError_t e = grow(&h->partials, &h->partials_cap, ((size_t)ngroups + nsum) * nstat);
    if (e == cudaSuccess) e = grow(&h->gcount, &h->c_gcount, (size_t)16);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        if (!h->gside[k]) e = cudaStreamCreateWithFlags(&h->gside[k], cudaStreamNonBlocking);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        if (!h->gev[k]) e = cudaEventCreateWithFlags(&h->gev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = vg::launch_init_status(h->status, h->bad, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->gcount, 0, sizeof(int) * 16, st);
    if (e == cudaSuccess && vg::uses_table(cov, prec))
        e = vg::launch_mtab_build(cov, covparms, h->mtab, prec ? h->mtabf : nullptr, st);
    if (e == cudaSuccess) e = cudaEventRecord(h->gev[0], st);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(h->gside[k], h->gev[0], 0);
    if (e != cudaSuccess) return cuda_fail(e, "grouped pass: set-up");
    // classes with the largest blocks first: their groups take longest
    int used = 0;
    for (int c = nclass - 1; c >= 0 && e == cudaSuccess; --c) {
        if (class_off[c + 1] == class_off[c]) continue;
        const vg::PassPlan& plan = plans[c];
        cudaStream_t sc = used % 3 == 0 ? st : h->gside[used % 3 - 1];
        ++used;
        vg::PassArgs a;
        a.locs = locs; a.y = y; a.X = X; a.NN = nullptr; a.covparms = covparms;
        a.mtab = h->mtab; a.mtabf = h->mtabf; a.partials = h->partials + (size_t)class_off[c] * nstat;
        a.status = h->status; a.bad = h->bad;
        a.n = n; a.d = d; a.p = p; a.m = class_kmax[c] - 1;
        a.nstat = plan.nstat; a.nv = plan.nv; a.slot_stride = plan.slot_stride;
        a.acc_per_lane = plan.acc_per_lane; a.tab_in_smem = plan.tab_smem;
        a.blk_off = reinterpret_cast<const long long*>(block_off); a.blk_idx = block_idx;
        a.nmemb = nmemb; a.gorder = gorder ? gorder + class_off[c] : nullptr;
        a.ngroups = class_off[c + 1] - class_off[c];
        a.ngroups_all = ngroups;
        a.gchunk = plan.gchunk;
        a.unit_counter = h->gcount + c;
        e = vg::launch_pass(cov, plan, a, sc);
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventRecord(h->gev[1 + k], h->gside[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->gev[1 + k], 0);
    }
    double* sums = h->partials + (size_t)ngroups * nstat;
    if (e == cudaSuccess)
        e = vg::launch_reduce_records(h->partials, (int)ngroups, nstat, rchunk, sums, st);
    if (e == cudaSuccess)
        e = vg::launch_profile(sums, nsum, nstat, p, q, n, covparms, h->status, h->bad, out,
                               reinterpret_cast<long long*>(dev_status), st);
    if (e != cudaSuccess) return cuda_fail(e, "launching the grouped pass");
    return VEC_OK;
}

vec_status vecchia_measure_peaks(vec_handle h, double* out) {
    if (!h || !out) return fail(VEC_ERR_ARG, "vecchia_measure_peaks: NULL argument");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaError_t e = vg::measure_peaks(h->nsm, h->stream, out);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_measure_peaks");
    return VEC_OK;
}

vec_status vecchia_covariance_pairs(vec_handle h, vec_covfun covfun, const double* covparms,
                                    int d, int64_t npairs, const double* la, const double* lb,
                                    const int32_t* same, double* C, double* dC, void* stream) {
    if (!h) return fail(VEC_ERR_ARG, "vecchia_covariance_pairs: NULL handle");
    if (vecchia_nparms_d(covfun, d) < 0)
        return fail(VEC_ERR_ARG, "covariance function %d does not take d = %d", (int)covfun, d);
    if (npairs < 0) return fail(VEC_ERR_ARG, "npairs < 0");
    if (npairs > 0 && (!covparms || !la || !lb || !same || !C || !dC))
        return fail(VEC_ERR_ARG, "a required pointer is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(VEC_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (covfun == VEC_MATERN_ISO) e = vg::launch_mtab_build(vg::COV_MATERN, covparms, h->mtab, nullptr, st);
    if (e == cudaSuccess)
        e = vg::launch_cov_pairs((int)covfun, covparms, h->mtab, d, npairs, la, lb, same, C, dC, st);
    if (e != cudaSuccess) return cuda_fail(e, "vecchia_covariance_pairs");
    return VEC_OK;
}

}  // extern "C"
