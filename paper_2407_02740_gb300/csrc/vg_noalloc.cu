// vg_noalloc.cu -- a pass entry point that allocates no device memory.
//
// Some callers cannot allocate device memory when they need a likelihood value: host
// programs whose GPU memory is owned entirely by another allocator (a framework's caching
// pool, an application that reserves the whole device at start-up) or held to a fixed
// budget, and latency-sensitive loops in which the implicit device synchronisation of an
// allocation is not acceptable.  For them, vecchia_loglik_grad_info_noalloc runs the same
// FP64 kernels as vecchia_loglik_grad_info but takes its scratch (per-block partial sums,
// the status word, the Matern table) from the file-scope device array below instead of a
// handle.  Every GPU that loads this library holds that array (1,102,592 bytes) until the
// process exits.
//
// Host code must not pass the array's name to a kernel: on the host the name is only a
// stand-in for the symbol.  Its device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, during the first call on the device;
// the same one-time set-up loads every kernel the entry point can launch.
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/vecchia.h"
#include "vg_internal.h"

namespace {

// Layout of the scratch array, in doubles; each region starts on a 256-byte boundary.
constexpr int kTabOff = 0;
constexpr int kTabLen = 6720;                     // reserved for the Matern table
static_assert(vg::MT_DOUBLES <= kTabLen, "the Matern table must fit its reserved region");
constexpr int kStatusOff = kTabOff + kTabLen;      // int status, then long long bad index
constexpr int kStatusLen = 32;
constexpr int kPartOff = kStatusOff + kStatusLen;
constexpr int kPartLen = 131072;                   // per-block partial records (1 MiB)
constexpr int kScratchDoubles = kPartOff + kPartLen;   // 137824 doubles = 1102592 bytes
static_assert(kScratchDoubles == 137824, "keep the size stated in include/vecchia.h in step");

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
int g_nsm[kMaxDevices] = {0};

// errors are reported through vecchia_last_error(), like every other entry point
vec_status nfail(vec_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
vec_status nfail(vec_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    vg::set_last_error(buf);
    return st;
}

}  // namespace

extern "C" {

VECCHIA_API vec_status vecchia_loglik_grad_info_noalloc(
    const double* locs, const double* y, const double* X, const int32_t* NNarray, int64_t n,
    int d, int p, int m, const double* covparms, vec_covfun covfun, vec_precision prec,
    void* stream, double* out, int64_t* dev_status) {
    if (!locs || !y || !X || !NNarray || !covparms || !out || !dev_status)
        return nfail(VEC_ERR_ARG, "a required pointer is NULL");
    if (n < 1 || n > (int64_t)INT_MAX) return nfail(VEC_ERR_ARG, "n = %lld out of range", (long long)n);
    if (vecchia_nparms_d(covfun, d) < 0)
        return nfail(VEC_ERR_ARG, "covariance function %d does not take d = %d", (int)covfun, d);
    if (p < 1 || p > vg::PMAX) return nfail(VEC_ERR_ARG, "p = %d out of range [1, %d]", p, vg::PMAX);
    if (m < 0 || m > vg::KMAX - 1)
        return nfail(VEC_ERR_UNSUPPORTED, "m = %d out of range [0, %d]", m, vg::KMAX - 1);
    if (prec != VEC_FP64) return nfail(VEC_ERR_UNSUPPORTED, "only VEC_FP64 is available here");

    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return nfail(VEC_ERR_CUDA, "no usable current device (%s)", cudaGetErrorString(e));
    double* base;
    int nsm;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            // one-time set-up on this device (the calling thread's current device)
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr)
                return nfail(VEC_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                             cudaGetErrorString(e));
            int sms = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess || sms < 1)
                return nfail(VEC_ERR_CUDA, "cannot query the SM count: %s", cudaGetErrorString(e));
            e = vg::load_pass_kernels_f64();
            if (e != cudaSuccess)
                return nfail(VEC_ERR_CUDA, "loading the pass kernels failed: %s", cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<double*>(ptr);
            g_nsm[dev] = sms;
        }
        base = g_scratch_ptr[dev];
        nsm = g_nsm[dev];
    }

    const int cov = (int)covfun;
    vg::PassPlan plan;
    int pr = vg::plan_pass(cov, m, d, p, nsm, 0, 0, &plan);
    if (pr == -1) return nfail(VEC_ERR_UNSUPPORTED, "no kernel mapping fits m = %d, p = %d", m, p);
    if (pr != 0) {
        // report the runtime's error and clear it, so that it does not surface in a later call
        e = cudaGetLastError();
        return nfail(VEC_ERR_CUDA, "planning the pass kernel failed: %s", cudaGetErrorString(e));
    }
    const long long need = (long long)plan.grid * plan.nstat;
    if (need > kPartLen)
        return nfail(VEC_ERR_UNSUPPORTED,
                     "the pass needs %lld doubles of partial sums (%d blocks x %d); the "
                     "allocation-free scratch holds %d", need, plan.grid, plan.nstat, kPartLen);

    double* tab = base + kTabOff;
    int* status = reinterpret_cast<int*>(base + kStatusOff);
    long long* bad = reinterpret_cast<long long*>(base + kStatusOff + 1);
    double* partials = base + kPartOff;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    // the status word and failing index restart from zero / "none" on every call; the
    // table and every partial record are rewritten in full by the kernels below
    e = vg::launch_init_status(status, bad, st);
    if (e == cudaSuccess && vg::uses_table(cov, 0)) e = vg::launch_mtab_build(cov, covparms, tab, nullptr, st);
    if (e != cudaSuccess) return nfail(VEC_ERR_CUDA, "launching the setup kernels: %s", cudaGetErrorString(e));
    vg::PassArgs a;
    a.locs = locs; a.y = y; a.X = X; a.NN = NNarray; a.covparms = covparms;
    a.mtab = tab; a.mtabf = nullptr; a.partials = partials; a.status = status; a.bad = bad;
    a.n = n; a.d = d; a.p = p; a.m = m;
    a.nstat = plan.nstat; a.nv = plan.nv; a.slot_stride = plan.slot_stride;
    a.acc_per_lane = plan.acc_per_lane; a.tab_in_smem = plan.tab_smem;
    e = vg::launch_pass(cov, plan, a, st);
    if (e != cudaSuccess) return nfail(VEC_ERR_CUDA, "launching the pass kernel: %s", cudaGetErrorString(e));
    e = vg::launch_profile(partials, plan.grid, plan.nstat, p, vg::nparms(cov, d), n, covparms, status, bad, out,
                           reinterpret_cast<long long*>(dev_status), st);
    if (e != cudaSuccess) return nfail(VEC_ERR_CUDA, "launching the profile kernel: %s", cudaGetErrorString(e));
    return VEC_OK;
}

}  // extern "C"
