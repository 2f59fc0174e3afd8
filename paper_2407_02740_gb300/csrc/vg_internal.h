// vg_internal.h -- host-side interface between the C ABI layer and the kernel launchers.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "vg_common.cuh"

namespace vg {


struct PassPlan {
    int L;             // lanes per observation
    int threads;       // threads per block
    int grid;          // persistent grid (blocks)
    size_t smem;       // dynamic shared memory per block
    int tab_smem;      // Matern table staged in shared memory
    int nstat;         // doubles per partial record
    int nv;            // per-observation value count
    int slot_stride;   // bytes per shared-memory slot
    int acc_per_lane;  // accumulator doubles per thread
    int prec;          // 0 = FP64 kernel, 1 = mixed (FP32 block) kernel
    int batched;       // plan made for the batched kernel
    int grouped;       // plan made for the grouped-conditioning kernel
    int gchunk;        // grouped: members whose terms are formed together (slot sized for it)
};

// Chooses the lanes-per-observation mapping that fits shared memory (or the forced one).
// Returns 0 on success, -1 if no mapping fits, -2 on a CUDA error.
// force_tab: -1 = Matern table in shared memory when it fits, 1 = shared memory only,
// 0 = global memory (read through L1).  Returns 0, -1 (no mapping fits) or -2 (CUDA error).
int plan_pass(int cov, int m, int d, int p, int nsm, int force_L, int force_threads,
              PassPlan* plan, int prec = 0, bool batched = false, int force_tab = -1,
              bool grouped = false, int force_gchunk = 0);
size_t pass_smem_bytes(int cov, int m, int d, int p, int L, int threads, bool tab_smem,
                       int prec = 0, bool grouped = false, int gchunk = 1);
const void* pass_kernel_f64(int cov, int L);
const void* pass_kernel_f32(int cov, int L);
const void* pass_batch_kernel_f64(int cov, int L);
const void* pass_batch_kernel_f32(int cov, int L);
const void* pass_group_kernel(int cov, int L, int prec);
cudaError_t launch_pass_batch(int cov, const PassPlan& plan, const BatchArgs& args, cudaStream_t st);
// Per-pass coefficient tables (the Matern family, or the exponential families' closed
// forms for any other cov); the FP32 copy only for the Matern family.
cudaError_t launch_mtab_build_batch(int cov, const double* covparms_b, int nbatch, int q,
                                    double* tabs, float* tabsf, const int* active, cudaStream_t st);
constexpr int VG_MAX_BINS = 64;  // largest number of semivariogram bins
size_t vario_smem_bytes(int nbins);
cudaError_t launch_field_moments(const double* Y, int n, int nfields, double* mean, double* var,
                                 cudaStream_t st);
cudaError_t launch_vario(const double* locs, int d, const int32_t* NN, int n, int m, const double* Y,
                         int nfields, const uint32_t* R, long long P, const double* edges2,
                         int nbins, int slices, double* psum, long long* pcnt, cudaStream_t st);
cudaError_t launch_vario_finish(const double* psum, const long long* pcnt, int slices, int nbins,
                                const double* var, int nfields, float* feat, double* bin_sum,
                                long long* bin_count, cudaStream_t st);
size_t mlp_smem_bytes();
int mlp_nparams();
int mlp_block_samples();
cudaError_t launch_mlp_fwdbwd(const float* P, const float* norm, const float* X, const float* T,
                              const int* index, int B, int mode, float* out, float* gpart,
                              float* lpart, cudaStream_t st);
cudaError_t launch_mlp_update(const float* gpart, const float* lpart, int nblk, float* P, float* m,
                              float* v, int step, float lr, float beta1, float beta2, float eps,
                              float* grad, float* loss, cudaStream_t st);
cudaError_t launch_col_moments(const float* X, int rows, int cols, float* mean, float* sd,
                               cudaStream_t st);
cudaError_t launch_theta_from_pred(const float* pred, const double* var, int nfields, double* theta,
                                   cudaStream_t st);
cudaError_t launch_targets_from_theta(const double* theta, const double* var, int nfields,
                                      const double* lo, const double* hi, float* T, cudaStream_t st);
cudaError_t launch_choose_start(const double* theta0, const double* dflt, const double* out0,
                                const long long* st0, const double* out1, const long long* st1,
                                int nfields, int q, int nout, double* start, int* used,
                                cudaStream_t st);
// qx == nullptr: ordered search (candidates j < i, rows [i, neighbours]); else the m
// nearest of the nq query locations qx among all n reference locations (rows of m).
cudaError_t launch_ordered_nn(const double* x, long long n, int d, int m, int G, void* scratch,
                              int32_t* NN, cudaStream_t st, const double* qx = nullptr,
                              long long nq = 0);
size_t ordered_nn_scratch_bytes(long long n, int d, int G);
// maxmin ordering (vg_maxmin.cu): co-resident blocks of its step kernel, the bounding box
// partials (nblk x 6), the grid over the box, the scratch size, and the launch (the error
// flag of the step kernel is copied to err_out, device memory)
int maxmin_blocks(int nsm);
cudaError_t launch_maxmin_bbox(const double* x, long long n, int d, int nblk, double* part,
                               cudaStream_t st);
void maxmin_grid(long long n, int d, const double* lo, const double* hi, double* h, int* nc,
                 long long* ncell);
size_t maxmin_scratch_bytes(long long n, int nblocks, long long ncell);
cudaError_t launch_maxmin(const double* x, long long n, int d, const double* lo, int nblk,
                          double h, const int* nc, long long ncell, void* scratch,
                          size_t scratch_bytes, long long* order, int* err_out, cudaStream_t st);
cudaError_t launch_predict(int cov, const double* locs, const double* y, const double* X,
                           const double* beta, long long n, const double* qlocs,
                           const double* qX, const int32_t* NN, long long nq, int d, int p,
                           int m, const double* covparms, const double* tab, int latent,
                           int nsm, double* mean, double* var, int* status, long long* bad,
                           cudaStream_t st);
cudaError_t launch_sim_recur(const double* factor, const int32_t* NN, int n, int m, int nfields,
                            const double* z, double* y, cudaStream_t st);
cudaError_t launch_batch_status(const int* status_b, const long long* bad_b, int nbatch,
                               long long* dev_status, cudaStream_t st);
cudaError_t launch_init_batch(int* status_b, long long* bad_b, int nbatch, int* tile_counter,
                              int ncounter, cudaStream_t st);
cudaError_t launch_profile_batch(const double* partials, const int* tile_off, int nbatch, int nstat,
                                 int p, int q, const DatasetDesc* desc, const double* covparms_b,
                                 const int* status_b, const long long* bad_b, double* out,
                                 long long* dev_status, cudaStream_t st);

cudaError_t launch_pass(int cov, const PassPlan& plan, const PassArgs& args, cudaStream_t st);
cudaError_t launch_init_status(int* status, long long* bad, cudaStream_t st);
cudaError_t launch_mtab_build(int cov, const double* covparms, double* tab, float* tabf,
                              cudaStream_t st);
// Loads (under lazy module loading) every kernel the single-dataset FP64 pass can launch.
cudaError_t load_pass_kernels_f64();
// out[k] = the sum of records k chunk .. (k+1) chunk - 1 of in, in order (nrec records of
// nstat doubles; ceil(nrec / chunk) outputs)
cudaError_t launch_reduce_records(const double* in, int nrec, int nstat, int chunk, double* out,
                                  cudaStream_t st);
cudaError_t launch_profile(const double* partials, int nblk, int nstat, int p, int q,
                           long long n, const double* covparms, const int* status,
                           const long long* bad, double* out, long long* dev_status,
                           cudaStream_t st);
// Measured throughputs (see vg_peaks.cu): out = {FP64 GFLOP/s, FP32 GFLOP/s, exponential
// covariance pairs/s, Matern covariance pairs/s}.  Synchronous on st.
cudaError_t measure_peaks(int nsm, cudaStream_t st, double* out);
cudaError_t launch_cov_pairs(int cov, const double* covparms, const double* tab, int d,
                             long long npairs, const double* la, const double* lb,
                             const int32_t* same, double* C, double* dC, cudaStream_t st);
int mtab_doubles();
int mtab_floats();

// Records the thread-local message returned by vecchia_last_error().
void set_last_error(const char* msg);

}  // namespace vg
