// vg_fit.h -- device state and launchers of the Fisher-scoring driver (vg_fit.cu).
#pragma once
#include <cuda_runtime.h>

#include "vg_common.cuh"

namespace vg {

enum : int { FIT_CONVERGED = 0, FIT_MAXIT = 1, FIT_NO_ASCENT = 2, FIT_START_FAILED = 3,
             FIT_RUNNING = -1 };

// Lives in device memory owned by the handle; copied back to the host after a fit.
struct FitState {
    double theta_cur[QMAX];     // accepted parameters
    double theta_trial[QMAX];   // parameters of the next pass
    double delta[QMAX];         // current log-scale step
    double loglik;              // at theta_cur
    double grad[QMAX];
    double info[QMAX * QMAX];
    double beta[PMAX];
    int iters;               // accepted Fisher steps
    int halvings;            // halvings of the current step
    int evals;               // passes run
    int accepted_any;
    int done;
    int status;              // FIT_*
    int pass_status;         // status of the last pass
    int pad;
};

cudaError_t launch_fit_init(FitState* fs, const double* start, int q, cudaStream_t st);
cudaError_t launch_fit_step(FitState* fs, const double* out, const long long* dev_status, int q,
                            int p, int cov, double tol, int maxit, int max_halvings,
                            cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st);
cudaError_t launch_fit_init_batch(FitState* fs, const double* start, int from_cur, int q,
                                  int nbatch, double* theta_b, int* active, cudaStream_t st);
cudaError_t launch_fit_step_batch(FitState* fs, const double* out, const long long* dev_status,
                                  int q, int p, int cov, double tol, int maxit, int max_halvings,
                                  int nbatch, double* theta_b, int* active, int* any_active,
                                  cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st);
cudaError_t launch_fit_export_batch(const FitState* fs, int nbatch, int q, int p, double* theta_out,
                                    double* out, cudaStream_t st);

}  // namespace vg
