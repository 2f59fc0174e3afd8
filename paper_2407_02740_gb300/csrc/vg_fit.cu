// vg_fit.cu -- Fisher scoring (Eq. 4) driven entirely on the device.
//
// One iteration = one likelihood pass at theta_trial (status reset, Matern table, the
// per-observation kernel, the profile kernel) followed by k_fit_step, a single-thread
// kernel that applies the fitting rules:
//   * work on log theta: g~ = theta (.) g, I~ = diag(theta) I diag(theta);
//   * Delta = I~^-1 g~; if I~ is not positive definite, add r * 1e-4 * max diag(I~) to its
//     diagonal, r = 1..8;
//   * stop (converged) when g~' Delta < tol, before stepping; stop after maxit accepted
//     steps;
//   * trial theta' = theta (.) exp(Delta / 2^h): accepted at the first h whose loglik is
//     finite and larger than the current one; a pass that fails (block not positive
//     definite, non-finite) counts as -inf; at most max_halvings halvings;
//   * the Matern smoothness is clamped to [0.05, 20].
// The iterations run inside a CUDA graph whose WHILE conditional node repeats the body
// until k_fit_step clears the condition, so the host is not involved between iterations.
// The batched form keeps one state per dataset: each iteration is one batched pass over
// the datasets still iterating, then k_fit_step_batch applies the same rules to each of
// them and keeps the loop going while any remains.
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "../../include/vecchia.h"
#include "vg_fit.h"

namespace vg {

__device__ static void fit_init_one(FitState* fs, const double* start, int q) {
    for (int j = 0; j < QMAX; ++j) {
        fs->theta_trial[j] = (j < q) ? start[j] : 0.0;
        fs->theta_cur[j] = fs->theta_trial[j];
        fs->delta[j] = 0.0;
        fs->grad[j] = 0.0;
    }
    for (int t = 0; t < QMAX * QMAX; ++t) fs->info[t] = 0.0;
    for (int t = 0; t < PMAX; ++t) fs->beta[t] = 0.0;
    fs->loglik = -INFINITY;
    fs->iters = 0;
    fs->halvings = 0;
    fs->evals = 0;
    fs->accepted_any = 0;
    fs->done = 0;
    fs->status = FIT_RUNNING;
    fs->pass_status = 0;
}

__global__ void k_fit_init(FitState* fs, const double* start, int q) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    fit_init_one(fs, start, q);
}

// Batch: dataset b starts from start[b*q..] or, when from_cur is set, from its own
// theta_cur (the second phase of a mixed-precision fit).  theta_b (nbatch x q) holds the
// parameters of the next batched pass and active[b] whether dataset b is still iterating.
__global__ void k_fit_init_batch(FitState* fs, const double* start, int from_cur, int q, int nbatch,
                                 double* theta_b, int* active) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbatch) return;
    double s0[QMAX];
    for (int j = 0; j < q; ++j) s0[j] = from_cur ? fs[b].theta_cur[j] : start[(size_t)b * q + j];
    fit_init_one(fs + b, s0, q);
    for (int j = 0; j < q; ++j) theta_b[(size_t)b * q + j] = fs[b].theta_trial[j];
    active[b] = 1;
}

// Solves A x = b for a small SPD matrix (n <= QMAX) by Cholesky; false if not PD.
__device__ static bool small_spd_solve(int n, const double* A, const double* b, double* x) {
    double L[QMAX * QMAX], z[QMAX];
    for (int i = 0; i < n * n; ++i) L[i] = A[i];
    for (int c = 0; c < n; ++c) {
        double v = L[c * n + c];
        for (int s = 0; s < c; ++s) v -= L[c * n + s] * L[c * n + s];
        if (!(v > 0.0) || !isfinite(v)) return false;
        L[c * n + c] = sqrt(v);
        for (int r = c + 1; r < n; ++r) {
            double u = L[r * n + c];
            for (int s = 0; s < c; ++s) u -= L[r * n + s] * L[c * n + s];
            L[r * n + c] = u / L[c * n + c];
        }
    }
    for (int a = 0; a < n; ++a) {
        double u = b[a];
        for (int s = 0; s < a; ++s) u -= L[a * n + s] * z[s];
        z[a] = u / L[a * n + a];
    }
    for (int a = n - 1; a >= 0; --a) {
        double u = z[a];
        for (int r = a + 1; r < n; ++r) u -= L[r * n + a] * x[r];
        x[a] = u / L[a * n + a];
    }
    return true;
}

__device__ static void set_trial(FitState* fs, int q, int cov, double scale) {
    for (int j = 0; j < q; ++j) fs->theta_trial[j] = fs->theta_cur[j] * exp(fs->delta[j] * scale);
    if (cov == COV_MATERN) fs->theta_trial[2] = fmin(20.0, fmax(0.05, fs->theta_trial[2]));
}

// One scoring decision for one dataset.  out = [loglik, grad(q), info(q*q), betahat(p)] of
// the pass at theta_trial; dev_status = [code, first failing observation].  On return
// fs->done tells whether the fit has ended; otherwise theta_trial holds the next point.
__device__ static void fit_step_one(FitState* fs, const double* out, const long long* dev_status,
                                    int q, int p, int cov, double tol, int maxit,
                                    int max_halvings) {
    const int max_evals = (maxit + 2) * (max_halvings + 2);
    if (fs->done || fs->evals >= max_evals) {
        if (!fs->done) { fs->done = 1; fs->status = FIT_MAXIT; }
        return;
    }
    fs->evals += 1;
    const long long st = dev_status[0];
    const double ll = out[0];
    const bool ok = (st == 0) && isfinite(ll);
    fs->pass_status = (int)st;
    bool accept;
    if (!fs->accepted_any) {
        if (!ok) {
            fs->done = 1;
            fs->status = FIT_START_FAILED;
            return;
        }
        accept = true;
    } else {
        accept = ok && ll > fs->loglik;
    }
    if (!accept) {
        fs->halvings += 1;
        if (fs->halvings > max_halvings) {
            fs->done = 1;
            fs->status = FIT_NO_ASCENT;
            return;
        }
        set_trial(fs, q, cov, ldexp(1.0, -fs->halvings));
        return;
    }
    // accept the trial point
    if (fs->accepted_any) fs->iters += 1;
    fs->accepted_any = 1;
    fs->halvings = 0;
    fs->loglik = ll;
    for (int j = 0; j < q; ++j) {
        fs->theta_cur[j] = fs->theta_trial[j];
        fs->grad[j] = out[1 + j];
    }
    for (int t = 0; t < q * q; ++t) fs->info[t] = out[1 + q + t];
    for (int a = 0; a < p; ++a) fs->beta[a] = out[1 + q + q * q + a];
    // Fisher step on the log scale
    double gt[QMAX], It[QMAX * QMAX], A[QMAX * QMAX], dl[QMAX];
    double maxd = 0.0;
    for (int j = 0; j < q; ++j) gt[j] = fs->theta_cur[j] * fs->grad[j];
    for (int j = 0; j < q; ++j)
        for (int l = 0; l < q; ++l) It[j * q + l] = fs->theta_cur[j] * fs->info[j * q + l] * fs->theta_cur[l];
    for (int j = 0; j < q; ++j) maxd = fmax(maxd, It[j * q + j]);
    bool solved = false;
    for (int r = 0; r < 9 && !solved; ++r) {
        for (int t = 0; t < q * q; ++t) A[t] = It[t];
        for (int j = 0; j < q; ++j) A[j * q + j] += r * 1e-4 * maxd;
        solved = small_spd_solve(q, A, gt, dl);
    }
    if (!solved) {
        fs->done = 1;
        fs->status = FIT_NO_ASCENT;
        return;
    }
    double dec = 0.0;
    for (int j = 0; j < q; ++j) { fs->delta[j] = dl[j]; dec += gt[j] * dl[j]; }
    if (dec < tol) {
        fs->done = 1;
        fs->status = FIT_CONVERGED;
    } else if (fs->iters >= maxit) {
        fs->done = 1;
        fs->status = FIT_MAXIT;
    } else {
        set_trial(fs, q, cov, 1.0);
    }
}

__global__ void k_fit_step(FitState* fs, const double* out, const long long* dev_status, int q,
                           int p, int cov, double tol, int maxit, int max_halvings,
                           cudaGraphConditionalHandle cond, int use_cond) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    fit_step_one(fs, out, dev_status, q, p, cov, tol, maxit, max_halvings);
    if (use_cond) cudaGraphSetConditional(cond, fs->done ? 0 : 1);
}

// Batch: one block; thread t steps datasets t, t + blockDim.x, ...  Datasets that have
// ended are left alone.  The loop condition (and *any_active) is 1 while any dataset
// still iterates.
__global__ void k_fit_step_batch(FitState* fs, const double* out, const long long* dev_status,
                                 int q, int p, int cov, double tol, int maxit, int max_halvings,
                                 int nbatch, double* theta_b, int* active, int* any_active,
                                 cudaGraphConditionalHandle cond, int use_cond) {
    const int nout = 1 + q + q * q + p;
    int mine = 0;
    for (int b = threadIdx.x; b < nbatch; b += blockDim.x) {
        if (!active[b]) continue;
        FitState* f = fs + b;
        fit_step_one(f, out + (size_t)b * nout, dev_status + 2 * (size_t)b, q, p, cov, tol, maxit,
                     max_halvings);
        if (f->done) {
            active[b] = 0;
        } else {
            for (int j = 0; j < q; ++j) theta_b[(size_t)b * q + j] = f->theta_trial[j];
            mine = 1;
        }
    }
    const int any = __syncthreads_or(mine);
    if (threadIdx.x == 0) {
        *any_active = any;
        if (use_cond) cudaGraphSetConditional(cond, any ? 1 : 0);
    }
}

// Batch results: theta_out (nbatch x q) and out (nbatch x (1+q+q*q+p)) = [loglik, grad,
// info, betahat] at each dataset's last accepted parameters.
__global__ void k_fit_export_batch(const FitState* fs, int nbatch, int q, int p, double* theta_out,
                                   double* out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbatch) return;
    const FitState& f = fs[b];
    const int nout = 1 + q + q * q + p;
    double* o = out + (size_t)b * nout;
    for (int j = 0; j < q; ++j) theta_out[(size_t)b * q + j] = f.theta_cur[j];
    o[0] = f.loglik;
    for (int j = 0; j < q; ++j) o[1 + j] = f.grad[j];
    for (int t = 0; t < q * q; ++t) o[1 + q + t] = f.info[t];
    for (int a = 0; a < p; ++a) o[1 + q + q * q + a] = f.beta[a];
}

cudaError_t launch_fit_export_batch(const FitState* fs, int nbatch, int q, int p, double* theta_out,
                                    double* out, cudaStream_t st) {
    k_fit_export_batch<<<(nbatch + 127) / 128, 128, 0, st>>>(fs, nbatch, q, p, theta_out, out);
    return cudaGetLastError();
}

cudaError_t launch_fit_init(FitState* fs, const double* start, int q, cudaStream_t st) {
    k_fit_init<<<1, 1, 0, st>>>(fs, start, q);
    return cudaGetLastError();
}

cudaError_t launch_fit_step(FitState* fs, const double* out, const long long* dev_status, int q,
                            int p, int cov, double tol, int maxit, int max_halvings,
                            cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st) {
    k_fit_step<<<1, 1, 0, st>>>(fs, out, dev_status, q, p, cov, tol, maxit, max_halvings, cond,
                                use_cond);
    return cudaGetLastError();
}

cudaError_t launch_fit_init_batch(FitState* fs, const double* start, int from_cur, int q,
                                  int nbatch, double* theta_b, int* active, cudaStream_t st) {
    k_fit_init_batch<<<(nbatch + 127) / 128, 128, 0, st>>>(fs, start, from_cur, q, nbatch, theta_b,
                                                         active);
    return cudaGetLastError();
}

cudaError_t launch_fit_step_batch(FitState* fs, const double* out, const long long* dev_status,
                                  int q, int p, int cov, double tol, int maxit, int max_halvings,
                                  int nbatch, double* theta_b, int* active, int* any_active,
                                  cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st) {
    k_fit_step_batch<<<1, 256, 0, st>>>(fs, out, dev_status, q, p, cov, tol, maxit, max_halvings,
                                        nbatch, theta_b, active, any_active, cond, use_cond);
    return cudaGetLastError();
}

}  // namespace vg
