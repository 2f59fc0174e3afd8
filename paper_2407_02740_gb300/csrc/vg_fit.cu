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
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "../../include/vecchia.h"
#include "vg_fit.h"

namespace vg {

__global__ void k_fit_init(FitState* fs, const double* start, int q) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int j = 0; j < 4; ++j) {
        fs->theta_trial[j] = (j < q) ? start[j] : 0.0;
        fs->theta_cur[j] = fs->theta_trial[j];
        fs->delta[j] = 0.0;
        fs->grad[j] = 0.0;
    }
    for (int t = 0; t < 16; ++t) fs->info[t] = 0.0;
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

// Solves A x = b for a small SPD matrix (n <= 4) by Cholesky; false if not PD.
__device__ static bool small_spd_solve(int n, const double* A, const double* b, double* x) {
    double L[16], z[4];
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

// out = [loglik, grad(q), info(q*q), betahat(p)] of the pass at theta_trial;
// dev_status = [code, first failing observation].
__global__ void k_fit_step(FitState* fs, const double* out, const long long* dev_status, int q,
                           int p, int cov, double tol, int maxit, int max_halvings,
                           cudaGraphConditionalHandle cond, int use_cond) {
    const int max_evals = (maxit + 2) * (max_halvings + 2);
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (fs->done || fs->evals >= max_evals) {
        if (!fs->done) { fs->done = 1; fs->status = FIT_MAXIT; }
        if (use_cond) cudaGraphSetConditional(cond, 0);
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
            if (use_cond) cudaGraphSetConditional(cond, 0);
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
            if (use_cond) cudaGraphSetConditional(cond, 0);
            return;
        }
        set_trial(fs, q, cov, ldexp(1.0, -fs->halvings));
        if (use_cond) cudaGraphSetConditional(cond, 1);
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
    double gt[4], It[16], A[16], dl[4];
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
        if (use_cond) cudaGraphSetConditional(cond, 0);
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
    if (use_cond) cudaGraphSetConditional(cond, fs->done ? 0 : 1);
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

}  // namespace vg
