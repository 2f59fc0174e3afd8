/*
 * vecchia_oracle.c -- plain, slow, FP64 CPU oracle for the Vecchia likelihood pass.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the CUDA
 * path is checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or constant
 * with the CUDA library (paper_2407_02740_gb300/), and the CUDA library never loads it.
 *
 * What it computes (James & Guinness, "Implementation and Analysis of GPU Algorithms
 * for Vecchia Approximation"):
 *   - Sec. 2.1, Eq. 3: the Vecchia density p(y) ~ prod_i p(y_i | y_{s_i}), where s_i is
 *     the list of at most m earlier-ordered nearest neighbours in NNarray row i.
 *   - Algorithm 1: per observation, gather the neighbour block, build the covariance
 *     matrix, Cholesky-factor it, forward-solve y and X, accumulate logdet, ySy, XSX,
 *     ySX and the derivative sums dlogdet, dySy, dXSX, dySX and ainfo.  The paper elides
 *     the derivative half ("remaining operations"); it is written out here from Gaussian
 *     conditioning and differentiation of the Cholesky factor (see derivation below).
 *   - Sec. 3 (the "separate function" after Algorithm 1): profile beta out and form the
 *     loglikelihood, gradient and Fisher information.
 *   - Eq. 4: Fisher scoring, run on log-parameters with step halving.
 *   - Sec. 4.3, Eq. 5-6: the exponential covariance with a relative nugget
 *     sigma^2 tau^2 -- isotropic, and with one range per coordinate (the form fitted to
 *     the Elevators attributes, q = d + 2) -- plus the isotropic Matern family and a
 *     space-time exponential.
 *
 * Derivation of the elided terms (per observation, block of size K = k+1 with the
 * observation itself last, L = chol(Sigma_block)):
 *   With M_j = L^-1 dSigma_j L^-T and Phi(M) = lower triangle of M with half diagonal,
 *   dL = L Phi(M_j) and d(L^-1) = -Phi(M_j) L^-1.  Let b = last row of L^-1 and
 *   m_j = L^-1 dSigma_j b^T (= last column of M_j).  Then
 *     d log L[K-1][K-1]^2            = m_j[K-1]
 *     d (last row of L^-1) . v       = -(m_j . hat(L^-1 v)),  hat() halves the last entry
 *   and the Fisher information of the conditional density is I(block) - I(neighbours)
 *     = 1/2 tr(M_j M_l) - 1/2 tr(leading k x k block)  = m_j . m_l - 1/2 m_j[K-1] m_l[K-1].
 *
 * Numerics: every quantity is FP64.  Sums over observations use Neumaier compensated
 * summation in fixed chunks of ORC_CHUNK observations, so the result does not depend on
 * the number of OpenMP threads.
 *
 * Matern function: M_nu(x) = 2^(1-nu)/Gamma(nu) x^nu K_nu(x) is evaluated through the
 * Gamma-mixture identity  M_nu(x) = (1/Gamma(nu)) int_0^inf u^(nu-1) exp(-u - x^2/(4u)) du
 * (obtained from the integral K_nu(x) = 1/2 (x/2)^nu int_0^inf exp(-t - x^2/(4t)) t^(-nu-1) dt
 * with t = x^2/(4u)).  Its nu- and x-derivatives are integrals of the same kind, taken by
 * the trapezoid rule in s = log u; the integrand is analytic in |Im s| < pi/2, so the
 * rule converges geometrically (error ~ exp(-2 pi d / h)).  Gamma(nu) is libm's tgamma;
 * the digamma function is computed here by upward recurrence and its asymptotic series.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXP_ISO 0       /* theta = (sigma2, rho, tau2)          Eq. 6, isotropic      */
#define ORC_MATERN_ISO 1    /* theta = (sigma2, rho, nu, tau2)      Matern, x = r/rho     */
#define ORC_EXP_SPACETIME 2 /* theta = (sigma2, rho_s, rho_t, tau2) d = 3: (lon, lat, t)  */
#define ORC_EXP_ANISO 3     /* theta = (sigma2, rho_1..rho_d, tau2), Eq. 6 with one range
                               per coordinate; 1 <= d <= ORC_DMAX_ANISO                   */
#define ORC_DMAX_ANISO 20
#define ORC_QMAX (ORC_DMAX_ANISO + 2)

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_NOT_PD 2
#define ORC_ERR_NONFINITE 3
#define ORC_ERR_NOMEM 4

#define ORC_CHUNK 256

/* Number of covariance parameters of a family in d dimensions (-1: unknown family, or a
 * dimension the family does not take). */
int orc_nparms_d(int covfun, int d)
{
    switch (covfun) {
    case ORC_EXP_ISO: return 3;
    case ORC_MATERN_ISO: return 4;
    case ORC_EXP_SPACETIME: return 4;
    case ORC_EXP_ANISO: return (d >= 1 && d <= ORC_DMAX_ANISO) ? d + 2 : -1;
    default: return -1;
    }
}

/* The same for the families whose parameter count does not depend on d. */
int orc_nparms(int covfun) { return covfun == ORC_EXP_ANISO ? -1 : orc_nparms_d(covfun, 1); }

/* Number of doubles in one Algorithm 1 record:
 * logdet, ySy, XSX[p][p], ySX[p], dlogdet[q], dySy[q], dXSX[q][p][p], dySX[q][p], ainfo[q][q] */
int orc_stats_len(int p, int q) { return 2 + p * p + p + q * (2 + p * p + p) + q * q; }

/* ------------------------------------------------------------------------------------ */
/* Special functions                                                                    */
/* ------------------------------------------------------------------------------------ */

/* digamma(x), x > 0: psi(x) = psi(x + n) - sum_{k<n} 1/(x+k), then the asymptotic series
 * psi(z) ~ ln z - 1/(2z) - sum_k B_2k / (2k z^2k) for z >= 10. */
double orc_digamma(double x)
{
    double acc = 0.0;
    while (x < 10.0) {
        acc -= 1.0 / x;
        x += 1.0;
    }
    double z2 = 1.0 / (x * x);
    /* B2/2 = 1/12, B4/4 = -1/120, B6/6 = 1/252, B8/8 = -1/240, B10/10 = 1/132,
       B12/12 = -691/32760, B14/14 = 1/12 */
    double series = z2 * (1.0 / 12 - z2 * (1.0 / 120 - z2 * (1.0 / 252 - z2 * (1.0 / 240
                    - z2 * (1.0 / 132 - z2 * (691.0 / 32760 - z2 * (1.0 / 12)))))));
    return acc + log(x) - 0.5 / x - series;
}

/* G(a, c, w) = int_{-inf}^{inf} exp(a s - e^s - c e^{-s}) w(s) ds with w(s) = 1 (wpow=0)
 * or w(s) = s (wpow=1), c > 0.  Trapezoid rule, step h, anchored at the peak of the
 * (concave) exponent and truncated where the exponent is 60 below its peak. */
static double gmix_integral(double a, double c, int wpow)
{
    const double h = 0.1;
    /* peak: a - e^s + c e^{-s} = 0  ->  e^s = (a + sqrt(a^2 + 4c)) / 2 */
    double disc = sqrt(a * a + 4.0 * c);
    double es = (a >= 0.0) ? 0.5 * (a + disc) : (2.0 * c) / (disc - a);
    double sp = log(es);
    double phip = a * sp - es - c / es;
    double sum = 0.0;
    for (int dir = 0; dir < 2; dir++) {
        for (long k = (dir == 0 ? 0 : 1);; k++) {
            double s = sp + (dir == 0 ? (double)k : -(double)k) * h;
            double phi = a * s - exp(s) - c * exp(-s);
            double f = exp(phi);
            sum += (wpow ? s * f : f);
            if (phi < phip - 60.0 && k > 4) break;
            if (k > 200000) break; /* never reached for c > 0; keeps the loop finite */
        }
    }
    return h * sum;
}

/* Matern correlation and derivatives for x > 0:
 *   M      = M_nu(x)
 *   xdMdx  = x dM/dx          (so rho dM/drho = -x dM/dx)
 *   dMdnu  = dM/dnu                                                              */
static void matern_eval(double nu, double x, double lg_nu, double psi_nu,
                        double* M, double* xdMdx, double* dMdnu)
{
    double c = 0.25 * x * x;
    double inv_gamma = exp(-lg_nu);
    double J0 = gmix_integral(nu, c, 0);       /* int u^(nu-1) e^{-u - c/u} du          */
    double J1 = gmix_integral(nu, c, 1);       /* int u^(nu-1) log u e^{-u - c/u} du    */
    double J2 = gmix_integral(nu - 1.0, c, 0); /* int u^(nu-2) e^{-u - c/u} du          */
    *M = J0 * inv_gamma;
    /* d/dx e^{-x^2/(4u)} = -(x/(2u)) e^{...}  ->  x dM/dx = -(x^2/2) J2 / Gamma(nu) */
    *xdMdx = -2.0 * c * J2 * inv_gamma;
    /* d/dnu [u^(nu-1)/Gamma(nu)] = (log u - psi(nu)) u^(nu-1)/Gamma(nu) */
    *dMdnu = J1 * inv_gamma - psi_nu * (*M);
}

/* Covariance between two locations and its derivatives with respect to theta.
 * same = 1 when the two entries are the same observation (diagonal: nugget added).
 * dC must hold nparms(covfun) values. */
typedef struct {
    int covfun, d;
    int q;
    double th[ORC_QMAX];
    double lg_nu, psi_nu; /* Matern only: log Gamma(nu), digamma(nu) */
} orc_cov;

static int orc_cov_init(orc_cov* cv, int covfun, int d, const double* theta)
{
    int q = orc_nparms_d(covfun, d);
    if (q < 0) return ORC_ERR_ARG;
    cv->covfun = covfun;
    cv->d = d;
    cv->q = q;
    for (int j = 0; j < q; j++) {
        if (!(theta[j] > 0.0) || !isfinite(theta[j])) return ORC_ERR_ARG;
        cv->th[j] = theta[j];
    }
    if (covfun == ORC_EXP_SPACETIME && d != 3) return ORC_ERR_ARG;
    if (covfun == ORC_MATERN_ISO) {
        double nu = theta[2];
        if (nu < 0.05 || nu > 20.0) return ORC_ERR_ARG;
        cv->lg_nu = lgamma(nu);
        cv->psi_nu = orc_digamma(nu);
    }
    return ORC_OK;
}

static double orc_cov_eval(const orc_cov* cv, const double* la, const double* lb, int same,
                           double* dC)
{
    const double* t = cv->th;
    int d = cv->d;
    double C = 0.0;
    switch (cv->covfun) {
    case ORC_EXP_ISO: { /* sigma2 exp(-r/rho) + [same] sigma2 tau2 */
        double r2 = 0.0;
        for (int k = 0; k < d; k++) r2 += (la[k] - lb[k]) * (la[k] - lb[k]);
        double x = sqrt(r2) / t[1];
        double e = exp(-x);
        C = t[0] * e;
        dC[0] = e;
        dC[1] = t[0] * e * x / t[1];
        dC[2] = 0.0;
        if (same) {
            C += t[0] * t[2];
            dC[0] += t[2];
            dC[2] = t[0];
        }
        break;
    }
    case ORC_MATERN_ISO: { /* sigma2 M_nu(r/rho) + [same] sigma2 tau2 */
        double r2 = 0.0;
        for (int k = 0; k < d; k++) r2 += (la[k] - lb[k]) * (la[k] - lb[k]);
        double M = 1.0, xdMdx = 0.0, dMdnu = 0.0;
        if (r2 > 0.0) {
            double x = sqrt(r2) / t[1];
            matern_eval(t[2], x, cv->lg_nu, cv->psi_nu, &M, &xdMdx, &dMdnu);
        }
        C = t[0] * M;
        dC[0] = M;
        dC[1] = -t[0] * xdMdx / t[1]; /* dM/drho = dM/dx * (-x/rho) */
        dC[2] = t[0] * dMdnu;
        dC[3] = 0.0;
        if (same) {
            C += t[0] * t[3];
            dC[0] += t[3];
            dC[3] = t[0];
        }
        break;
    }
    case ORC_EXP_SPACETIME: { /* sigma2 exp(-sqrt((dlon^2+dlat^2)/rs^2 + dt^2/rt^2)) */
        double ds2 = (la[0] - lb[0]) * (la[0] - lb[0]) + (la[1] - lb[1]) * (la[1] - lb[1]);
        double dt2 = (la[2] - lb[2]) * (la[2] - lb[2]);
        double D = sqrt(ds2 / (t[1] * t[1]) + dt2 / (t[2] * t[2]));
        double e = exp(-D);
        C = t[0] * e;
        dC[0] = e;
        if (D > 0.0) {
            /* dD/drho_s = -ds2/(rho_s^3 D), dD/drho_t = -dt2/(rho_t^3 D) */
            dC[1] = t[0] * e * ds2 / (t[1] * t[1] * t[1] * D);
            dC[2] = t[0] * e * dt2 / (t[2] * t[2] * t[2] * D);
        } else {
            dC[1] = 0.0;
            dC[2] = 0.0;
        }
        dC[3] = 0.0;
        if (same) {
            C += t[0] * t[3];
            dC[0] += t[3];
            dC[3] = t[0];
        }
        break;
    }
    case ORC_EXP_ANISO: { /* sigma2 exp(-sqrt(sum_k (dz_k / rho_k)^2)) + [same] sigma2 tau2 */
        double D2 = 0.0;
        for (int k = 0; k < d; k++) {
            double u = (la[k] - lb[k]) / t[1 + k];
            D2 += u * u;
        }
        double D = sqrt(D2);
        double e = exp(-D);
        C = t[0] * e;
        dC[0] = e;
        /* dD/drho_k = -(dz_k / rho_k)^2 / (rho_k D), so dC/drho_k = sigma2 e u_k^2 / (rho_k D) */
        for (int k = 0; k < d; k++) {
            double u = (la[k] - lb[k]) / t[1 + k];
            dC[1 + k] = (D > 0.0) ? t[0] * e * u * u / (t[1 + k] * D) : 0.0;
        }
        dC[d + 1] = 0.0;
        if (same) {
            C += t[0] * t[d + 1];
            dC[0] += t[d + 1];
            dC[d + 1] = t[0];
        }
        break;
    }
    }
    return C;
}

/* Exported: covariance and derivatives for npairs location pairs (used by the oracle's
 * own unit tests to pin the covariance functions against closed forms and scipy). */
int orc_cov_pairs(int covfun, int d, const double* theta, int64_t npairs, const double* la,
                  const double* lb, const int32_t* same, double* C, double* dC)
{
    orc_cov cv;
    int st = orc_cov_init(&cv, covfun, d, theta);
    if (st) return st;
    int q = cv.q;
    for (int64_t i = 0; i < npairs; i++)
        C[i] = orc_cov_eval(&cv, la + i * d, lb + i * d, same[i], dC + i * q);
    return ORC_OK;
}

/* Exported: digamma (for its pin against scipy). */
double orc_psi(double x) { return orc_digamma(x); }

/* ------------------------------------------------------------------------------------ */
/* Neumaier compensated accumulation                                                    */
/* ------------------------------------------------------------------------------------ */
static inline void neu_add(double* s, double* comp, double v)
{
    double t = *s + v;
    if (fabs(*s) >= fabs(v))
        *comp += (*s - t) + v;
    else
        *comp += (v - t) + *s;
    *s = t;
}

/* ------------------------------------------------------------------------------------ */
/* One observation of Algorithm 1                                                       */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int Kmax, d, p, q;
    int32_t* idx;  /* K          block indices: neighbours (farthest first), then i */
    double* locsub;/* K x d                                                         */
    double* ysub;  /* K                                                             */
    double* Xsub;  /* K x p                                                         */
    double* covmat;/* K x K, Cholesky factor in place (lower)                       */
    double* dcov;  /* q x K x K                                                     */
    double* Liy;   /* K                                                             */
    double* LiX;   /* K x p                                                         */
    double* bvec;  /* K   last row of L^-1                                          */
    double* g;     /* K                                                             */
    double* mj;    /* q x K                                                         */
    double* rec;   /* stats record of one observation                               */
} orc_work;

static int work_alloc(orc_work* w, int Kmax, int d, int p, int q)
{
    w->Kmax = Kmax; w->d = d; w->p = p; w->q = q;
    w->idx = (int32_t*)malloc(sizeof(int32_t) * Kmax);
    size_t nd = (size_t)Kmax * d + Kmax + (size_t)Kmax * p + (size_t)Kmax * Kmax
                + (size_t)q * Kmax * Kmax + Kmax + (size_t)Kmax * p + Kmax + Kmax
                + (size_t)q * Kmax + orc_stats_len(p, q);
    double* buf = (double*)calloc(nd, sizeof(double));
    if (!w->idx || !buf) { free(w->idx); free(buf); return ORC_ERR_NOMEM; }
    w->locsub = buf; buf += (size_t)Kmax * d;
    w->ysub = buf; buf += Kmax;
    w->Xsub = buf; buf += (size_t)Kmax * p;
    w->covmat = buf; buf += (size_t)Kmax * Kmax;
    w->dcov = buf; buf += (size_t)q * Kmax * Kmax;
    w->Liy = buf; buf += Kmax;
    w->LiX = buf; buf += (size_t)Kmax * p;
    w->bvec = buf; buf += Kmax;
    w->g = buf; buf += Kmax;
    w->mj = buf; buf += (size_t)q * Kmax;
    w->rec = buf;
    return ORC_OK;
}
static void work_free(orc_work* w) { free(w->idx); free(w->locsub); }

/* Computes the Algorithm 1 contribution of observation i into w->rec.
 * Returns ORC_OK, ORC_ERR_ARG (bad NNarray row) or ORC_ERR_NOT_PD. */
static int one_point(const orc_cov* cv, const double* locs, const double* y, const double* X,
                     const int32_t* NN, int64_t i, int m, orc_work* w)
{
    const int d = w->d, p = w->p, q = w->q;
    const int32_t* row = NN + i * (int64_t)(m + 1);
    if (row[0] != (int32_t)i) return ORC_ERR_ARG;
    int k = 0;
    while (k < m && row[1 + k] >= 0) {
        if (row[1 + k] >= i) return ORC_ERR_ARG; /* neighbours must precede i */
        k++;
    }
    for (int j = k; j < m; j++)
        if (row[1 + j] != -1) return ORC_ERR_ARG; /* padding is -1 after the last neighbour */
    const int K = k + 1;

    /* Algorithm 1: substitute the neighbours (reversed, so that i is last). */
    for (int a = 0; a < K; a++) w->idx[a] = row[K - 1 - a];
    for (int a = 0; a < K; a++) {
        int64_t r = w->idx[a];
        for (int c = 0; c < d; c++) w->locsub[a * d + c] = locs[r * d + c];
        w->ysub[a] = y[r];
        for (int c = 0; c < p; c++) w->Xsub[a * p + c] = X[r * p + c];
    }

    /* covariance matrix and its derivatives (full symmetric storage) */
    double dC[ORC_QMAX];
    for (int a = 0; a < K; a++) {
        for (int b = 0; b <= a; b++) {
            double C = orc_cov_eval(cv, w->locsub + a * d, w->locsub + b * d, a == b, dC);
            w->covmat[a * K + b] = C;
            w->covmat[b * K + a] = C;
            for (int j = 0; j < q; j++) {
                w->dcov[(j * K + a) * K + b] = dC[j];
                w->dcov[(j * K + b) * K + a] = dC[j];
            }
        }
    }

    /* Cholesky in place (lower triangle), textbook column-by-column */
    double* L = w->covmat;
    for (int c = 0; c < K; c++) {
        double v = L[c * K + c];
        for (int s = 0; s < c; s++) v -= L[c * K + s] * L[c * K + s];
        if (!(v > 0.0) || !isfinite(v)) return ORC_ERR_NOT_PD;
        double lcc = sqrt(v);
        L[c * K + c] = lcc;
        for (int r = c + 1; r < K; r++) {
            double u = L[r * K + c];
            for (int s = 0; s < c; s++) u -= L[r * K + s] * L[c * K + s];
            L[r * K + c] = u / lcc;
        }
    }

    /* Liy = L^-1 ysub, LiX = L^-1 Xsub (forward substitution) */
    for (int a = 0; a < K; a++) {
        double u = w->ysub[a];
        for (int s = 0; s < a; s++) u -= L[a * K + s] * w->Liy[s];
        w->Liy[a] = u / L[a * K + a];
        for (int c = 0; c < p; c++) {
            double v = w->Xsub[a * p + c];
            for (int s = 0; s < a; s++) v -= L[a * K + s] * w->LiX[s * p + c];
            w->LiX[a * p + c] = v / L[a * K + a];
        }
    }

    /* record layout */
    double* rec = w->rec;
    double* logdet = rec;
    double* ySy = rec + 1;
    double* XSX = rec + 2;
    double* ySX = XSX + p * p;
    double* dlogdet = ySX + p;
    double* dySy = dlogdet + q;
    double* dXSX = dySy + q;
    double* dySX = dXSX + q * p * p;
    double* ainfo = dySX + q * p;

    const int last = K - 1;
    const double ell = w->Liy[last];
    const double* xl = w->LiX + last * p;
    *logdet = 2.0 * log(L[last * K + last]);
    *ySy = ell * ell;
    for (int a = 0; a < p; a++)
        for (int b = 0; b < p; b++) XSX[a * p + b] = xl[a] * xl[b];
    for (int a = 0; a < p; a++) ySX[a] = ell * xl[a];

    /* remaining operations: b = last row of L^-1 (solve L^T b^T = e_last) */
    for (int a = K - 1; a >= 0; a--) {
        double u = (a == last) ? 1.0 : 0.0;
        for (int r = a + 1; r < K; r++) u -= L[r * K + a] * w->bvec[r];
        w->bvec[a] = u / L[a * K + a];
    }
    for (int j = 0; j < q; j++) {
        const double* dS = w->dcov + (size_t)j * K * K;
        double* mj = w->mj + j * K;
        /* g = dSigma_j b^T, then m_j = L^-1 g */
        for (int a = 0; a < K; a++) {
            double u = 0.0;
            for (int b = 0; b < K; b++) u += dS[a * K + b] * w->bvec[b];
            w->g[a] = u;
        }
        for (int a = 0; a < K; a++) {
            double u = w->g[a];
            for (int s = 0; s < a; s++) u -= L[a * K + s] * mj[s];
            mj[a] = u / L[a * K + a];
        }
        /* d ell = -(m_j . hat(Liy)),  d x = -(m_j^T hat(LiX)) */
        double dell = 0.0;
        for (int a = 0; a < K; a++) dell -= mj[a] * w->Liy[a] * (a == last ? 0.5 : 1.0);
        double dx[64];
        for (int c = 0; c < p; c++) {
            double u = 0.0;
            for (int a = 0; a < K; a++) u -= mj[a] * w->LiX[a * p + c] * (a == last ? 0.5 : 1.0);
            dx[c] = u;
        }
        dlogdet[j] = mj[last];
        dySy[j] = 2.0 * ell * dell;
        for (int c = 0; c < p; c++) dySX[j * p + c] = dell * xl[c] + ell * dx[c];
        for (int a = 0; a < p; a++)
            for (int b = 0; b < p; b++)
                dXSX[(j * p + a) * p + b] = dx[a] * xl[b] + xl[a] * dx[b];
    }
    for (int j = 0; j < q; j++)
        for (int l = 0; l < q; l++) {
            double u = 0.0;
            for (int a = 0; a < K; a++) u += w->mj[j * K + a] * w->mj[l * K + a];
            ainfo[j * q + l] = u - 0.5 * w->mj[j * K + last] * w->mj[l * K + last];
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 1 over all observations                                                    */
/* ------------------------------------------------------------------------------------ */

/* Runs Algorithm 1 over observations [0, n) and writes the summed record (length
 * orc_stats_len(p, q)) to stats.  Observations are processed in fixed chunks; each chunk
 * is summed with Neumaier compensation, then the chunk sums are added in chunk order.
 * bad_index receives the smallest observation index whose block is not positive
 * definite (or -1).  nthreads <= 0 means the OpenMP default. */
int orc_vecchia_stats(const double* locs, const double* y, const double* X, const int32_t* NN,
                      int64_t n, int d, int p, int m, const double* theta, int covfun,
                      double* stats, int64_t* bad_index, int nthreads)
{
    if (n < 1 || d < 1 || p < 1 || p > 64 || m < 0) return ORC_ERR_ARG;
    orc_cov cv;
    int st = orc_cov_init(&cv, covfun, d, theta);
    if (st) return st;
    const int q = cv.q;
    const int S = orc_stats_len(p, q);
    const int64_t nchunk = (n + ORC_CHUNK - 1) / ORC_CHUNK;
    double* csum = (double*)calloc((size_t)nchunk * S * 2, sizeof(double));
    if (!csum) return ORC_ERR_NOMEM;
    int64_t bad = -1;
    int err = ORC_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        orc_work w;
        int wst = work_alloc(&w, m + 1, d, p, q);
        if (wst) {
#pragma omp critical
            err = wst;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t ch = 0; ch < nchunk; ch++) {
            if (wst) continue;
            double* s = csum + (size_t)ch * S * 2;
            double* comp = s + S;
            int64_t i1 = (ch + 1) * ORC_CHUNK < n ? (ch + 1) * ORC_CHUNK : n;
            for (int64_t i = ch * ORC_CHUNK; i < i1; i++) {
                int pst = one_point(&cv, locs, y, X, NN, i, m, &w);
                if (pst != ORC_OK) {
#pragma omp critical
                    {
                        if (pst == ORC_ERR_NOT_PD) {
                            if (bad < 0 || i < bad) bad = i;
                            if (err == ORC_OK) err = ORC_ERR_NOT_PD;
                        } else {
                            err = pst;
                        }
                    }
                    continue;
                }
                for (int t = 0; t < S; t++) neu_add(&s[t], &comp[t], w.rec[t]);
            }
        }
        if (!wst) work_free(&w);
    }
    for (int t = 0; t < S; t++) {
        double acc = 0.0, comp = 0.0;
        for (int64_t ch = 0; ch < nchunk; ch++) {
            neu_add(&acc, &comp, csum[(size_t)ch * S * 2 + t]);
            neu_add(&acc, &comp, csum[(size_t)ch * S * 2 + S + t]);
        }
        stats[t] = acc + comp;
    }
    free(csum);
    if (bad_index) *bad_index = bad;
    if (err == ORC_OK) {
        for (int t = 0; t < S; t++)
            if (!isfinite(stats[t])) return ORC_ERR_NONFINITE;
    }
    return err;
}

/* Per-observation records (n x S), for tests on tiny inputs. */
int orc_vecchia_records(const double* locs, const double* y, const double* X, const int32_t* NN,
                        int64_t n, int d, int p, int m, const double* theta, int covfun,
                        double* recs)
{
    orc_cov cv;
    int st = orc_cov_init(&cv, covfun, d, theta);
    if (st) return st;
    const int q = cv.q;
    const int S = orc_stats_len(p, q);
    orc_work w;
    if (work_alloc(&w, m + 1, d, p, q)) return ORC_ERR_NOMEM;
    int err = ORC_OK;
    for (int64_t i = 0; i < n && err == ORC_OK; i++) {
        err = one_point(&cv, locs, y, X, NN, i, m, &w);
        if (err == ORC_OK) memcpy(recs + i * S, w.rec, sizeof(double) * S);
    }
    work_free(&w);
    return err;
}

/* ------------------------------------------------------------------------------------ */
/* The "separate function": profile beta, form loglik, gradient and Fisher information   */
/* ------------------------------------------------------------------------------------ */

/* Cholesky solve of a small SPD system A x = b (A n x n, row-major); returns 0 if PD. */
static int small_chol_solve(int n, const double* A, const double* b, double* x)
{
    double L[64 * 64];
    if (n > 64) return -1;
    for (int i = 0; i < n * n; i++) L[i] = A[i];
    for (int c = 0; c < n; c++) {
        double v = L[c * n + c];
        for (int s = 0; s < c; s++) v -= L[c * n + s] * L[c * n + s];
        if (!(v > 0.0)) return -1;
        L[c * n + c] = sqrt(v);
        for (int r = c + 1; r < n; r++) {
            double u = L[r * n + c];
            for (int s = 0; s < c; s++) u -= L[r * n + s] * L[c * n + s];
            L[r * n + c] = u / L[c * n + c];
        }
    }
    double z[64];
    for (int a = 0; a < n; a++) {
        double u = b[a];
        for (int s = 0; s < a; s++) u -= L[a * n + s] * z[s];
        z[a] = u / L[a * n + a];
    }
    for (int a = n - 1; a >= 0; a--) {
        double u = z[a];
        for (int r = a + 1; r < n; r++) u -= L[r * n + a] * x[r];
        x[a] = u / L[a * n + a];
    }
    return 0;
}

/* From the summed record: betahat = XSX^-1 ySX;
 *   loglik = -n/2 log(2 pi) - 1/2 logdet - 1/2 (ySy - ySX^T betahat)
 *   grad_j = -1/2 (dlogdet_j + dySy_j - 2 betahat^T dySX_j + betahat^T dXSX_j betahat)
 *   info   = ainfo                                                                    */
int orc_profile(const double* stats, int64_t n, int p, int q, double* loglik, double* grad,
                double* info, double* betahat)
{
    const double* logdet = stats;
    const double* ySy = stats + 1;
    const double* XSX = stats + 2;
    const double* ySX = XSX + p * p;
    const double* dlogdet = ySX + p;
    const double* dySy = dlogdet + q;
    const double* dXSX = dySy + q;
    const double* dySX = dXSX + q * p * p;
    const double* ainfo = dySX + q * p;
    double beta[64];
    if (small_chol_solve(p, XSX, ySX, beta)) return ORC_ERR_NOT_PD;
    double quad = *ySy;
    for (int a = 0; a < p; a++) quad -= ySX[a] * beta[a];
    *loglik = -0.5 * (double)n * log(2.0 * M_PI) - 0.5 * (*logdet) - 0.5 * quad;
    for (int j = 0; j < q; j++) {
        double t = dlogdet[j] + dySy[j];
        for (int a = 0; a < p; a++) t -= 2.0 * beta[a] * dySX[j * p + a];
        for (int a = 0; a < p; a++)
            for (int b = 0; b < p; b++) t += beta[a] * dXSX[(j * p + a) * p + b] * beta[b];
        grad[j] = -0.5 * t;
    }
    for (int t = 0; t < q * q; t++) info[t] = ainfo[t];
    for (int a = 0; a < p; a++) betahat[a] = beta[a];
    return ORC_OK;
}

int orc_loglik_grad_info(const double* locs, const double* y, const double* X,
                         const int32_t* NN, int64_t n, int d, int p, int m, const double* theta,
                         int covfun, double* loglik, double* grad, double* info,
                         double* betahat, int64_t* bad_index, int nthreads)
{
    int q = orc_nparms_d(covfun, d);
    if (q < 0 || p < 1 || p > 64) return ORC_ERR_ARG;
    double* stats = (double*)malloc(sizeof(double) * orc_stats_len(p, q));
    if (!stats) return ORC_ERR_NOMEM;
    int st = orc_vecchia_stats(locs, y, X, NN, n, d, p, m, theta, covfun, stats, bad_index,
                               nthreads);
    if (st == ORC_OK) st = orc_profile(stats, n, p, q, loglik, grad, info, betahat);
    free(stats);
    return st;
}

/* ------------------------------------------------------------------------------------ */
/* Fisher scoring (Eq. 4) on log-parameters                                             */
/* ------------------------------------------------------------------------------------ */

/* Rules:
 *   work on log theta: g~ = theta (.) g,  I~ = diag(theta) I diag(theta);
 *   if I~ is not positive definite, add 1e-4 * max diag(I~) to its diagonal (repeat, up to 8x);
 *   Delta = I~^-1 g~; stop (converged) when g~^T Delta < tol, before taking the step;
 *   trial theta' = theta (.) exp(Delta / 2^h), h = 0..10, accepted at the first h whose
 *   loglik is finite and larger than the current one; a trial that fails (not PD,
 *   non-finite, or outside the parameter domain because a parameter underflowed to 0 or
 *   overflowed) counts as -inf; nu is clamped to [0.05, 20];
 *   at most maxit accepted steps.
 * Outputs the final theta, betahat, loglik, grad, info; *iters = accepted steps;
 * *status = 0 converged, 1 iteration limit, 2 no ascent step found, else an error code. */
int orc_fisher_fit(const double* locs, const double* y, const double* X, const int32_t* NN,
                   int64_t n, int d, int p, int m, int covfun, const double* start, double tol,
                   int maxit, double* theta_out, double* betahat, double* loglik, double* grad,
                   double* info, int* iters, int* status, int nthreads)
{
    int q = orc_nparms_d(covfun, d);
    if (q < 0) return ORC_ERR_ARG;
    double th[ORC_QMAX], ll, g[ORC_QMAX], I[ORC_QMAX * ORC_QMAX], bh[64];
    for (int j = 0; j < q; j++) th[j] = start[j];
    int64_t bad;
    int st = orc_loglik_grad_info(locs, y, X, NN, n, d, p, m, th, covfun, &ll, g, I, bh, &bad,
                                  nthreads);
    if (st) return st;
    int it = 0;
    *status = 1;
    for (;;) {
        double gt[ORC_QMAX], It[ORC_QMAX * ORC_QMAX], delta[ORC_QMAX];
        for (int j = 0; j < q; j++) gt[j] = th[j] * g[j];
        for (int j = 0; j < q; j++)
            for (int l = 0; l < q; l++) It[j * q + l] = th[j] * I[j * q + l] * th[l];
        double maxd = 0.0;
        for (int j = 0; j < q; j++) maxd = fmax(maxd, It[j * q + j]);
        int ok = -1;
        for (int r = 0; r < 9 && ok; r++) {
            double A[ORC_QMAX * ORC_QMAX];
            for (int t = 0; t < q * q; t++) A[t] = It[t];
            for (int j = 0; j < q; j++) A[j * q + j] += r * 1e-4 * maxd;
            ok = small_chol_solve(q, A, gt, delta);
        }
        if (ok) { *status = 2; break; }
        double dec = 0.0;
        for (int j = 0; j < q; j++) dec += gt[j] * delta[j];
        if (dec < tol) { *status = 0; break; }
        if (it >= maxit) { *status = 1; break; }
        int accepted = 0;
        for (int h = 0; h <= 10 && !accepted; h++) {
            double tn[ORC_QMAX], lln, gn[ORC_QMAX], In[ORC_QMAX * ORC_QMAX], bhn[64];
            double scale = ldexp(1.0, -h);
            for (int j = 0; j < q; j++) tn[j] = th[j] * exp(delta[j] * scale);
            if (covfun == ORC_MATERN_ISO) tn[2] = fmin(20.0, fmax(0.05, tn[2]));
            int s2 = orc_loglik_grad_info(locs, y, X, NN, n, d, p, m, tn, covfun, &lln, gn, In,
                                          bhn, &bad, nthreads);
            if (s2 == ORC_OK && isfinite(lln) && lln > ll) {
                accepted = 1;
                for (int j = 0; j < q; j++) { th[j] = tn[j]; g[j] = gn[j]; }
                for (int t = 0; t < q * q; t++) I[t] = In[t];
                for (int a = 0; a < p; a++) bh[a] = bhn[a];
                ll = lln;
            }
            /* any other outcome is a failed trial: the step is halved */
        }
        if (!accepted) { *status = 2; break; }
        it++;
    }
    for (int j = 0; j < q; j++) { theta_out[j] = th[j]; grad[j] = g[j]; }
    for (int t = 0; t < q * q; t++) info[t] = I[t];
    for (int a = 0; a < p; a++) betahat[a] = bh[a];
    *loglik = ll;
    *iters = it;
    return ORC_OK;
}
