/*
 * prep.c -- input preprocessing and field generation for Vecchia workloads: maxmin
 * ordering, ordered nearest neighbours (NNarray), and the pieces of the sequential draw
 * of synthetic fields (regression weights from closed-form covariances, recurrence).
 *
 * This is input generation, shared by both sides that consume the inputs (the CPU
 * oracle and the CUDA library), and used by neither to compute anything: it evaluates
 * no likelihood or derivative, and its covariance code exists only to draw y.
 *
 *   Ordering (Sec. 2.1; maxmin heuristic of Guinness 2018): the first point is the one
 *   nearest to the centroid; each next point is the one whose minimum distance to the
 *   points already chosen is largest.  Ties go to the lowest original index.  Exact.
 *   Implemented with a uniform grid (range queries) and a lazily updated max-heap.
 *
 *   Ordered nearest neighbours (Sec. 3, NNarray): row i lists i, then the min(i, m)
 *   points of index < i that are closest to point i, nearest first, padded with -1.
 *   Ties go to the lowest index.  Exact, grid accelerated (expanding shells).
 *
 * All distances are squared Euclidean distances in FP64, summed in coordinate order;
 * the build uses -ffp-contract=off so the result is the same on every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <omp.h>
#include <string.h>

#define PREP_OK 0
#define PREP_ERR_ARG 1
#define PREP_ERR_NOMEM 2

static double sqdist(const double* a, const double* b, int d)
{
    double s = 0.0;
    for (int k = 0; k < d; k++) {
        double t = a[k] - b[k];
        s += t * t;
    }
    return s;
}

/* ---------------------------------- uniform grid ----------------------------------- */
typedef struct {
    int d;
    int64_t nc[3];    /* cells per dimension (1 for unused dims) */
    double lo[3], h;  /* origin and cell size                    */
    int64_t ncell;
    int64_t* start;   /* ncell + 1 (CSR over cells)              */
    int64_t* items;   /* point indices sorted by cell            */
} grid_t;

static void cell_of(const grid_t* g, const double* x, int64_t* c)
{
    for (int k = 0; k < 3; k++) {
        if (k >= g->d) { c[k] = 0; continue; }
        int64_t v = (int64_t)floor((x[k] - g->lo[k]) / g->h);
        if (v < 0) v = 0;
        if (v >= g->nc[k]) v = g->nc[k] - 1;
        c[k] = v;
    }
}

/* Builds a grid over the given points with about `per_cell` points per cell on
 * average (by bounding-box volume).  If `ids` is NULL all n points are inserted. */
static int grid_build(grid_t* g, const double* x, int64_t n, int d, double per_cell)
{
    memset(g, 0, sizeof(*g));
    g->d = d;
    double hi[3] = {0, 0, 0};
    for (int k = 0; k < 3; k++) { g->lo[k] = 0.0; hi[k] = 0.0; }
    for (int k = 0; k < d; k++) { g->lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < d; k++) {
            double v = x[i * d + k];
            if (v < g->lo[k]) g->lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
    double vol = 1.0, maxext = 0.0;
    for (int k = 0; k < d; k++) {
        double e = hi[k] - g->lo[k];
        if (e > maxext) maxext = e;
    }
    if (!(maxext > 0.0)) maxext = 1.0;
    for (int k = 0; k < d; k++) {
        double e = hi[k] - g->lo[k];
        vol *= (e > 1e-12 * maxext ? e : 1e-12 * maxext);
    }
    double h = pow(vol * per_cell / (double)(n > 0 ? n : 1), 1.0 / d);
    if (!(h > 0.0) || !isfinite(h)) h = maxext;
    /* cap the number of cells at ~4 n */
    for (;;) {
        double cells = 1.0;
        for (int k = 0; k < d; k++) cells *= floor((hi[k] - g->lo[k]) / h) + 1.0;
        if (cells <= 4.0 * (double)n + 64.0) break;
        h *= 1.25;
    }
    g->h = h;
    g->ncell = 1;
    for (int k = 0; k < 3; k++) {
        g->nc[k] = (k < d) ? (int64_t)floor((hi[k] - g->lo[k]) / h) + 1 : 1;
        g->ncell *= g->nc[k];
    }
    g->start = (int64_t*)calloc((size_t)g->ncell + 1, sizeof(int64_t));
    g->items = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* cid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!g->start || !g->items || !cid) {
        free(g->start); free(g->items); free(cid);
        return PREP_ERR_NOMEM;
    }
    for (int64_t i = 0; i < n; i++) {
        int64_t c[3];
        cell_of(g, x + i * d, c);
        cid[i] = (c[2] * g->nc[1] + c[1]) * g->nc[0] + c[0];
        g->start[cid[i] + 1]++;
    }
    for (int64_t c = 0; c < g->ncell; c++) g->start[c + 1] += g->start[c];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->ncell);
    if (!fill) { free(g->start); free(g->items); free(cid); return PREP_ERR_NOMEM; }
    memcpy(fill, g->start, sizeof(int64_t) * (size_t)g->ncell);
    for (int64_t i = 0; i < n; i++) g->items[fill[cid[i]]++] = i; /* ascending index per cell */
    free(fill);
    free(cid);
    return PREP_OK;
}
static void grid_free(grid_t* g) { free(g->start); free(g->items); }

/* ------------------------------------ max-heap -------------------------------------- */
typedef struct { double key; int64_t id; } hent;
/* a before b in the heap order: larger key first, then smaller id */
static int hbefore(const hent* a, const hent* b)
{
    return a->key > b->key || (a->key == b->key && a->id < b->id);
}
typedef struct { hent* v; int64_t n, cap; } heap_t;
static int heap_push(heap_t* h, double key, int64_t id)
{
    if (h->n == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 1024;
        hent* nv = (hent*)realloc(h->v, sizeof(hent) * (size_t)nc);
        if (!nv) return PREP_ERR_NOMEM;
        h->v = nv; h->cap = nc;
    }
    int64_t i = h->n++;
    h->v[i].key = key; h->v[i].id = id;
    while (i > 0) {
        int64_t par = (i - 1) / 2;
        if (!hbefore(&h->v[i], &h->v[par])) break;
        hent t = h->v[i]; h->v[i] = h->v[par]; h->v[par] = t;
        i = par;
    }
    return PREP_OK;
}
static hent heap_pop(heap_t* h)
{
    hent top = h->v[0];
    h->v[0] = h->v[--h->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, b = i;
        if (l < h->n && hbefore(&h->v[l], &h->v[b])) b = l;
        if (r < h->n && hbefore(&h->v[r], &h->v[b])) b = r;
        if (b == i) break;
        hent t = h->v[i]; h->v[i] = h->v[b]; h->v[b] = t;
        i = b;
    }
    return top;
}

/* ------------------------------------ maxmin ---------------------------------------- */
/* order[k] = original index of the k-th point in maxmin order. */
int prep_maxmin(const double* x, int64_t n, int d, int64_t* order)
{
    if (n < 1 || d < 1 || d > 3) return PREP_ERR_ARG;
    double cen[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < d; k++) cen[k] += x[i * d + k];
    for (int k = 0; k < d; k++) cen[k] /= (double)n;
    int64_t first = 0;
    double best = INFINITY;
    for (int64_t i = 0; i < n; i++) {
        double s = sqdist(x + i * d, cen, d);
        if (s < best) { best = s; first = i; }
    }
    double* dist = (double*)malloc(sizeof(double) * (size_t)n);
    unsigned char* sel = (unsigned char*)calloc((size_t)n, 1);
    grid_t g;
    heap_t hp = {0, 0, 0};
    if (!dist || !sel || grid_build(&g, x, n, d, 2.0)) {
        free(dist); free(sel);
        return PREP_ERR_NOMEM;
    }
    int rc = PREP_OK;
    for (int64_t i = 0; i < n; i++) {
        dist[i] = sqdist(x + i * d, x + first * d, d);
        if (i != first && heap_push(&hp, dist[i], i)) rc = PREP_ERR_NOMEM;
    }
    order[0] = first;
    sel[first] = 1;
    int64_t k = 1;
    while (k < n && rc == PREP_OK) {
        if (hp.n == 0) { rc = PREP_ERR_ARG; break; }
        hent e = heap_pop(&hp);
        if (sel[e.id] || e.key != dist[e.id]) continue; /* stale entry */
        int64_t j = e.id;
        order[k++] = j;
        sel[j] = 1;
        /* update points that are closer to j than to the chosen set: they lie within
           distance sqrt(dist[j]) of j because dist[k] <= dist[j] for every k */
        double R = sqrt(dist[j]);
        int64_t c0[3], c1[3];
        double lo[3], hi[3];
        for (int t = 0; t < 3; t++) {
            lo[t] = (t < d) ? x[j * d + t] - R : 0.0;
            hi[t] = (t < d) ? x[j * d + t] + R : 0.0;
        }
        cell_of(&g, lo, c0);
        cell_of(&g, hi, c1);
        for (int64_t cz = c0[2]; cz <= c1[2]; cz++)
            for (int64_t cy = c0[1]; cy <= c1[1]; cy++)
                for (int64_t cx = c0[0]; cx <= c1[0]; cx++) {
                    int64_t c = (cz * g.nc[1] + cy) * g.nc[0] + cx;
                    for (int64_t t = g.start[c]; t < g.start[c + 1]; t++) {
                        int64_t u = g.items[t];
                        if (sel[u]) continue;
                        double s = sqdist(x + u * d, x + j * d, d);
                        if (s < dist[u]) {
                            dist[u] = s;
                            if (heap_push(&hp, s, u)) rc = PREP_ERR_NOMEM;
                        }
                    }
                }
    }
    free(hp.v);
    grid_free(&g);
    free(dist);
    free(sel);
    return rc;
}

/* Exact maxmin by brute force, O(n^2 d); pins prep_maxmin on small inputs and orders
 * points of more than 3 coordinates (1 <= d <= 64), where the grid is not used. */
int prep_maxmin_brute(const double* x, int64_t n, int d, int64_t* order)
{
    if (n < 1 || d < 1 || d > 64) return PREP_ERR_ARG;
    double cen[64] = {0};
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < d; k++) cen[k] += x[i * d + k];
    for (int k = 0; k < d; k++) cen[k] /= (double)n;
    int64_t first = 0;
    double best = INFINITY;
    for (int64_t i = 0; i < n; i++) {
        double s = sqdist(x + i * d, cen, d);
        if (s < best) { best = s; first = i; }
    }
    double* dist = (double*)malloc(sizeof(double) * (size_t)n);
    unsigned char* sel = (unsigned char*)calloc((size_t)n, 1);
    if (!dist || !sel) { free(dist); free(sel); return PREP_ERR_NOMEM; }
    for (int64_t i = 0; i < n; i++) dist[i] = sqdist(x + i * d, x + first * d, d);
    order[0] = first;
    sel[first] = 1;
    for (int64_t k = 1; k < n; k++) {
        int64_t j = -1;
        double bd = -1.0;
        for (int64_t i = 0; i < n; i++)
            if (!sel[i] && dist[i] > bd) { bd = dist[i]; j = i; }
        order[k] = j;
        sel[j] = 1;
        for (int64_t i = 0; i < n; i++) {
            double s = sqdist(x + i * d, x + j * d, d);
            if (s < dist[i]) dist[i] = s;
        }
    }
    free(dist);
    free(sel);
    return PREP_OK;
}

/* ------------------------------ ordered nearest neighbours -------------------------- */
/* Candidate list kept sorted by (distance, index), at most m long. */
static void cand_insert(double* cd, int64_t* ci, int* cnt, int m, double s, int64_t id)
{
    int c = *cnt;
    if (c == m && !(s < cd[m - 1] || (s == cd[m - 1] && id < ci[m - 1]))) return;
    int pos = (c < m) ? c : m - 1;
    while (pos > 0 && (s < cd[pos - 1] || (s == cd[pos - 1] && id < ci[pos - 1]))) {
        cd[pos] = cd[pos - 1];
        ci[pos] = ci[pos - 1];
        pos--;
    }
    cd[pos] = s;
    ci[pos] = id;
    if (c < m) *cnt = c + 1;
}

/* x holds the points already in maxmin order.  NN is n x (m+1), int32. */
int prep_ordered_nn(const double* x, int64_t n, int d, int m, int32_t* NN)
{
    if (n < 1 || d < 1 || d > 3 || m < 0 || n > 2147483647LL) return PREP_ERR_ARG;
    const int64_t W = (int64_t)m + 1;
    for (int64_t i = 0; i < n * W; i++) NN[i] = -1;
    if (m == 0) {
        for (int64_t i = 0; i < n; i++) NN[i] = (int32_t)i;
        return PREP_OK;
    }
    grid_t g;
    if (grid_build(&g, x, n, d, 2.0)) return PREP_ERR_NOMEM;
    /* rows are independent: OpenMP over i, one candidate buffer per thread */
    const int nthr = omp_get_max_threads();
    double* cd_all = (double*)malloc(sizeof(double) * (size_t)m * (size_t)nthr);
    int64_t* ci_all = (int64_t*)malloc(sizeof(int64_t) * (size_t)m * (size_t)nthr);
    if (!cd_all || !ci_all) { free(cd_all); free(ci_all); grid_free(&g); return PREP_ERR_NOMEM; }
    const int64_t brute_upto = 4 * (int64_t)m + 64;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) {
        double* cd = cd_all + (size_t)m * (size_t)omp_get_thread_num();
        int64_t* ci = ci_all + (size_t)m * (size_t)omp_get_thread_num();
        int cnt = 0;
        NN[i * W] = (int32_t)i;
        if (i <= brute_upto) {
            for (int64_t j = 0; j < i; j++)
                cand_insert(cd, ci, &cnt, m, sqdist(x + i * d, x + j * d, d), j);
        } else {
            int64_t c[3];
            cell_of(&g, x + i * d, c);
            int64_t maxr = 0;
            for (int t = 0; t < d; t++) {
                int64_t r = c[t] > g.nc[t] - 1 - c[t] ? c[t] : g.nc[t] - 1 - c[t];
                if (r > maxr) maxr = r;
            }
            for (int64_t r = 0; r <= maxr; r++) {
                /* visit the cells at Chebyshev distance exactly r from cell c */
                int64_t lo[3], hi[3];
                for (int t = 0; t < 3; t++) {
                    lo[t] = (t < d) ? c[t] - r : 0;
                    hi[t] = (t < d) ? c[t] + r : 0;
                }
                for (int64_t cz = lo[2]; cz <= hi[2]; cz++) {
                    if (cz < 0 || cz >= g.nc[2]) continue;
                    for (int64_t cy = lo[1]; cy <= hi[1]; cy++) {
                        if (cy < 0 || cy >= g.nc[1]) continue;
                        int edge_zy = (d >= 3 && (cz == lo[2] || cz == hi[2])) ||
                                      (d >= 2 && (cy == lo[1] || cy == hi[1]));
                        for (int64_t cx = lo[0]; cx <= hi[0]; cx++) {
                            if (cx < 0 || cx >= g.nc[0]) continue;
                            if (!edge_zy && !(cx == lo[0] || cx == hi[0])) {
                                /* interior of the shell: jump to the far face */
                                if (cx < hi[0]) cx = hi[0] - 1;
                                continue;
                            }
                            int64_t cc = (cz * g.nc[1] + cy) * g.nc[0] + cx;
                            for (int64_t t = g.start[cc]; t < g.start[cc + 1]; t++) {
                                int64_t j = g.items[t];
                                if (j >= i) break; /* items ascend within a cell */
                                cand_insert(cd, ci, &cnt, m, sqdist(x + i * d, x + j * d, d), j);
                            }
                        }
                    }
                }
                /* every unvisited cell is at least r*h away (minus rounding slack) */
                if (cnt == m) {
                    double bound = ((double)r - 1e-6) * g.h;
                    if (bound > 0.0 && cd[m - 1] < bound * bound) break;
                }
            }
        }
        for (int t = 0; t < cnt; t++) NN[i * W + 1 + t] = (int32_t)ci[t];
    }
    free(cd_all);
    free(ci_all);
    grid_free(&g);
    return PREP_OK;
}

/* Brute-force ordered NN, O(n^2 d); pins prep_ordered_nn on small inputs and searches
 * points of more than 3 coordinates.  Rows are independent (OpenMP over rows). */
int prep_ordered_nn_brute(const double* x, int64_t n, int d, int m, int32_t* NN)
{
    if (n < 1 || d < 1 || m < 0 || n > 2147483647LL) return PREP_ERR_ARG;
    const int64_t W = (int64_t)m + 1;
    for (int64_t i = 0; i < n * W; i++) NN[i] = -1;
    int fail = 0;
#pragma omp parallel
    {
        double* cd = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
        int64_t* ci = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        const int have = cd && ci;
        if (!have) {
#pragma omp atomic write
            fail = 1;
        }
        /* every thread reaches the work-sharing loop; one without buffers skips its rows */
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; i++) {
            if (!have) continue;
            int cnt = 0;
            NN[i * W] = (int32_t)i;
            if (m > 0)
                for (int64_t j = 0; j < i; j++)
                    cand_insert(cd, ci, &cnt, m, sqdist(x + i * d, x + j * d, d), j);
            for (int t = 0; t < cnt; t++) NN[i * W + 1 + t] = (int32_t)ci[t];
        }
        free(cd);
        free(ci);
    }
    return fail ? PREP_ERR_NOMEM : PREP_OK;
}

/* Sequential simulation recurrence: for i = 0..n-1 in order,
 *   e[i] = sum_k W[i][k] * e[NN[i][1+k]] + sd[i] * z[i]
 * (k over the valid neighbours; W and sd are given).  Used by the workload generators to
 * draw a field from a sequential (Vecchia) model; W and sd come from the generator. */
int prep_seq_recurrence(int64_t n, int m, const int32_t* NN, const double* W, const double* sd,
                        const double* z, double* e)
{
    const int64_t Wd = (int64_t)m + 1;
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int k = 0; k < m; k++) {
            int32_t j = NN[i * Wd + 1 + k];
            if (j < 0) break;
            if (j >= i) return PREP_ERR_ARG;
            s += W[i * m + k] * e[j];
        }
        e[i] = s + sd[i] * z[i];
    }
    return PREP_OK;
}

/* ------------------------------ sequential-draw weights ------------------------------ */
/* Generator-side Gaussian-process regression weights for drawing fields from a sequential
 * model: for each i with listed earlier neighbours N(i), W[i] = S_NN^-1 S_Ni and
 * sd[i] = sqrt(S_ii - S_iN W[i]) for the covariance S = sigma2 (R + tau2 I).
 * kind: 0 exponential exp(-r/rho); 1 Matern nu = 3/2 (1 + x) e^-x; 2 Matern nu = 5/2
 * (1 + x + x^2/3) e^-x (x = r/rho); 3 space-time exponential (d = 3, theta =
 * (sigma2, rho_s, rho_t, tau2)).  theta for kinds 0-2: (sigma2, rho, tau2).
 * W is n x m (unused entries 0).  Returns PREP_ERR_ARG if a block is not positive definite. */
static double gen_corr(int kind, const double* a, const double* b, int d, const double* th)
{
    if (kind == 3) {
        double s = ((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1])) / (th[1] * th[1]);
        s += (a[2] - b[2]) * (a[2] - b[2]) / (th[2] * th[2]);
        return exp(-sqrt(s));
    }
    double x = sqrt(sqdist(a, b, d)) / th[1];
    if (kind == 1) return (1.0 + x) * exp(-x);
    if (kind == 2) return (1.0 + x + x * x / 3.0) * exp(-x);
    return exp(-x);
}

int prep_seq_weights(int64_t n, int d, int m, const int32_t* NN, const double* x, int kind,
                     const double* theta, double* W, double* sd)
{
    if (n < 1 || d < 1 || m < 0 || kind < 0 || kind > 3) return PREP_ERR_ARG;
    const double sig2 = theta[0];
    const double tau2 = theta[kind == 3 ? 3 : 2];
    int err = PREP_OK;
#pragma omp parallel
    {
        const int K = m + 1;
        double* S = (double*)malloc(sizeof(double) * (size_t)K * K);
        double* z = (double*)malloc(sizeof(double) * (size_t)K);
        int32_t* ix = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
#pragma omp for schedule(dynamic, 1024)
        for (int64_t i = 0; i < n; i++) {
            const int32_t* row = NN + i * (int64_t)K;
            int k = 0;
            while (k < m && row[1 + k] >= 0) { ix[k] = row[1 + k]; k++; }
            ix[k] = (int32_t)i;
            const int Kp = k + 1;
            for (int a = 0; a < Kp; a++)
                for (int b = 0; b <= a; b++) {
                    double c = sig2 * gen_corr(kind, x + (int64_t)ix[a] * d, x + (int64_t)ix[b] * d, d, theta);
                    if (a == b) c += sig2 * tau2;
                    S[a * Kp + b] = c;
                }
            /* Cholesky of the (k+1) block; its last row gives L_N^-1 S_Ni and the sd */
            int bad = 0;
            for (int c = 0; c < Kp && !bad; c++) {
                double v = S[c * Kp + c];
                for (int s = 0; s < c; s++) v -= S[c * Kp + s] * S[c * Kp + s];
                if (!(v > 0.0)) { bad = 1; break; }
                double l = sqrt(v);
                S[c * Kp + c] = l;
                for (int r = c + 1; r < Kp; r++) {
                    double u = S[r * Kp + c];
                    for (int s = 0; s < c; s++) u -= S[r * Kp + s] * S[c * Kp + s];
                    S[r * Kp + c] = u / l;
                }
            }
            if (bad) {
#pragma omp critical
                err = PREP_ERR_ARG;
                continue;
            }
            /* W = L_N^-T (last row of L restricted to the neighbours) */
            for (int a = k - 1; a >= 0; a--) {
                double u = S[k * Kp + a];
                for (int r = a + 1; r < k; r++) u -= S[r * Kp + a] * z[r];
                z[a] = u / S[a * Kp + a];
            }
            for (int a = 0; a < m; a++) W[i * (int64_t)m + a] = (a < k) ? z[a] : 0.0;
            sd[i] = S[k * Kp + k];
        }
        free(S);
        free(z);
        free(ix);
    }
    return err;
}
