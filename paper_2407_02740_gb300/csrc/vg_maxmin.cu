// vg_maxmin.cu -- the maxmin ordering on the device (the ordering Sec. 2.1 uses, the
// heuristic of Guinness 2018; the paper computes it on the CPU).
//
// Definition (the one the CPU generator in workloads/prep.c implements): the first point is
// the one nearest to the centroid (lowest index on a tie); each next point is the
// unselected one whose smallest squared distance to the selected points is largest, ties to
// the lowest index.  Squared distances are sums over coordinates, in order, of (x_k - y_k)^2
// with every product and sum rounded separately in FP64, so any FP64 implementation of the
// definition takes the same decisions.
//
// The sequential rule picks one point per step.  Here a step accepts a whole prefix of the
// candidates at once, exactly: with the unselected points sorted by (dist desc, index asc),
// the sequential rule picks c_0, then c_1 if adding c_0 leaves dist(c_1) unchanged (that is
// |c_1 - c_0|^2 >= dist(c_1); every other point's dist can only have dropped and was not
// larger), and so on: c_t is the next pick as long as |c_t - c_s|^2 >= dist(c_t) for every
// earlier c_s of the prefix.  The first c_t that fails ends the step.
//
// Candidates come from a pool: the unselected points whose key (dist, -index) is at least
// a threshold key chosen when the pool is (re)built, so that every point outside the pool
// ranks below every pool entry whose key is still at or above the threshold (dists only
// decrease).  A step takes the pool's entries at or above the threshold, sorted; when none
// is left the pool is rebuilt from all points.  After a step the accepted points lower the
// dist of the points within sqrt(dist(c_s)) of each c_s, found through a uniform grid
// (an atomic minimum on the FP64 bit pattern, which orders like the value for
// non-negative numbers; selected points hold -1 and keep it).
//
// Data that other blocks change during the step kernel (distances, the pool, the accepted
// lists, the control block) is read past the non-coherent L1 (ld.global.cg or volatile).
//
// Kernels: set-up (centroid, first point, initial distances, grid as CSR) as ordinary
// launches, then one persistent cooperative kernel runs every step, its phases separated
// by a grid barrier of its own whose waits are bounded (a wait that runs out sets an error
// flag, and every block leaves at the next barrier).
#include <climits>
#include <cstdint>

#include "vg_internal.h"

namespace vg {

namespace {

constexpr int MM_THREADS = 512;
constexpr int MM_PMAX = 2048;      // pool capacity (one block sorts it in shared memory)
constexpr int MM_TACC = 256;       // candidates examined per step
constexpr int MM_TCHUNK = 64;      // candidates checked together (the prefix ends at the first conflict)
constexpr long long MM_SPIN_LIMIT = 1ll << 26;   // ~seconds of waiting per barrier

enum : int { MODE_UPDATE = 0, MODE_REBUILD = 1, MODE_DONE = 2 };

struct MMCtl {
    unsigned long long maxbits;   // rebuild: largest dist (bit pattern)
    long long k;                  // points selected so far
    unsigned bar_count, bar_gen;  // grid barrier
    int mode, err;
    int pool_n;                   // pool entries
    int nacc;                     // points accepted in the current step
    int count;                    // rebuild: points at or above the trial threshold
    long long total_work;         // (accepted point, cell) items of the update
    double thr_d;                 // pool threshold key (thr_d, thr_i)
    long long thr_i;
    double alpha;                 // rebuild: threshold as a fraction of the largest dist
};

struct MMArgs {
    const double* x;
    long long n;
    int d;
    double* dist;                 // n (selected: -1)
    long long* order;             // n (out)
    const int* cell_start;        // ncell + 1
    const int* cell_items;        // n
    int nc[3];
    double lo[3], h;
    int* pool;                    // MM_PMAX
    int* acc_idx;                 // MM_TACC accepted points of the step
    double* acc_r2;               // their dist at acceptance
    int* acc_box;                 // per accepted point: c0[3], c1[3]
    long long* acc_work;          // prefix sums of the boxes' cell counts (MM_TACC + 1)
    int* blk_count;               // gridDim.x (tie rule)
    MMCtl* ctl;
};

__device__ __forceinline__ double sqdist_rn(const double* a, const double* b, int d) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        const double t = __dsub_rn(a[k], b[k]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

__device__ __forceinline__ int cell_coord(double v, double lo, double h, int nc) {
    const double f = floor((v - lo) / h);
    int c = f < 0.0 ? 0 : (f >= (double)nc ? nc - 1 : (int)f);
    return c;
}

// (dist desc, index asc): true when key a ranks before key b.  Distances are compared as
// their FP64 bit patterns, which order like the values for non-negative numbers (selected
// points hold -1 and padding LLONG_MIN: negative patterns, after every valid key); an
// integer comparison keeps the one-block sort off the GPU's narrow FP64 unit.
__device__ __forceinline__ bool ranks_before(long long da, int ia, long long db, int ib) {
    return da > db || (da == db && ia < ib);
}

// Grid barrier with bounded waits: a block that waits too long sets ctl->err and goes on.
// Returns the error flag as read after the barrier, the same value for every thread of the
// block (so that a block leaves a phase as a whole).
__device__ bool grid_barrier(MMCtl* ctl) {
    __shared__ int s_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = &ctl->bar_gen;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(&ctl->bar_count, 1u) == gridDim.x - 1) {
            ctl->bar_count = 0;
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            long long it = 0;
            while (*gen == g) {
                if (++it > MM_SPIN_LIMIT) { atomicExch(&ctl->err, 1); break; }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_err = *(volatile int*)&ctl->err;
    }
    __syncthreads();
    return s_err != 0;
}

// ---------------------------------------------------------------- set-up kernels
// per-block partial sums of the coordinates (fixed order within and across blocks)
__global__ void k_mm_centroid_partial(const double* __restrict__ x, long long n, int d,
                                      double* __restrict__ part) {
    __shared__ double red[MM_THREADS];
    for (int k = 0; k < d; ++k) {
        double s = 0.0;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x)
            s += x[i * d + k];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * 3 + k] = red[0];
        __syncthreads();
    }
}

// centroid, then per-block nearest point to it (smallest (d2, index))
__global__ void k_mm_first_partial(const double* __restrict__ x, long long n, int d,
                                   const double* __restrict__ part, int nblk,
                                   double* __restrict__ bestd, long long* __restrict__ besti) {
    __shared__ double cen[3];
    __shared__ double sd[MM_THREADS];
    __shared__ long long si[MM_THREADS];
    if (threadIdx.x < 3) {
        double s = 0.0;
        if ((int)threadIdx.x < d)
            for (int b = 0; b < nblk; ++b) s += part[(size_t)b * 3 + threadIdx.x];
        cen[threadIdx.x] = s / (double)n;
    }
    __syncthreads();
    double bd = 1.0 / 0.0;
    long long bi = LLONG_MAX;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double s = sqdist_rn(x + i * d, cen, d);
        if (s < bd || (s == bd && i < bi)) { bd = s; bi = i; }
    }
    sd[threadIdx.x] = bd;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            const double od = sd[threadIdx.x + o];
            const long long oi = si[threadIdx.x + o];
            if (od < sd[threadIdx.x] || (od == sd[threadIdx.x] && oi < si[threadIdx.x])) {
                sd[threadIdx.x] = od;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { bestd[blockIdx.x] = sd[0]; besti[blockIdx.x] = si[0]; }
}

// the first point, the initial distances, the bounding box (in the control block's spare
// fields: lo/hi per coordinate as min / max over the points)
__global__ void k_mm_init(const double* __restrict__ x, long long n, int d,
                          const double* __restrict__ bestd, const long long* __restrict__ besti,
                          int nblk, double* __restrict__ dist, long long* __restrict__ order,
                          MMCtl* ctl) {
    __shared__ long long first;
    if (threadIdx.x == 0) {
        double bd = 1.0 / 0.0;
        long long bi = LLONG_MAX;
        for (int b = 0; b < nblk; ++b)
            if (bestd[b] < bd || (bestd[b] == bd && besti[b] < bi)) { bd = bestd[b]; bi = besti[b]; }
        first = bi;
    }
    __syncthreads();
    const long long f = first;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dist[i] = (i == f) ? -1.0 : sqdist_rn(x + i * d, x + f * d, d);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        order[0] = f;
        ctl->k = 1;
        ctl->mode = MODE_REBUILD;
        ctl->err = 0;
        ctl->pool_n = 0;
        ctl->nacc = 0;
        ctl->bar_count = 0;
        ctl->bar_gen = 0;
        ctl->alpha = 0.5;
    }
}

__global__ void k_mm_cells(const double* __restrict__ x, long long n, int d, int nc0, int nc1,
                           int nc2, double lo0, double lo1, double lo2, double h,
                           int* __restrict__ cell_of, int* __restrict__ counts) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c0 = cell_coord(x[i * d], lo0, h, nc0);
        const int c1 = d > 1 ? cell_coord(x[i * d + 1], lo1, h, nc1) : 0;
        const int c2 = d > 2 ? cell_coord(x[i * d + 2], lo2, h, nc2) : 0;
        const int c = (c2 * nc1 + c1) * nc0 + c0;
        cell_of[i] = c;
        atomicAdd(&counts[c], 1);
    }
}

// exclusive scan of ncell counts into start (one block, chunked), start[ncell] = n
__global__ void k_mm_scan(const int* __restrict__ counts, int ncell, int* __restrict__ start,
                          int* __restrict__ cursor) {
    __shared__ int part[MM_THREADS];
    const int T = blockDim.x;
    const int per = (ncell + T - 1) / T;
    const int b0 = threadIdx.x * per, b1 = min(ncell, b0 + per);
    int s = 0;
    for (int c = b0; c < b1; ++c) s += counts[c];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int t = 0; t < T; ++t) { const int v = part[t]; part[t] = run; run += v; }
        start[ncell] = run;
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int c = b0; c < b1; ++c) { start[c] = run; cursor[c] = run; run += counts[c]; }
}

__global__ void k_mm_fill(long long n, const int* __restrict__ cell_of, int* __restrict__ cursor,
                          int* __restrict__ items) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        items[atomicAdd(&cursor[cell_of[i]], 1)] = (int)i;
}

// ---------------------------------------------------------------- the steps
// Phase A (block 0): sort the pool by (dist desc, index asc), accept the exact prefix,
// record the accepted points and their update boxes.
__device__ void mm_phase_a(const MMArgs& a) {
    __shared__ long long sk[MM_PMAX];   // dist as its bit pattern
    __shared__ int si[MM_PMAX];
    __shared__ int s_first_conflict;
    __shared__ int s_nvalid;
    MMCtl* ctl = a.ctl;
    const int tid = threadIdx.x;
    const int np = *(volatile int*)&ctl->pool_n;
    int P2 = 1;
    while (P2 < np) P2 <<= 1;
    for (int t = tid; t < P2; t += blockDim.x) {
        if (t < np) {
            const int i = __ldcg(a.pool + t);
            sk[t] = __ldcg(reinterpret_cast<const long long*>(a.dist) + i);  // selected: -1, last
            si[t] = i;
        } else {
            sk[t] = LLONG_MIN;
            si[t] = INT_MAX;
        }
    }
    __syncthreads();
    // bitonic sort, descending by rank
    for (int kk = 2; kk <= P2; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int t = tid; t < P2; t += blockDim.x) {
                const int u = t ^ j;
                if (u > t) {
                    const bool up = (t & kk) == 0;
                    const bool before = ranks_before(sk[u], si[u], sk[t], si[t]);
                    if (before == up) {
                        const long long td = sk[t]; sk[t] = sk[u]; sk[u] = td;
                        const int ti = si[t]; si[t] = si[u]; si[u] = ti;
                    }
                }
            }
            __syncthreads();
        }
    // entries still at or above the threshold key form the valid head of the sorted pool
    if (tid == 0) { s_nvalid = 0; s_first_conflict = INT_MAX; }
    __syncthreads();
    const long long thr_d = __double_as_longlong(*(volatile double*)&ctl->thr_d);   // >= 0
    const long long thr_i = *(volatile long long*)&ctl->thr_i;
    for (int t = tid; t < np; t += blockDim.x) {
        const bool ok = sk[t] > thr_d || (sk[t] == thr_d && (long long)si[t] <= thr_i);
        const bool okn = (t + 1 < np) && (sk[t + 1] > thr_d || (sk[t + 1] == thr_d && (long long)si[t + 1] <= thr_i));
        if (ok && !okn) s_nvalid = t + 1;
    }
    __syncthreads();
    const int nvalid = s_nvalid;
    const long long k = *(volatile long long*)&ctl->k;
    if (nvalid == 0) {
        if (tid == 0) ctl->mode = (k >= a.n) ? MODE_DONE : MODE_REBUILD;
        return;
    }
    const int T = nvalid < MM_TACC ? nvalid : MM_TACC;
    // c_t conflicts when an earlier candidate is closer to it than its dist.  The prefix
    // ends at the first conflict, so the candidates are checked MM_TCHUNK at a time, each
    // against every earlier one, and the check stops after the first chunk with a conflict
    // (squared distances and dists are non-negative: compared as bit patterns).
    for (int t0 = 0; t0 < T; t0 += MM_TCHUNK) {
        const int t1 = t0 + MM_TCHUNK < T ? t0 + MM_TCHUNK : T;
        for (int w = tid; w < (t1 - t0) * t1; w += blockDim.x) {
            const int t = t0 + w / t1, s = w - (w / t1) * t1;
            if (s < t) {
                const double s2 = sqdist_rn(a.x + (long long)si[t] * a.d, a.x + (long long)si[s] * a.d, a.d);
                if (__double_as_longlong(s2) < sk[t]) atomicMin(&s_first_conflict, t);
            }
        }
        __syncthreads();
        if (s_first_conflict < t1) break;
    }
    const int p = s_first_conflict < T ? s_first_conflict : T;
    for (int t = tid; t < p; t += blockDim.x) {
        const int i = si[t];
        a.order[k + t] = i;
        a.acc_idx[t] = i;
        const double r2 = __longlong_as_double(sk[t]);
        a.acc_r2[t] = r2;
        a.dist[i] = -1.0;
        // cells within sqrt(dist) of the point, one cell of margin on each side
        const double R = sqrt(r2);
        long long cnt = 1;
        for (int q = 0; q < 3; ++q) {
            int c0 = 0, c1 = 0;
            if (q < a.d) {
                const double v = a.x[(long long)i * a.d + q];
                c0 = cell_coord(v - R, a.lo[q], a.h, a.nc[q]) - 1;
                c1 = cell_coord(v + R, a.lo[q], a.h, a.nc[q]) + 1;
                c0 = c0 < 0 ? 0 : c0;
                c1 = c1 >= a.nc[q] ? a.nc[q] - 1 : c1;
            }
            a.acc_box[t * 6 + q] = c0;
            a.acc_box[t * 6 + 3 + q] = c1;
            cnt *= (c1 - c0 + 1);
        }
        a.acc_work[t + 1] = cnt;
    }
    // the pool keeps its sorted remainder
    for (int t = tid; t < np - p; t += blockDim.x) a.pool[t] = si[p + t];
    __syncthreads();
    if (tid == 0) {
        a.acc_work[0] = 0;
        for (int t = 0; t < p; ++t) a.acc_work[t + 1] += a.acc_work[t];
        ctl->total_work = a.acc_work[p];
        ctl->nacc = p;
        ctl->pool_n = np - p;
        ctl->k = k + p;
        ctl->mode = MODE_UPDATE;
    }
    __syncthreads();
}

// Phase B (all blocks): the accepted points lower the dist of the points around them.
__device__ void mm_phase_b(const MMArgs& a) {
    const MMCtl* ctl = a.ctl;
    const int nacc = *(volatile const int*)&ctl->nacc;
    const long long W = *(volatile const long long*)&ctl->total_work;
    const long long G = (long long)gridDim.x * blockDim.x;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < W; w += G) {
        int lo = 0, hi = nacc - 1;               // accepted point s: acc_work[s] <= w < acc_work[s+1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldcg(a.acc_work + mid) <= w) lo = mid; else hi = mid - 1;
        }
        const int s = lo;
        int bx[6];
        for (int q = 0; q < 6; ++q) bx[q] = __ldcg(a.acc_box + s * 6 + q);
        long long r = w - __ldcg(a.acc_work + s);
        const int n0 = bx[3] - bx[0] + 1, n1 = bx[4] - bx[1] + 1;
        const int c0 = bx[0] + (int)(r % n0);
        r /= n0;
        const int c1 = bx[1] + (int)(r % n1);
        const int c2 = bx[2] + (int)(r / n1);
        const int cell = (c2 * a.nc[1] + c1) * a.nc[0] + c0;
        const double* xs = a.x + (long long)__ldcg(a.acc_idx + s) * a.d;
        for (int t = a.cell_start[cell]; t < a.cell_start[cell + 1]; ++t) {
            const int u = a.cell_items[t];
            // compared as bit patterns (non-negative values order like their patterns)
            const long long du = __ldcg(reinterpret_cast<const long long*>(a.dist) + u);
            if (du <= 0) continue;               // selected (-1), or already at 0
            const long long s2 = __double_as_longlong(sqdist_rn(a.x + (long long)u * a.d, xs, a.d));
            if (s2 < du) atomicMin(reinterpret_cast<long long*>(a.dist + u), s2);
        }
    }
}

// Rebuild (all blocks): threshold key so that at most MM_PMAX unselected points are at or
// above it, then the pool = those points.
__device__ void mm_rebuild(const MMArgs& a) {
    MMCtl* ctl = a.ctl;
    __shared__ unsigned long long s_max;
    __shared__ int s_cnt;
    const long long G = (long long)gridDim.x * blockDim.x;
    const long long g0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) { ctl->maxbits = 0ull; ctl->pool_n = 0; }
    if (grid_barrier(ctl)) return;
    if (threadIdx.x == 0) s_max = 0ull;
    __syncthreads();
    unsigned long long mb = 0ull;
    for (long long i = g0; i < a.n; i += G) {
        const double v = __ldcg(a.dist + i);
        if (v >= 0.0) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(v);
            mb = b > mb ? b : mb;
        }
    }
    atomicMax(&s_max, mb);
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(&ctl->maxbits, s_max);
    if (grid_barrier(ctl)) return;
    const double M = __longlong_as_double((long long)*(volatile unsigned long long*)&ctl->maxbits);
    // threshold dist: alpha M, alpha raised (towards 1) until at most MM_PMAX points reach
    // it; at alpha = 1 with more than MM_PMAX ties at the largest dist, the tie rule below
    bool tie = false;
    for (int trial = 0; trial < 80; ++trial) {
        const double thr = *(volatile double*)&ctl->alpha * M;
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->count = 0;
        if (grid_barrier(ctl)) return;
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        int c = 0;
        for (long long i = g0; i < a.n; i += G) {
            const double v = __ldcg(a.dist + i);
            c += (v >= 0.0 && v >= thr) ? 1 : 0;
        }
        atomicAdd(&s_cnt, c);
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&ctl->count, s_cnt);
        if (grid_barrier(ctl)) return;
        const int cnt = *(volatile int*)&ctl->count;
        const double al = *(volatile double*)&ctl->alpha;
        const bool accept = cnt <= MM_PMAX || thr == M;
        tie = cnt > MM_PMAX;
        if (grid_barrier(ctl)) return;      // everyone has read count and alpha
        if (accept) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const double na = 0.5 * (al + 1.0);
            ctl->alpha = (na * M > al * M && na < 1.0) ? na : 1.0;   // 1 once no progress is left
        }
        if (grid_barrier(ctl)) return;
    }
    if (!tie) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctl->thr_d = *(volatile double*)&ctl->alpha * M;
            ctl->thr_i = LLONG_MAX;
            // the next rebuild starts a little lower, so that pools do not shrink over time
            ctl->alpha = 0.75 * ctl->alpha;
        }
    } else {
        // ties at the largest dist: the MM_PMAX lowest indices among them (blocks take
        // contiguous index ranges; counts per block, then the cut inside one block)
        const long long per = (a.n + gridDim.x - 1) / gridDim.x;
        const long long b0 = (long long)blockIdx.x * per, b1 = b0 + per < a.n ? b0 + per : a.n;
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        int c = 0;
        for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) c += (__ldcg(a.dist + i) == M) ? 1 : 0;
        atomicAdd(&s_cnt, c);
        __syncthreads();
        if (threadIdx.x == 0) a.blk_count[blockIdx.x] = s_cnt;
        if (grid_barrier(ctl)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            long long run = 0, cut = LLONG_MAX;
            for (int b = 0; b < (int)gridDim.x && cut == LLONG_MAX; ++b) {
                const long long bb0 = (long long)b * per, bb1 = bb0 + per < a.n ? bb0 + per : a.n;
                const int bc = __ldcg(a.blk_count + b);
                if (run + bc < MM_PMAX) { run += bc; continue; }
                for (long long i = bb0; i < bb1; ++i)
                    if (__ldcg(a.dist + i) == M && ++run == MM_PMAX) { cut = i; break; }
            }
            ctl->thr_d = M;
            ctl->thr_i = cut;
            ctl->alpha = 0.75;
        }
    }
    if (grid_barrier(ctl)) return;
    const double td = *(volatile double*)&ctl->thr_d;
    const long long ti = *(volatile long long*)&ctl->thr_i;
    for (long long i = g0; i < a.n; i += G) {
        const double v = __ldcg(a.dist + i);
        if (v >= 0.0 && (v > td || (v == td && i <= ti))) {
            const int slot = atomicAdd(&ctl->pool_n, 1);
            if (slot < MM_PMAX) a.pool[slot] = (int)i;
        }
    }
    if (grid_barrier(ctl)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0 && *(volatile int*)&ctl->pool_n > MM_PMAX) {
        ctl->pool_n = MM_PMAX;
        atomicExch(&ctl->err, 2);            // cannot happen: the count was checked
    }
}

__global__ void __launch_bounds__(MM_THREADS) k_mm_steps(MMArgs a) {
    MMCtl* ctl = a.ctl;
    __shared__ int s_mode;
    // every step accepts at least one point, or rebuilds the pool after which the next step
    // does: at most 2 n + 2 iterations
    for (long long guard = 0; guard < 2 * a.n + 16; ++guard) {
        // the mode is UPDATE (sort the pool and accept a prefix) or REBUILD here; it was
        // written before the last barrier, and every thread of a block sees one value
        if (threadIdx.x == 0) s_mode = *(volatile int*)&ctl->mode;
        __syncthreads();
        if (blockIdx.x == 0 && s_mode == MODE_UPDATE) mm_phase_a(a);
        if (grid_barrier(ctl)) break;
        if (threadIdx.x == 0) s_mode = *(volatile int*)&ctl->mode;
        __syncthreads();
        if (s_mode == MODE_DONE) break;
        if (s_mode == MODE_REBUILD) {
            mm_rebuild(a);
            __syncthreads();
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl->mode = MODE_UPDATE;
        } else {
            mm_phase_b(a);
        }
        if (grid_barrier(ctl)) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && *(volatile int*)&ctl->err == 0 && ctl->k < a.n) ctl->err = 3;
}

// bounding box: per-block minima and maxima of each coordinate (part: nblk x 6)
__global__ void k_mm_bbox(const double* __restrict__ x, long long n, int d, double* __restrict__ part) {
    __shared__ double smin[MM_THREADS], smax[MM_THREADS];
    for (int k = 0; k < d; ++k) {
        double lo = 1.0 / 0.0, hi = -1.0 / 0.0;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            lo = fmin(lo, x[i * d + k]);
            hi = fmax(hi, x[i * d + k]);
        }
        smin[threadIdx.x] = lo;
        smax[threadIdx.x] = hi;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) {
                smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
                smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            part[(size_t)blockIdx.x * 6 + k] = smin[0];
            part[(size_t)blockIdx.x * 6 + 3 + k] = smax[0];
        }
        __syncthreads();
    }
}

}  // namespace

int maxmin_blocks(int nsm) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mm_steps, MM_THREADS, 0) != cudaSuccess ||
        per_sm < 1)
        return 0;
    return nsm * (per_sm < 2 ? per_sm : 2);
}

cudaError_t launch_maxmin_bbox(const double* x, long long n, int d, int nblk, double* part,
                               cudaStream_t st) {
    k_mm_bbox<<<nblk, MM_THREADS, 0, st>>>(x, n, d, part);
    return cudaGetLastError();
}

// uniform grid over the bounding box with about two points per cell (at most 4 n + 64 cells)
void maxmin_grid(long long n, int d, const double* lo, const double* hi, double* h_out, int* nc,
                 long long* ncell) {
    double ext[3] = {1.0, 1.0, 1.0}, vol = 1.0;
    for (int k = 0; k < d; ++k) {
        ext[k] = hi[k] - lo[k];
        if (!(ext[k] > 0.0)) ext[k] = 1e-300;
        vol *= ext[k];
    }
    const double cells = (double)n / 2.0 > 1.0 ? (double)n / 2.0 : 1.0;
    double h = pow(vol / cells, 1.0 / d);
    if (!(h > 0.0) || !std::isfinite(h)) h = 1.0;
    long long nce = 1;
    for (int k = 0; k < 3; ++k) {
        long long c = 1;
        if (k < d) {
            const double f = ceil(ext[k] / h);
            c = f < 1.0 ? 1 : (f > 1e7 ? 10000000 : (long long)f);
        }
        nc[k] = (int)c;
        nce *= c;
    }
    while (nce > 4 * n + 64) {          // degenerate extents: coarser cells
        h *= 2.0;
        nce = 1;
        for (int k = 0; k < d; ++k) {
            const double f = ceil(ext[k] / h);
            nc[k] = f < 1.0 ? 1 : (int)f;
            nce *= nc[k];
        }
    }
    *h_out = h;
    *ncell = nce;
}

size_t maxmin_scratch_bytes(long long n, int nblocks, long long ncell) {
    // dist, cell_of, items (n each), start/counts/cursor (ncell + 1 each), pool, accepted
    // lists, block counts, partial sums and the control block
    size_t b = 0;
    auto add = [&](size_t bytes) { b += (bytes + 255) / 256 * 256; };
    add(sizeof(double) * n);
    add(sizeof(int) * n);
    add(sizeof(int) * n);
    add(sizeof(int) * (ncell + 1));
    add(sizeof(int) * (ncell + 1));
    add(sizeof(int) * (ncell + 1));
    add(sizeof(int) * MM_PMAX);
    add(sizeof(int) * MM_TACC);
    add(sizeof(double) * MM_TACC);
    add(sizeof(int) * MM_TACC * 6);
    add(sizeof(long long) * (MM_TACC + 1));
    add(sizeof(int) * nblocks);
    add(sizeof(double) * 3 * nblocks + sizeof(double) * nblocks + sizeof(long long) * nblocks);
    add(sizeof(MMCtl));
    return b;
}

cudaError_t launch_maxmin(const double* x, long long n, int d, const double* lo, int nblk,
                          double h, const int* nc, long long ncell, void* scratch,
                          size_t scratch_bytes, long long* order, int* err_out, cudaStream_t st) {
    if (n < 1 || d < 1 || d > 3 || nblk < 1) return cudaErrorInvalidValue;
    if (ncell > (long long)INT_MAX / 2 || maxmin_scratch_bytes(n, nblk, ncell) > scratch_bytes)
        return cudaErrorInvalidValue;
    MMArgs a;
    for (int k = 0; k < 3; ++k) {
        a.nc[k] = nc[k];
        a.lo[k] = k < d ? lo[k] : 0.0;
    }
    char* p = static_cast<char*>(scratch);
    auto take = [&](size_t bytes) { char* r = p; p += (bytes + 255) / 256 * 256; return r; };
    a.x = x;
    a.n = n;
    a.d = d;
    a.h = h;
    a.dist = reinterpret_cast<double*>(take(sizeof(double) * n));
    int* cell_of = reinterpret_cast<int*>(take(sizeof(int) * n));
    int* items = reinterpret_cast<int*>(take(sizeof(int) * n));
    int* start = reinterpret_cast<int*>(take(sizeof(int) * (ncell + 1)));
    int* counts = reinterpret_cast<int*>(take(sizeof(int) * (ncell + 1)));
    int* cursor = reinterpret_cast<int*>(take(sizeof(int) * (ncell + 1)));
    a.pool = reinterpret_cast<int*>(take(sizeof(int) * MM_PMAX));
    a.acc_idx = reinterpret_cast<int*>(take(sizeof(int) * MM_TACC));
    a.acc_r2 = reinterpret_cast<double*>(take(sizeof(double) * MM_TACC));
    a.acc_box = reinterpret_cast<int*>(take(sizeof(int) * MM_TACC * 6));
    a.acc_work = reinterpret_cast<long long*>(take(sizeof(long long) * (MM_TACC + 1)));
    a.blk_count = reinterpret_cast<int*>(take(sizeof(int) * nblk));
    double* part = reinterpret_cast<double*>(take(sizeof(double) * 3 * nblk + sizeof(double) * nblk +
                                                  sizeof(long long) * nblk));
    double* bestd = part + 3 * nblk;
    long long* besti = reinterpret_cast<long long*>(bestd + nblk);
    a.ctl = reinterpret_cast<MMCtl*>(take(sizeof(MMCtl)));
    a.order = order;
    a.cell_start = start;
    a.cell_items = items;
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (ncell + 1), st);
    if (e != cudaSuccess) return e;
    k_mm_centroid_partial<<<nblk, MM_THREADS, 0, st>>>(x, n, d, part);
    k_mm_first_partial<<<nblk, MM_THREADS, 0, st>>>(x, n, d, part, nblk, bestd, besti);
    k_mm_init<<<nblk, MM_THREADS, 0, st>>>(x, n, d, bestd, besti, nblk, a.dist, order, a.ctl);
    k_mm_cells<<<nblk, MM_THREADS, 0, st>>>(x, n, d, a.nc[0], a.nc[1], a.nc[2], a.lo[0], a.lo[1],
                                            a.lo[2], h, cell_of, counts);
    k_mm_scan<<<1, MM_THREADS, 0, st>>>(counts, (int)ncell, start, cursor);
    k_mm_fill<<<nblk, MM_THREADS, 0, st>>>(n, cell_of, cursor, items);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (n > 1) {
        void* params[] = {&a};
        e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_mm_steps), dim3(nblk),
                                        dim3(MM_THREADS), params, 0, st);
        if (e != cudaSuccess) return e;
    }
    // the step kernel's error flag, for the caller
    return cudaMemcpyAsync(err_out, &a.ctl->err, sizeof(int), cudaMemcpyDeviceToDevice, st);
}

}  // namespace vg
