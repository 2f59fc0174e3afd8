// vg_nn.cu -- nearest-neighbour search on the device: for each observation i of an
// ordering, its m nearest among the observations 0..i-1 (the NNarray of Sec. 2.1 and
// Algorithm 1's input; the paper computes it on the CPU and names a GPU version as future
// work); and, for prediction, the m nearest observations of each query location.
//
// Definition (exact): neighbours of i = the m smallest keys (d2(i, j), j) over j < i in
// lexicographic order, d2 = sum over coordinates, in order, of (x_ik - x_jk)^2 in FP64 with
// every product and sum rounded separately (no fused multiply-add), so that any FP64
// implementation ranks identically; nearest first; rows of i < m padded with -1.
//
// Kernels:
//   k_nn_bbox     bounding box of the first two coordinates (one block, fixed-order reduction)
//   k_nn_cells    cell of every observation on a G x G grid over that box; cell counts
//   k_nn_scan     exclusive scan of the counts (one block)
//   k_nn_scatter  observations listed by cell (order within a cell is irrelevant)
//   k_nn_search   one warp per observation: brute force over j < i while i is small,
//                 else rings of cells around i's cell, the lanes taking cells of a ring in
//                 turn; candidates with j < i are appended (warp ballot) to a per-warp
//                 buffer in shared memory that is bitonic-sorted and cut to the m best when
//                 it fills and after each ring; the search stops once the m-th best d2 is
//                 below the squared distance to the unvisited rings, with one ring of
//                 margin against rounding in the cell assignment.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>

#include "vg_internal.h"

namespace vg {

constexpr int NN_WARPS = 4;      // warps (observations) per block of the search
constexpr int NN_CAP = 512;      // candidate buffer per warp (power of two)

struct NNGrid {
    double x0, y0, hx, hy;       // origin and cell sizes
    int gx, gy;
};

__device__ __forceinline__ double nn_d2(const double* a, const double* b, int d) {
    double s = __dmul_rn(__dsub_rn(a[0], b[0]), __dsub_rn(a[0], b[0]));
    for (int k = 1; k < d; ++k) {
        const double t = __dsub_rn(a[k], b[k]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

__device__ __forceinline__ bool key_less(double da, int ja, double db, int jb) {
    return da < db || (da == db && ja < jb);
}

__global__ void __launch_bounds__(1024) k_nn_bbox(const double* __restrict__ x, long long n, int d,
                                                  int G, NNGrid* grid) {
    __shared__ double red[4][1024];
    const int t = threadIdx.x;
    double v[4] = {INFINITY, -INFINITY, INFINITY, -INFINITY};
    for (long long i = t; i < n; i += blockDim.x) {
        const double a = x[i * d], b = d > 1 ? x[i * d + 1] : 0.0;
        v[0] = fmin(v[0], a); v[1] = fmax(v[1], a);
        v[2] = fmin(v[2], b); v[3] = fmax(v[3], b);
    }
    for (int k = 0; k < 4; ++k) red[k][t] = v[k];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) {
            red[0][t] = fmin(red[0][t], red[0][t + o]);
            red[1][t] = fmax(red[1][t], red[1][t + o]);
            red[2][t] = fmin(red[2][t], red[2][t + o]);
            red[3][t] = fmax(red[3][t], red[3][t + o]);
        }
        __syncthreads();
    }
    if (t == 0) {
        NNGrid g;
        g.gx = G;
        g.gy = d > 1 ? G : 1;
        g.x0 = red[0][0];
        g.y0 = red[2][0];
        const double wx = red[1][0] - red[0][0], wy = red[3][0] - red[2][0];
        g.hx = wx > 0.0 ? wx / g.gx : 1.0;
        g.hy = wy > 0.0 ? wy / g.gy : 1.0;
        *grid = g;
    }
}

__device__ __forceinline__ void nn_cell_of(const NNGrid& g, const double* p, int d, int& cx, int& cy) {
    cx = (int)floor((p[0] - g.x0) / g.hx);
    cy = d > 1 ? (int)floor((p[1] - g.y0) / g.hy) : 0;
    cx = cx < 0 ? 0 : (cx >= g.gx ? g.gx - 1 : cx);
    cy = cy < 0 ? 0 : (cy >= g.gy ? g.gy - 1 : cy);
}

__global__ void k_nn_cells(const double* __restrict__ x, long long n, int d,
                           const NNGrid* __restrict__ grid, int* __restrict__ cell,
                           int* __restrict__ count) {
    const NNGrid g = *grid;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int cx, cy;
        nn_cell_of(g, x + i * d, d, cx, cy);
        const int c = cy * g.gx + cx;
        cell[i] = c;
        atomicAdd(count + c, 1);
    }
}

// Exclusive scan of count[0..nc) into start[0..nc] (start[nc] = total) and cursor = start.
__global__ void __launch_bounds__(1024) k_nn_scan(const int* __restrict__ count, int nc,
                                                  int* __restrict__ start, int* __restrict__ cursor) {
    __shared__ long long part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int per = (nc + T - 1) / T;
    const int a = t * per, b = min(nc, a + per);
    long long s = 0;
    for (int c = a; c < b; ++c) s += count[c];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {   // inclusive Hillis-Steele scan of the chunk sums
        const long long v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = t > 0 ? part[t - 1] : 0;
    for (int c = a; c < b; ++c) {
        start[c] = (int)run;
        cursor[c] = (int)run;
        run += count[c];
    }
    if (t == T - 1) start[nc] = (int)part[T - 1];
}

__global__ void k_nn_scatter(const int* __restrict__ cell, long long n, int* __restrict__ cursor,
                             int* __restrict__ items) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        items[atomicAdd(cursor + cell[i], 1)] = (int)i;
}

// Bitonic sort of the warp's buffer (cnt entries, padded to a power of two) and cut to m.
__device__ void nn_sort_cut(double* bd, int* bj, int& cnt, int m, int lane) {
    int P = 1;
    while (P < cnt) P <<= 1;
    for (int t = cnt + lane; t < P; t += 32) { bd[t] = INFINITY; bj[t] = INT_MAX; }
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int t = lane; t < P; t += 32) {
                const int u = t ^ jj;
                if (u > t) {
                    const bool up = (t & k) == 0;
                    const bool gt = key_less(bd[u], bj[u], bd[t], bj[t]);  // buf[t] > buf[u]
                    if (gt == up) {
                        const double td = bd[t]; bd[t] = bd[u]; bd[u] = td;
                        const int tj = bj[t]; bj[t] = bj[u]; bj[u] = tj;
                    }
                }
            }
            __syncwarp();
        }
    }
    if (cnt > m) cnt = m;
}

// ordered = 1: queries are the reference points themselves, candidates j < i, rows
// [i, neighbours] (m + 1 columns).  ordered = 0: queries qx (nq of them) against all n
// reference points, rows [neighbours] (m columns).
__global__ void __launch_bounds__(NN_WARPS * 32) k_nn_search(
    const double* __restrict__ x, long long n, int d, int m, const NNGrid* __restrict__ grid,
    const int* __restrict__ start, const int* __restrict__ items, long long brute_upto,
    int32_t* __restrict__ NN, const double* __restrict__ qx, long long nq, int ordered) {
    __shared__ double s_d[NN_WARPS][NN_CAP];
    __shared__ int s_j[NN_WARPS][NN_CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double* bd = s_d[w];
    int* bj = s_j[w];
    const NNGrid g = *grid;
    const int W = ordered ? m + 1 : m;
    const double hmin = fmin(g.hx, g.hy);
    const long long nw = (long long)gridDim.x * NN_WARPS;
    const long long nquery = ordered ? n : nq;
    for (long long i = blockIdx.x * (long long)NN_WARPS + w; i < nquery; i += nw) {
        const double* xi = ordered ? x + i * d : qx + i * d;
        const long long lim = ordered ? i : n;   // candidates j < lim
        int cnt = 0;
        double thr_d = INFINITY;   // key of the current m-th best (when cnt == m after a cut)
        int thr_j = INT_MAX;
        // offers one candidate per lane (valid lanes only) to the buffer
        auto offer = [&](bool valid, double d2, int j) {
            bool take = valid && key_less(d2, j, thr_d, thr_j);
            if (cnt + 32 > NN_CAP) {
                nn_sort_cut(bd, bj, cnt, m, lane);
                if (cnt == m) { thr_d = bd[m - 1]; thr_j = bj[m - 1]; }
                take = take && key_less(d2, j, thr_d, thr_j);
            }
            const unsigned mask = __ballot_sync(0xffffffffu, take);
            if (take) {
                const int pos = cnt + __popc(mask & ((1u << lane) - 1u));
                bd[pos] = d2;
                bj[pos] = j;
            }
            cnt += __popc(mask);
            __syncwarp();
        };
        if (m > 0 && lim > 0) {
            if (lim <= brute_upto) {
                for (long long j0 = 0; j0 < lim; j0 += 32) {
                    const long long j = j0 + lane;
                    const bool valid = j < lim;
                    offer(valid, valid ? nn_d2(xi, x + j * d, d) : 0.0, (int)j);
                }
            } else {
                int cx, cy;
                nn_cell_of(g, xi, d, cx, cy);
                const int rmax = max(g.gx, g.gy);
                for (int r = 0; r <= rmax; ++r) {
                    // the cells at Chebyshev distance r: lane l takes cells l, l+32, ...
                    const int ncell = r == 0 ? 1 : 8 * r;
                    for (int c0 = 0; c0 < ncell; c0 += 32) {
                        const int ci = c0 + lane;
                        int ccx = 0, ccy = 0, beg = 0, end = 0;
                        if (ci < ncell) {
                            if (r == 0) { ccx = cx; ccy = cy; }
                            else if (ci < 2 * r + 1) { ccx = cx - r + ci; ccy = cy - r; }
                            else if (ci < 4 * r + 2) { ccx = cx - r + (ci - 2 * r - 1); ccy = cy + r; }
                            else if (ci < 6 * r + 1) { ccx = cx - r; ccy = cy - r + 1 + (ci - 4 * r - 2); }
                            else { ccx = cx + r; ccy = cy - r + 1 + (ci - 6 * r - 1); }
                            if (ccx >= 0 && ccx < g.gx && ccy >= 0 && ccy < g.gy) {
                                const int c = ccy * g.gx + ccx;
                                beg = start[c];
                                end = start[c + 1];
                            }
                        }
                        // walk the lanes' cells in step, one point per lane per round
                        for (;;) {
                            const bool more = beg < end;
                            if (__ballot_sync(0xffffffffu, more) == 0u) break;
                            int j = -1;
                            double d2 = 0.0;
                            bool valid = false;
                            if (more) {
                                j = items[beg++];
                                valid = j < lim;
                                if (valid) d2 = nn_d2(xi, x + (long long)j * d, d);
                            }
                            offer(valid, d2, j);
                        }
                    }
                    if (cnt >= m) {
                        nn_sort_cut(bd, bj, cnt, m, lane);
                        thr_d = bd[m - 1];
                        thr_j = bj[m - 1];
                    }
                    // unvisited points lie in rings >= r + 1: farther than r cells from i's
                    // cell; one ring of margin covers points assigned to a neighbouring cell
                    const double bound = (double)(r - 1) * hmin;
                    if (cnt == m && r >= 1 && thr_d < bound * bound) break;
                }
            }
            nn_sort_cut(bd, bj, cnt, m, lane);
        }
        int32_t* row = NN + i * W;
        if (ordered) {
            for (int k = lane; k < W; k += 32)
                row[k] = k == 0 ? (int32_t)i : (k - 1 < cnt ? (int32_t)bj[k - 1] : -1);
        } else {
            for (int k = lane; k < W; k += 32) row[k] = k < cnt ? (int32_t)bj[k] : -1;
        }
        __syncwarp();
    }
}

cudaError_t launch_ordered_nn(const double* x, long long n, int d, int m, int G, void* scratch,
                              int32_t* NN, cudaStream_t st, const double* qx, long long nq) {
    // scratch layout: NNGrid | cell[n] | count[G*G] | start[G*G+1] | cursor[G*G] | items[n]
    char* p = static_cast<char*>(scratch);
    NNGrid* grid = reinterpret_cast<NNGrid*>(p);
    p += 64;
    const long long nc = (long long)G * (d > 1 ? G : 1);
    int* cell = reinterpret_cast<int*>(p);       p += sizeof(int) * n;
    int* count = reinterpret_cast<int*>(p);      p += sizeof(int) * nc;
    int* start = reinterpret_cast<int*>(p);      p += sizeof(int) * (nc + 1);
    int* cursor = reinterpret_cast<int*>(p);     p += sizeof(int) * nc;
    int* items = reinterpret_cast<int*>(p);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * nc, st);
    if (e != cudaSuccess) return e;
    k_nn_bbox<<<1, 1024, 0, st>>>(x, n, d, G, grid);
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_nn_cells<<<blocks, 256, 0, st>>>(x, n, d, grid, cell, count);
    k_nn_scan<<<1, 1024, 0, st>>>(count, (int)nc, start, cursor);
    k_nn_scatter<<<blocks, 256, 0, st>>>(cell, n, cursor, items);
    // brute force while the candidates are few: below sqrt(m n) it is cheaper than rings
    const long long brute = (long long)std::max(2.0 * m, std::sqrt((double)m * (double)n));
    const int ordered = qx ? 0 : 1;
    const long long nquery = ordered ? n : nq;
    const long long sblocks = (nquery + NN_WARPS - 1) / NN_WARPS;
    k_nn_search<<<(unsigned)(sblocks < 65535LL * 8 ? sblocks : 65535LL * 8), NN_WARPS * 32, 0, st>>>(
        x, n, d, m, grid, start, items, brute, NN, qx, nq, ordered);
    return cudaGetLastError();
}

size_t ordered_nn_scratch_bytes(long long n, int d, int G) {
    const long long nc = (long long)G * (d > 1 ? G : 1);
    return 64 + sizeof(int) * (size_t)(2 * n + 3 * nc + 1);
}

}  // namespace vg
