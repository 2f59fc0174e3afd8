// vg_pass.cuh -- K1: the fused per-observation Vecchia pass, FP64.
//
// Algorithm 1 of the paper, one observation at a time per "group" of L lanes of a warp
// (L = 1, 2, 4, 8, 16 or 32 lanes per observation, chosen per block size).  The
// conditioning block of an observation lives in a shared-memory slot owned by its group;
// every step is done by the L lanes together:
//
//   gather      NNarray row -> block indices (neighbours reversed, observation last),
//               locations, y and X rows                              (Algorithm 1, l. 4-5)
//   assembly    lower triangle of the covariance, nugget on the diagonal       (l. 6)
//   factor      left-looking Cholesky; y and X ride along as extra rows, so the same
//               column sweep produces Liy = L^-1 y and LiX = L^-1 X            (l. 7-9)
//   terms       logdet_i, Liy[last], LiX[last, :]                              (l. 10-13)
//   derivative  b = last row of L^-1 (back substitution), g_j = dSigma_j b^T with each
//               pair (a, c) evaluated once (a conflict-free round-robin pair schedule lets
//               the lanes scatter into g without atomics), m_j = L^-1 g_j, then the dot
//               products that give dlogdet, dySy, dySX, dXSX and the information (l. 14-15,
//               written out from dL = L Phi(L^-1 dSigma L^-T))
//   accumulate  per-observation values into per-lane running sums (shared memory), then a
//               fixed-order block reduction into one partial record per block.
//
// FP64 on this GPU issues one warp instruction per 64 cycles per SM sub-partition whatever
// the number of active lanes, so the mapping keeps all 32 lanes busy: rows, pairs and
// vector entries are spread round-robin over the L lanes of a group, and each pivot costs
// an FP32 seed plus two short FP64 Newton steps instead of a square root and a division.
#pragma once
#include "vg_common.cuh"
#include "vg_matern.cuh"

namespace vg {

// sizes (in doubles) of the parts of one slot; K = m + 1
struct SlotLayout {
    int K, A, Y, inv, loc, bacc, b, G, D1, V, total;
    __host__ __device__ void init(int m, int d, int p, int cov, int nv) {
        K = m + 1;
        int Q = npair_derivs(cov) + 1;
        A = 0;
        Y = A + K * (K + 1) / 2;
        inv = Y + (1 + p) * K;
        loc = inv + K;
        bacc = loc + d * K;
        b = bacc + K;
        G = b + K;
        D1 = G + Q * K;
        V = D1 + (cov == COV_MATERN ? 0 : K * (K - 1) / 2);
        total = V + nv;
        total |= 1;  // odd stride spreads the slots of a warp over the shared-memory banks
    }
};

// Synchronises the lanes of a group and orders their shared-memory accesses.  Also
// issued for one-lane groups: it is then a memory barrier between the phases.
template <int L>
__device__ __forceinline__ void gsync(unsigned mask) {
    __syncwarp(mask);
}

// sums over the L lanes of a group (xor partners stay inside the group)
template <int L>
__device__ __forceinline__ double gsum(double v, unsigned mask) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}
template <int L>
__device__ __forceinline__ int gsum_i(int v, unsigned mask) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// Pair k of round r of the round-robin (circle) schedule on Nv = Kp or Kp+1 vertices.
// Within a round all pairs are vertex-disjoint.  Returns false for pairs with the dummy
// vertex (odd Kp).  The pair is returned with a > c.
__device__ __forceinline__ bool circle_pair(int Kp, int Nv, int r, int k, int& a, int& c) {
    int u, v;
    if (k == 0) { u = Nv - 1; v = r; }
    else {
        u = r + k; if (u >= Nv - 1) u -= Nv - 1;
        v = r - k; if (v < 0) v += Nv - 1;
    }
    if (u >= Kp || v >= Kp) return false;
    a = u > v ? u : v;
    c = u > v ? v : u;
    return true;
}

template <int COV, int L>
__global__ void __launch_bounds__(256) k_pass_fp64(PassArgs args) {
    extern __shared__ __align__(16) double smem[];
    constexpr int NG = npair_derivs(COV);
    constexpr int Q = NG + 1;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int gl = lane & (L - 1);
    const int grp = tid / L;
    const int ngrp = blockDim.x / L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (lane & ~(L - 1)));
    const int d = args.d, p = args.p, m = args.m;
    const int Kmax = m + 1;

    // ---- shared-memory carve-up: [Matern table][stat index table][acc][slots][int slots]
    double* sp = smem;
    const double* tab = args.mtab;
    if (COV == COV_MATERN && args.tab_in_smem) {
        for (int t = tid; t < MT_DOUBLES; t += blockDim.x) sp[t] = args.mtab[t];
        tab = sp;
        sp += MT_DOUBLES;
    }
    uint32_t* sidx = reinterpret_cast<uint32_t*>(sp);
    sp += (args.nstat + 1) / 2;
    double* acc = sp + (size_t)tid * args.acc_per_lane;
    sp += (size_t)blockDim.x * args.acc_per_lane;
    SlotLayout SL;
    SL.init(m, d, p, COV, args.nv);
    double* slot = sp + (size_t)grp * args.slot_stride;
    int* idx = reinterpret_cast<int*>(sp + (size_t)ngrp * args.slot_stride) + grp * Kmax;
    double* A = slot + SL.A;
    double* Yg = slot + SL.Y;
    double* invd = slot + SL.inv;
    double* loc = slot + SL.loc;
    double* bacc = slot + SL.bacc;
    double* bv = slot + SL.b;
    double* G = slot + SL.G;
    double* D1 = slot + SL.D1;
    double* V = slot + SL.V;

    // ---- per-observation value vector V and the record formulas (see RecLayout)
    //   V[0] = 1, V[1] = 0, V[2] = logdet_i, V[3] = ell, V[4..4+p) = x,
    //   V[vb_j + 0] = md_j, +1 = dell_j, +2.. = dx_j (p), +2+p = -md_j/2,
    //   then mm_jl = m_j . m_l for j <= l.
    // Record entry t = V[u1] V[v1] + V[u2] V[v2], indices packed in sidx[t].
    RecLayout RL;
    RL.init(p, Q);
    const int vb0 = 4 + p, vstep = 3 + p, vmm = vb0 + Q * vstep;
    if (tid == 0) {
        auto pk = [](int a, int b, int c, int e) {
            return (uint32_t)a | ((uint32_t)b << 8) | ((uint32_t)c << 16) | ((uint32_t)e << 24);
        };
        int t = 0;
        sidx[t++] = pk(2, 0, 1, 1);                       // logdet
        sidx[t++] = pk(3, 3, 1, 1);                       // ySy
        for (int a = 0; a < p; ++a)
            for (int b = a; b < p; ++b) sidx[t++] = pk(4 + a, 4 + b, 1, 1);  // XSX
        for (int a = 0; a < p; ++a) sidx[t++] = pk(3, 4 + a, 1, 1);          // ySX
        for (int j = 0; j < Q; ++j) {
            int vb = vb0 + j * vstep;
            sidx[t++] = pk(vb, 0, 1, 1);                  // dlogdet_j
            sidx[t++] = pk(3, vb + 1, vb + 1, 3);         // dySy_j = 2 ell dell_j
            for (int a = 0; a < p; ++a) sidx[t++] = pk(vb + 1, 4 + a, 3, vb + 2 + a);  // dySX
            for (int a = 0; a < p; ++a)
                for (int b = a; b < p; ++b)
                    sidx[t++] = pk(vb + 2 + a, 4 + b, 4 + a, vb + 2 + b);           // dXSX
        }
        int mm = vmm;
        for (int j = 0; j < Q; ++j)
            for (int l = j; l < Q; ++l) {
                sidx[t++] = pk(mm++, 0, vb0 + j * vstep, vb0 + l * vstep + 2 + p);  // info
            }
    }
    for (int k = 0; k < args.acc_per_lane; ++k) acc[k] = 0.0;

    // ---- covariance parameters
    const double* th = args.covparms;
    const double sig2 = th[0];
    const double tau2 = th[nparms(COV) - 1];
    bool ok = sig2 > 0.0 && tau2 > 0.0 && th[1] > 0.0 && th[2] > 0.0 &&
              isfinite(sig2) && isfinite(tau2) && isfinite(th[1]) && isfinite(th[2]);
    if (COV != COV_EXP) ok = ok && th[3] > 0.0 && isfinite(th[3]);
    if (COV == COV_MATERN) ok = ok && th[2] >= 0.05 && th[2] <= 20.0;
    if (!ok) {
        if (blockIdx.x == 0 && tid == 0) report(args.status, args.bad, ST_ARG, -1);
    }
    const double diagC = sig2 * (1.0 + tau2);
    // EXP: rho = th[1]; MATERN: rho = th[1], nu = th[2]; ST: rho_s = th[1], rho_t = th[2]
    const double inv_r1 = 1.0 / th[1];
    const double inv_r2 = (COV == COV_ST) ? 1.0 / th[2] : 1.0;
    double m_psi = 0.0, m_lg = 0.0;
    if (COV == COV_MATERN && ok) { m_psi = dev_digamma(th[2]); m_lg = lgamma(th[2]); }
    __syncthreads();

    const long long n = args.n;
    const long long gstride = (long long)gridDim.x * ngrp;
    for (long long i = (long long)blockIdx.x * ngrp + grp; ok && i < n; i += gstride) {
        // ---------------- gather ----------------
        const int32_t* row = args.NN + i * (long long)(m + 1);
        int cnt = 0, badrow = 0;
        for (int c = gl; c <= m; c += L) {
            int v = row[c];
            if (c == 0) badrow |= (v != (int)i);
            else if (v >= 0) {
                cnt++;
                badrow |= (v >= i) | (c >= 2 && row[c - 1] < 0);
            } else if (v != -1) badrow = 1;
        }
        cnt = gsum_i<L>(cnt, gmask);
        badrow = gsum_i<L>(badrow, gmask);
        if (badrow) {
            if (gl == 0) report(args.status, args.bad, ST_ARG, i);
            continue;
        }
        const int Kp = cnt + 1;
        for (int a = gl; a < Kp; a += L) {
            int j = row[Kp - 1 - a];
            idx[a] = j;
            // coordinates are stored divided by their range parameter, so that squared
            // distances come out already scaled
            for (int k = 0; k < d; ++k)
                loc[k * Kmax + a] = args.locs[(long long)j * d + k] * ((COV == COV_ST && k == 2) ? inv_r2 : inv_r1);
            Yg[a] = args.y[j];
            for (int t = 0; t < p; ++t) Yg[(1 + t) * Kmax + a] = args.X[(long long)j * p + t];
        }
        gsync<L>(gmask);

        // ---------------- covariance assembly (packed lower triangle) ----------------
        const int ntri = Kp * (Kp + 1) / 2;
        for (int e = gl; e < ntri; e += L) {
            int a = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
            while (a * (a + 1) / 2 > e) --a;
            while ((a + 1) * (a + 2) / 2 <= e) ++a;
            int c = e - a * (a + 1) / 2;
            double C;
            if (a == c) {
                C = diagC;
            } else if (COV == COV_EXP) {
                double s = 0.0;
                for (int k = 0; k < d; ++k) {
                    double t = loc[k * Kmax + a] - loc[k * Kmax + c];
                    s = fma(t, t, s);
                }
                double x = sqrt(s);
                double ex = sig2 * exp(-x);
                C = ex;
                D1[a * (a - 1) / 2 + c] = ex * x;          // rho dC/drho
            } else if (COV == COV_ST) {
                double t0 = loc[a] - loc[c];
                double t1 = loc[Kmax + a] - loc[Kmax + c];
                double t2 = loc[2 * Kmax + a] - loc[2 * Kmax + c];
                double u = fma(t0, t0, fma(t1, t1, t2 * t2));
                double D = sqrt(u);
                double ex = sig2 * exp(-D);
                C = ex;
                D1[a * (a - 1) / 2 + c] = D > 0.0 ? ex / D : 0.0;
            } else {  // Matern
                double s = 0.0;
                for (int k = 0; k < d; ++k) {
                    double t = loc[k * Kmax + a] - loc[k * Kmax + c];
                    s = fma(t, t, s);
                }
                C = sig2 * matern_F0(tab, s, th[2], m_psi, m_lg);
            }
            A[e] = C;
        }
        gsync<L>(gmask);

        // ---------------- Cholesky + forward solves of y and X ----------------
        // combined rows: r < Kp -> matrix row r (packed), r >= Kp -> augmented row r - Kp
        const int R = Kp + 1 + p;
        bool pd = true;
        for (int c = 0; c < Kp; ++c) {
            const double* Lc = A + c * (c + 1) / 2;
            const int r0 = c + ((gl - c) & (L - 1));
            for (int r = r0; r < R; r += L) {
                double* Rr = r < Kp ? A + r * (r + 1) / 2 : Yg + (r - Kp) * Kmax;
                double v0 = Rr[c], v1 = 0.0;
                int s = 0;
                for (; s + 1 < c; s += 2) {
                    v0 = fma(-Rr[s], Lc[s], v0);
                    v1 = fma(-Rr[s + 1], Lc[s + 1], v1);
                }
                if (s < c) v0 = fma(-Rr[s], Lc[s], v0);
                Rr[c] = v0 + v1;
            }
            gsync<L>(gmask);
            const double vc = Lc[c];
            if (!(vc > 0.0) || !isfinite(vc)) { pd = false; break; }
            const double ic = rsqrt_newton(vc);
            if (r0 == c) invd[c] = ic;
            for (int r = (r0 == c ? r0 + L : r0); r < R; r += L) {
                double* Rr = r < Kp ? A + r * (r + 1) / 2 : Yg + (r - Kp) * Kmax;
                Rr[c] *= ic;
            }
            gsync<L>(gmask);
        }
        if (!pd) {
            if (gl == 0) report(args.status, args.bad, ST_NOT_PD, i);
            gsync<L>(gmask);
            continue;
        }
        const int last = Kp - 1;

        // ---------------- b = last row of L^-1 (L^T b^T = e_last) ----------------
        for (int a = gl; a < Kp; a += L) bacc[a] = (a == last) ? 1.0 : 0.0;
        gsync<L>(gmask);
        for (int c = last; c >= 0; --c) {
            const double bc = bacc[c] * invd[c];
            if (((c - gl) & (L - 1)) == 0) bv[c] = bc;
            const double* Lr = A + c * (c + 1) / 2;
            for (int a = gl; a < c; a += L) bacc[a] = fma(-Lr[a], bc, bacc[a]);
            gsync<L>(gmask);
        }

        // ---------------- g_j = dSigma_j b^T ----------------
        // g for the pair-derivative parameters starts at 0; the nugget one is sigma2 b.
        for (int a = gl; a < Kp; a += L) {
#pragma unroll
            for (int j = 0; j < NG; ++j) G[j * Kmax + a] = 0.0;
            G[NG * Kmax + a] = sig2 * bv[a];
        }
        gsync<L>(gmask);
        {
            const int Nv = (Kp & 1) ? Kp + 1 : Kp;
            const int npr = Nv / 2;
            for (int r = 0; r < Nv - 1; ++r) {
                for (int k = gl; k < npr; k += L) {
                    int a, c;
                    if (!circle_pair(Kp, Nv, r, k, a, c)) continue;
                    double dv[NG];
                    if (COV == COV_EXP) {
                        dv[0] = D1[a * (a - 1) / 2 + c] * inv_r1;
                    } else if (COV == COV_ST) {
                        double t0 = loc[a] - loc[c];
                        double t1 = loc[Kmax + a] - loc[Kmax + c];
                        double t2 = loc[2 * Kmax + a] - loc[2 * Kmax + c];
                        double w = D1[a * (a - 1) / 2 + c];
                        dv[0] = w * fma(t0, t0, t1 * t1) * inv_r1;
                        if (NG > 1) dv[NG - 1] = w * t2 * t2 * inv_r2;
                    } else {
                        double s = 0.0;
                        for (int kk = 0; kk < d; ++kk) {
                            double t = loc[kk * Kmax + a] - loc[kk * Kmax + c];
                            s = fma(t, t, s);
                        }
                        double F1, F2;
                        matern_F12(tab, s, th[2], m_psi, m_lg, F1, F2);
                        dv[0] = sig2 * F1 * inv_r1;
                        if (NG > 1) dv[NG - 1] = sig2 * F2;
                    }
                    const double ba = bv[a], bc = bv[c];
#pragma unroll
                    for (int j = 0; j < NG; ++j) {
                        G[j * Kmax + a] = fma(dv[j], bc, G[j * Kmax + a]);
                        G[j * Kmax + c] = fma(dv[j], ba, G[j * Kmax + c]);
                    }
                }
                gsync<L>(gmask);
            }
        }

        // ---------------- m_j = L^-1 g_j (in place, column sweep) ----------------
        // Column c: every lane reads the finished residual g_j[c] and scales it; after a
        // group barrier the owner of c stores m_j[c] and each lane updates its rows a > c.
        for (int c = 0; c < Kp; ++c) {
            const double ic = invd[c];
            double mc[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) mc[j] = G[j * Kmax + c] * ic;
            gsync<L>(gmask);
            if (((c - gl) & (L - 1)) == 0) {
#pragma unroll
                for (int j = 0; j < Q; ++j) G[j * Kmax + c] = mc[j];
            }
            const int a0 = c + 1 + ((gl - c - 1) & (L - 1));
            for (int a = a0; a < Kp; a += L) {
                const double lac = A[a * (a + 1) / 2 + c];
#pragma unroll
                for (int j = 0; j < Q; ++j) G[j * Kmax + a] = fma(-lac, mc[j], G[j * Kmax + a]);
            }
            gsync<L>(gmask);
        }

        // ---------------- per-observation values ----------------
        {
            // partial dot products over this lane's entries, last entry of hat() halved
            double dl[Q], dx[Q][PMAX], mm[Q * (Q + 1) / 2];
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                dl[j] = 0.0;
                for (int t = 0; t < p; ++t) dx[j][t] = 0.0;
            }
#pragma unroll
            for (int t = 0; t < Q * (Q + 1) / 2; ++t) mm[t] = 0.0;
            for (int a = gl; a < Kp; a += L) {
                const double hf = (a == last) ? 0.5 : 1.0;
                const double ly = Yg[a] * hf;
                double mj[Q];
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    mj[j] = G[j * Kmax + a];
                    dl[j] = fma(mj[j], ly, dl[j]);
                }
                for (int t = 0; t < p; ++t) {
                    const double lx = Yg[(1 + t) * Kmax + a] * hf;
#pragma unroll
                    for (int j = 0; j < Q; ++j) dx[j][t] = fma(mj[j], lx, dx[j][t]);
                }
                int u = 0;
#pragma unroll
                for (int j = 0; j < Q; ++j)
#pragma unroll
                    for (int l = j; l < Q; ++l) { mm[u] = fma(mj[j], mj[l], mm[u]); ++u; }
            }
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                dl[j] = gsum<L>(dl[j], gmask);
                for (int t = 0; t < p; ++t) dx[j][t] = gsum<L>(dx[j][t], gmask);
            }
#pragma unroll
            for (int t = 0; t < Q * (Q + 1) / 2; ++t) mm[t] = gsum<L>(mm[t], gmask);
            if (gl == 0) {
                V[0] = 1.0;
                V[1] = 0.0;
                V[2] = -2.0 * log(invd[last]);
                V[3] = Yg[last];
                for (int t = 0; t < p; ++t) V[4 + t] = Yg[(1 + t) * Kmax + last];
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    const int vb = vb0 + j * vstep;
                    const double md = G[j * Kmax + last];
                    V[vb] = md;
                    V[vb + 1] = -dl[j];
                    for (int t = 0; t < p; ++t) V[vb + 2 + t] = -dx[j][t];
                    V[vb + 2 + p] = -0.5 * md;
                }
#pragma unroll
                for (int t = 0; t < Q * (Q + 1) / 2; ++t) V[vmm + t] = mm[t];
            }
            gsync<L>(gmask);
        }

        // ---------------- accumulate the record ----------------
        for (int t = gl, k = 0; t < args.nstat; t += L, ++k) {
            const uint32_t w = sidx[t];
            const double v1 = V[w & 255u] * V[(w >> 8) & 255u];
            acc[k] += fma(V[(w >> 16) & 255u], V[w >> 24], v1);
        }
        gsync<L>(gmask);
    }

    // ---------------- block reduction (fixed order) ----------------
    __syncthreads();
    double* accbase = sp - (size_t)blockDim.x * args.acc_per_lane;
    for (int t = tid; t < args.nstat; t += blockDim.x) {
        const int lr = t % L, k = t / L;
        double s = 0.0;
        for (int g = 0; g < ngrp; ++g) s += accbase[(size_t)(g * L + lr) * args.acc_per_lane + k];
        args.partials[(size_t)blockIdx.x * args.nstat + t] = s;
    }
}

}  // namespace vg
