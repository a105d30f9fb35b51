// Shared pieces of the blocked Householder QR (FP64): the compact-WY trailing update on the
// FP64 pipe, the panel reflectors and the whole panel step, used by the one-kernel QR (k_qrb) and
// by the QR whose trailing updates run on the tensor cores (k_qrt_*).
#pragma once

#include <cfloat>

#include "slmc_internal.cuh"

namespace {


constexpr int kThreads = 256;
constexpr int kWarps = 8;
constexpr int kCT = 8;   // trailing columns per warp group
constexpr int kRC = 2;   // row chunks (of 32 rows) per lane in the rank-BP update

template <int BP>
struct QrSmem {
    static size_t bytes(int N) {
        return sizeof(double) * ((size_t)N * (BP + 1) + BP * BP + kWarps * BP * kCT + 4 * (size_t)N + 2 * BP) +
               sizeof(int) * (size_t)N;
    }
};

// Rows r0 + lane + 32 q (q < RC) of the kCT columns cptr: y -= V[r][0:nb] W'[0:nb][c].
template <int RC, int BP, typename T, typename CT>
__device__ __forceinline__ void wy_rows(const T* __restrict__ Vp, const T* __restrict__ W, const CT (&cptr)[kCT], int N,
                                        int r0, int nb, int lane) {
    constexpr int BPS = BP + 1;
    T y[RC][kCT];
#pragma unroll
    for (int q = 0; q < RC; ++q) {
        const int r = r0 + lane + 32 * q;
#pragma unroll
        for (int c = 0; c < kCT; ++c) y[q][c] = (r < N && cptr[c]) ? cptr[c][r] : T(0);
    }
    for (int mm = 0; mm < nb; ++mm) {
        T wv[kCT];
#pragma unroll
        for (int c = 0; c < kCT; ++c) wv[c] = W[mm * kCT + c];
#pragma unroll
        for (int q = 0; q < RC; ++q) {
            const int r = r0 + lane + 32 * q;
            const T v = (r < N) ? Vp[r * BPS + mm] : T(0);
#pragma unroll
            for (int c = 0; c < kCT; ++c) y[q][c] = fma(-v, wv[c], y[q][c]);
        }
    }
#pragma unroll
    for (int q = 0; q < RC; ++q) {
        const int r = r0 + lane + 32 * q;
        if (r < N) {
#pragma unroll
            for (int c = 0; c < kCT; ++c)
                if (cptr[c]) cptr[c][r] = y[q][c];
        }
    }
}

// Rank-BP update of ncols columns, rows [p, N), of a column-major matrix A (column jj stored at
// col(jj)): A <- (I - V op(S) V^T) A, op(S) = S^T for the QR trailing update (Q_p^T A) and S
// for the backward formation of Q (Q_p A). V is the clean panel in shared memory (rows
// p..N-1, unit diagonal, zeros above), row stride BP+1.
template <int BP, bool TRANS, typename T, typename ColFn>
__device__ __forceinline__ void wy_update(const T* __restrict__ Vp, const T* __restrict__ Ssm, T* __restrict__ Wsm,
                                          int N, int p, int nb, int ncols, ColFn col) {
    constexpr int BPS = BP + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T* W = Wsm + warp * BP * kCT;
    using CT = decltype(col(0));  // column pointer: same precision as T (no conversions in the loops)
    for (int g = warp * kCT; g < ncols; g += kWarps * kCT) {
        CT cptr[kCT];
#pragma unroll
        for (int c = 0; c < kCT; ++c) cptr[c] = (g + c < ncols) ? col(g + c) : nullptr;
        // W[m][c] = sum_r V[r][m] A[r][c]: lane (m, h) owns reflector m = lane % BP and the
        // CPL columns of half h = lane / BP (A rows are broadcast to the warp)
        constexpr int CPL = kCT * BP / 32;
        const int m = lane % BP, h = lane / BP;
        CT mine[CPL];
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) mine[cc] = (h == 0) ? cptr[cc] : cptr[(CPL < kCT ? CPL : 0) + cc];
        T acc[CPL];
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) acc[cc] = T(0);
        for (int r = p; r < N; ++r) {
            const T v = Vp[r * BPS + m];
#pragma unroll
            for (int cc = 0; cc < CPL; ++cc)
                if (mine[cc]) acc[cc] = fma(v, mine[cc][r], acc[cc]);
        }
        __syncwarp();
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) W[m * kCT + h * CPL + cc] = (m < nb) ? acc[cc] : T(0);
        __syncwarp();
        // W' = op(S) W, op(S) triangular. Lane (c = lane % kCT, g = lane / kCT) owns the
        // reflectors m = g + 4 t: the four lane groups then run nearly equal triangular loops
        // (a lane-per-reflector layout would idle half the lanes on average).
        {
            constexpr int MT = BP / 4;
            const int c = lane % kCT, g = lane / kCT;
            T w2[MT];
#pragma unroll
            for (int t = 0; t < MT; ++t) {
                const int mr = g + 4 * t;
                T a = T(0);
                if (mr < nb) {
                    if (TRANS) {
                        for (int q = 0; q <= mr; ++q) a = fma(Ssm[q * BP + mr], W[q * kCT + c], a);
                    } else {
                        for (int q = mr; q < nb; ++q) a = fma(Ssm[mr * BP + q], W[q * kCT + c], a);
                    }
                }
                w2[t] = a;
            }
            __syncwarp();
#pragma unroll
            for (int t = 0; t < MT; ++t) W[(g + 4 * t) * kCT + c] = w2[t];
            __syncwarp();
        }
        // A[r][c] -= sum_m V[r][m] W'[m][c]   (lanes over rows; chunks of 64 rows, then 32)
        int r0 = p;
        for (; r0 + 32 * kRC <= N; r0 += 32 * kRC) wy_rows<kRC, BP>(Vp, W, cptr, N, r0, nb, lane);
        for (; r0 < N; r0 += 32) wy_rows<1, BP>(Vp, W, cptr, N, r0, nb, lane);
        __syncwarp();
    }
}

// Warp sums of K values per lane (K a power of two <= 32) with K - 1 + log2(32 / K) additions per
// lane instead of 5 K: at each butterfly level a lane keeps half of its values and adds the
// partner's copy of that half. Returns the sum of value index j in lane j * (32 / K).
template <int K>
__device__ __forceinline__ double warp_transpose_sum(double (&v)[K], int lane) {
#pragma unroll
    for (int size = K, o = 16; size > 1; size >>= 1, o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < size / 2; ++i) {
            const double keep = upper ? v[i + size / 2] : v[i];
            const double other = upper ? v[i] : v[i + size / 2];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, other, o);
        }
    }
    double sum = v[0];
#pragma unroll
    for (int o = 16 / K; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    return sum;
}

template <int N>
struct Pow2Ceil {
    static constexpr int value = N <= 1 ? 1 : (N <= 2 ? 2 : (N <= 4 ? 4 : (N <= 8 ? 8 : (N <= 16 ? 16 : 32))));
};

// Householder reflector of panel column c (logical row k = p + c) by one warp: beta, tau and
// v = x / (alpha - beta) below the diagonal, written back into the panel.
template <int BP>
__device__ __forceinline__ void panel_reflector(double* __restrict__ Vp, int k, int c, int N, int lane,
                                                double* s_tau, double* s_beta, double* __restrict__ tau_f,
                                                int* s_ntriv) {
    constexpr int BPS = BP + 1;
    const double alpha = Vp[k * BPS + c];
    double sig = 0.0;
    for (int r = k + 1 + lane; r < N; r += 32) {
        const double v = Vp[r * BPS + c];
        sig = fma(v, v, sig);
    }
    sig = slmc::warp_allsum(sig);
    double tau = 0.0, beta = alpha, scal = 0.0;
    if (sig != 0.0) {
        const double nrm = sqrt(fma(alpha, alpha, sig));
        beta = (alpha >= 0.0) ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
    }
    for (int r = k + 1 + lane; r < N; r += 32) Vp[r * BPS + c] *= scal;
    if (lane == 0) {
        s_tau[c] = tau;
        s_beta[c] = beta;
        tau_f[k] = tau;
        if (tau != 0.0) *s_ntriv += 1;
    }
}

// Applies reflector c (rows k.., v_k = 1) to the NC panel columns c0, c0 + cs, ... by one warp:
// a -= tau (v . a) v, with the NC dot products and reductions interleaved.
template <int BP, int NC>
__device__ __forceinline__ void panel_apply(double* __restrict__ Vp, int k, int c, double tau, int c0, int cs, int N,
                                            int lane) {
    constexpr int BPS = BP + 1;
    int cols[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) cols[j] = c0 + j * cs;
    double d[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) d[j] = (lane == 0) ? Vp[k * BPS + cols[j]] : 0.0;
    for (int r = k + 1 + lane; r < N; r += 32) {
        const double v = Vp[r * BPS + c];
#pragma unroll
        for (int j = 0; j < NC; ++j) d[j] = fma(v, Vp[r * BPS + cols[j]], d[j]);
    }
    {  // all NC dot products reduced together, then broadcast
        constexpr int K = Pow2Ceil<NC>::value;
        double t[K];
#pragma unroll
        for (int j = 0; j < K; ++j) t[j] = (j < NC) ? d[j] : 0.0;
        const double sum = warp_transpose_sum<K>(t, lane);
#pragma unroll
        for (int j = 0; j < NC; ++j) d[j] = __shfl_sync(0xffffffffu, sum, j * (32 / K)) * tau;
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NC; ++j) Vp[k * BPS + cols[j]] -= d[j];
    }
    for (int r = k + 1 + lane; r < N; r += 32) {
        const double v = Vp[r * BPS + c];
#pragma unroll
        for (int j = 0; j < NC; ++j) Vp[r * BPS + cols[j]] = fma(-d[j], v, Vp[r * BPS + cols[j]]);
    }
}

__device__ __forceinline__ int k_of(int p, int c) { return p + c; }

// Compact-WY triangle of a panel of nb reflectors, by one warp (lane = row): S_cc = tau_c,
// S[0:c, c] = -tau_c S[0:c, 0:c] G[0:c, c], from the strictly upper part of the Gram matrix
// G = V^T V (row stride ldg). S (BP x BP, row-major) is zero below the diagonal and beyond nb.
template <int BP>
__device__ __forceinline__ void wy_triangle(const double* G, int ldg, const double* tau, double* Ssm, int nb,
                                            int lane) {
    for (int c = 0; c < nb; ++c) {
        const double tc = tau[c];
        double v = 0.0;
        if (lane < c) {  // four independent partial sums (short dependency chains)
            double v4[4] = {0.0, 0.0, 0.0, 0.0};
            int q = lane;
            for (; q + 4 <= c; q += 4) {
#pragma unroll
                for (int j = 0; j < 4; ++j) v4[j] = fma(Ssm[lane * BP + q + j], G[(q + j) * ldg + c], v4[j]);
            }
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (q + j < c) v4[j] = fma(Ssm[lane * BP + q + j], G[(q + j) * ldg + c], v4[j]);
            v = -tc * ((v4[0] + v4[1]) + (v4[2] + v4[3]));
        } else if (lane == c) {
            v = tc;
        }
        if (lane < BP) Ssm[lane * BP + c] = (lane <= c) ? v : 0.0;
        __syncwarp();
    }
    for (int c = nb; c < BP; ++c) {
        if (lane < BP) Ssm[lane * BP + c] = 0.0;
    }
    __syncwarp();
}

// Factors panel t (logical columns p .. p + nb - 1, already updated by the earlier panels) of one
// field by one CTA: loads it from Y in pre-pivoted order, forms its Householder reflectors in shared
// memory (tau), the new scales ln D'_k = ln|beta_k| + ln D_{perm(k)} of its rows, writes logical
// columns p .. p + nb - 1 of the packed output (Rt above the diagonal, v below), then leaves the clean
// reflectors V (unit diagonal, zeros above) in Vp and the compact-WY triangle S of the panel in Ssm
// and in Sall_f. G (BP x BP) is scratch. Rows i < p of the output use the scales s_lnDn / s_g of the
// earlier panels. NT threads (8 or more warps; the arithmetic of every column does not depend on NT).
// want_wy = false stops after V is clean: no Gram matrix, no S (the caller forms them).
template <int BP, int NT = kThreads>
__device__ __forceinline__ void panel_step(const double* __restrict__ Y, double* __restrict__ QR,
                                           double* __restrict__ tau_f, double* __restrict__ Sall_f, double* Vp,
                                           double* Ssm, double* G, const double* s_lnd, double* s_lnDn, double* s_g,
                                           double* s_tau, double* s_beta, const int* s_perm, int* s_ntriv,
                                           int* s_wide, int N, int p, int nb, bool want_wy = true) {
    constexpr int BPS = BP + 1;
    constexpr int NW = NT / 32;  // warps of the CTA
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int idx = tid; idx < nb * (N - p); idx += NT) {
        const int c = idx / (N - p), rr = idx - c * (N - p);
        Vp[(p + rr) * BPS + c] = Y[(size_t)s_perm[p + c] * N + p + rr];
    }
    __syncthreads();
    // Householder on the panel (shared memory), one block barrier per column: warp 0 applies
    // reflector c to column c+1 and forms reflector c+1 from it, while warps 1.. apply
    // reflector c to columns c+2.. (their dot products and reductions interleaved).
    if (warp == 0) panel_reflector<BP>(Vp, k_of(p, 0), 0, N, lane, s_tau, s_beta, tau_f, s_ntriv);
    __syncthreads();
    for (int c = 0; c < nb; ++c) {
        const int k = p + c;
        const double tau = s_tau[c];
        if (warp == 0) {
            if (c + 1 < nb) {
                if (tau != 0.0) panel_apply<BP, 1>(Vp, k, c, tau, c + 1, 1, N, lane);
                __syncwarp();
                panel_reflector<BP>(Vp, k + 1, c + 1, N, lane, s_tau, s_beta, tau_f, s_ntriv);
            }
        } else if (tau != 0.0) {
            // columns c0, c0 + NW - 1, ... below nb (warp-uniform count nv <= 5 for NW >= 8)
            const int c0 = c + 2 + (warp - 1), cs = NW - 1;
            const int nv = (c0 < nb) ? (nb - 1 - c0) / cs + 1 : 0;
            switch (nv) {
                case 0: break;
                case 1: panel_apply<BP, 1>(Vp, k, c, tau, c0, cs, N, lane); break;
                case 2: panel_apply<BP, 2>(Vp, k, c, tau, c0, cs, N, lane); break;
                case 3: panel_apply<BP, 3>(Vp, k, c, tau, c0, cs, N, lane); break;
                case 4: panel_apply<BP, 4>(Vp, k, c, tau, c0, cs, N, lane); break;
                default: panel_apply<BP, 5>(Vp, k, c, tau, c0, cs, N, lane); break;
            }
        }
        __syncthreads();
    }
    // new scales of this panel's rows
    if (tid < nb) {
        const int k = p + tid;
        const double l = log(fabs(s_beta[tid])) + s_lnd[s_perm[k]];
        s_lnDn[k] = l;
        s_g[k] = exp(-l);
        if (fabs(l) > 600.0) *s_wide = 1;
    }
    __syncthreads();
    // write logical columns p..p+nb-1 of the packed output (Rt above, v below)
    const bool wide = *s_wide != 0;
    for (int c = warp; c < nb; c += NW) {
        const int k = p + c;
        const int pc = s_perm[k];
        const double lk = s_lnd[pc];
        const double ek = wide ? 0.0 : exp(lk);
        for (int i = lane; i < N; i += 32) {
            double o;
            if (i < k) {
                const double rv = (i < p) ? Y[(size_t)pc * N + i] : Vp[i * BPS + c];
                o = wide ? rv * exp(lk - s_lnDn[i]) : rv * ek * s_g[i];
            } else if (i == k) {
                o = (s_beta[c] >= 0.0) ? 1.0 : -1.0;
            } else {
                o = Vp[i * BPS + c];
            }
            QR[(size_t)k * N + i] = o;
        }
    }
    __syncthreads();
    // clean V (unit diagonal, zeros above) and the Gram matrix G = V^T V
    for (int idx = tid; idx < nb * nb; idx += NT) {
        const int a = idx / nb, c = idx - a * nb;  // Vp row p+a, column c
        if (a < c) Vp[(p + a) * BPS + c] = 0.0;
        else if (a == c) Vp[(p + a) * BPS + c] = 1.0;
    }
    __syncthreads();
    if (!want_wy) return;  // the Gram matrix and S are formed elsewhere
    {   // G[a][c] = v_a . v_c for a < c; each warp interleaves four pairs (independent chains)
        const int npairs = nb * (nb - 1) / 2;
        for (int q0 = warp * 4; q0 < npairs; q0 += NW * 4) {
            int pa[4], pc[4];
            double d[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int q = q0 + j, cc = 1;
                while (q >= cc) {  // pair index -> (a, c): pairs ordered by c, then a
                    q -= cc;
                    ++cc;
                }
                pa[j] = q;
                pc[j] = (q0 + j < npairs) ? cc : N;  // N: empty range
                d[j] = 0.0;
            }
            const int rmax = N - p - pc[0];
            for (int t = 0; t * 32 < rmax; ++t) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = p + pc[j] + lane + 32 * t;
                    if (r < N) d[j] = fma(Vp[r * BPS + pa[j]], Vp[r * BPS + pc[j]], d[j]);
                }
            }
            const double sum = warp_transpose_sum<4>(d, lane);  // pair j's sum in lane 8 j
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (lane == 8 * j && q0 + j < npairs) G[pa[j] * BP + pc[j]] = sum;
        }
    }
    __syncthreads();
    if (warp == 0) wy_triangle<BP>(G, BP, s_tau, Ssm, nb, lane);
    __syncthreads();
    for (int idx = tid; idx < nb * BP; idx += NT) {
        const int a = idx / BP, b = idx - a * BP;
        Sall_f[(size_t)(p + a) * BP + b] = (b < nb) ? Ssm[a * BP + b] : 0.0;
    }
}

}  // namespace
