// Blocked UDT stabilisation in FP64: pre-pivoted blocked Householder QR, blocked formation
// of Q, and the T update as a tiled triangular GEMM.
//
// On this part the FP64 pipe is the scarce unit, so every FP64 issue slot should be an FMA
// of the factorisation itself. A column-by-column (BLAS-2) QR spends most slots on
// reduction trees and norm downdates; here the columns are ordered once by their scaled
// norms ||y_j|| D_j (pre-pivoting, the ordering full column pivoting starts from), and the
// unpivoted QR is blocked: a panel of BP columns is factored in shared memory, then the
// trailing columns receive the panel's reflectors at once through the compact WY form
// Q_p = I - V S V^T as three small GEMMs (W = V^T C, W' = S^T W, C -= V W') whose inner loops
// are plain FMAs. Each warp updates its own groups of 8 trailing columns with no block
// synchronisation. The graded structure that makes this as accurate as per-step pivoting for
// products of this kind is the column scaling by D, which the pre-sort already captures.
//
// As in the unblocked kernel, the QR factors Y itself and carries D as logarithms
// (pivot keys ||y_j||^2 exp(2 (lnD_j - max lnD)), new scales ln D'_k = ln|R_kk| + lnD_{p_k}).
// Outputs match the unblocked kernel (logical column order): QR = Rt on/above the diagonal and
// v_k below it, tau, perm, lnD', sgnU, plus the panels' WY triangles S for the formation of Q.
//
// Few large fields (fewer fields than SMs) are factored by a thread-block cluster of C CTAs per
// field: panel t belongs to CTA t mod C, which also owns (and alone updates) the columns of
// every panel t' = t mod C. The owner factors the panel in its shared memory; after a cluster
// barrier the other CTAs copy V, S and the new scales from the owner's shared memory
// (distributed shared memory) and update their own trailing columns. One cluster barrier per
// panel suffices: a CTA overwrites its panel buffer only C panels later, after every CTA has
// passed the barriers in between (and so finished its copies). C = 1 is the one-CTA kernel.
#include <algorithm>
#include <cfloat>

#include <cooperative_groups.h>

#include "qr_panel.cuh"

namespace cg = cooperative_groups;

namespace {

template <int BP>
__global__ void __launch_bounds__(kThreads, 2) k_qrb(double* __restrict__ Yall, double* __restrict__ lnD_all,
                                                  double* __restrict__ QRall, double* __restrict__ tau_all,
                                                  int* __restrict__ perm_all, int* __restrict__ sgnU,
                                                  double* __restrict__ Sall, unsigned int* __restrict__ err, int N) {
    constexpr int BPS = BP + 1;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
    const int f = blockIdx.x / C;
    const size_t NN = (size_t)N * N;
    double* __restrict__ Y = Yall + f * NN;
    double* __restrict__ QR = QRall + f * NN;
    extern __shared__ __align__(16) unsigned char smraw[];
    double* Vp = reinterpret_cast<double*>(smraw);
    double* Ssm = Vp + (size_t)N * BPS;
    double* Wsm = Ssm + BP * BP;
    double* s_key = Wsm + kWarps * BP * kCT;
    double* s_lnd = s_key + N;
    double* s_lnDn = s_lnd + N;
    double* s_g = s_lnDn + N;
    double* s_tau = s_g + N;
    double* s_beta = s_tau + BP;
    int* s_perm = reinterpret_cast<int*>(s_beta + BP);
    __shared__ double s_mx;
    __shared__ int s_ntriv, s_wide;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- scaled column norms and the pre-pivoting order ----
    for (int j = tid; j < N; j += kThreads) s_lnd[j] = lnD_all[(size_t)f * N + j];
    if (tid == 0) {
        s_ntriv = 0;
        s_wide = 0;
    }
    __syncthreads();
    if (warp == 0) {
        double mx = -DBL_MAX;
        for (int j = lane; j < N; j += 32) mx = fmax(mx, s_lnd[j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_mx = mx;
    }
    __syncthreads();
    for (int j = warp; j < N; j += kWarps) {
        double a = 0.0;
        for (int i = lane; i < N; i += 32) {
            const double y = Y[(size_t)j * N + i];
            a = fma(y, y, a);
        }
        a = slmc::warp_allsum(a);
        if (lane == 0) {
            const double key = a * exp(2.0 * (s_lnd[j] - s_mx));
            s_key[j] = (key >= 0.0) ? key : -1.0;  // NaN sorts last and keeps ranks unique
        }
    }
    __syncthreads();
    for (int j = tid; j < N; j += kThreads) {
        // keys are >= +0 or -1: their bit patterns as 64-bit integers order as the values do, and
        // the integer compares leave the FP64 pipe to the factorisation
        const long long kj = __double_as_longlong(s_key[j]);
        int r = 0;
        for (int i = 0; i < N; ++i) {
            const long long ki = __double_as_longlong(s_key[i]);
            r += (ki > kj) || (ki == kj && i < j);
        }
        s_perm[r] = j;
    }
    __syncthreads();
    for (int k = tid; k < N; k += kThreads)
        if (fabs(s_lnd[k]) > 600.0) s_wide = 1;

    // ---- panels ----
    const int npanels = (N + BP - 1) / BP;
    for (int t = 0; t < npanels; ++t) {
        const int p = t * BP, nb = min(BP, N - p), owner = t % C;
        __syncthreads();
        if (rank == owner)
            panel_step<BP>(Y, QR, tau_all + (size_t)f * N, Sall + (size_t)f * N * BP, Vp, Ssm, Wsm, s_lnd, s_lnDn, s_g,
                           s_tau, s_beta, s_perm, &s_ntriv, &s_wide, N, p, nb);
        if (C > 1) {
            cluster.sync();  // panel t: V, S and the new scales are in the owner's shared memory
            if (rank != owner) {
                const double* oV = cluster.map_shared_rank(Vp, owner);
                const double* oS = cluster.map_shared_rank(Ssm, owner);
                const double* oL = cluster.map_shared_rank(s_lnDn, owner);
                const double* oG = cluster.map_shared_rank(s_g, owner);
                for (int idx = tid; idx < (N - p) * nb; idx += kThreads) {
                    const int rr = idx / nb, c = idx - rr * nb;
                    Vp[(p + rr) * BPS + c] = oV[(p + rr) * BPS + c];
                }
                for (int idx = tid; idx < BP * BP; idx += kThreads) Ssm[idx] = oS[idx];
                if (tid < nb) {
                    const double l = oL[p + tid];
                    s_lnDn[p + tid] = l;
                    s_g[p + tid] = oG[p + tid];
                    if (fabs(l) > 600.0) s_wide = 1;
                }
            }
        }
        __syncthreads();
        // trailing update C <- Q_p^T C on this CTA's logical columns beyond the panel: the columns
        // of panels t1, t1 + C, ... (t1 the first panel after t that this CTA owns)
        const int t1 = t + 1 + ((rank - (t + 1)) % C + C) % C;
        int ncols = 0;
        for (int u = t1; u < npanels; u += C) ncols += min(BP, N - u * BP);
        wy_update<BP, true>(Vp, Ssm, Wsm, N, p, nb, ncols, [&](int jj) {
            const int j = (t1 + (jj / BP) * C) * BP + jj % BP;
            return Y + (size_t)s_perm[j] * N;
        });
    }
    if (C > 1) cluster.sync();  // every CTA holds all scales; the ranks' reflector counts are final
    __syncthreads();
    if (rank == 0) {
        bool bad = false;
        for (int k = tid; k < N; k += kThreads) {
            lnD_all[(size_t)f * N + k] = s_lnDn[k];
            perm_all[(size_t)f * N + k] = s_perm[k];
            bad |= !isfinite(s_lnDn[k]);
        }
        if (tid == 0) {
            int ntriv = s_ntriv;
            for (int r = 1; r < C; ++r) ntriv += *cluster.map_shared_rank(&s_ntriv, r);
            sgnU[f] = (ntriv & 1) ? -1 : 1;
        }
        if (bad) atomicOr(err, SLMC_EBIT_NONFINITE);
    }
    if (C > 1) cluster.sync();  // shared memory stays alive until rank 0 has read the counts
}

// Q = Q_0 Q_1 ... (Q_p = I - V_p S_p V_p^T), accumulated backwards into U (column-major),
// computed in T: FP64, or FP32 when Q only feeds reduced-precision slice products (which round
// it to FP32 on entry anyway).
// Columns of Q are independent: CTA (field, blockIdx.y) forms columns [j0, j1) of gridDim.y
// blocks (several CTAs per field when there are few fields).
template <int BP, typename T>
__global__ void __launch_bounds__(kThreads, 2) k_formq_b(const double* __restrict__ QRall, const double* __restrict__ Sall,
                                                      T* __restrict__ Uall, int N) {
    constexpr int BPS = BP + 1;
    const int f = blockIdx.x;
    const int j0 = (int)((long long)blockIdx.y * N / gridDim.y), j1 = (int)((long long)(blockIdx.y + 1) * N / gridDim.y);
    const size_t NN = (size_t)N * N;
    const double* __restrict__ QR = QRall + f * NN;
    T* __restrict__ U = Uall + f * NN;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Vp = reinterpret_cast<T*>(smraw);
    T* Ssm = Vp + (size_t)N * BPS;
    T* Wsm = Ssm + BP * BP;
    const int tid = threadIdx.x;
    for (size_t idx = (size_t)j0 * N + tid; idx < (size_t)j1 * N; idx += kThreads)
        U[idx] = (idx % (N + 1) == 0) ? T(1) : T(0);
    for (int p = ((N - 1) / BP) * BP; p >= 0; p -= BP) {
        const int nb = min(BP, N - p);
        __syncthreads();
        for (int idx = tid; idx < nb * (N - p); idx += kThreads) {
            const int c = idx / (N - p), r = p + idx - c * (N - p);
            const int k = p + c;
            Vp[r * BPS + c] = (T)((r > k) ? QR[(size_t)k * N + r] : (r == k ? 1.0 : 0.0));
        }
        for (int idx = tid; idx < nb * BP; idx += kThreads) {
            const int a = idx / BP, b = idx - a * BP;
            Ssm[a * BP + b] = (T)Sall[(size_t)f * N * BP + (size_t)(p + a) * BP + b];
        }
        __syncthreads();
        const int jb = max(p, j0);  // columns left of the panel are still unit vectors
        if (jb < j1) wy_update<BP, false>(Vp, Ssm, Wsm, N, p, nb, j1 - jb, [&](int jj) { return U + (size_t)(jb + jj) * N; });
    }
}

// T_new = Rt P^T T_old, T row-major: T_new[i][j] = sum_{k >= i} Rt[i][k] T_old[perm[k]][j].
// 64x64 output tile per CTA, 4x4 per thread, K chunks of 16 staged in shared memory; chunks
// entirely below the diagonal of Rt are skipped.
__global__ void __launch_bounds__(256) k_tupd(const double* __restrict__ QRall, const double* __restrict__ Told,
                                              const int* __restrict__ perm_all, double* __restrict__ Tnew, int N) {
    constexpr int TM = 64, TK = 16;
    __shared__ double As[TK][TM + 4];
    __shared__ double Bs[TK][TM + 4];
    const int f = blockIdx.z;
    const size_t NN = (size_t)N * N;
    const double* __restrict__ A = QRall + f * NN;
    const double* __restrict__ B = Told + f * NN;
    const int* __restrict__ perm = perm_all + (size_t)f * N;
    const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TM;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int k0 = (i0 / TK) * TK; k0 < N; k0 += TK) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < TK * TM; idx += 256) {
            const int kk = idx / TM, ii = idx - kk * TM;
            const int k = k0 + kk, i = i0 + ii, j = j0 + ii;
            As[kk][ii] = (k < N && i < N && k >= i) ? A[(size_t)k * N + i] : 0.0;
            Bs[kk][ii] = (k < N && j < N) ? B[(size_t)perm[k] * N + j] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty * 4 + q];
                b[q] = Bs[kk][tx * 4 + q];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
        }
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int i = i0 + ty * 4 + x;
        if (i >= N) continue;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int j = j0 + tx * 4 + y;
            if (j < N) Tnew[f * NN + (size_t)i * N + j] = acc[x][y];
        }
    }
}

// CTAs per field for the QR and the formation of Q: 1, 2 or 4, so that few fields still
// occupy most SMs (tuned value if set).
int qr_cluster_size(const slmc_ctx* c, int nf) {
    if (c->tune_qr_cluster) return c->tune_qr_cluster;
    if (c->N < 128 || c->num_sms <= 0 || nf <= 0) return 1;
    const int r = c->num_sms / nf;
    return r >= 4 ? 4 : (r >= 2 ? 2 : 1);
}

template <int BP>
cudaError_t launch_qrb(slmc_ctx* c, int nf, cudaStream_t s) {
    const size_t smem = QrSmem<BP>::bytes(c->N);
    cudaError_t e = cudaFuncSetAttribute(k_qrb<BP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int C = qr_cluster_size(c, nf);
    if (C == 1) {
        k_qrb<BP><<<nf, kThreads, smem, s>>>(c->Y, c->lnD, c->QR, c->tau, c->perm, c->sgnU, c->Sws, c->err, c->N);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nf * C));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_qrb<BP>, c->Y, c->lnD, c->QR, c->tau, c->perm, c->sgnU, c->Sws, c->err, c->N);
}

template <int BP, typename T>
cudaError_t launch_formq_b(slmc_ctx* c, int nf, cudaStream_t s) {
    const size_t smem = sizeof(T) * ((size_t)c->N * (BP + 1) + BP * BP + kWarps * BP * kCT);
    cudaError_t e = cudaFuncSetAttribute(k_formq_b<BP, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    T* U;
    if constexpr (sizeof(T) == 4) U = c->U32;
    else U = c->U;
    // column blocks per field: at least the QR's cluster size, and enough for about two CTAs per SM
    int cb = qr_cluster_size(c, nf);
    if (c->num_sms > 0 && nf > 0) cb = std::max(cb, std::min(4, (2 * c->num_sms + nf - 1) / nf));
    dim3 grid(nf, cb);
    k_formq_b<BP, T><<<grid, kThreads, smem, s>>>(c->QR, c->Sws, U, c->N);
    return cudaGetLastError();
}

}  // namespace

namespace slmc {

// Panel width: the tuned value if set and its shared memory fits, else 32 up to N = 256 and 16 above.
int qr_panel_width(const slmc_ctx* c) {
    const int want = c->tune_qr_panel ? c->tune_qr_panel : (c->N <= 256 ? 32 : 16);
    if (want == 32 && QrSmem<32>::bytes(c->N) > 220 * 1024) return 16;
    return want;
}

cudaError_t qr_blocked(slmc_ctx* c, int nf, cudaStream_t s) {
    return qr_panel_width(c) == 32 ? launch_qrb<32>(c, nf, s) : launch_qrb<16>(c, nf, s);
}

cudaError_t form_q_blocked(slmc_ctx* c, int nf, bool fp32, cudaStream_t s) {
    if (fp32) return qr_panel_width(c) == 32 ? launch_formq_b<32, float>(c, nf, s) : launch_formq_b<16, float>(c, nf, s);
    return qr_panel_width(c) == 32 ? launch_formq_b<32, double>(c, nf, s) : launch_formq_b<16, double>(c, nf, s);
}

cudaError_t t_update_tiled(slmc_ctx* c, int nf, cudaStream_t s) {
    const int nt = (c->N + 63) / 64;
    dim3 grid(nt, nt, nf);
    k_tupd<<<grid, 256, 0, s>>>(c->QR, c->Ta, c->perm, c->Tb, c->N);
    double* t = c->Ta;
    c->Ta = c->Tb;
    c->Tb = t;
    return cudaGetLastError();
}

}  // namespace slmc
