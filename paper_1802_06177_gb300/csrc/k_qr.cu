// UDT stabilisation step in FP64: pivoted Householder QR of C = Y diag(D) and formation of Q.
//
// The paper leaves stabilisation to the DQMC literature; this is the standard UDT chain
// (every n_s slices the product Y D T is re-factored as Q D' T'). Because a Householder
// reflector does not change when the column that defines it is scaled, the QR of Y diag(D)
// with column pivoting applies exactly the reflectors of Y itself, chosen in the order of
// the scaled trailing norms ||y_j^(k)|| D_j. The kernel therefore factors the O(1)-ranged Y
// and keeps D only as logarithms: pivots compare ||y_j^(k)||^2 exp(2 (lnD_j - max lnD)),
// the new scales are ln D'_k = ln|R^Y_kk| + lnD_{p_k}, and the scaled triangle is
//   Rt_ik = R^Y_ik exp(lnD_{p_k} - ln D'_i)   (|Rt_ik| <= 1 for k > i, |Rt_kk| = 1).
// Trailing norms are downdated and recomputed when cancellation makes them unreliable.
//
// Output (column-major, logical column order): QR holds Rt on and above the diagonal and
// the Householder vectors v_k (v_k[k] = 1 implied) below it; tau[k]; perm[k] = original
// column placed at position k; lnD[k] overwritten with ln D'_k; sgnU = det(Q) = +-1.
#include <cfloat>
#include <climits>

#include "slmc_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ bool better(double v, int j, double bv, int bj) {
    return v > bv || (v == bv && j < bj);
}

template <int MAXR>
__global__ void __launch_bounds__(kThreads) k_qrp(double* __restrict__ Yall, double* __restrict__ lnD_all,
                                                  double* __restrict__ QRall, double* __restrict__ tau_all,
                                                  int* __restrict__ perm_all, int* __restrict__ sgnU,
                                                  unsigned int* __restrict__ err, int N) {
    const int f = blockIdx.x;
    const size_t NN = (size_t)N * N;
    double* __restrict__ Y = Yall + f * NN;
    double* __restrict__ QR = QRall + f * NN;
    extern __shared__ __align__(16) unsigned char smraw[];
    double* s_v = reinterpret_cast<double*>(smraw);
    double* s_nrm = s_v + N;
    double* s_nrm0 = s_nrm + N;
    double* s_w = s_nrm0 + N;
    double* s_lnd = s_w + N;
    double* s_lnDn = s_lnd + N;
    double* s_e = s_lnDn + N;
    double* s_g = s_e + N;
    int* s_map = reinterpret_cast<int*>(s_g + N);
    int* s_pos = s_map + N;
    __shared__ double s_redv[kWarps];
    __shared__ int s_redi[kWarps];
    __shared__ double s_tau, s_mx;
    __shared__ int s_ntriv, s_wide;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int j = tid; j < N; j += kThreads) {
        s_lnd[j] = lnD_all[(size_t)f * N + j];
        s_map[j] = j;
        s_pos[j] = j;
    }
    if (tid == 0) s_ntriv = 0;
    __syncthreads();
    if (warp == 0) {
        double m = -DBL_MAX;
        for (int j = lane; j < N; j += 32) m = fmax(m, s_lnd[j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_mx = m;
    }
    __syncthreads();
    for (int j = tid; j < N; j += kThreads) s_w[j] = exp(2.0 * (s_lnd[j] - s_mx));
    __syncthreads();

    // Column norms and each warp's best pivot candidate for step 0.
    double best = -1.0;
    int bestj = INT_MAX;
    for (int j = warp; j < N; j += kWarps) {
        double acc = 0.0;
#pragma unroll
        for (int r = 0; r < MAXR; ++r) {
            const int i = lane + 32 * r;
            if (i < N) {
                const double y = Y[(size_t)j * N + i];
                acc = fma(y, y, acc);
            }
        }
        acc = slmc::warp_allsum(acc);
        if (lane == 0) {
            s_nrm[j] = acc;
            s_nrm0[j] = acc;
        }
        const double val = acc * s_w[j];
        if (better(val, j, best, bestj)) {
            best = val;
            bestj = j;
        }
    }
    if (lane == 0) {
        s_redv[warp] = best;
        s_redi[warp] = bestj;
    }
    __syncthreads();

    for (int k = 0; k < N; ++k) {
        const int m = N - k;
        // ---- pivot choice and Householder reflector of the pivot column (warp 0) ----
        if (warp == 0) {
            double bv = (lane < kWarps) ? s_redv[lane] : -1.0;
            int bi = (lane < kWarps) ? s_redi[lane] : INT_MAX;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (better(ov, oi, bv, bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            const int pc = (bi == INT_MAX) ? s_map[k] : bi;  // all candidates NaN: keep order
            if (lane == 0) {
                const int q = s_pos[pc];
                const int other = s_map[k];
                s_map[k] = pc;
                s_map[q] = other;
                s_pos[pc] = k;
                s_pos[other] = q;
            }
            __syncwarp();
            double y[MAXR];
#pragma unroll
            for (int r = 0; r < MAXR; ++r) {
                const int ii = lane + 32 * r;
                y[r] = (ii < m) ? Y[(size_t)pc * N + k + ii] : 0.0;
            }
            const double alpha = __shfl_sync(0xffffffffu, y[0], 0);
            double sig = 0.0;
#pragma unroll
            for (int r = 0; r < MAXR; ++r) {
                const int ii = lane + 32 * r;
                if (ii >= 1 && ii < m) sig = fma(y[r], y[r], sig);
            }
            sig = slmc::warp_allsum(sig);
            double tau = 0.0, beta = alpha, scal = 0.0;
            if (sig != 0.0) {
                const double nrm = sqrt(fma(alpha, alpha, sig));
                beta = (alpha >= 0.0) ? -nrm : nrm;
                tau = (beta - alpha) / beta;
                scal = 1.0 / (alpha - beta);
            }
#pragma unroll
            for (int r = 0; r < MAXR; ++r) {
                const int ii = lane + 32 * r;
                if (ii < m) {
                    if (ii == 0) {
                        s_v[k] = 1.0;
                        Y[(size_t)pc * N + k] = beta;
                    } else {
                        const double v = y[r] * scal;
                        s_v[k + ii] = v;
                        Y[(size_t)pc * N + k + ii] = v;
                    }
                }
            }
            if (lane == 0) {
                s_tau = tau;
                tau_all[(size_t)f * N + k] = tau;
                if (tau != 0.0) s_ntriv += 1;
            }
        }
        __syncthreads();

        // ---- apply the reflector to every remaining column; downdate norms ----
        const double tau = s_tau;
        best = -1.0;
        bestj = INT_MAX;
        for (int j = warp; j < N; j += kWarps) {
            if (s_pos[j] <= k) continue;
            double y[MAXR];
#pragma unroll
            for (int r = 0; r < MAXR; ++r) {
                const int ii = lane + 32 * r;
                y[r] = (ii < m) ? Y[(size_t)j * N + k + ii] : 0.0;
            }
            if (tau != 0.0) {
                double d = 0.0;
#pragma unroll
                for (int r = 0; r < MAXR; ++r) {
                    const int ii = lane + 32 * r;
                    if (ii < m) d = fma(s_v[k + ii], y[r], d);
                }
                d = slmc::warp_allsum(d) * tau;
#pragma unroll
                for (int r = 0; r < MAXR; ++r) {
                    const int ii = lane + 32 * r;
                    if (ii < m) {
                        y[r] = fma(-d, s_v[k + ii], y[r]);
                        Y[(size_t)j * N + k + ii] = y[r];
                    }
                }
            }
            const double rkj = __shfl_sync(0xffffffffu, y[0], 0);
            if (k < N - 1) {
                const double nr = s_nrm[j], nr0 = s_nrm0[j];
                __syncwarp();
                double temp = (nr > 0.0) ? 1.0 - (rkj * rkj) / nr : 0.0;
                temp = fmax(temp, 0.0);
                double nrnew;
                if (temp * nr <= 1.4901161193847656e-08 * nr0) {  // sqrt(eps): recompute
                    double a = 0.0;
#pragma unroll
                    for (int r = 0; r < MAXR; ++r) {
                        const int ii = lane + 32 * r;
                        if (ii >= 1 && ii < m) a = fma(y[r], y[r], a);
                    }
                    nrnew = slmc::warp_allsum(a);
                    if (lane == 0) s_nrm0[j] = nrnew;
                } else {
                    nrnew = nr * temp;
                }
                if (lane == 0) s_nrm[j] = nrnew;
                const double val = nrnew * s_w[j];
                if (better(val, j, best, bestj)) {
                    best = val;
                    bestj = j;
                }
            }
        }
        if (lane == 0) {
            s_redv[warp] = best;
            s_redi[warp] = bestj;
        }
        __syncthreads();
    }

    // ---- new scales, scaled triangle in logical column order ----
    bool bad = false;
    for (int k = tid; k < N; k += kThreads) {
        const int pc = s_map[k];
        const double l = log(fabs(Y[(size_t)pc * N + k])) + s_lnd[pc];
        s_lnDn[k] = l;
        bad |= !isfinite(l);
    }
    if (tid == 0) s_wide = 0;
    __syncthreads();
    for (int k = tid; k < N; k += kThreads)
        if (fabs(s_lnDn[k]) > 600.0 || fabs(s_lnd[s_map[k]]) > 600.0) s_wide = 1;
    __syncthreads();
    const bool wide = s_wide != 0;
    if (!wide) {
        for (int k = tid; k < N; k += kThreads) {
            s_e[k] = exp(s_lnd[s_map[k]]);
            s_g[k] = exp(-s_lnDn[k]);
        }
    }
    __syncthreads();
    for (int k = warp; k < N; k += kWarps) {
        const int pc = s_map[k];
#pragma unroll
        for (int r = 0; r < MAXR; ++r) {
            const int i = lane + 32 * r;
            if (i >= N) continue;
            const double yv = Y[(size_t)pc * N + i];
            double o;
            if (i < k) o = wide ? yv * exp(s_lnd[pc] - s_lnDn[i]) : yv * s_e[k] * s_g[i];
            else if (i == k) o = (yv >= 0.0) ? 1.0 : -1.0;
            else o = yv;
            QR[(size_t)k * N + i] = o;
        }
    }
    for (int k = tid; k < N; k += kThreads) {
        lnD_all[(size_t)f * N + k] = s_lnDn[k];
        perm_all[(size_t)f * N + k] = s_map[k];
    }
    if (tid == 0) sgnU[f] = (s_ntriv & 1) ? -1 : 1;
    if (bad) atomicOr(err, SLMC_EBIT_NONFINITE);
}

// Q = H_0 H_1 ... H_{N-1}: column j equals H_0 ... H_j e_j (reflectors k > j leave e_j
// unchanged), so every column is formed independently by one warp without block syncs.
template <int MAXR>
__global__ void __launch_bounds__(256) k_formq(const double* __restrict__ QRall, const double* __restrict__ tau_all,
                                               double* __restrict__ Uall, int N) {
    const int f = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * 8 + warp;
    if (j >= N) return;
    const size_t NN = (size_t)N * N;
    const double* __restrict__ QR = QRall + f * NN;
    const double* __restrict__ tau = tau_all + (size_t)f * N;
    double q[MAXR];
#pragma unroll
    for (int r = 0; r < MAXR; ++r) q[r] = (lane + 32 * r == j) ? 1.0 : 0.0;
    for (int k = j; k >= 0; --k) {
        const double t = __ldg(tau + k);
        if (t == 0.0) continue;
        const double* __restrict__ vk = QR + (size_t)k * N;
        double v[MAXR];
        double d = 0.0;
#pragma unroll
        for (int r = 0; r < MAXR; ++r) {
            const int i = lane + 32 * r;
            v[r] = (i > k && i < N) ? __ldg(vk + i) : (i == k ? 1.0 : 0.0);
            d = fma(v[r], q[r], d);
        }
        d = slmc::warp_allsum(d) * t;
#pragma unroll
        for (int r = 0; r < MAXR; ++r) q[r] = fma(-d, v[r], q[r]);
    }
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
        const int i = lane + 32 * r;
        if (i < N) Uall[f * NN + (size_t)j * N + i] = q[r];
    }
}

template <int MAXR>
cudaError_t launch_qr(slmc_ctx* c, int nf, cudaStream_t s) {
    const int N = c->N;
    const size_t smem = (size_t)N * (8 * sizeof(double) + 2 * sizeof(int));
    cudaError_t e = cudaFuncSetAttribute(k_qrp<MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_qrp<MAXR><<<nf, kThreads, smem, s>>>(c->Y, c->lnD, c->QR, c->tau, c->perm, c->sgnU, c->err, N);
    return cudaGetLastError();
}

template <int MAXR>
cudaError_t launch_formq(slmc_ctx* c, int nf, cudaStream_t s) {
    dim3 grid((c->N + 7) / 8, nf);
    k_formq<MAXR><<<grid, 256, 0, s>>>(c->QR, c->tau, c->U, c->N);
    return cudaGetLastError();
}

}  // namespace

namespace slmc {

cudaError_t qr_pivoted(slmc_ctx* c, int nf, cudaStream_t s) {
    switch (rows_per_lane_class(c->N)) {
        case 1: return launch_qr<1>(c, nf, s);
        case 2: return launch_qr<2>(c, nf, s);
        case 4: return launch_qr<4>(c, nf, s);
        case 5: return launch_qr<5>(c, nf, s);
        case 8: return launch_qr<8>(c, nf, s);
        case 12: return launch_qr<12>(c, nf, s);
        case 18: return launch_qr<18>(c, nf, s);
        default: return launch_qr<32>(c, nf, s);
    }
}

cudaError_t form_q(slmc_ctx* c, int nf, cudaStream_t s) {
    switch (rows_per_lane_class(c->N)) {
        case 1: return launch_formq<1>(c, nf, s);
        case 2: return launch_formq<2>(c, nf, s);
        case 4: return launch_formq<4>(c, nf, s);
        case 5: return launch_formq<5>(c, nf, s);
        case 8: return launch_formq<8>(c, nf, s);
        case 12: return launch_formq<12>(c, nf, s);
        case 18: return launch_formq<18>(c, nf, s);
        default: return launch_formq<32>(c, nf, s);
    }
}

}  // namespace slmc
