// Final step of the stabilised determinant [Suppl. Eq. (S2), (S3)], FP64.
// With B_L ... B_1 = U D T and D = D_b D_s (D_b = max(D, 1), D_s = min(D, 1)):
//   I + U D T = U D_b M,   M = D_b^-1 U^T + D_s T,
//   ln|det(I + B_L ... B_1)| = sum ln D_b + ln|det M|,  sign = det(U) sign(det M),
//   G = (I + B_L ... B_1)^-1 = M^-1 D_b^-1 U^T.
// M is factored by a blocked right-looking LU with partial pivoting (one CTA per field; the
// unblocked kernel covers N > 842, whose panel does not fit in shared memory); G is
// solved by blocked triangular solves, 32 right-hand sides per CTA (for N > 842, whose
// right-hand sides do not fit in shared memory, one warp per column).
#include <cfloat>
#include <climits>

#include "slmc_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// M (column-major, written over Y) from U (column-major), T (row-major) and lnD.
__global__ void __launch_bounds__(kThreads) k_assemble_M(const double* __restrict__ Uall, const double* __restrict__ Tall,
                                                         const double* __restrict__ lnD_all, double* __restrict__ Mall,
                                                         int N) {
    const int f = blockIdx.x;
    const size_t NN = (size_t)N * N;
    extern __shared__ double sm[];
    double* sb = sm;      // D_b^-1
    double* ss = sm + N;  // D_s
    for (int i = threadIdx.x; i < N; i += kThreads) {
        const double l = lnD_all[(size_t)f * N + i];
        sb[i] = exp(-fmax(l, 0.0));
        ss[i] = exp(fmin(l, 0.0));
    }
    __syncthreads();
    const double* U = Uall + f * NN;
    const double* T = Tall + f * NN;
    double* M = Mall + f * NN;
    for (size_t idx = threadIdx.x; idx < NN; idx += kThreads) {  // M column-major, T row-major
        const int j = (int)(idx / N), i = (int)(idx - (size_t)j * N);
        M[idx] = fma(sb[i], U[(size_t)i * N + j], ss[i] * T[(size_t)i * N + j]);
    }
}

template <int MAXR>
__global__ void __launch_bounds__(kThreads) k_lu(double* __restrict__ Mall, int* __restrict__ piv_all,
                                                 const double* __restrict__ lnD_all, const int* __restrict__ sgnU,
                                                 double* __restrict__ lndet, int* __restrict__ sign,
                                                 unsigned int* __restrict__ err, int N) {
    const int f = blockIdx.x;
    const size_t NN = (size_t)N * N;
    double* __restrict__ M = Mall + f * NN;
    extern __shared__ double s_l[];  // [N] multipliers of the current step
    __shared__ int s_p;
    __shared__ double s_logabs;
    __shared__ int s_neg, s_sing;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_logabs = 0.0;
        s_neg = 0;
        s_sing = 0;
    }
    __syncthreads();
    for (int k = 0; k < N; ++k) {
        const int m = N - k;
        if (warp == 0) {
            double col[MAXR];
            double bv = -1.0;
            int bi = INT_MAX;
#pragma unroll
            for (int r = 0; r < MAXR; ++r) {
                const int ii = lane + 32 * r;
                col[r] = (ii < m) ? M[(size_t)k * N + k + ii] : 0.0;
                const double a = fabs(col[r]);
                if (ii < m && (a > bv || (a == bv && ii < bi))) {
                    bv = a;
                    bi = ii;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            if (bi == INT_MAX) bi = 0;  // NaN column: no swap
            // pivot value (row k+bi) and the current diagonal element (row k) it swaps with
            double pval = 0.0;
#pragma unroll
            for (int r = 0; r < MAXR; ++r) {
                const double vb = __shfl_sync(0xffffffffu, col[r], bi & 31);
                if (r == bi / 32) pval = vb;
            }
            const double top = __shfl_sync(0xffffffffu, col[0], 0);
            const double rinv = (pval != 0.0) ? 1.0 / pval : 0.0;
#pragma unroll
            for (int r = 0; r < MAXR; ++r) {
                const int ii = lane + 32 * r;
                if (ii >= m) continue;
                double v = col[r];
                if (ii == 0) v = pval;
                else if (ii == bi) v = top;
                if (ii == 0) {
                    M[(size_t)k * N + k] = v;
                } else {
                    const double l = v * rinv;
                    s_l[k + ii] = l;
                    M[(size_t)k * N + k + ii] = l;
                }
            }
            if (lane == 0) {
                s_p = k + bi;
                piv_all[(size_t)f * N + k] = k + bi;
                if (pval == 0.0) s_sing = 1;
                s_logabs += log(fabs(pval));
                s_neg ^= (pval < 0.0) ^ (bi != 0);
            }
        }
        __syncthreads();
        const int p = s_p;
        for (int j = warp; j < N; j += kWarps) {
            if (j == k) continue;
            double* Mj = M + (size_t)j * N;
            if (p != k && lane == 0) {
                const double a = Mj[k];
                Mj[k] = Mj[p];
                Mj[p] = a;
            }
            if (j < k) continue;
            __syncwarp();
            const double u = Mj[k];
#pragma unroll
            for (int r = 0; r < MAXR; ++r) {
                const int ii = lane + 32 * r;
                if (ii >= 1 && ii < m) Mj[k + ii] = fma(-s_l[k + ii], u, Mj[k + ii]);
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        double ld = s_logabs;
        for (int i = 0; i < N; ++i) ld += fmax(lnD_all[(size_t)f * N + i], 0.0);
        const bool ok = !s_sing && isfinite(ld);
        lndet[f] = ok ? ld : __longlong_as_double(0x7ff8000000000000ll);
        sign[f] = ok ? (sgnU[f] * (s_neg ? -1 : 1)) : 0;
        if (s_sing) atomicOr(err, SLMC_EBIT_SINGULAR);
        else if (!ok) atomicOr(err, SLMC_EBIT_NONFINITE);
    }
}

// G[:, j] = M^-1 (D_b^-1 U^T)[:, j] with the LU factors of M; one warp per column, the
// right-hand side kept in shared memory. Output row-major G[f][i][j].
template <int MAXR>
__global__ void __launch_bounds__(256) k_greens(const double* __restrict__ LUall, const int* __restrict__ piv_all,
                                                const double* __restrict__ Uall, const double* __restrict__ lnD_all,
                                                double* __restrict__ Gout, int N) {
    const int f = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * 8 + warp;
    extern __shared__ double sm[];
    double* b = sm + (size_t)warp * N;
    if (j >= N) return;
    const size_t NN = (size_t)N * N;
    const double* __restrict__ LU = LUall + f * NN;
    const double* __restrict__ U = Uall + f * NN;
    const double* __restrict__ lnD = lnD_all + (size_t)f * N;
    const int* __restrict__ piv = piv_all + (size_t)f * N;
    for (int i = lane; i < N; i += 32) b[i] = exp(-fmax(lnD[i], 0.0)) * U[(size_t)i * N + j];
    __syncwarp();
    if (lane == 0) {
        for (int k = 0; k < N; ++k) {
            const int p = piv[k];
            if (p != k) {
                const double a = b[k];
                b[k] = b[p];
                b[p] = a;
            }
        }
    }
    __syncwarp();
    for (int k = 0; k < N - 1; ++k) {  // unit lower triangle
        const double yk = b[k];
        const double* __restrict__ col = LU + (size_t)k * N;
#pragma unroll
        for (int r = 0; r < MAXR; ++r) {
            const int i = lane + 32 * r;
            if (i > k && i < N) b[i] = fma(-col[i], yk, b[i]);
        }
        __syncwarp();
    }
    for (int k = N - 1; k >= 0; --k) {  // upper triangle
        const double* __restrict__ col = LU + (size_t)k * N;
        const double gk = b[k] / col[k];
        __syncwarp();
        if (lane == 0) b[k] = gk;
#pragma unroll
        for (int r = 0; r < MAXR; ++r) {
            const int i = lane + 32 * r;
            if (i < k) b[i] = fma(-col[i], gk, b[i]);
        }
        __syncwarp();
    }
    for (int i = lane; i < N; i += 32) Gout[f * NN + (size_t)i * N + j] = b[i];
}

// Right-looking blocked LU with partial pivoting of M (column-major, in global memory), one CTA
// per field, panels of 32 columns. The panel is factored in shared memory one column at a time
// (pivot search by warp 0, ties to the lowest row); its row interchanges are then applied to the
// other columns, the panel's 32 rows of U to its right are solved against its unit lower
// triangle (one thread per column, values in registers), and the trailing matrix receives the
// rank-32 update (one thread per row and 8 columns, plain FMAs). Same factors (LAPACK
// convention: piv[k] = row interchanged with row k at step k) as the unblocked kernel, up to
// rounding; ln|det M| and the sign are accumulated from the pivots.
constexpr int kLB = 32;  // panel width
constexpr int kLS = 33;  // padded row stride of the panel in shared memory

__global__ void __launch_bounds__(256) k_lu_blk(double* __restrict__ Mall, int* __restrict__ piv_all,
                                                const double* __restrict__ lnD_all, const int* __restrict__ sgnU,
                                                double* __restrict__ lndet, int* __restrict__ sign,
                                                unsigned int* __restrict__ err, int N) {
    const int f = blockIdx.x;
    const size_t NN = (size_t)N * N;
    double* __restrict__ M = Mall + f * NN;
    int* __restrict__ piv = piv_all + (size_t)f * N;
    extern __shared__ __align__(16) unsigned char smraw[];
    double* P = reinterpret_cast<double*>(smraw);  // panel rows p0..N-1: P[(r - p0) * kLS + c]
    __shared__ int s_piv[kLB];
    __shared__ double s_logabs;
    __shared__ int s_neg, s_sing;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_logabs = 0.0;
        s_neg = 0;
        s_sing = 0;
    }
    for (int p0 = 0; p0 < N; p0 += kLB) {
        const int nb = min(kLB, N - p0), R = N - p0;
        __syncthreads();
        for (int idx = tid; idx < R * nb; idx += 256) {
            const int c = idx / R, rr = idx - c * R;
            P[rr * kLS + c] = M[(size_t)(p0 + c) * N + p0 + rr];
        }
        __syncthreads();
        // ---- panel ----
        for (int c = 0; c < nb; ++c) {
            if (warp == 0) {
                double bv = -1.0;
                int bi = R;
                for (int rr = c + lane; rr < R; rr += 32) {
                    const double a = fabs(P[rr * kLS + c]);
                    if (a > bv) {  // rows ascend per lane: ties keep the lower row
                        bv = a;
                        bi = rr;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (ov > bv || (ov == bv && oi < bi)) {
                        bv = ov;
                        bi = oi;
                    }
                }
                if (bi >= R) bi = c;  // no comparable entry (NaN column): no interchange
                if (lane == 0) {
                    const double pval = P[bi * kLS + c];
                    s_piv[c] = bi;
                    piv[p0 + c] = p0 + bi;
                    if (pval == 0.0) s_sing = 1;
                    s_logabs += log(fabs(pval));
                    s_neg ^= (pval < 0.0) ^ (bi != c);
                }
            }
            __syncthreads();
            const int bi = s_piv[c];
            if (bi != c && tid < nb) {
                const double a = P[c * kLS + tid];
                P[c * kLS + tid] = P[bi * kLS + tid];
                P[bi * kLS + tid] = a;
            }
            __syncthreads();
            const double pv = P[c * kLS + c];
            const double rinv = (pv != 0.0) ? 1.0 / pv : 0.0;
            for (int rr = c + 1 + tid; rr < R; rr += 256) {  // multiplier and rank-1 update of the row
                const double l = P[rr * kLS + c] * rinv;
                P[rr * kLS + c] = l;
                for (int j = c + 1; j < nb; ++j) P[rr * kLS + j] = fma(-l, P[c * kLS + j], P[rr * kLS + j]);
            }
            __syncthreads();
        }
        for (int idx = tid; idx < R * nb; idx += 256) {
            const int c = idx / R, rr = idx - c * R;
            M[(size_t)(p0 + c) * N + p0 + rr] = P[rr * kLS + c];
        }
        // ---- interchanges on the other columns; rows of U to the right of the panel ----
        for (int j = tid; j < N; j += 256) {
            if (j >= p0 && j < p0 + nb) continue;
            double* __restrict__ Mj = M + (size_t)j * N;
            for (int c = 0; c < nb; ++c) {
                const int bi = s_piv[c];
                if (bi != c) {
                    const double a = Mj[p0 + c];
                    Mj[p0 + c] = Mj[p0 + bi];
                    Mj[p0 + bi] = a;
                }
            }
            if (j >= p0 + nb) {  // U12[:, j] = L11^-1 A12[:, j]
                double x[kLB];
#pragma unroll
                for (int i = 0; i < kLB; ++i) x[i] = (i < nb) ? Mj[p0 + i] : 0.0;
#pragma unroll
                for (int c = 0; c < kLB - 1; ++c) {
#pragma unroll
                    for (int i = c + 1; i < kLB; ++i)
                        if (i < nb) x[i] = fma(-P[i * kLS + c], x[c], x[i]);
                }
#pragma unroll
                for (int i = 0; i < kLB; ++i)
                    if (i < nb) Mj[p0 + i] = x[i];
            }
        }
        __syncthreads();
        // ---- trailing update A22 -= L21 U12 ----
        const int nr = N - p0 - nb;
        const int ncg = (nr + 7) / 8;
        for (int item = tid; item < nr * ncg; item += 256) {
            const int rr = item % nr, g = item / nr;
            const int i = p0 + nb + rr, j0 = p0 + nb + 8 * g;
            double acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = (j0 + q < N) ? M[(size_t)(j0 + q) * N + i] : 0.0;
            for (int c = 0; c < nb; ++c) {
                const double l = P[(nb + rr) * kLS + c];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (j0 + q < N) acc[q] = fma(-l, M[(size_t)(j0 + q) * N + p0 + c], acc[q]);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (j0 + q < N) M[(size_t)(j0 + q) * N + i] = acc[q];
        }
    }
    __syncthreads();
    if (tid == 0) {
        double ld = s_logabs;
        for (int i = 0; i < N; ++i) ld += fmax(lnD_all[(size_t)f * N + i], 0.0);
        const bool ok = !s_sing && isfinite(ld);
        lndet[f] = ok ? ld : __longlong_as_double(0x7ff8000000000000ll);
        sign[f] = ok ? (sgnU[f] * (s_neg ? -1 : 1)) : 0;
        if (s_sing) atomicOr(err, SLMC_EBIT_SINGULAR);
        else if (!ok) atomicOr(err, SLMC_EBIT_NONFINITE);
    }
}

// G[:, j0..j0+31] = M^-1 (D_b^-1 U^T)[:, j0..j0+31] with the LU factors of M (P M = L U'),
// blocked over rows in blocks of 32. One CTA owns 32 right-hand-side columns of one field,
// held in shared memory row-major with a padded row stride (X[i][c] at i * 33 + c):
//   forward (unit L):  for each row block: solve the 32 x 32 diagonal block (warp w owns
//                      columns 4w..4w+3, lane = row, values in registers, shuffles only), then
//                      subtract its contribution from every row below (a rank-32 update, each
//                      thread one row and 8 columns: plain FMAs, no reductions);
//   backward (U'):     the same from the bottom block up, with the diagonal reciprocals.
// Output row-major G[f][i][j].
constexpr int kGB = 32;   // rows per block = right-hand sides per CTA
constexpr int kGS = 33;   // padded row stride of X (doubles)

__global__ void __launch_bounds__(256) k_greens_blk(const double* __restrict__ LUall, const int* __restrict__ piv_all,
                                                    const double* __restrict__ Uall, const double* __restrict__ lnD_all,
                                                    double* __restrict__ Gout, int N) {
    const int f = blockIdx.y, j0 = blockIdx.x * kGB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t NN = (size_t)N * N;
    const double* __restrict__ LU = LUall + f * NN;
    const double* __restrict__ U = Uall + f * NN;
    const double* __restrict__ lnD = lnD_all + (size_t)f * N;
    extern __shared__ __align__(16) unsigned char smraw[];
    double* X = reinterpret_cast<double*>(smraw);          // [N][kGS]
    double* rdiag = X + (size_t)N * kGS;                    // [N]
    int* src = reinterpret_cast<int*>(rdiag + N);           // [N] row of B that lands in row i of P B
    if (tid == 0) {
        for (int i = 0; i < N; ++i) src[i] = i;
        const int* piv = piv_all + (size_t)f * N;
        for (int k = 0; k < N; ++k) {
            const int p = piv[k];
            if (p != k) {
                const int a = src[k];
                src[k] = src[p];
                src[p] = a;
            }
        }
    }
    for (int i = tid; i < N; i += 256) rdiag[i] = 1.0 / LU[(size_t)i * N + i];
    __syncthreads();
    // X = P D_b^-1 U^T restricted to the CTA's columns (columns beyond N are zero)
    for (int idx = tid; idx < N * kGB; idx += 256) {
        const int i = idx / kGB, c = idx - i * kGB, j = j0 + c;
        const int r = src[i];
        X[i * kGS + c] = (j < N) ? exp(-fmax(lnD[r], 0.0)) * U[(size_t)r * N + j] : 0.0;
    }
    __syncthreads();
    const int nblk = (N + kGB - 1) / kGB;
    // ---- forward substitution with the unit lower factor ----
    for (int b = 0; b < nblk; ++b) {
        const int kb = b * kGB, nb = min(kGB, N - kb);
        {   // diagonal block: warp w owns columns 4w..4w+3, lane = row kb + lane
            const int i = kb + lane;
            double x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = (lane < nb) ? X[i * kGS + 4 * warp + q] : 0.0;
            for (int k = 0; k < nb - 1; ++k) {
                const double l = (lane > k && lane < nb) ? LU[(size_t)(kb + k) * N + i] : 0.0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double xk = __shfl_sync(0xffffffffu, x[q], k);
                    if (lane > k) x[q] = fma(-l, xk, x[q]);
                }
            }
            if (lane < nb) {
#pragma unroll
                for (int q = 0; q < 4; ++q) X[i * kGS + 4 * warp + q] = x[q];
            }
        }
        __syncthreads();
        // rows below the block: X[i][:] -= L[i][kb:kb+nb] X[kb:kb+nb][:]; item = (row, 8 columns)
        const int r0 = kb + nb, nrows = N - r0;
        for (int item = tid; item < nrows * 4; item += 256) {
            const int i = r0 + (item >> 2), c0 = (item & 3) * 8;
            double acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = X[i * kGS + c0 + q];
            for (int k = 0; k < nb; ++k) {
                const double l = LU[(size_t)(kb + k) * N + i];
                const double* xk = X + (kb + k) * kGS + c0;
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[q] = fma(-l, xk[q], acc[q]);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) X[i * kGS + c0 + q] = acc[q];
        }
        __syncthreads();
    }
    // ---- backward substitution with the upper factor ----
    for (int b = nblk - 1; b >= 0; --b) {
        const int kb = b * kGB, nb = min(kGB, N - kb);
        {
            const int i = kb + lane;
            double x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = (lane < nb) ? X[i * kGS + 4 * warp + q] : 0.0;
            const double rd = (lane < nb) ? rdiag[i] : 0.0;
            for (int k = nb - 1; k >= 0; --k) {
                const double u = (lane < k) ? LU[(size_t)(kb + k) * N + i] : 0.0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (lane == k) x[q] *= rd;
                    const double xk = __shfl_sync(0xffffffffu, x[q], k);
                    if (lane < k) x[q] = fma(-u, xk, x[q]);
                }
            }
            if (lane < nb) {
#pragma unroll
                for (int q = 0; q < 4; ++q) X[i * kGS + 4 * warp + q] = x[q];
            }
        }
        __syncthreads();
        // rows above the block: X[i][:] -= U'[i][kb:kb+nb] X[kb:kb+nb][:]
        for (int item = tid; item < kb * 4; item += 256) {
            const int i = item >> 2, c0 = (item & 3) * 8;
            double acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = X[i * kGS + c0 + q];
            for (int k = 0; k < nb; ++k) {
                const double u = LU[(size_t)(kb + k) * N + i];
                const double* xk = X + (kb + k) * kGS + c0;
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[q] = fma(-u, xk[q], acc[q]);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) X[i * kGS + c0 + q] = acc[q];
        }
        __syncthreads();
    }
    for (int idx = tid; idx < N * kGB; idx += 256) {
        const int i = idx / kGB, c = idx - i * kGB, j = j0 + c;
        if (j < N) Gout[f * NN + (size_t)i * N + j] = X[i * kGS + c];
    }
}

template <int MAXR>
cudaError_t launch_final(slmc_ctx* c, int nf, double* lndet, int* sign, cudaStream_t s, bool assemble) {
    const int N = c->N;
    if (assemble) k_assemble_M<<<nf, kThreads, 2 * N * sizeof(double), s>>>(c->U, c->Ta, c->lnD, c->Y, N);
    const size_t smem = (size_t)N * kLS * sizeof(double);
    if (smem <= 227 * 1024) {  // blocked LU (the panel fits in shared memory)
        cudaError_t e = cudaFuncSetAttribute(k_lu_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_lu_blk<<<nf, 256, smem, s>>>(c->Y, c->piv, c->lnD, c->sgnU, lndet, sign, c->err, N);
        return cudaGetLastError();
    }
    k_lu<MAXR><<<nf, kThreads, N * sizeof(double), s>>>(c->Y, c->piv, c->lnD, c->sgnU, lndet, sign, c->err, N);
    return cudaGetLastError();
}

template <int MAXR>
cudaError_t launch_greens(slmc_ctx* c, int nf, double* G, cudaStream_t s) {
    const int N = c->N;
    const size_t smem = (size_t)8 * N * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_greens<MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((N + 7) / 8, nf);
    k_greens<MAXR><<<grid, 256, smem, s>>>(c->Y, c->piv, c->U, c->lnD, G, N);
    return cudaGetLastError();
}

}  // namespace

namespace slmc {

namespace {
cudaError_t final_dispatch(slmc_ctx* c, int nf, double* lndet, int* sign, cudaStream_t s, bool assemble) {
    switch (rows_per_lane_class(c->N)) {
        case 1: return launch_final<1>(c, nf, lndet, sign, s, assemble);
        case 2: return launch_final<2>(c, nf, lndet, sign, s, assemble);
        case 4: return launch_final<4>(c, nf, lndet, sign, s, assemble);
        case 5: return launch_final<5>(c, nf, lndet, sign, s, assemble);
        case 8: return launch_final<8>(c, nf, lndet, sign, s, assemble);
        case 12: return launch_final<12>(c, nf, lndet, sign, s, assemble);
        case 18: return launch_final<18>(c, nf, lndet, sign, s, assemble);
        default: return launch_final<32>(c, nf, lndet, sign, s, assemble);
    }
}
}  // namespace

cudaError_t final_logdet(slmc_ctx* c, int nf, double* lndet, int* sign, cudaStream_t s) {
    return final_dispatch(c, nf, lndet, sign, s, true);
}

cudaError_t final_lu(slmc_ctx* c, int nf, double* lndet, int* sign, cudaStream_t s) {
    return final_dispatch(c, nf, lndet, sign, s, false);
}

cudaError_t final_greens(slmc_ctx* c, int nf, double* G, cudaStream_t s) {
    const int N = c->N;
    const size_t smem = (size_t)N * kGS * sizeof(double) + (size_t)N * (sizeof(double) + sizeof(int));
    if (smem <= 227 * 1024) {  // blocked solve (the column-per-warp kernel below covers larger N)
        cudaError_t e = cudaFuncSetAttribute(k_greens_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        dim3 grid((N + kGB - 1) / kGB, nf);
        k_greens_blk<<<grid, 256, smem, s>>>(c->Y, c->piv, c->U, c->lnD, G, N);
        return cudaGetLastError();
    }
    switch (rows_per_lane_class(c->N)) {
        case 1: return launch_greens<1>(c, nf, G, s);
        case 2: return launch_greens<2>(c, nf, G, s);
        case 4: return launch_greens<4>(c, nf, G, s);
        case 5: return launch_greens<5>(c, nf, G, s);
        case 8: return launch_greens<8>(c, nf, G, s);
        case 12: return launch_greens<12>(c, nf, G, s);
        case 18: return launch_greens<18>(c, nf, G, s);
        default: return launch_greens<32>(c, nf, G, s);
    }
}

}  // namespace slmc
