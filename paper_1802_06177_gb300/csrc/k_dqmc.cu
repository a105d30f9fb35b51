// Conventional DQMC updates of the phonon field [Supplemental Material, Eqs. (S3)-(S6) and
// the block update described after them], the baseline the self-learning method is compared
// with.
//
// Local updates: at time slice l the equal-time Green's function G(l) (row-major, one chain
// per CTA) decides the move of x_{i,l-1} through the fast ratio R = 1 + (1 - G_ii) Delta_ii,
// Delta_ii = exp(-dtau lam d) - 1 (Eq. (S5)); with both spin species the weight ratio is
// R^2 exp(d ln w_bose). An accepted move updates G by Sherman-Morrison,
// G -= (Delta_ii / R) G[:, i] (e_i - G[i, :]) (Eq. (S6)). Between slices G(l) = B_l G(l-1) B_l^-1
// with B_l = diag(s) exp(-dtau K); at the start of every group of n_s slices G is recomputed
// from two stabilised products (dqmc_combine below).
//
// FP64 issue is the scarce resource on this GPU (about two FMAs per clock per SM), so the
// kernel spends it only on the arithmetic the method needs:
//  * exp(-dtau K) of the periodic square lattice factorises exactly into
//    e^{dtau mu} (E_x kron E_y), E_x and E_y symmetric circulant (the hopping along x and
//    along y commute); the mu factors of B_l and B_l^-1 cancel, and the wrap becomes four
//    in-place circulant transforms along the lines of G: 2 N^2 (Lx + Ly) FMAs instead of
//    the 2 N^3 of two dense products;
//  * G stays in shared memory when it fits (N <= 160), else in global memory (L2-resident). There the
//    accepted moves of a slice are delayed in batches of up to 32 (Ad, Bd in shared memory, with the
//    running diagonal of G for the decisions; the batch size is what the shared memory left holds):
//    each new move needs only the current column and row of G, and the batch is added to G in one
//    register-tiled pass. Every entry is formed by the same FMA chain in the same order as immediate
//    rank-1 updates, so the results are bit-identical, for one read and write of G per batch
//    instead of per move;
//  * the proposal, Delta_ii, exp(d ln w_bose) and both uniforms of every site of a slice are
//    computed in parallel before the slice's sites are visited; each thread then takes the
//    site's decision itself (u < R^2 exp(d ln w_bose), the same test as
//    ln(R^2) + d ln w_bose compared with ln u up to rounding), so a rejected move costs no
//    barrier and an accepted one costs the N^2 FMAs of the rank-1 update and two barriers.
// Sites of a slice are visited in order; the proposal x' = x + U[-Delta, Delta] and the
// acceptance uniform come from Philox counter (i L + l - 1, sweep, chain, 3). The new field is
// rounded step by step as in the oracle, so accepted moves leave identical fields.
//
// Block updates reflect one site's whole column (x -> -x) and are accepted with the ratio of
// full weights (computed by the determinant path); the site and the uniform come from Philox
// counter (k, sweep, chain, 4).
#include "slmc_internal.cuh"

#include <algorithm>

namespace {

constexpr int kThreads = 256;

// G0 += sum_{q < cnt} A_q B_q^T in place (rows by warps, 4 columns per lane per pass), each entry by the
// FMA chain of cnt immediate rank-1 updates in their order: the result equals theirs bit for bit, for
// one read and one write of G per batch instead of per accepted move.
__device__ __forceinline__ void dqmc_flush(double* G, const double* Ad, const double* Bd, int cnt, int N, int lane,
                                           int warp) {
    for (int j = warp; j < N; j += kThreads / 32) {
        double* Gj = G + (size_t)j * N;
        for (int m0 = 0; m0 < N; m0 += 128) {
            double acc[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int m = m0 + lane + 32 * t;
                acc[t] = m < N ? Gj[m] : 0.0;
            }
            for (int q = 0; q < cnt; ++q) {
                const double aj = Ad[q * N + j];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int m = m0 + lane + 32 * t;
                    if (m < N) acc[t] = fma(aj, Bd[q * N + m], acc[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int m = m0 + lane + 32 * t;
                if (m < N) Gj[m] = acc[t];
            }
        }
    }
}

template <int LMAX>
__global__ void __launch_bounds__(kThreads) k_dqmc_slices(double* __restrict__ x, double* __restrict__ Gall, int Lx,
                                                          int Ly, int L, int l0, int nsl, double dtau,
                                                          const double* __restrict__ kron,
                                                          double lam, double w02, double delta, uint32_t key0,
                                                          uint32_t key1, uint32_t sweep, int chain0, int g_in_smem,
                                                          int kd, unsigned long long* __restrict__ n_acc) {
    extern __shared__ double dsm[];
    constexpr int QMAX = (LMAX * LMAX + 31) / 32;  // columns per lane in the rank-1 update
    const int N = Lx * Ly;
    const int f = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t NN = (size_t)N * N;
    double* G = g_in_smem ? dsm : Gall + f * NN;
    double* p = g_in_smem ? dsm + NN : dsm;
    double* s = p;                 // [N] slice scales exp(-dtau lam x_{i,l-1})
    double* sinv = p + N;          // [N] 1 / s
    double* xn = p + 2 * N;        // [N] proposed field
    double* dl = p + 3 * N;        // [N] Delta_ii
    double* eb = p + 4 * N;        // [N] exp(d ln w_bose)
    double* ua = p + 5 * N;        // [N] acceptance uniform
    double* ac = p + 6 * N;        // [N] -(Delta_ii / R) G[:, i]
    double* rw = p + 7 * N;        // [N] e_i - G[i, :]
    double* ex = p + 8 * N;        // [2 Lx] E_x
    double* exi = ex + slmc::kKronTab;   // [2 Lx] E_x^-1
    double* ey = exi + slmc::kKronTab;   // [2 Ly] E_y
    double* eyi = ey + slmc::kKronTab;   // [2 Ly] E_y^-1
    // delayed updates (kd > 0, G in global memory): accepted moves q < cnt of the current batch as
    // G = G0 + sum_q A_q B_q^T, A_q = -(Delta/R) G[:, i_q], B_q = e_i - G[i_q, :] ([kd][N] each), and the
    // running diagonal of G
    double* Ad = eyi + slmc::kKronTab;
    double* Bd = Ad + (size_t)kd * N;
    double* dg = Bd + (size_t)kd * N;
    double* xf = x + (size_t)f * N * L;
    const uint32_t chain = (uint32_t)(chain0 + f);

    for (int k = tid; k < 4 * slmc::kKronTab; k += kThreads) ex[k] = kron[k];  // ex, exi, ey, eyi are contiguous
    if (g_in_smem) {
        const double2* src = reinterpret_cast<const double2*>(Gall + f * NN);
        double2* dst = reinterpret_cast<double2*>(G);
        for (size_t k = tid; k < NN / 2; k += kThreads) dst[k] = src[k];
        if ((NN & 1) && tid == 0) G[NN - 1] = Gall[f * NN + NN - 1];
    }
    int accepted = 0;
    for (int l = l0 + 1; l <= l0 + nsl; ++l) {
        const int c = l - 1;
        const int cu = c + 1 == L ? 0 : c + 1, cd = c == 0 ? L - 1 : c - 1;
        for (int i = tid; i < N; i += kThreads) {
            const double v = xf[(size_t)i * L + c];
            const slmc::u32x4 w = slmc::philox4x32_10(slmc::u32x4{(uint32_t)(i * L + c), sweep, chain, 3u}, key0, key1);
            const double u1 = slmc::uniform53(w.x, w.y);
            const double xp = __dadd_rn(v, __dmul_rn(delta, __dadd_rn(__dmul_rn(2.0, u1), -1.0)));
            const double up = xf[(size_t)i * L + cu], dn = xf[(size_t)i * L + cd];
            const double kin = ((up - xp) * (up - xp) + (xp - dn) * (xp - dn) - (up - v) * (up - v) -
                                (v - dn) * (v - dn)) / (2.0 * dtau * dtau);
            const double dlb = dtau * lam * (xp - v) - dtau * (0.5 * w02 * (xp * xp - v * v) + kin);
            s[i] = exp(-dtau * lam * v);
            sinv[i] = exp(dtau * lam * v);
            xn[i] = xp;
            dl[i] = exp(-dtau * lam * (xp - v)) - 1.0;
            eb[i] = exp(dlb);
            ua[i] = slmc::uniform53(w.z, w.w);
        }
        __syncthreads();
        // wrap: G <- diag(s) (E_x kron E_y) G (E_x kron E_y)^-1 diag(1/s), site i = ix + Lx iy
        for (int q = tid; q < N * Lx; q += kThreads)  // right factor along y: lines (i, jx)
            slmc::circ_line<LMAX, false>(G, (q / Lx) * N + q % Lx, Lx, Ly, eyi, nullptr, 0, nullptr, 0, 1.0);
        __syncthreads();
        for (int q = tid; q < N * Ly; q += kThreads)  // right factor along x: lines (i, jy)
            slmc::circ_line<LMAX, false>(G, (q / Ly) * N + (q % Ly) * Lx, 1, Lx, exi, nullptr, 0, nullptr, 0, 1.0);
        __syncthreads();
        for (int q = tid; q < Ly * N; q += kThreads)  // left factor along x: lines (iy, j)
            slmc::circ_line<LMAX, true>(G, (q / N) * Lx * N + q % N, N, Lx, ex, nullptr, 0, nullptr, 0, 1.0);
        __syncthreads();
        for (int q = tid; q < Lx * N; q += kThreads) {  // left factor along y, then the scales
            const int ix = q / N, j = q % N;
            slmc::circ_line<LMAX, true>(G, ix * N + j, Lx * N, Ly, ey, nullptr, 0, s + ix, Lx, sinv[j]);  // row ix + Lx d
        }
        __syncthreads();
        if (kd > 0) {
            for (int j = tid; j < N; j += kThreads) dg[j] = G[(size_t)j * N + j];
            __syncthreads();
        }
        int cnt = 0;  // delayed moves of the current batch (block-uniform)
        for (int i = 0; i < N; ++i) {
            // every thread takes the same decision from the same G_ii
            const double gii = kd > 0 ? dg[i] : G[(size_t)i * N + i];
            const double R = __dadd_rn(1.0, __dmul_rn(__dadd_rn(1.0, -gii), dl[i]));
            if (!(ua[i] < R * R * eb[i])) continue;
            const double a = dl[i] * __drcp_rn(R);
            if (kd > 0) {
                // the current column G[:, i] and row G[i, :] from G0 and the batch, each entry by the
                // same FMA chain the immediate update would have applied to it
                for (int j = tid; j < N; j += kThreads) {
                    double cj = G[(size_t)j * N + i], rj = G[(size_t)i * N + j];
                    for (int q = 0; q < cnt; ++q) {
                        cj = fma(Ad[q * N + j], Bd[q * N + i], cj);
                        rj = fma(Ad[q * N + i], Bd[q * N + j], rj);
                    }
                    const double aj = -a * cj;
                    const double bj = (j == i ? 1.0 : 0.0) - rj;
                    Ad[cnt * N + j] = aj;
                    Bd[cnt * N + j] = bj;
                    dg[j] = fma(aj, bj, dg[j]);
                }
                if (tid == 0) {
                    xf[(size_t)i * L + c] = xn[i];
                    ++accepted;
                }
                __syncthreads();
                if (++cnt == kd) {
                    dqmc_flush(G, Ad, Bd, cnt, N, lane, warp);
                    cnt = 0;
                    __syncthreads();
                }
                continue;
            }
            for (int j = tid; j < N; j += kThreads) {
                ac[j] = -a * G[(size_t)j * N + i];
                rw[j] = (j == i ? 1.0 : 0.0) - G[(size_t)i * N + j];
            }
            if (tid == 0) {
                xf[(size_t)i * L + c] = xn[i];
                ++accepted;
            }
            __syncthreads();
            // rank-1 update, one row per warp at a time: the row's coefficient is loaded once and
            // the lane's entries of e_i - G[i, :] stay in registers (N <= LMAX^2 = 32 QMAX)
            double r[QMAX];
#pragma unroll
            for (int q = 0; q < QMAX; ++q) r[q] = lane + 32 * q < N ? rw[lane + 32 * q] : 0.0;
            for (int j = warp; j < N; j += kThreads / 32) {
                const double cj = ac[j];
                double* Gj = G + (size_t)j * N;
#pragma unroll
                for (int q = 0; q < QMAX; ++q)
                    if (lane + 32 * q < N) Gj[lane + 32 * q] = fma(cj, r[q], Gj[lane + 32 * q]);
            }
            __syncthreads();
        }
        if (cnt > 0) dqmc_flush(G, Ad, Bd, cnt, N, lane, warp);  // the slice's last batch
        __syncthreads();  // rejected sites take no barrier: the next slice's tables wait for all threads here
    }
    if (tid == 0 && n_acc) n_acc[f] += (unsigned long long)accepted;
}

// Block update k: reflect the whole column of one site of every chain (in place) and draw the
// acceptance uniform u[f].
__global__ void k_block_propose(double* __restrict__ x, int N, int L, uint32_t key0, uint32_t key1, uint32_t sweep,
                                uint32_t k, int chain0, double* __restrict__ u) {
    const int f = blockIdx.x;
    const slmc::u32x4 w = slmc::philox4x32_10(slmc::u32x4{k, sweep, (uint32_t)(chain0 + f), 4u}, key0, key1);
    const int s0 = (int)(slmc::uniform53(w.x, w.y) * (double)N);
    const int site = s0 < N - 1 ? s0 : N - 1;
    double* xs = x + ((size_t)f * N + site) * L;
    for (int l = threadIdx.x; l < L; l += blockDim.x) xs[l] = -xs[l];
    if (threadIdx.x == 0) u[f] = slmc::uniform53(w.z, w.w);
}

// G(g0) from two stabilised products. With B(g0, 0) = U_R D_R T_R (the running chain of the
// slices already visited in this sweep) and B(L, g0)^T = U_L D_L T_L (the transposed chain of
// the slices still to come, kept from the start of the sweep), D = D_b D_s (D_b = max(D, 1),
// D_s = min(D, 1)):
//   I + B(g0, 0) B(L, g0) = U_R D_bR M D_bL U_L^T,
//   M = D_bR^-1 (U_R^T U_L) D_bL^-1 + D_sR (T_R T_L^T) D_sL,
//   G(g0) = U_L D_bL^-1 M^-1 D_bR^-1 U_R^T,
// M bounded entry-wise by the scale split, so its LU carries no exponentially large or small
// numbers (the same split as the final step of the determinant path).
struct GemmTerm {
    const double* A;   // A(i, k): A[i N + k] (kAik) or A[k N + i]
    const double* B;   // B(k, j): B[j N + k] (kBjk) or B[k N + j]
    const double* ra;  // optional row scales of A, [nf][sstride]
    const double* sk;  // optional scales of the summation index, applied to B
    const double* cb;  // optional column scales of B
};
struct GemmArgs {
    GemmTerm t[2];
    int nterms;
};

// C = sum over terms of diag(ra) A diag(sk) B diag(cb), one field per blockIdx.z, a TM x TM
// tile per CTA (4 x 4 outputs per thread), k-tiles of 16 staged in shared memory.
template <int TM, bool kAik, bool kBjk, bool kCrow>
__global__ void __launch_bounds__((TM / 4) * (TM / 4)) k_gemm64(GemmArgs g, double* __restrict__ C, int N,
                                                                int sstride) {
    constexpr int TT = TM / 4, NT = TT * TT, BK = 16;
    __shared__ __align__(16) double As[BK][TM];
    __shared__ __align__(16) double Bs[BK][TM];
    const int f = blockIdx.z, i0 = blockIdx.y * TM, j0 = blockIdx.x * TM;
    const int tid = threadIdx.x, tx = tid % TT, ty = tid / TT;
    const size_t NN = (size_t)N * N;
    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = 0.0;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        if (t >= g.nterms) break;
        const double* A = g.t[t].A + f * NN;
        const double* B = g.t[t].B + f * NN;
        const double* ra = g.t[t].ra ? g.t[t].ra + (size_t)f * sstride : nullptr;
        const double* sk = g.t[t].sk ? g.t[t].sk + (size_t)f * sstride : nullptr;
        const double* cb = g.t[t].cb ? g.t[t].cb + (size_t)f * sstride : nullptr;
        for (int k0 = 0; k0 < N; k0 += BK) {
            for (int q = tid; q < TM * BK; q += NT) {
                const int ii = kAik ? q / BK : q % TM, kk = kAik ? q % BK : q / TM;
                const int i = i0 + ii, k = k0 + kk;
                double v = 0.0;
                if (i < N && k < N) {
                    v = kAik ? A[(size_t)i * N + k] : A[(size_t)k * N + i];
                    if (ra) v *= ra[i];
                }
                As[kk][ii] = v;
            }
            for (int q = tid; q < TM * BK; q += NT) {
                const int jj = kBjk ? q / BK : q % TM, kk = kBjk ? q % BK : q / TM;
                const int j = j0 + jj, k = k0 + kk;
                double v = 0.0;
                if (j < N && k < N) {
                    v = kBjk ? B[(size_t)j * N + k] : B[(size_t)k * N + j];
                    if (sk) v *= sk[k];
                    if (cb) v *= cb[j];
                }
                Bs[kk][jj] = v;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const double2 a01 = *reinterpret_cast<const double2*>(&As[kk][ty * 4]);
                const double2 a23 = *reinterpret_cast<const double2*>(&As[kk][ty * 4 + 2]);
                const double2 b01 = *reinterpret_cast<const double2*>(&Bs[kk][tx * 4]);
                const double2 b23 = *reinterpret_cast<const double2*>(&Bs[kk][tx * 4 + 2]);
                const double a[4] = {a01.x, a01.y, a23.x, a23.y}, b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty * 4 + r;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + tx * 4 + q;
            if (i < N && j < N) C[f * NN + (kCrow ? (size_t)i * N + j : (size_t)j * N + i)] = acc[r][q];
        }
    }
}

// S[f] = [D_bR^-1 | D_sR | D_bL^-1 | D_sL], each [N], from the ln D of both products
__global__ void k_split_scales(const double* __restrict__ lnR, const double* __restrict__ lnL, double* __restrict__ S,
                               int N) {
    const int f = blockIdx.x;
    double* Sf = S + (size_t)f * 4 * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double r = lnR[(size_t)f * N + i], l = lnL[(size_t)f * N + i];
        Sf[i] = exp(-fmax(r, 0.0));
        Sf[N + i] = exp(fmin(r, 0.0));
        Sf[2 * N + i] = exp(-fmax(l, 0.0));
        Sf[3 * N + i] = exp(fmin(l, 0.0));
    }
}

template <int TM, bool kAik, bool kBjk, bool kCrow>
cudaError_t launch_gemm(const GemmArgs& g, double* C, int N, int nf, int sstride, cudaStream_t s) {
    dim3 grid((N + TM - 1) / TM, (N + TM - 1) / TM, nf);
    k_gemm64<TM, kAik, kBjk, kCrow><<<grid, (TM / 4) * (TM / 4), 0, s>>>(g, C, N, sstride);
    return cudaGetLastError();
}

// the tile (32, 48 or 64) that pads N least, the larger on ties
template <bool kAik, bool kBjk, bool kCrow>
cudaError_t gemm64(const GemmArgs& g, double* C, int N, int nf, int sstride, cudaStream_t s) {
    const int p32 = (N + 31) / 32 * 32, p48 = (N + 47) / 48 * 48, p64 = (N + 63) / 64 * 64;
    if (p64 <= p48 && p64 <= p32) return launch_gemm<64, kAik, kBjk, kCrow>(g, C, N, nf, sstride, s);
    if (p48 <= p32) return launch_gemm<48, kAik, kBjk, kCrow>(g, C, N, nf, sstride, s);
    return launch_gemm<32, kAik, kBjk, kCrow>(g, C, N, nf, sstride, s);
}

size_t dqmc_smem_bytes(int N, bool g_in_smem, int kd = 0) {
    return ((g_in_smem ? (size_t)N * N : 0) + 8 * (size_t)N + 4 * slmc::kKronTab + (kd > 0 ? (2 * (size_t)kd + 1) * N : 0)) *
           sizeof(double);
}

constexpr int kDelayMax = 32;  // accepted moves per delayed batch (G in global memory)

bool dqmc_supported(const slmc_ctx* c) { return c->L >= 2 && c->kron != nullptr; }

template <int LMAX>
cudaError_t launch_slices(slmc_ctx* c, double* x, double* G, int nf, int chain0, int l0, int nsl, uint64_t sweep,
                          long long* n_acc, cudaStream_t s) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const bool in_smem = dqmc_smem_bytes(c->N, true) <= (size_t)optin;
    // G in global memory: batch up to kd accepted moves in shared memory (delayed updates). With G in
    // shared memory the immediate rank-1 updates were faster (12x12: 463 against 418 chain-sweeps/s
    // with batches of 16), since there a pass over G costs no L2 traffic.
    int kd = 0;
    if (!in_smem) {
        kd = kDelayMax;
        while (kd > 1 && dqmc_smem_bytes(c->N, false, kd) > (size_t)optin) kd /= 2;
        if (dqmc_smem_bytes(c->N, false, kd) > (size_t)optin) kd = 0;
    }
    const size_t bytes = dqmc_smem_bytes(c->N, in_smem, kd);
    e = cudaFuncSetAttribute(k_dqmc_slices<LMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_dqmc_slices<LMAX><<<nf, kThreads, bytes, s>>>(
        x, G, c->p.Lx, c->p.Ly, c->L, l0, nsl, c->p.dtau, c->kron, c->p.lambda, c->p.omega0 * c->p.omega0,
        c->p.sweep_delta, (uint32_t)(c->p.seed & 0xffffffffu), (uint32_t)(c->p.seed >> 32), (uint32_t)sweep, chain0,
        in_smem ? 1 : 0, kd, reinterpret_cast<unsigned long long*>(n_acc));
    return cudaGetLastError();
}

}  // namespace

namespace slmc {

bool dqmc_ok(const slmc_ctx* c) { return dqmc_supported(c); }

cudaError_t dqmc_combine(slmc_ctx* c, const double* Ul, const double* lnDl, const double* Tl, int nf, double* G,
                         double* lndet_scratch, int* sign_scratch, cudaStream_t s) {
    const int N = c->N;
    double* S = c->Sws;  // [nf][4][N]: free between the steps of a chain
    k_split_scales<<<nf, 256, 0, s>>>(c->lnD, lnDl, S, N);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    GemmArgs m{};
    m.nterms = 2;
    m.t[0] = GemmTerm{c->U, Ul, S, nullptr, S + 2 * N};     // D_bR^-1 U_R^T U_L D_bL^-1
    m.t[1] = GemmTerm{c->Ta, Tl, S + N, nullptr, S + 3 * N};  // D_sR T_R T_L^T D_sL
    e = gemm64<true, true, false>(m, c->Y, N, nf, 4 * N, s);  // M column-major, as the LU expects
    if (e != cudaSuccess) return e;
    e = final_lu(c, nf, lndet_scratch, sign_scratch, s);
    if (e != cudaSuccess) return e;
    e = final_greens(c, nf, c->Tb, s);  // X = M^-1 D_bR^-1 U_R^T, row-major, in the idle T buffer
    if (e != cudaSuccess) return e;
    GemmArgs gg{};
    gg.nterms = 1;
    gg.t[0] = GemmTerm{Ul, c->Tb, nullptr, S + 2 * N, nullptr};  // U_L D_bL^-1 X
    return gemm64<false, false, true>(gg, G, N, nf, 4 * N, s);
}

cudaError_t dqmc_slices(slmc_ctx* c, double* x, double* G, int nf, int chain0, int l0, int nsl, uint64_t sweep,
                        long long* n_acc, cudaStream_t s) {
    const int lm = std::max(c->p.Lx, c->p.Ly);
    if (lm <= 8) return launch_slices<8>(c, x, G, nf, chain0, l0, nsl, sweep, n_acc, s);
    if (lm <= 16) return launch_slices<16>(c, x, G, nf, chain0, l0, nsl, sweep, n_acc, s);
    return launch_slices<32>(c, x, G, nf, chain0, l0, nsl, sweep, n_acc, s);
}

cudaError_t dqmc_block_propose(slmc_ctx* c, double* x, int nf, int chain0, uint64_t sweep, int k, double* u,
                               cudaStream_t s) {
    k_block_propose<<<nf, 128, 0, s>>>(x, c->N, c->L, (uint32_t)(c->p.seed & 0xffffffffu), (uint32_t)(c->p.seed >> 32),
                                       (uint32_t)sweep, (uint32_t)k, chain0, u);
    return cudaGetLastError();
}

}  // namespace slmc
