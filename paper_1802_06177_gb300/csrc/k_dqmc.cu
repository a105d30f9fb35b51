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
// from scratch by the stabilised determinant path on the time-rotated field.
//
// FP64 issue is the scarce resource on this GPU (about two FMAs per clock per SM), so the
// kernel spends it only on the arithmetic the method needs:
//  * exp(-dtau K) of the periodic square lattice factorises exactly into
//    e^{dtau mu} (E_x kron E_y), E_x and E_y symmetric circulant (the hopping along x and
//    along y commute); the mu factors of B_l and B_l^-1 cancel, and the wrap becomes four
//    in-place circulant transforms along the lines of G: 2 N^2 (Lx + Ly) FMAs instead of
//    the 2 N^3 of two dense products;
//  * G stays in shared memory when it fits (N <= 160), else in global memory (L2-resident);
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

// xr[f][i][c] = x[f][i][(c + g0) mod L]: column c of xr is the field of B_{g0 + c + 1}, so the
// Green's function G(L) of xr is G(g0) of x.
__global__ void k_rotate(const double* __restrict__ x, double* __restrict__ xr, int N, int L, int g0, size_t total) {
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t row = idx / L;
        const int c = (int)(idx - row * L);
        const int src = c + g0 < L ? c + g0 : c + g0 - L;
        xr[idx] = x[row * L + src];
    }
}

template <int LMAX>
__global__ void __launch_bounds__(kThreads) k_dqmc_slices(double* __restrict__ x, double* __restrict__ Gall, int Lx,
                                                          int Ly, int L, int l0, int nsl, double dtau,
                                                          const double* __restrict__ kron,
                                                          double lam, double w02, double delta, uint32_t key0,
                                                          uint32_t key1, uint32_t sweep, int chain0, int g_in_smem,
                                                          unsigned long long* __restrict__ n_acc) {
    extern __shared__ double dsm[];
    const int N = Lx * Ly;
    const int f = blockIdx.x, tid = threadIdx.x;
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
        for (int i = 0; i < N; ++i) {
            // every thread takes the same decision from the same G_ii
            const double R = __dadd_rn(1.0, __dmul_rn(__dadd_rn(1.0, -G[(size_t)i * N + i]), dl[i]));
            if (!(ua[i] < R * R * eb[i])) continue;
            const double a = dl[i] * __drcp_rn(R);
            for (int j = tid; j < N; j += kThreads) {
                ac[j] = -a * G[(size_t)j * N + i];
                rw[j] = (j == i ? 1.0 : 0.0) - G[(size_t)i * N + j];
            }
            if (tid == 0) {
                xf[(size_t)i * L + c] = xn[i];
                ++accepted;
            }
            __syncthreads();
            int j = tid / N, k = tid - (tid / N) * N;
            for (size_t idx = tid; idx < NN; idx += kThreads) {
                G[idx] = fma(ac[j], rw[k], G[idx]);
                k += kThreads;
                while (k >= N) {
                    k -= N;
                    ++j;
                }
            }
            __syncthreads();
        }
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

size_t dqmc_smem_bytes(int N, bool g_in_smem) {
    return ((g_in_smem ? (size_t)N * N : 0) + 8 * (size_t)N + 4 * slmc::kKronTab) * sizeof(double);
}

bool dqmc_supported(const slmc_ctx* c) { return c->L >= 2 && c->kron != nullptr; }

template <int LMAX>
cudaError_t launch_slices(slmc_ctx* c, double* x, double* G, int nf, int chain0, int l0, int nsl, uint64_t sweep,
                          long long* n_acc, cudaStream_t s) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const bool in_smem = dqmc_smem_bytes(c->N, true) <= (size_t)optin;
    const size_t bytes = dqmc_smem_bytes(c->N, in_smem);
    e = cudaFuncSetAttribute(k_dqmc_slices<LMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_dqmc_slices<LMAX><<<nf, kThreads, bytes, s>>>(
        x, G, c->p.Lx, c->p.Ly, c->L, l0, nsl, c->p.dtau, c->kron, c->p.lambda, c->p.omega0 * c->p.omega0,
        c->p.sweep_delta, (uint32_t)(c->p.seed & 0xffffffffu), (uint32_t)(c->p.seed >> 32), (uint32_t)sweep, chain0,
        in_smem ? 1 : 0, reinterpret_cast<unsigned long long*>(n_acc));
    return cudaGetLastError();
}

}  // namespace

namespace slmc {

cudaError_t dqmc_rotate(slmc_ctx* c, const double* x, double* xr, int nf, int g0, cudaStream_t s) {
    const size_t total = (size_t)nf * c->N * c->L;
    k_rotate<<<(unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096), 256, 0, s>>>(x, xr, c->N, c->L, g0,
                                                                                                  total);
    return cudaGetLastError();
}

bool dqmc_ok(const slmc_ctx* c) { return dqmc_supported(c); }

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
