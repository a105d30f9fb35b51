// Conventional DQMC updates of the phonon field [Supplemental Material, Eqs. (S3)-(S6) and
// the block update described after them], the baseline the self-learning method is compared
// with.
//
// Local updates: at time slice l the equal-time Green's function G(l) (row-major, one chain
// per CTA, in global memory: one N x N matrix per chain stays L2-resident) decides the move
// of x_{i,l-1} through the fast ratio R = 1 + (1 - G_ii) Delta_ii, Delta_ii =
// exp(-dtau lam d) - 1 (Eq. (S5)); with both spin species the weight ratio is
// R^2 exp(d ln w_bose). An accepted move updates G by Sherman-Morrison,
// G -= (Delta_ii / R) G[:, i] (e_i - G[i, :]) (Eq. (S6)), a rank-1 update spread over the CTA.
// Between slices G(l) = B_l G(l-1) B_l^-1 with B_l = diag(s) E (two N^3 products through a
// per-chain scratch matrix); at the start of every group of n_s slices G is recomputed from
// scratch by the stabilised determinant path on the time-rotated field.
// Sites of a slice are visited in order; the proposal x' = x + U[-Delta, Delta] and the
// acceptance uniform come from Philox counter (i L + l - 1, sweep, chain, 3). The new field is
// rounded step by step as in the oracle, so accepted moves leave identical fields.
//
// Block updates reflect one site's whole column (x -> -x) and are accepted with the ratio of
// full weights (computed by the determinant path); the site and the uniform come from Philox
// counter (k, sweep, chain, 4).
#include "slmc_internal.cuh"

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

__global__ void __launch_bounds__(kThreads) k_dqmc_slices(double* __restrict__ x, double* __restrict__ Gall,
                                                          double* __restrict__ Wall, const double* __restrict__ E,
                                                          const double* __restrict__ Einv, int N, int L, int l0, int nsl,
                                                          double dtau, double lam, double w02, double delta,
                                                          uint32_t key0, uint32_t key1, uint32_t sweep, int chain0,
                                                          unsigned long long* __restrict__ n_acc) {
    extern __shared__ double dsm[];
    double* s = dsm;          // [N] slice scales
    double* col = dsm + N;    // [N] G[:, i]
    double* row = dsm + 2 * N;  // [N] e_i - G[i, :]
    __shared__ double s_coef;
    __shared__ int s_acc[2];  // decision of site i in s_acc[i & 1]: thread 0 writes the next one while
                              // others may still be reading this one
    const int f = blockIdx.x, tid = threadIdx.x;
    const size_t NN = (size_t)N * N;
    double* __restrict__ G = Gall + f * NN;
    double* __restrict__ W = Wall + f * NN;
    double* __restrict__ xf = x + (size_t)f * N * L;
    const uint32_t chain = (uint32_t)(chain0 + f);
    int accepted = 0;
    for (int l = l0 + 1; l <= l0 + nsl; ++l) {
        const int c = l - 1;
        for (int i = tid; i < N; i += kThreads) s[i] = exp(-dtau * lam * xf[(size_t)i * L + c]);
        // wrap: W = G Einv, G = diag(s) E W diag(1/s)
        for (size_t idx = tid; idx < NN; idx += kThreads) {
            const int i = (int)(idx / N), j = (int)(idx - (size_t)i * N);
            const double* gi = G + (size_t)i * N;
            double acc = 0.0;
            for (int m = 0; m < N; ++m) acc = fma(gi[m], Einv[(size_t)m * N + j], acc);
            W[idx] = acc;
        }
        __syncthreads();
        for (size_t idx = tid; idx < NN; idx += kThreads) {
            const int i = (int)(idx / N), j = (int)(idx - (size_t)i * N);
            const double* ei = E + (size_t)i * N;
            double acc = 0.0;
            for (int k = 0; k < N; ++k) acc = fma(ei[k], W[(size_t)k * N + j], acc);
            G[idx] = s[i] * acc / s[j];
        }
        __syncthreads();
        for (int i = 0; i < N; ++i) {
            if (tid == 0) {
                const slmc::u32x4 w =
                    slmc::philox4x32_10(slmc::u32x4{(uint32_t)(i * L + c), sweep, chain, 3u}, key0, key1);
                const double u1 = slmc::uniform53(w.x, w.y), u2 = slmc::uniform53(w.z, w.w);
                const double v = xf[(size_t)i * L + c];
                const double xn = __dadd_rn(v, __dmul_rn(delta, __dadd_rn(__dmul_rn(2.0, u1), -1.0)));
                const double dl = exp(-dtau * lam * (xn - v)) - 1.0;
                const double R = 1.0 + (1.0 - G[(size_t)i * N + i]) * dl;
                const double up = xf[(size_t)i * L + (c + 1 == L ? 0 : c + 1)];
                const double dn = xf[(size_t)i * L + (c == 0 ? L - 1 : c - 1)];
                const double kin = ((up - xn) * (up - xn) + (xn - dn) * (xn - dn) - (up - v) * (up - v) -
                                    (v - dn) * (v - dn)) / (2.0 * dtau * dtau);
                const double dlb = dtau * lam * (xn - v) - dtau * (0.5 * w02 * (xn * xn - v * v) + kin);
                const double lnr = log(R * R) + dlb;
                const int acc = (lnr >= 0.0 || u2 < exp(lnr)) ? 1 : 0;
                if (acc) {
                    xf[(size_t)i * L + c] = xn;
                    s_coef = dl / R;
                    ++accepted;
                }
                s_acc[i & 1] = acc;
            }
            __syncthreads();
            if (s_acc[i & 1]) {  // Sherman-Morrison (block-uniform branch)
                for (int j = tid; j < N; j += kThreads) {
                    col[j] = G[(size_t)j * N + i];
                    row[j] = (j == i ? 1.0 : 0.0) - G[(size_t)i * N + j];
                }
                __syncthreads();
                const double a = s_coef;
                for (size_t idx = tid; idx < NN; idx += kThreads) {
                    const int j = (int)(idx / N), k = (int)(idx - (size_t)j * N);
                    G[idx] = fma(-a * col[j], row[k], G[idx]);
                }
                __syncthreads();
            }
        }
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

}  // namespace

namespace slmc {

cudaError_t dqmc_rotate(slmc_ctx* c, const double* x, double* xr, int nf, int g0, cudaStream_t s) {
    const size_t total = (size_t)nf * c->N * c->L;
    k_rotate<<<(unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096), 256, 0, s>>>(x, xr, c->N, c->L, g0,
                                                                                                  total);
    return cudaGetLastError();
}

cudaError_t dqmc_slices(slmc_ctx* c, double* x, double* G, double* W, int nf, int chain0, int l0, int nsl,
                        uint64_t sweep, long long* n_acc, cudaStream_t s) {
    k_dqmc_slices<<<nf, kThreads, 3 * c->N * sizeof(double), s>>>(
        x, G, W, c->E64, c->Einv64, c->N, c->L, l0, nsl, c->p.dtau, c->p.lambda, c->p.omega0 * c->p.omega0,
        c->p.sweep_delta, (uint32_t)(c->p.seed & 0xffffffffu), (uint32_t)(c->p.seed >> 32), (uint32_t)sweep, chain0,
        reinterpret_cast<unsigned long long*>(n_acc));
    return cudaGetLastError();
}

cudaError_t dqmc_block_propose(slmc_ctx* c, double* x, int nf, int chain0, uint64_t sweep, int k, double* u,
                               cudaStream_t s) {
    k_block_propose<<<nf, 128, 0, s>>>(x, c->N, c->L, (uint32_t)(c->p.seed & 0xffffffffu), (uint32_t)(c->p.seed >> 32),
                                       (uint32_t)sweep, (uint32_t)k, chain0, u);
    return cudaGetLastError();
}

}  // namespace slmc
