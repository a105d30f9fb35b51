// FP64 slice-group products through the separable hopping exponential [Suppl. Eq. (S2)].
//
// On the periodic Lx x Ly lattice exp(-dtau K) = e^{dtau mu} E_x kron E_y exactly (the
// hopping along x and along y commute; E_x, E_y are symmetric circulant). Applying it to a
// column of the running product therefore takes N (Lx + Ly) FMAs, a circulant transform
// along every x line and every y line of the column, instead of the N^2 of a dense product:
// 8x fewer at 16 x 16. FP64 issue is the scarce resource of the FP64 path on this GPU, so
// this is the slice kernel of the FP64 mode.
//
//   plain:       Y = B_{l0+nsl} ... B_{l0+1} U,          B_l   = diag(s_l) E
//   transposed:  Y = B_{l0+1}^T ... B_{l0+nsl}^T U,      B_l^T = E diag(s_l)
// with s_l = exp(-dtau lambda x[:, l-1]). The transposed chain accumulates the products
// B(L, g0)^T = B_{g0+1}^T ... B_L^T that the DQMC updates combine with B(g0, 0) to obtain
// G(g0) without a full chain per recomputation.
//
// One CTA owns a panel of NB columns of one field in shared memory for all nsl slices (as
// the dense panel kernel does); within a slice, one pass transforms the x lines and one the
// y lines of every column, each thread one line at a time with the outputs in registers.
// Layout: column-major N x N, element (i, j) at j*N + i, site i = ix + Lx iy.
#include "slmc_internal.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kNB = 32;  // columns per CTA

template <int LMAX, bool kTrans>
__global__ void __launch_bounds__(kThreads) k_slice_kron(const double* __restrict__ U, double* __restrict__ Y,
                                                         const double* __restrict__ x,
                                                         const double* __restrict__ kron, int Lx, int Ly, int L,
                                                         int l0, int nsl, double dtlam, double emu) {
    extern __shared__ double sm[];
    const int N = Lx * Ly;
    double* P = sm;                 // [kNB][N] panel, column-major
    double* sc = sm + kNB * N;      // [N] e^{dtau mu} s_l
    double* tx = sc + N;            // E_x, twice over
    double* ty = tx + slmc::kKronTab;  // E_y, twice over
    const int f = blockIdx.y, j0 = blockIdx.x * kNB, tid = threadIdx.x;
    const int nb = min(kNB, N - j0);
    const size_t NN = (size_t)N * N;
    const double* Uf = U + f * NN + (size_t)j0 * N;
    for (int k = tid; k < slmc::kKronTab; k += kThreads) {
        tx[k] = kron[k];
        ty[k] = kron[2 * slmc::kKronTab + k];
    }
    for (int idx = tid; idx < nb * N; idx += kThreads) P[idx] = Uf[idx];
    const double* xf = x + (size_t)f * N * L;
    for (int step = 0; step < nsl; ++step) {
        const int c = kTrans ? l0 + nsl - 1 - step : l0 + step;  // field column of the slice
        for (int i = tid; i < N; i += kThreads) sc[i] = exp(-dtlam * xf[(size_t)i * L + c]) * emu;
        __syncthreads();
        // x lines (jj, iy): contiguous; the transposed slice scales its input here
        for (int q = tid; q < nb * Ly; q += kThreads) {
            const int jj = q / Ly, iy = q - jj * Ly;
            slmc::circ_line<LMAX, true>(P, jj * N + iy * Lx, 1, Lx, tx, kTrans ? sc + iy * Lx : nullptr, 1, nullptr,
                                        0, 1.0);
        }
        __syncthreads();
        // y lines (jj, ix): stride Lx; the plain slice scales its output here
        for (int q = tid; q < nb * Lx; q += kThreads) {
            const int jj = q / Lx, ix = q - jj * Lx;
            slmc::circ_line<LMAX, true>(P, jj * N + ix, Lx, Ly, ty, nullptr, 0, kTrans ? nullptr : sc + ix, Lx,
                                        1.0);
        }
        __syncthreads();
    }
    double* Yf = Y + f * NN + (size_t)j0 * N;
    for (int idx = tid; idx < nb * N; idx += kThreads) Yf[idx] = P[idx];
}

template <int LMAX, bool kTrans>
cudaError_t launch_kron(slmc_ctx* c, const double* x, int nf, int l0, int nsl, cudaStream_t s) {
    const int N = c->N;
    const size_t smem = ((size_t)kNB * N + N + 2 * slmc::kKronTab) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_slice_kron<LMAX, kTrans>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((N + kNB - 1) / kNB, nf);
    k_slice_kron<LMAX, kTrans><<<grid, kThreads, smem, s>>>(c->U, c->Y, x, c->kron, c->p.Lx, c->p.Ly, c->L, l0, nsl,
                                                            c->p.dtau * c->p.lambda, exp(c->p.dtau * c->p.mu));
    return cudaGetLastError();
}

template <bool kTrans>
cudaError_t dispatch_kron(slmc_ctx* c, const double* x, int nf, int l0, int nsl, cudaStream_t s) {
    const int lm = c->p.Lx > c->p.Ly ? c->p.Lx : c->p.Ly;
    if (lm <= 8) return launch_kron<8, kTrans>(c, x, nf, l0, nsl, s);
    if (lm <= 16) return launch_kron<16, kTrans>(c, x, nf, l0, nsl, s);
    return launch_kron<32, kTrans>(c, x, nf, l0, nsl, s);
}

}  // namespace

namespace slmc {

cudaError_t slice_group_kron(slmc_ctx* c, const double* x, int nf, int l0, int nsl, bool transposed, cudaStream_t s) {
    if (!c->kron) return cudaErrorInvalidValue;
    return transposed ? dispatch_kron<true>(c, x, nf, l0, nsl, s) : dispatch_kron<false>(c, x, nf, l0, nsl, s);
}

}  // namespace slmc
