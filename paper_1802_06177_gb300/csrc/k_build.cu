// E = exp(-dtau K) for the periodic square lattice [Eq. (2), Suppl. Eq. (S2)], built on the
// device from the plane-wave eigenbasis of K:
//   E_ij = (1/N) sum_k cos(k . (r_i - r_j)) exp(-dtau eps_k),  eps_k = -2t (cos kx + cos ky) - mu,
// k = 2 pi (nx/Lx, ny/Ly). Phases are formed as exact rationals and evaluated with cospi.
// Reduced-precision modes multiply by F = E - I (identity added exactly afterwards); its
// FP32 copy and the stencil of its FP32 rounding residual are derived from the FP64 matrix.

#include "slmc_internal.cuh"

namespace {

__global__ void k_hopping_exp(double* __restrict__ E, int Lx, int Ly, double dtau, double t, double mu) {
    const int N = Lx * Ly;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * N) return;
    const int i = idx / N, j = idx - (idx / N) * N;
    const int dx = ((i % Lx) - (j % Lx) + Lx) % Lx;
    const int dy = ((i / Lx) - (j / Lx) + Ly) % Ly;
    double acc = 0.0;
    for (int ny = 0; ny < Ly; ++ny) {
        for (int nx = 0; nx < Lx; ++nx) {
            const double eps = -2.0 * t * (cospi(2.0 * nx / Lx) + cospi(2.0 * ny / Ly)) - mu;
            const int px = (nx * dx) % Lx, py = (ny * dy) % Ly;
            const double phase = (double)px / Lx + (double)py / Ly;  // in [0, 2)
            acc += cospi(2.0 * phase) * exp(-dtau * eps);
        }
    }
    E[idx] = acc / N;
}

// The one-dimensional factors of the plane-wave sum above: for a side of Ld sites,
// e[d] = (1/Ld) sum_n cos(2 pi n d / Ld) exp(+-2 dtau t cos(2 pi n / Ld)); the sums over
// x and y separate because the hopping along x and along y commute. Block q of tab holds
// [E_x | E_x^-1 | E_y | E_y^-1][q], each written twice over.
__global__ void k_kron_tables(double* __restrict__ tab, int Lx, int Ly, double dtau_t2) {
    const int q = blockIdx.x, d = threadIdx.x;
    const int Ld = q < 2 ? Lx : Ly;
    const double a = (q & 1) ? -dtau_t2 : dtau_t2;
    if (d >= Ld) return;
    double acc = 0.0;
    for (int n = 0; n < Ld; ++n) acc += cospi(2.0 * ((n * d) % Ld) / Ld) * exp(a * cospi(2.0 * n / Ld));
    tab[q * slmc::kKronTab + d] = acc / Ld;
    tab[q * slmc::kKronTab + d + Ld] = acc / Ld;
}

__global__ void k_split_F(const double* __restrict__ E, float* __restrict__ F32, int N) {
    const int NN = N * N;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= NN) return;
    F32[idx] = (float)(E[idx] - ((idx % (N + 1) == 0) ? 1.0 : 0.0));
}

// F is translation invariant on the periodic lattice (E_ij depends on r_i - r_j only), so its
// FP32 rounding residual F_lo = F - fl32(F) is a stencil: F_lo(i, k) = F_lo(0, j) for
// r_k = r_i + r_j. The S displacements j with the largest |F(0, j)| are kept (rank by |F|,
// ties to the lower index; slot = rank); on the others |F_lo| <= 2^-24 |F| is below
// 2^-24 of the S-th largest entry and is dropped.
__global__ void k_lo_select(const double* __restrict__ E, int N, int S, int* __restrict__ sel,
                            float* __restrict__ lo_val) {
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double fd = E[j] - (j == 0 ? 1.0 : 0.0);
        const double a = fabs(fd);
        int r = 0;
        for (int q = 0; q < N; ++q) {
            const double b = fabs(E[q] - (q == 0 ? 1.0 : 0.0));
            r += (b > a) || (b == a && q < j);
        }
        if (r < S) {
            sel[r] = j;
            lo_val[r] = (float)(fd - (double)(float)fd);
        }
    }
}

__global__ void k_lo_fill(const int* __restrict__ sel, int Lx, int Ly, int S, int* __restrict__ kidx) {
    const int N = Lx * Ly;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= S * N) return;
    const int s = idx / N, i = idx - s * N, j = sel[s];
    const int kx = (i % Lx + j % Lx) % Lx, ky = (i / Lx + j / Lx) % Ly;
    kidx[idx] = kx + Lx * ky;
}

}  // namespace

namespace slmc {

cudaError_t build_hopping_exp(slmc_ctx* c, cudaStream_t s) {
    const int N = c->N;
    const int NN = N * N;
    k_hopping_exp<<<(NN + 255) / 256, 256, 0, s>>>(c->E64, c->p.Lx, c->p.Ly, c->p.dtau, c->p.t, c->p.mu);
    if (c->Einv64)  // exp(+dtau K): the same plane-wave sum with -dtau
        k_hopping_exp<<<(NN + 255) / 256, 256, 0, s>>>(c->Einv64, c->p.Lx, c->p.Ly, -c->p.dtau, c->p.t, c->p.mu);
    if (c->kron) k_kron_tables<<<4, kKronMaxLine, 0, s>>>(c->kron, c->p.Lx, c->p.Ly, 2.0 * c->p.dtau * c->p.t);
    k_split_F<<<(NN + 255) / 256, 256, 0, s>>>(c->E64, c->F32, N);
    if (c->lo_kidx) {
        int* sel = c->lo_kidx + (size_t)c->lo_S * N;
        k_lo_select<<<1, 1024, 0, s>>>(c->E64, N, c->lo_S, sel, c->lo_val);
        k_lo_fill<<<(c->lo_S * N + 255) / 256, 256, 0, s>>>(sel, c->p.Lx, c->p.Ly, c->lo_S, c->lo_kidx);
    }
    return cudaGetLastError();
}

}  // namespace slmc
