// Bosonic parts of the weight, the symmetric effective model and its Markov chain, the
// cumulative-update acceptance, the CDW structure factor and the E_eff regression.
//
//   ln w       = 2 ln|det| + dtau lam sum x - dtau sum [w0^2 x^2/2 + (x_{l+1}-x_l)^2/(2 dtau^2)]
//                                                             [Sec. "Model", Suppl. Eq. (S2)]
//   ln w_eff   = -dtau (E0 + J_k F_k + J_p F_p + J_p' F_p' + J_nn F_nn + J_nn' F_nn')
//                                                             [Eq. (4) / (S7)]
//   acceptance = min{1, [w(x')/w(x)] [w_eff(x)/w_eff(x')]}   [Eq. (6)]
//   S(pi,pi)   = (1/N) sum_ij s_i s_j [4 (1-G_ii)(1-G_jj) + 2 (d_ij - G_ji) G_ij]  [Sec. "Results"]
//   fit        = least squares of ln w on [1, F]               [Eq. (5)]
//
// Site i = ix + Lx iy, field element (i, l) at i*L + l. All reductions use a fixed
// order (per-thread strided partial sums, then a shared-memory tree), so results are
// reproducible run to run.
#include <cfloat>

#include "slmc_internal.cuh"

namespace {

constexpr int kThreads = 256;

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red /* [NV][kThreads] */) {
#pragma unroll
    for (int q = 0; q < NV; ++q) red[q * kThreads + threadIdx.x] = v[q];
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
#pragma unroll
            for (int q = 0; q < NV; ++q) red[q * kThreads + threadIdx.x] += red[q * kThreads + threadIdx.x + h];
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = red[q * kThreads];
}

__global__ void __launch_bounds__(kThreads) k_bose(const double* __restrict__ x, int N, int L, double dtau, double lam,
                                                   double w02, const double* __restrict__ lndet, double* __restrict__ lnw) {
    __shared__ double red[kThreads];
    const int f = blockIdx.x;
    const double* xf = x + (size_t)f * N * L;
    const double inv2dt2 = 1.0 / (2.0 * dtau * dtau);
    double acc[1] = {0.0};
    for (int idx = threadIdx.x; idx < N * L; idx += kThreads) {
        const int i = idx / L, l = idx - i * L;
        const double v = xf[idx];
        const double vn = xf[(size_t)i * L + (l + 1 == L ? 0 : l + 1)];
        const double d = vn - v;
        acc[0] += dtau * lam * v - dtau * (0.5 * w02 * v * v + d * d * inv2dt2);
    }
    block_sum<1>(acc, red);
    if (threadIdx.x == 0) lnw[f] = (lndet ? 2.0 * lndet[f] : 0.0) + acc[0];
}

__global__ void __launch_bounds__(kThreads) k_features(const double* __restrict__ x, int Lx, int Ly, int L, double a2,
                                                       double dtau, const double* __restrict__ J,
                                                       double* __restrict__ F, int ldF, double* __restrict__ lnw_eff) {
    __shared__ double red[5 * kThreads];
    const int f = blockIdx.x;
    const int N = Lx * Ly;
    const double* xf = x + (size_t)f * N * L;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int idx = threadIdx.x; idx < N * L; idx += kThreads) {
        const int i = idx / L, l = idx - i * L;
        const int ix = i % Lx, iy = i / Lx;
        const double v = xf[idx];
        const double vt = xf[(size_t)i * L + (l + 1 == L ? 0 : l + 1)];
        const double vx = xf[(size_t)((ix + 1 == Lx ? 0 : ix + 1) + Lx * iy) * L + l];
        const double vy = xf[(size_t)(ix + Lx * (iy + 1 == Ly ? 0 : iy + 1)) * L + l];
        const double v2 = v * v;
        const double d = vt - v;
        acc[0] += d * d;
        acc[1] += v2 * v2 * 0.25 - a2 * v2 * 0.5;
        acc[2] += v2 * v2 * v2 * (1.0 / 6.0) - a2 * v2 * v2 * 0.25;
        acc[3] += v * (vx + vy);
        acc[4] += v * vt;
    }
    block_sum<5>(acc, red);
    if (threadIdx.x == 0) {
        if (F)
            for (int q = 0; q < 5; ++q) F[(size_t)f * ldF + q] = acc[q];
        if (lnw_eff) {
            const double e = J[0] + J[1] * acc[0] + J[2] * acc[1] + J[3] * acc[2] + J[4] * acc[3] + J[5] * acc[4];
            lnw_eff[f] = -dtau * e;
        }
    }
}

// Terms of E0 + J.F that contain one site value v.
__device__ __forceinline__ double local_energy(const double* J, double a2, double v, double up, double dn, double nb) {
    const double v2 = v * v;
    const double du = up - v, dd = v - dn;
    return J[1] * (du * du + dd * dd) + J[2] * (v2 * v2 * 0.25 - a2 * v2 * 0.5) +
           J[3] * (v2 * v2 * v2 * (1.0 / 6.0) - a2 * v2 * v2 * 0.25) + J[4] * v * nb + J[5] * v * (up + dn);
}

// Loads of the field: plain (cached) in the per-colour kernels, L2-only (ld.global.cg) in the
// persistent queue kernel, whose CTAs read values that other CTAs of the same launch wrote.
template <bool kL2>
__device__ __forceinline__ double ldx(const double* p) {
    if (kL2) return __ldcg(p);
    return *p;
}

// Metropolis update of site pair s of colour c in one chain's field (thread s of the half-sweep
// owns site i = s / (L/2) and the slice l of colour c in the pair (2 (s mod L/2), 2 (s mod L/2) + 1)).
// Returns 1 if the move was accepted (and written).
template <bool kL2>
__device__ __forceinline__ int site_update(double* xfield, int Lx, int Ly, int L, const double* J, double dtau,
                                           double a2, double delta, uint32_t key0, uint32_t key1, uint32_t sweep,
                                           int c, int s, uint32_t chain) {
    const int half = L / 2;
    const int i = s / half, lp = s - i * half;
    const int ix = i % Lx, iy = i / Lx;
    const int l = 2 * lp + ((ix + iy + c) & 1);
    const double v = ldx<kL2>(xfield + (size_t)i * L + l);
    const double up = ldx<kL2>(xfield + (size_t)i * L + (l + 1 == L ? 0 : l + 1));
    const double dn = ldx<kL2>(xfield + (size_t)i * L + (l == 0 ? L - 1 : l - 1));
    const int xp = (ix + 1 == Lx ? 0 : ix + 1) + Lx * iy, xm = (ix == 0 ? Lx - 1 : ix - 1) + Lx * iy;
    const int yp = ix + Lx * (iy + 1 == Ly ? 0 : iy + 1), ym = ix + Lx * (iy == 0 ? Ly - 1 : iy - 1);
    const double nb = ldx<kL2>(xfield + (size_t)xp * L + l) + ldx<kL2>(xfield + (size_t)xm * L + l) +
                      ldx<kL2>(xfield + (size_t)yp * L + l) + ldx<kL2>(xfield + (size_t)ym * L + l);
    const slmc::u32x4 w = slmc::philox4x32_10(slmc::u32x4{(uint32_t)(i * L + l), sweep, chain, 0u}, key0, key1);
    const double u1 = slmc::uniform53(w.x, w.y);
    // x' = x + delta (2 u1 - 1), rounded step by step (no contraction) as in the oracle
    const double xn = __dadd_rn(v, __dmul_rn(delta, __dadd_rn(__dmul_rn(2.0, u1), -1.0)));
    // Fast decision in FP32: dE = d [2 J_k (s - up - dn) + s (J_p ((x'^2 + x^2)/4 - a^2/2)
    //   + J_p' ((x'^4 + x'^2 x^2 + x^4)/6 - a^2 (x'^2 + x^2)/4)) + J_nn nb + J_nn' (up + dn)],
    // d = x' - x, s = x' + x (the exact difference of the local energies, factored). The FP32
    // verdict is used only when the log-ratio is further from log u than a margin bounding
    // (i) the FP32 rounding of the bracket (1e-5 of the sum of the magnitudes of its terms,
    // about 170 units of FP32 rounding), (ii) the rounding of x, x' to FP32, which moves d by
    // up to 2^-24 (|x| + |x'|), and (iii) the truncation of u to 24 bits (log u is known to
    // within 2^-24 / u); otherwise the exact FP64 rule of the oracle decides.
    const float vf = (float)v, xf = (float)xn, upf = (float)up, dnf = (float)dn, nbf = (float)nb;
    const float d = xf - vf, sm = xf + vf, x2 = xf * xf, v2 = vf * vf, a2f = (float)a2;
    const float tk = 2.f * (float)J[1] * (sm - upf - dnf);
    const float tp = sm * (float)J[2] * (0.25f * (x2 + v2) - 0.5f * a2f);
    const float tpp = sm * (float)J[3] * ((x2 * x2 + x2 * v2 + v2 * v2) * (1.f / 6.f) - 0.25f * a2f * (x2 + v2));
    const float tn = (float)J[4] * nbf + (float)J[5] * (upf + dnf);
    const float mag = 2.f * fabsf((float)J[1]) * (fabsf(sm) + fabsf(upf) + fabsf(dnf)) +
                      fabsf(sm) * (fabsf((float)J[2]) * (x2 + v2 + a2f) +
                                   fabsf((float)J[3]) * (x2 * x2 + x2 * v2 + v2 * v2 + a2f * (x2 + v2))) +
                      fabsf((float)J[4] * nbf) + fabsf((float)J[5]) * (fabsf(upf) + fabsf(dnf));
    const float dlnw32 = -(float)dtau * d * (tk + tp + tpp + tn);
    const float uf = (float)(w.z >> 8) * 5.9604644775390625e-8f;  // top 24 bits of the acceptance uniform
    int decided = 0, acc = 0;
    if (uf > 0.f && isfinite(dlnw32) && isfinite(mag)) {
        const float lu = logf(uf);
        const float margin =
            1e-5f + (float)dtau * mag * (1e-5f * fabsf(d) + 2e-7f * (fabsf(xf) + fabsf(vf))) + 1.2e-7f / uf;
        if (dlnw32 > lu + margin) {
            decided = 1;
            acc = 1;
        } else if (dlnw32 < lu - margin) {
            decided = 1;
            acc = 0;
        }
    }
    if (!decided) {  // exact FP64 rule of the oracle
        const double u2 = slmc::uniform53(w.z, w.w);
        const double dE = local_energy(J, a2, xn, up, dn, nb) - local_energy(J, a2, v, up, dn, nb);
        const double dlnw = -dtau * dE;
        acc = (dlnw >= 0.0 || u2 < exp(dlnw)) ? 1 : 0;
    }
    if (acc) xfield[(size_t)i * L + l] = xn;
    return acc;
}

// One checkerboard half-sweep over all chains: thread s of chain f updates site pair s.
__global__ void __launch_bounds__(kThreads) k_half_sweep(double* __restrict__ x, int Lx, int Ly, int L,
                                                         const double* __restrict__ Jg, double dtau, double a2,
                                                         double delta, uint32_t key0, uint32_t key1, uint32_t sweep_arg,
                                                         int colour, const int* __restrict__ colour_pc, int cxor,
                                                         int chain0, unsigned long long* __restrict__ n_acc,
                                                         const unsigned long long* __restrict__ dctr, int nsweeps) {
    __shared__ double J[6];
    __shared__ int s_cnt;
    if (threadIdx.x < 6) J[threadIdx.x] = Jg[threadIdx.x];
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int f = blockIdx.y;
    const int N = Lx * Ly, half = L / 2;
    const int s = blockIdx.x * kThreads + threadIdx.x;
    // cumulative updates: sweep counter (update * nsweeps + sweep_arg), update from the device counter
    const uint32_t sweep = dctr ? (uint32_t)((*dctr) * (unsigned long long)nsweeps + sweep_arg) : sweep_arg;
    int accepted = 0;
    if (s < N * half) {
        const int c = colour_pc ? (colour_pc[f] ^ cxor) : colour;
        accepted = site_update<false>(x + (size_t)f * N * L, Lx, Ly, L, J, dtau, a2, delta, key0, key1, sweep, c, s,
                                      (uint32_t)(chain0 + f));
    }
    const unsigned int ballot = __ballot_sync(0xffffffffu, accepted);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(&s_cnt, __popc(ballot));
    __syncthreads();
    if (threadIdx.x == 0 && n_acc && s_cnt) atomicAdd(n_acc + f, (unsigned long long)s_cnt);
}

// Modified Wolff cluster update of E_eff [Sec. "Wolff update of the effective Hamiltonian",
// Eq. (S9)], one CTA per chain. Bond term b = 2i, (i, i + x^), or 2i + 1, (i, i + y^), of J_nn F_nn
// is activated with probability max(0, 1 - exp(t_b)), t_b = 2 dtau J_nn sum_l x_il x_jl: reflecting
// the whole column of one endpoint multiplies the term's weight by exp(t_b). The sum runs over l
// in order with products and sums rounded separately (as in the oracle, so both take the same
// decisions); the uniform is that of Philox counter (b, ctr, chain, 2), the seed site that of
// (2N, ctr, chain, 2), ctr = (sweep counter) * nwolff + k. The seed's connected component over
// the activated bonds is found by label propagation in shared memory (marks only go from 0 to 1,
// so at most N + 1 rounds) and its columns are reflected, x -> -x. Every other term of E_eff is
// invariant under reflecting whole columns: the move is always accepted.
// One Wolff cluster update of one chain's field xf by the whole CTA (blockDim.x threads); act and
// in_c are 2N and N bytes of shared memory; counter ctr, Philox chain index chain.
template <bool kL2>
__device__ __forceinline__ void wolff_chain(double* xf, int Lx, int Ly, int L, const double* __restrict__ Jg,
                                            double dtau, uint32_t key0, uint32_t key1, uint32_t ctr, uint32_t chain,
                                            unsigned char* act, unsigned char* in_c, int* s_seed, int* s_cnt,
                                            unsigned long long* __restrict__ n_sites) {
    const int N = Lx * Ly, tid = threadIdx.x;
    const double cfac = __dmul_rn(__dmul_rn(2.0, dtau), Jg[4]);
    for (int b = tid; b < 2 * N; b += blockDim.x) {
        const int i = b >> 1, ix = i % Lx, iy = i / Lx;
        const int j = (b & 1) ? ix + Lx * (iy + 1 == Ly ? 0 : iy + 1) : (ix + 1 == Lx ? 0 : ix + 1) + Lx * iy;
        const double* xi = xf + (size_t)i * L;
        const double* xj = xf + (size_t)j * L;
        double sb = 0.0;
        for (int l = 0; l < L; ++l) sb = __dadd_rn(sb, __dmul_rn(ldx<kL2>(xi + l), ldx<kL2>(xj + l)));
        const double t = __dmul_rn(cfac, sb);
        unsigned char a = 0;
        if (t < 0.0) {
            const slmc::u32x4 w = slmc::philox4x32_10(slmc::u32x4{(uint32_t)b, ctr, chain, 2u}, key0, key1);
            a = slmc::uniform53(w.x, w.y) < __dadd_rn(1.0, -exp(t));
        }
        act[b] = a;
    }
    if (tid == 0) {
        const slmc::u32x4 w = slmc::philox4x32_10(slmc::u32x4{(uint32_t)(2 * N), ctr, chain, 2u}, key0, key1);
        const int s0 = (int)(slmc::uniform53(w.x, w.y) * (double)N);
        *s_seed = s0 < N - 1 ? s0 : N - 1;
        *s_cnt = 0;
    }
    __syncthreads();
    for (int i = tid; i < N; i += blockDim.x) in_c[i] = (i == *s_seed);
    __syncthreads();
    for (int round = 0; round <= N; ++round) {
        int changed = 0;
        for (int b = tid; b < 2 * N; b += blockDim.x) {
            if (!act[b]) continue;
            const int i = b >> 1, ix = i % Lx, iy = i / Lx;
            const int j = (b & 1) ? ix + Lx * (iy + 1 == Ly ? 0 : iy + 1) : (ix + 1 == Lx ? 0 : ix + 1) + Lx * iy;
            if (in_c[i] != in_c[j]) {
                in_c[i] = 1;
                in_c[j] = 1;
                changed = 1;
            }
        }
        if (!__syncthreads_or(changed)) break;
    }
    int cnt = 0;
    for (int i = tid; i < N; i += blockDim.x) cnt += in_c[i];
    for (size_t idx = tid; idx < (size_t)N * L; idx += blockDim.x)
        if (in_c[idx / L]) xf[idx] = -ldx<kL2>(xf + idx);
    if (n_sites) {
        atomicAdd(s_cnt, cnt);
        __syncthreads();
        if (tid == 0) atomicAdd(n_sites, (unsigned long long)*s_cnt);
    }
}

__global__ void __launch_bounds__(256) k_wolff(double* __restrict__ x, int Lx, int Ly, int L,
                                               const double* __restrict__ Jg, double dtau, uint32_t key0,
                                               uint32_t key1, uint32_t sweep_arg,
                                               const unsigned long long* __restrict__ dctr, int nsweeps, int nwolff,
                                               int k, int chain0, unsigned long long* __restrict__ n_sites) {
    extern __shared__ unsigned char wsm[];
    const int N = Lx * Ly;
    __shared__ int s_seed, s_cnt;
    const int f = blockIdx.x;
    const uint32_t sweep = dctr ? (uint32_t)((*dctr) * (unsigned long long)nsweeps + sweep_arg) : sweep_arg;
    const uint32_t ctr = sweep * (uint32_t)nwolff + (uint32_t)k;
    wolff_chain<false>(x + (size_t)f * N * L, Lx, Ly, L, Jg, dtau, key0, key1, ctr, (uint32_t)(chain0 + f), wsm,
                       wsm + 2 * N, &s_seed, &s_cnt, n_sites);
}

// Persistent E_eff sweep queue: the half-sweep slabs and Wolff updates of every chain of several
// lattice classes, pulled in queue order by the CTAs of one launch. The queue lists, phase after
// phase (colour 0, the Wolff updates, colour 1 of each sweep), the items of every chain in order of
// decreasing N L (longest first), so every item depends only on earlier ones: item q of chain g
// waits until g's completion counter reaches its count of g's earlier items. A CTA takes an item
// only while it runs, so all items it waits on are held by running CTAs, and the launch cannot
// deadlock whatever the grid size. Values written by other CTAs of the launch are read through L2
// (__ldcg); a CTA publishes an item after a barrier and a device-scope fence. The arithmetic of a
// site update or a Wolff update is the one of k_half_sweep / k_wolff (shared device functions), so
// the chains are bit-identical to the kernel-per-half-sweep path.
//
// Every wait is bounded: after wait_cycles the CTA sets SLMC_EBIT_TIMEOUT in the error word of
// every class and the abort word ctl[1]; every CTA stops taking items once it sees the abort.
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(kThreads) k_sweep_queue(const slmc::QueueClass* __restrict__ cls, int ncls,
                                                          const int4* __restrict__ items, int nitems,
                                                          unsigned int* __restrict__ done, unsigned int* __restrict__ ctl,
                                                          uint32_t u, long long wait_cycles) {
    extern __shared__ unsigned char qsm[];
    __shared__ double J[6];
    __shared__ int s_item, s_cnt, s_seed, s_wcnt;
    for (;;) {
        if (threadIdx.x == 0) {
            int q = -1;
            if (ld_acquire_u32(ctl + 1) == 0u) q = (int)atomicAdd(ctl, 1u);
            if (q >= nitems) q = -1;
            if (q >= 0) {
                const int4 it = items[q];
                const slmc::QueueClass& C = cls[it.x >> 24];
                const unsigned int* cnt = done + C.done0 + (it.x & 0xffffff);
                const long long t0 = clock64();
                while (ld_acquire_u32(cnt) < (unsigned int)it.w) {
                    if (ld_acquire_u32(ctl + 1) != 0u) {
                        q = -1;
                        break;
                    }
                    if (clock64() - t0 > wait_cycles) {
                        for (int k = 0; k < ncls; ++k) atomicOr(cls[k].err, SLMC_EBIT_TIMEOUT);
                        atomicExch(ctl + 1, 1u);
                        q = -1;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            s_item = q;
            s_cnt = 0;
        }
        __syncthreads();
        const int q = s_item;
        if (q < 0) break;
        const int4 it = items[q];
        const slmc::QueueClass& C = cls[it.x >> 24];
        const int f = it.x & 0xffffff;
        if (threadIdx.x < 6) J[threadIdx.x] = C.J[threadIdx.x];
        __syncthreads();
        const int N = C.Lx * C.Ly;
        double* xf = C.x + (size_t)f * N * C.L;
        const int sw = it.y >> 8, sub = it.y & 0x7f;
        const uint32_t chain = (uint32_t)f;
        const uint32_t sweep = (uint32_t)((*C.dctr) * (unsigned long long)C.nsweeps +
                                          (unsigned long long)u * C.nsweeps + sw);
        if (it.y & 0x80) {
            const uint32_t ctr = sweep * (uint32_t)C.nwolff + (uint32_t)sub;
            wolff_chain<true>(xf, C.Lx, C.Ly, C.L, J, C.dtau, C.key0, C.key1, ctr, chain, qsm, qsm + 2 * N, &s_seed,
                              &s_wcnt, C.wolff_sites);
        } else {
            const int sites = N * (C.L / 2);
            const int c = C.first_colour[f] ^ sub;
            int accepted = 0;
            for (int j = 0; j < slmc::kQueueSlab / kThreads; ++j) {
                const int st = it.z * slmc::kQueueSlab + j * kThreads + threadIdx.x;
                if (st < sites)
                    accepted += site_update<true>(xf, C.Lx, C.Ly, C.L, J, C.dtau, C.a2, C.delta, C.key0, C.key1,
                                                  sweep, c, st, chain);
            }
            if (accepted) atomicAdd(&s_cnt, accepted);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (!(it.y & 0x80) && C.n_acc && s_cnt) atomicAdd(C.n_acc + f, (unsigned long long)s_cnt);
            __threadfence();
            atomicAdd(done + C.done0 + f, 1u);
        }
    }
}

__global__ void k_update_draws(int nf, int chain0, uint32_t u_off, const unsigned long long* __restrict__ dctr,
                               uint32_t key0, uint32_t key1, int* __restrict__ first, double* __restrict__ u) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const uint32_t update = (uint32_t)(*dctr + u_off);
    const slmc::u32x4 w = slmc::philox4x32_10(slmc::u32x4{update, 0u, (uint32_t)(chain0 + f), 1u}, key0, key1);
    first[f] = (int)(w.x & 1u);
    u[f] = slmc::uniform53(w.z, w.w);
}

__global__ void k_accept(int nf, const double* __restrict__ lnw_new, const double* __restrict__ lnweff_old,
                         const double* __restrict__ lnweff_new, const double* __restrict__ u, double* __restrict__ lnw,
                         int* __restrict__ accepted, unsigned long long* __restrict__ n_acc) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const double lnA = (lnw_new[f] - lnw[f]) - (lnweff_new[f] - lnweff_old[f]);
    const bool acc = lnA >= 0.0 || u[f] < exp(lnA);
    accepted[f] = acc ? 1 : 0;
    if (acc) {
        lnw[f] = lnw_new[f];
        if (n_acc) n_acc[f] += 1ull;
    }
}

__global__ void k_restore(double* __restrict__ x, const double* __restrict__ x_old, const int* __restrict__ accepted,
                          int NL) {
    const int f = blockIdx.y;
    if (accepted[f]) return;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < NL; idx += gridDim.x * blockDim.x)
        x[(size_t)f * NL + idx] = x_old[(size_t)f * NL + idx];
}

__global__ void __launch_bounds__(kThreads) k_cdw(const double* __restrict__ G, int Lx, int Ly, double* __restrict__ S,
                                                  const int* __restrict__ only_if, double* __restrict__ obs) {
    __shared__ double red[3 * kThreads];
    const int f = blockIdx.x;
    const int N = Lx * Ly;
    const size_t NN = (size_t)N * N;
    const bool update = !only_if || only_if[f];
    if (update) {
        const double* Gf = G + f * NN;
        double acc[3] = {0.0, 0.0, 0.0};  // sum s_i (1 - G_ii), sum G_ii, sum s_i s_j G_ij G_ji
        for (int i = threadIdx.x; i < N; i += kThreads) {
            const double si = (((i % Lx) + (i / Lx)) & 1) ? -1.0 : 1.0;
            const double g = Gf[(size_t)i * N + i];
            acc[0] += si * (1.0 - g);
            acc[1] += g;
        }
        for (size_t idx = threadIdx.x; idx < NN; idx += kThreads) {
            const int i = (int)(idx / N), j = (int)(idx - (size_t)i * N);
            const double sij = ((((i % Lx) + (i / Lx)) ^ ((j % Lx) + (j / Lx))) & 1) ? -1.0 : 1.0;
            acc[2] += sij * Gf[idx] * Gf[(size_t)j * N + i];
        }
        block_sum<3>(acc, red);  // block-uniform branch: `update` depends on f only
        if (threadIdx.x == 0) S[f] = (4.0 * acc[0] * acc[0] + 2.0 * acc[1] - 2.0 * acc[2]) / N;
    }
    if (obs && threadIdx.x == 0) obs[f] = S[f];
}

// ---- regression: Givens-rotation QR of the rows [1, (F - F_ref)/sc, y - y_ref] into a 7x7 R ----
// fitR layout: R[7][7] row-major (0..48), ref[6] (49..54: F_ref[5], y_ref), flag (55), count (56).
__global__ void k_fit_begin(double* __restrict__ R) {
    for (int q = threadIdx.x; q < 64; q += blockDim.x) R[q] = 0.0;
}

// Absorbs one row (lane m < 7 holds its element m) into the triangular factor held by the warp
// (lane m holds column m of every row of R) with Givens rotations.
__device__ __forceinline__ void givens_absorb(double (&Rrow)[7], double a, int lane) {
    for (int k = 0; k < 7; ++k) {
        const double ak = __shfl_sync(0xffffffffu, a, k);
        const double rkk = __shfl_sync(0xffffffffu, Rrow[k], k);
        if (ak == 0.0) continue;
        const double r = hypot(rkk, ak);
        const double cs = rkk / r, sn = ak / r;
        if (lane == k) {
            Rrow[k] = r;
            a = 0.0;
        } else if (lane > k && lane < 7) {
            const double rk = Rrow[k];
            Rrow[k] = cs * rk + sn * a;
            a = -sn * rk + cs * a;
        }
    }
}

// Warps take consecutive chunks of the configurations (the first warp starts from the current
// triangle), reduce them to partial triangles, and the partial triangles are merged pairwise
// in shared memory (all rows are taken relative to the same reference, so no shift is needed).
__global__ void k_fit_accumulate(double* __restrict__ R, const double* __restrict__ feat, int ldF,
                                 const double* __restrict__ lnw, int nconf, double sc) {
    __shared__ double sR[32][49];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0 && R[55] == 0.0) {
        for (int q = 0; q < 5; ++q) R[49 + q] = feat[q];
        R[54] = lnw[0];
        R[55] = 1.0;
    }
    __syncthreads();
    double Rrow[7];  // lane m < 7 holds column m of every row
    for (int k = 0; k < 7; ++k) Rrow[k] = (warp == 0 && lane < 7) ? R[k * 7 + lane] : 0.0;
    const int per = (nconf + nw - 1) / nw;
    const int c0 = warp * per, c1 = min(nconf, c0 + per);
    for (int c = c0; c < c1; ++c) {
        double a;
        if (lane == 0) a = 1.0;
        else if (lane < 6) a = (feat[(size_t)c * ldF + lane - 1] - R[49 + lane - 1]) / sc;
        else if (lane == 6) a = lnw[c] - R[54];
        else a = 0.0;
        givens_absorb(Rrow, a, lane);
    }
    for (int st = 1; st < nw; st <<= 1) {
        if (warp % (2 * st) == st)
            for (int k = 0; k < 7; ++k)
                if (lane < 7) sR[warp][k * 7 + lane] = Rrow[k];
        __syncthreads();
        if (warp % (2 * st) == 0 && warp + st < nw)
            for (int k = 0; k < 7; ++k) givens_absorb(Rrow, (lane < 7) ? sR[warp + st][k * 7 + lane] : 0.0, lane);
        __syncthreads();
    }
    if (warp == 0) {
        for (int k = 0; k < 7; ++k)
            if (lane < 7) R[k * 7 + lane] = Rrow[k];
        if (lane == 0) R[56] += nconf;
    }
}

// Merges partial states (same layout as R) into R. Each state's factor is first moved to the
// reference of the first non-empty state: its rows [1, (F - F_b)/sc, y - y_b] equal the rows
// [1, (F - F_c)/sc, y - y_c] minus row 0 times d, d = ((F_b - F_c)/sc, y_b - y_c), i.e. the
// columns change by a unit upper-triangular matrix, which touches only row 0 of R.
__global__ void k_fit_merge(const double* __restrict__ states, int nparts, double* __restrict__ R, double sc) {
    const int lane = threadIdx.x;
    int ref = -1;
    for (int p = 0; p < nparts; ++p)
        if (states[(size_t)p * SLMC_FIT_STATE_DOUBLES + 55] != 0.0) {
            ref = p;
            break;
        }
    const double* C = states + (size_t)(ref < 0 ? 0 : ref) * SLMC_FIT_STATE_DOUBLES;
    double Rrow[7];
    for (int k = 0; k < 7; ++k) Rrow[k] = 0.0;
    double count = 0.0;
    for (int p = 0; p < nparts; ++p) {
        const double* S = states + (size_t)p * SLMC_FIT_STATE_DOUBLES;
        if (S[55] == 0.0) continue;
        count += S[56];
        for (int k = 0; k < 7; ++k) {
            double a = (lane < 7) ? S[k * 7 + lane] : 0.0;
            if (k == 0 && lane >= 1 && lane < 7) {
                const double d = (lane < 6) ? (S[49 + lane - 1] - C[49 + lane - 1]) / sc : S[54] - C[54];
                a = fma(S[0], d, a);
            }
            givens_absorb(Rrow, a, lane);
        }
    }
    for (int k = 0; k < 7; ++k)
        if (lane < 7) R[k * 7 + lane] = Rrow[k];
    if (lane < 6) R[49 + lane] = (ref < 0) ? 0.0 : C[49 + lane];
    if (lane == 0) {
        R[55] = (ref < 0) ? 0.0 : 1.0;
        R[56] = count;
    }
    if (lane >= 7 && lane < 14) R[57 + lane - 7] = 0.0;
}

__global__ void k_fit_finish(const double* __restrict__ R, double dtau, double sc, double* __restrict__ J,
                             double* __restrict__ resid, unsigned int* __restrict__ err) {
    if (threadIdx.x != 0) return;
    double c[6];
    bool ok = true;
    for (int k = 5; k >= 0; --k) {
        double s = R[k * 7 + 6];
        for (int m = k + 1; m < 6; ++m) s -= R[k * 7 + m] * c[m];
        if (R[k * 7 + k] == 0.0) ok = false;
        c[k] = s / R[k * 7 + k];
    }
    double icpt = c[0] + R[54];
    for (int q = 0; q < 5; ++q) icpt -= c[q + 1] * R[49 + q] / sc;
    J[0] = -icpt / dtau;
    for (int q = 0; q < 5; ++q) J[q + 1] = -(c[q + 1] / sc) / dtau;
    if (resid) resid[0] = fabs(R[6 * 7 + 6]) / sqrt(fmax(R[56], 1.0));
    if (!ok) atomicOr(err, SLMC_EBIT_SINGULAR);
}

}  // namespace

namespace slmc {

cudaError_t bose_log_weight(slmc_ctx* c, const double* x, int nf, const double* lndet, double* lnw, cudaStream_t s) {
    k_bose<<<nf, kThreads, 0, s>>>(x, c->N, c->L, c->p.dtau, c->p.lambda, c->p.omega0 * c->p.omega0, lndet, lnw);
    return cudaGetLastError();
}

cudaError_t eff_features(slmc_ctx* c, const double* x, int nf, const double* J, double* F, int ldF, double* lnw_eff,
                         cudaStream_t s) {
    const double a = c->p.lambda / (c->p.omega0 * c->p.omega0);
    k_features<<<nf, kThreads, 0, s>>>(x, c->p.Lx, c->p.Ly, c->L, a * a, c->p.dtau, J, F, ldF, lnw_eff);
    return cudaGetLastError();
}

cudaError_t eff_half_sweep(slmc_ctx* c, double* x, int nf, int chain0, const double* J, uint64_t sweep, int colour,
                           const int* colour_per_chain, int colour_xor, long long* n_acc, cudaStream_t s,
                           const unsigned long long* dctr, int nsweeps) {
    const double a = c->p.lambda / (c->p.omega0 * c->p.omega0);
    const int sites = c->N * (c->L / 2);
    dim3 grid((sites + kThreads - 1) / kThreads, nf);
    k_half_sweep<<<grid, kThreads, 0, s>>>(x, c->p.Lx, c->p.Ly, c->L, J, c->p.dtau, a * a, c->p.sweep_delta,
                                           (uint32_t)(c->p.seed & 0xffffffffu), (uint32_t)(c->p.seed >> 32),
                                           (uint32_t)sweep, colour, colour_per_chain, colour_xor, chain0,
                                           reinterpret_cast<unsigned long long*>(n_acc), dctr, nsweeps);
    return cudaGetLastError();
}

cudaError_t update_draws(slmc_ctx* c, int nf, int chain0, uint64_t u_off, int* first_colour, double* u_acc,
                         cudaStream_t s) {
    k_update_draws<<<(nf + 127) / 128, 128, 0, s>>>(nf, chain0, (uint32_t)u_off, c->dctr, (uint32_t)(c->p.seed & 0xffffffffu),
                                                    (uint32_t)(c->p.seed >> 32), first_colour, u_acc);
    return cudaGetLastError();
}

cudaError_t accept_update(slmc_ctx* c, int nf, double* x, const double* x_old, const double* lnw_new,
                          const double* lnweff_old, const double* lnweff_new, const double* u_acc, double* lnw,
                          int* accepted, long long* n_acc, cudaStream_t s) {
    k_accept<<<(nf + 127) / 128, 128, 0, s>>>(nf, lnw_new, lnweff_old, lnweff_new, u_acc, lnw, accepted,
                                              reinterpret_cast<unsigned long long*>(n_acc));
    const int NL = c->N * c->L;
    dim3 grid((NL + 255) / 256 < 64 ? (NL + 255) / 256 : 64, nf);
    k_restore<<<grid, 256, 0, s>>>(x, x_old, accepted, NL);
    return cudaGetLastError();
}

cudaError_t eff_wolff(slmc_ctx* c, double* x, int nf, int chain0, const double* J, uint64_t sweep, int k,
                      cudaStream_t s, const unsigned long long* dctr, int nsweeps) {
    k_wolff<<<nf, 256, 3 * c->N, s>>>(x, c->p.Lx, c->p.Ly, c->L, J, c->p.dtau, (uint32_t)(c->p.seed & 0xffffffffu),
                                      (uint32_t)(c->p.seed >> 32), (uint32_t)sweep, dctr, nsweeps, c->nwolff, k,
                                      chain0, c->wolff_sites);
    return cudaGetLastError();
}

int sweep_queue_grid() {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_queue, kThreads, 3 * 1024) != cudaSuccess)
        return 0;
    return sms * (per_sm < 1 ? 1 : per_sm);
}

cudaError_t sweep_queue(const QueueClass* classes, int ncls, const int4* items, int nitems, unsigned int* done,
                        unsigned int* ctl, int max_N, uint32_t u, long long wait_cycles, int grid, cudaStream_t s) {
    k_sweep_queue<<<grid, kThreads, 3 * max_N, s>>>(classes, ncls, items, nitems, done, ctl, u, wait_cycles);
    return cudaGetLastError();
}

cudaError_t cdw_measure(slmc_ctx* c, const double* G, int nf, double* S, const int* only_if, double* obs,
                        cudaStream_t s) {
    k_cdw<<<nf, kThreads, 0, s>>>(G, c->p.Lx, c->p.Ly, S, only_if, obs);
    return cudaGetLastError();
}

__global__ void k_counter(unsigned long long* __restrict__ ctr, unsigned long long v, int add) {
    if (threadIdx.x == 0) *ctr = add ? *ctr + v : v;
}

cudaError_t counter_op(slmc_ctx* c, uint64_t v, bool add, cudaStream_t s) {
    k_counter<<<1, 32, 0, s>>>(c->dctr, (unsigned long long)v, add ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t fit_begin(slmc_ctx* c, double* R, cudaStream_t s) {
    (void)c;
    k_fit_begin<<<1, 64, 0, s>>>(R);
    return cudaGetLastError();
}

cudaError_t fit_accumulate(slmc_ctx* c, double* R, const double* feat, const double* lnw, int nconf, cudaStream_t s) {
    const int warps = nconf >= 32 * 16 ? 32 : (nconf + 15) / 16;  // about 16 configurations per warp
    k_fit_accumulate<<<1, 32 * (warps < 1 ? 1 : warps), 0, s>>>(R, feat, 8, lnw, nconf, (double)c->N * c->L);
    return cudaGetLastError();
}

cudaError_t fit_merge(slmc_ctx* c, const double* states, int nparts, cudaStream_t s) {
    k_fit_merge<<<1, 32, 0, s>>>(states, nparts, c->fitR, (double)c->N * c->L);
    return cudaGetLastError();
}

cudaError_t fit_finish(slmc_ctx* c, int nconf, double* J_out, double* resid, cudaStream_t s) {
    (void)nconf;
    k_fit_finish<<<1, 32, 0, s>>>(c->fitR, c->p.dtau, (double)c->N * c->L, J_out, resid, c->err);
    return cudaGetLastError();
}

}  // namespace slmc
