// SIMT panel kernel of the slice-group product.
//
// Slice group [Suppl. Eq. (S2)]: for one stabilisation group of nsl slices starting at l0,
//   Y = B_{l0+nsl} ... B_{l0+1} U,   B_l = diag(exp(-dtau lambda x[:, l-1])) E.
// In reduced precision each slice is applied as D_l (Y + F Y) with F = E - I: the rounding
// error of the operand that is reused in every slice (and so adds up coherently along the
// whole chain) is then relative to |F|, whose diagonal is about 100x smaller than E's,
// and the identity part is added exactly in the epilogue.
// Left multiplication acts on every column of U independently, so one CTA owns a panel
// of NB columns of one field, keeps it in shared memory across all nsl slices and streams
// E (symmetric, L2-resident) once per slice; the diagonal phonon scaling of each slice is
// applied in the epilogue before the panel is reused. Only U is read from and Y written to
// global memory, once per group.
//
// Layout: every N x N matrix is column-major, element (i, j) at j*N + i.
#include "slmc_internal.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kTS = 32;  // products accumulated in FP32 between two TwoSum steps of the FP32 slice kernel

template <typename T>
__device__ __forceinline__ T slice_scale(double xv, double dtlam);
template <>
__device__ __forceinline__ double slice_scale<double>(double xv, double dtlam) { return exp(-dtlam * xv); }

template <typename T, int MAXR, int CPT, bool TRI>
__global__ void __launch_bounds__(256) k_panel(const T* __restrict__ A, size_t a_stride,
                                               const double* __restrict__ B, const int* __restrict__ perm,
                                               double* __restrict__ out, const double* __restrict__ x,
                                               int N, int L, int l0, int nsl, double dtlam, int add_identity) {
    constexpr int NB = kWarps * CPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* P0 = reinterpret_cast<T*>(smem_raw);
    T* P1 = P0 + (size_t)NB * N;
    T* sc = P1 + (size_t)NB * N;
    const int f = blockIdx.y, j0 = blockIdx.x * NB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t NN = (size_t)N * N;
    const T* Af = A + (size_t)f * a_stride;
    const double* Bf = B + (size_t)f * NN;
    const int* pf = perm ? perm + (size_t)f * N : nullptr;

    for (int idx = tid; idx < NB * N; idx += 256) {
        const int jj = idx / N, k = idx - jj * N, j = j0 + jj;
        T v = T(0);
        if (j < N) v = (T)Bf[(size_t)j * N + (pf ? pf[k] : k)];
        P0[idx] = v;
    }
    T* Pin = P0;
    T* Pout = P1;
    for (int s = 0; s < nsl; ++s) {
        if (x) {
            const double* xf = x + (size_t)f * N * L + l0 + s;
            for (int i = tid; i < N; i += 256) sc[i] = slice_scale<T>(xf[(size_t)i * L], dtlam);
        }
        __syncthreads();
        T acc[MAXR][CPT];
#pragma unroll
        for (int r = 0; r < MAXR; ++r)
#pragma unroll
            for (int c = 0; c < CPT; ++c) acc[r][c] = T(0);
        for (int k = 0; k < N; ++k) {
            T pv[CPT];
#pragma unroll
            for (int c = 0; c < CPT; ++c) pv[c] = Pin[(warp + kWarps * c) * N + k];
            const T* Ak = Af + (size_t)k * N;
#pragma unroll
            for (int r = 0; r < MAXR; ++r) {
                if (TRI && 32 * r > k) continue;  // rows below the diagonal of Rt
                const int i = lane + 32 * r;
                const T a = (i < N && (!TRI || i <= k)) ? __ldg(Ak + i) : T(0);
#pragma unroll
                for (int c = 0; c < CPT; ++c) acc[r][c] = fma(a, pv[c], acc[r][c]);
            }
        }
        const bool last = (s == nsl - 1);
#pragma unroll
        for (int r = 0; r < MAXR; ++r) {
            const int i = lane + 32 * r;
            if (i >= N) continue;
            const T si = x ? sc[i] : T(1);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int jj = warp + kWarps * c;
                const T v = (add_identity ? acc[r][c] + Pin[jj * N + i] : acc[r][c]) * si;
                if (last) {
                    if (j0 + jj < N) out[(size_t)f * NN + (size_t)(j0 + jj) * N + i] = (double)v;
                } else {
                    Pout[jj * N + i] = v;
                }
            }
        }
        T* tmp = Pin;
        Pin = Pout;
        Pout = tmp;
        __syncthreads();
    }
}

template <typename T, int MAXR, int CPT, bool TRI>
cudaError_t launch_panel(const T* A, size_t a_stride, const double* B, const int* perm, double* out,
                         const double* x, int N, int L, int l0, int nsl, double dtlam, int add_identity, int nf,
                         cudaStream_t s) {
    constexpr int NB = kWarps * CPT;
    const size_t smem = (size_t)(2 * NB * N + N) * sizeof(T);
    auto kern = k_panel<T, MAXR, CPT, TRI>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((N + NB - 1) / NB, nf);
    kern<<<grid, 256, smem, s>>>(A, a_stride, B, perm, out, x, N, L, l0, nsl, dtlam, add_identity);
    return cudaGetLastError();
}

template <typename T, bool TRI>
cudaError_t dispatch_panel(const T* A, size_t a_stride, const double* B, const int* perm, double* out,
                           const double* x, int N, int L, int l0, int nsl, double dtlam, int ai, int nf,
                           cudaStream_t s) {
    switch (slmc::rows_per_lane_class(N)) {
        case 1: return launch_panel<T, 1, 4, TRI>(A, a_stride, B, perm, out, x, N, L, l0, nsl, dtlam, ai, nf, s);
        case 2: return launch_panel<T, 2, 4, TRI>(A, a_stride, B, perm, out, x, N, L, l0, nsl, dtlam, ai, nf, s);
        case 4: return launch_panel<T, 4, 4, TRI>(A, a_stride, B, perm, out, x, N, L, l0, nsl, dtlam, ai, nf, s);
        case 5: return launch_panel<T, 5, 4, TRI>(A, a_stride, B, perm, out, x, N, L, l0, nsl, dtlam, ai, nf, s);
        case 8: return launch_panel<T, 8, 4, TRI>(A, a_stride, B, perm, out, x, N, L, l0, nsl, dtlam, ai, nf, s);
        case 12: return launch_panel<T, 12, 2, TRI>(A, a_stride, B, perm, out, x, N, L, l0, nsl, dtlam, ai, nf, s);
        case 18: return launch_panel<T, 18, 1, TRI>(A, a_stride, B, perm, out, x, N, L, l0, nsl, dtlam, ai, nf, s);
        default: return launch_panel<T, 32, 1, TRI>(A, a_stride, B, perm, out, x, N, L, l0, nsl, dtlam, ai, nf, s);
    }
}


// Reduced-precision (FP32 SIMT) slice group, accuracy-preserving form. Each slice computes
//   Y' = D_l (Y + F Y),  F = F_hi + F_lo (two FP32 terms of E - I),
// with the products of one block of 32 k accumulated in FP32 and the block sums combined by
// TwoSum (Knuth) into a compensated pair, so small far-field contributions are not rounded
// away against the large running sum. The F_lo products (2^-24 smaller) are accumulated into
// the compensation term, on the S displacements of the translation-invariant F where |F| is
// largest (a stencil: F_lo(i, k) for r_k = r_i + r_j; the dropped part of F_lo is below
// 2^-24 of the S-th largest |F| entry, far below the FP32 rounding of the kept terms).
// Thread (row i, column group) owns rows i, i+256, ... and NBT columns of the CTA's panel;
// the panel sits in shared memory k-major with a row stride of NB + 4 floats (four columns
// per 128-bit load; rows of consecutive threads fall in distinct bank groups), and the rows
// k0..k0+KB-1 of F_hi (contiguous in global memory) are double-buffered into shared memory
// with cp.async while the previous block is multiplied.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// rows [k0, k0 + nk) of F_hi into Fs[KB][N]
__device__ __forceinline__ void stage_F(float* Fs, const float* __restrict__ Fhi, int N, int k0, int nk) {
    const size_t n = (size_t)nk * N;
    const float* gh = Fhi + (size_t)k0 * N;
    if ((N & 3) == 0) {
        for (size_t q = threadIdx.x; q < n / 4; q += blockDim.x) cp_async16(Fs + 4 * q, gh + 4 * q);
    } else {
        for (size_t q = threadIdx.x; q < n; q += blockDim.x) cp_async4(Fs + q, gh + q);
    }
}

template <int RPT, int NBT, int KB, int NCG, int TR>
__global__ void __launch_bounds__(TR * NCG, (TR * NCG == 256 ? 2 : 1)) k_slice_f32(const float* __restrict__ Fhi, const int* __restrict__ lo_kidx,
                                                   const float* __restrict__ lo_val, int S,
                                                   const float* __restrict__ U, double* __restrict__ out,
                                                   const float* __restrict__ sc32, int N, int L, int l0, int nsl) {
    constexpr int NB = NCG * NBT;  // NCG column groups of NBT columns; thread = (row, group)
    constexpr int NBP = NB + 4;    // padded row stride of the panel
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* P0 = reinterpret_cast<float*>(smem_raw);  // [N][NBP]
    float* P1 = P0 + (size_t)N * NBP;
    float* Fs0 = P1 + (size_t)N * NBP;  // two stages of [KB][N]
    float* Fs1 = Fs0 + (size_t)KB * N;
    const int f = blockIdx.y, j0 = blockIdx.x * NB, tid = threadIdx.x % TR, cg = (threadIdx.x / TR) * NBT;
    const size_t NN = (size_t)N * N;
    const int nblk = (N + KB - 1) / KB;
    for (int idx = threadIdx.x; idx < NB * N; idx += TR * NCG) {
        const int jj = idx / N, k = idx - jj * N, j = j0 + jj;
        P0[k * NBP + jj] = (j < N) ? U[(size_t)f * NN + (size_t)j * N + k] : 0.f;
    }
    float* Pin = P0;
    float* Pout = P1;
    for (int s = 0; s < nsl; ++s) {
        __syncthreads();
        stage_F(Fs0, Fhi, N, 0, min(KB, N));
        cp_async_commit();
        float hi[RPT][NBT], cp[RPT][NBT], blk[RPT][NBT];
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int c = 0; c < NBT; ++c) hi[r][c] = cp[r][c] = blk[r][c] = 0.f;
        for (int b = 0; b < nblk; ++b) {
            float* Fcur = (b & 1) ? Fs1 : Fs0;
            if (b + 1 < nblk) stage_F((b & 1) ? Fs0 : Fs1, Fhi, N, (b + 1) * KB, min(KB, N - (b + 1) * KB));
            cp_async_commit();
            cp_async_wait1();
            __syncthreads();
            const int k0 = b * KB, nk = min(KB, N - k0);
            const float* Fh = Fcur;
            for (int kk = 0; kk < nk; ++kk) {
                const int k = k0 + kk;
                float pv[NBT];
#pragma unroll
                for (int c = 0; c < NBT; c += 4) {
                    const float4 q = *reinterpret_cast<const float4*>(Pin + k * NBP + cg + c);
                    pv[c] = q.x;
                    pv[c + 1] = q.y;
                    pv[c + 2] = q.z;
                    pv[c + 3] = q.w;
                }
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const int i = tid + TR * r;
                    const float ah = (i < N) ? Fh[kk * N + i] : 0.f;
#pragma unroll
                    for (int c = 0; c < NBT; ++c) blk[r][c] = fmaf(ah, pv[c], blk[r][c]);
                }
            }
            if (((b + 1) * KB) % kTS == 0 || b + 1 == nblk) {  // blocks of kTS products per TwoSum
#pragma unroll
                for (int r = 0; r < RPT; ++r)
#pragma unroll
                    for (int c = 0; c < NBT; ++c) {  // TwoSum(hi, blk) -> hi + error into cp
                        const float t = __fadd_rn(hi[r][c], blk[r][c]);
                        const float bp = __fsub_rn(t, hi[r][c]);
                        const float e = __fadd_rn(__fsub_rn(hi[r][c], __fsub_rn(t, bp)), __fsub_rn(blk[r][c], bp));
                        cp[r][c] = __fadd_rn(cp[r][c], e);
                        hi[r][c] = t;
                        blk[r][c] = 0.f;
                    }
            }
            __syncthreads();  // the stage just read is refilled two blocks later
        }
        // F_lo on its stencil (rows of the panel already in shared memory)
        for (int q = 0; q < S; ++q) {
            const float v = __ldg(lo_val + q);
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int i = tid + TR * r;
                if (i < N) {
                    const int k = __ldg(lo_kidx + (size_t)q * N + i);
#pragma unroll
                    for (int c = 0; c < NBT; c += 4) {
                        const float4 y = *reinterpret_cast<const float4*>(Pin + k * NBP + cg + c);
                        cp[r][c] = fmaf(v, y.x, cp[r][c]);
                        cp[r][c + 1] = fmaf(v, y.y, cp[r][c + 1]);
                        cp[r][c + 2] = fmaf(v, y.z, cp[r][c + 2]);
                        cp[r][c + 3] = fmaf(v, y.w, cp[r][c + 3]);
                    }
                }
            }
        }
        const bool last = (s == nsl - 1);
        const float* scl = sc32 + ((size_t)f * L + l0 + s) * N;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int i = tid + TR * r;
            if (i >= N) continue;
            const float sc = scl[i];
#pragma unroll
            for (int c = 0; c < NBT; c += 4) {
                const float4 y = *reinterpret_cast<const float4*>(Pin + i * NBP + cg + c);
                float4 v;
                v.x = __fmul_rn(__fadd_rn(y.x, __fadd_rn(hi[r][c], cp[r][c])), sc);
                v.y = __fmul_rn(__fadd_rn(y.y, __fadd_rn(hi[r][c + 1], cp[r][c + 1])), sc);
                v.z = __fmul_rn(__fadd_rn(y.z, __fadd_rn(hi[r][c + 2], cp[r][c + 2])), sc);
                v.w = __fmul_rn(__fadd_rn(y.w, __fadd_rn(hi[r][c + 3], cp[r][c + 3])), sc);
                if (last) {
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (j0 + cg + c + q < N) out[(size_t)f * NN + (size_t)(j0 + cg + c + q) * N + i] = (double)vv[q];
                } else {
                    *reinterpret_cast<float4*>(Pout + i * NBP + cg + c) = v;
                }
            }
        }
        float* t = Pin;
        Pin = Pout;
        Pout = t;
    }
}

constexpr size_t kSmemBudget = 220 * 1024;

template <int RPT, int NBT, int KB, int NCG, int TR>
cudaError_t launch_slice_f32_kb(const slmc_ctx* c, int nf, int l0, int nsl, cudaStream_t s) {
    const int N = c->N;
    constexpr int NBP = NCG * NBT + 4;
    const size_t smem = ((size_t)2 * N * NBP + (size_t)2 * KB * N) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_slice_f32<RPT, NBT, KB, NCG, TR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    constexpr int NB = NCG * NBT;
    dim3 grid((N + NB - 1) / NB, nf);
    k_slice_f32<RPT, NBT, KB, NCG, TR><<<grid, TR * NCG, smem, s>>>(c->F32, c->lo_kidx, c->lo_val, c->lo_S, c->U32, c->Y, c->sc32, N,
                                                      c->L, l0, nsl);
    return cudaGetLastError();
}

// Largest staged block (32, 16 or 8 rows of F) that fits the shared-memory budget. With one
// column group (256 threads, about half the registers and shared memory of two groups) a CTA
// leaves room on its SM for a CTA of the FP64 stabilisation kernels of another sub-batch.
template <int RPT, int NBT, int NCG, int TR = 256>
cudaError_t launch_slice_f32_g(const slmc_ctx* c, int nf, int l0, int nsl, cudaStream_t s) {
    const size_t budget = TR * NCG == 256 ? kSmemBudget / 2 : kSmemBudget;
    const size_t panel = (size_t)2 * c->N * (NCG * NBT + 4) * sizeof(float);
    const size_t per_row = (size_t)2 * c->N * sizeof(float);
    if (panel + 32 * per_row <= budget) return launch_slice_f32_kb<RPT, NBT, 32, NCG, TR>(c, nf, l0, nsl, s);
    if (panel + 16 * per_row <= budget) return launch_slice_f32_kb<RPT, NBT, 16, NCG, TR>(c, nf, l0, nsl, s);
    return launch_slice_f32_kb<RPT, NBT, 8, NCG, TR>(c, nf, l0, nsl, s);
}

template <int RPT, int NBT>
cudaError_t launch_slice_f32(const slmc_ctx* c, const double* x, int nf, int l0, int nsl, cudaStream_t s) {
    (void)x;
    if (c->tune_slice_groups == 2) return launch_slice_f32_g<RPT, NBT, 2>(c, nf, l0, nsl, s);
    if ((c->tune_slice_groups == 4 || c->tune_slice_groups == 0) && c->N <= 256) {
        // default for N <= 256: 64 row threads x 4 column groups of 8, up to 4 rows each
        switch ((c->N + 63) / 64) {
            case 1: return launch_slice_f32_g<1, 8, 4, 64>(c, nf, l0, nsl, s);
            case 2: return launch_slice_f32_g<2, 8, 4, 64>(c, nf, l0, nsl, s);
            case 3: return launch_slice_f32_g<3, 8, 4, 64>(c, nf, l0, nsl, s);
            default: return launch_slice_f32_g<4, 8, 4, 64>(c, nf, l0, nsl, s);
        }
    }
    return launch_slice_f32_g<RPT, NBT, 1>(c, nf, l0, nsl, s);
}

// exp(-dtau lambda x[f][i][l]) in FP64, rounded once to FP32, stored [f][l][i]: the slice
// scales of the reduced-precision modes (an FP32 exp of an FP32 argument carries a small
// systematic bias that every slice would repeat).
__global__ void k_scales(const double* __restrict__ x, float* __restrict__ sc, int N, int L, double dtlam,
                         size_t total) {
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t f = idx / ((size_t)N * L);
        const size_t rem = idx - f * N * L;
        const int i = (int)(rem / L), l = (int)(rem - (size_t)i * L);
        sc[(f * L + l) * N + i] = (float)exp(-dtlam * x[idx]);
    }
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, size_t total) {
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x)
        b[idx] = (float)a[idx];
}

__global__ void k_identity(double* __restrict__ U, float* __restrict__ U32, double* __restrict__ T,
                           double* __restrict__ lnD, int N) {
    const int f = blockIdx.y;
    const size_t NN = (size_t)N * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
        const double v = (idx % (N + 1) == 0) ? 1.0 : 0.0;
        U[(size_t)f * NN + idx] = v;
        if (U32) U32[(size_t)f * NN + idx] = (float)v;
        T[(size_t)f * NN + idx] = v;
        if (idx < (size_t)N) lnD[(size_t)f * N + idx] = 0.0;
    }
}

}  // namespace

namespace slmc {

cudaError_t slice_group(slmc_ctx* c, const double* x, int nf, int l0, int nsl, cudaStream_t s) {
    const double dtlam = c->p.dtau * c->p.lambda;
    if (c->p.precision == SLMC_PREC_FP32) {  // F = E - I as two FP32 terms, identity added in the epilogue
        const int rpt = (c->N + 255) / 256;
        if (rpt == 1 && c->tune_slice_cols == 8) return launch_slice_f32<1, 8>(c, x, nf, l0, nsl, s);
        if (rpt == 1) return launch_slice_f32<1, 16>(c, x, nf, l0, nsl, s);
        if (rpt == 2) return launch_slice_f32<2, 8>(c, x, nf, l0, nsl, s);
        if (rpt == 3) return launch_slice_f32<3, 8>(c, x, nf, l0, nsl, s);
        return launch_slice_f32<4, 4>(c, x, nf, l0, nsl, s);
    }
    if (c->kron && !c->dense_slices) return slice_group_kron(c, x, nf, l0, nsl, false, s);
    return dispatch_panel<double, false>(c->E64, 0, c->U, nullptr, c->Y, x, c->N, c->L, l0, nsl, dtlam, 0, nf, s);
}

cudaError_t slice_scales(slmc_ctx* c, const double* x, int nf, cudaStream_t s) {
    const size_t total = (size_t)nf * c->N * c->L;
    k_scales<<<(unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096), 256, 0, s>>>(
        x, c->sc32, c->N, c->L, c->p.dtau * c->p.lambda, total);
    return cudaGetLastError();
}

cudaError_t u_to_f32(slmc_ctx* c, int nf, cudaStream_t s) {
    const size_t total = (size_t)nf * c->N * c->N;
    k_to_f32<<<(unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096), 256, 0, s>>>(c->U, c->U32, total);
    return cudaGetLastError();
}

cudaError_t set_identity(slmc_ctx* c, int nf, cudaStream_t s) {
    dim3 grid(64, nf);
    k_identity<<<grid, 256, 0, s>>>(c->U, c->U32, c->Ta, c->lnD, c->N);
    return cudaGetLastError();
}

}  // namespace slmc
