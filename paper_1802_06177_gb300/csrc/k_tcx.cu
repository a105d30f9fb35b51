// Slice-group products on the tensor cores with exact accumulation [Suppl. Eq. (S2)]
// (precision mode SLMC_PREC_BF16X9).
//
// Each slice of a stabilisation group is applied as Y' = D_l (Y + F Y), F = E - I, as in the
// FP32 kernel. The product F Y runs on the tensor cores (tcgen05.mma kind::f16, BF16 operands,
// FP32 accumulators in tensor memory) in fixed-point slices:
//   F[i][k] = 2^(eF_i - 6) (f0 + f1 2^-7 + f2 2^-14 + f3 2^-21)      (per row i of F)
//   Y[k][j] = 2^(eY_j - 6) (y0 + y1 2^-7 + y2 2^-14)                 (per column j of Y)
// with integer slices |f0|, |y0| <= 128 and |f1..3|, |y1..2| <= 64 (round-to-nearest remainders),
// all exact in BF16; 2^eY_j is the power of two of the largest |Y[k][j]| and 2^eF_i the same
// for the row of F. The nine products f_a y_b with a + b <= 3 are summed by level a + b into four
// accumulators. Every term of a level shares one unit, and the worst case of a level's sum of
// absolute values is at most N 2^14 <= 2^24 for N <= 1024 (checked at set-up on the actual F
// slices), so every partial sum is an integer the FP32 accumulator holds exactly: the tensor
// cores add with no rounding at all, and the only roundings are those of the slicing (to
// nearest, unbiased) and of the FP32 epilogue. The levels are combined smallest first in FP32,
// Y is added exactly as in the FP32 kernel, and the row is scaled by exp(-dtau lambda x_il)
// (computed in FP64 and rounded once).
//
// Fusion: one CTA owns all N rows of NT columns of one field for every slice of the group. The
// three Y slices stay in shared memory (K-major, 128-byte swizzle, written by the epilogue in
// the layout TMA would produce), Y itself stays in the epilogue threads' registers, and only the
// F slices stream in (TMA ring of four 16-KB tiles; F is L2-resident: every CTA reads the same F). Roles: warps
// 0-7 epilogue (warp w reads tensor-memory lanes 32 (w % 4).. for half w / 4 of the NT columns,
// so each thread keeps MT x NT / 2 <= 64 values of Y in registers and two warps per SM
// sub-partition hide each other's latencies), warp 8 lane 0 issues the TMA copies, warp 9 lane 0
// the MMAs. Every mbarrier wait is bounded:
// on timeout the kernel flags SLMC_ERR_TIMEOUT, stops, waits (bounded) for its own copies and
// MMAs and frees its tensor memory.
#include <cuda_bf16.h>

#include <algorithm>

#include "tc_ptx.cuh"

namespace {

using namespace slmc::tc;

constexpr int kW = 7;                   // bits per slice
constexpr int kFS = 4, kYS = 3;         // slices of F and of Y
constexpr int kLevels = 4;              // a + b = 0..3
constexpr int kMaxStages = 4;           // ring of F tiles (8 measured no faster)
constexpr int kThreads = 320;           // 8 epilogue warps, producer warp, MMA warp
constexpr uint32_t kStageBytes = 128 * 128;  // 128 rows of F x 64 BF16
constexpr uint32_t kIdesc = idesc_f32acc(1, 128, 0);  // N field added per instantiation

__host__ __device__ constexpr uint32_t tmem_cols(int c) {
    return c <= 32 ? 32 : (c <= 64 ? 64 : (c <= 128 ? 128 : (c <= 256 ? 256 : 512)));
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// Exponent of the power of two of the largest |v| whose bit pattern is m (clamped so that
// every scale 2^(6 - e) and 2^(eF + e - 12) stays a normal FP32 number).
__device__ __forceinline__ int col_exponent(uint32_t m) {
    if (m == 0u) return 0;
    int e = (int)(m >> 23) - 127;
    return e < -100 ? -100 : (e > 100 ? 100 : e);
}

template <int MT, int NT>
__global__ void __launch_bounds__(kThreads, 1)
    k_tcx_group(const __grid_constant__ CUtensorMap tmF, const int* __restrict__ eF, const float* __restrict__ U32,
                double* __restrict__ Yout, const float* __restrict__ sc32, int N, int Npad, int L, int l0, int nsl,
                int kStages, unsigned int* __restrict__ err) {
    constexpr uint32_t TCOLS = tmem_cols(kLevels * MT * NT);
    constexpr uint32_t IDESC = kIdesc | ((uint32_t)(NT >> 3) << 17);
    const int f = blockIdx.y, j0 = blockIdx.x * NT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = Npad / 64;
    const uint32_t tileB = NT * 128u;         // one (Y slice, 64-row K chunk) tile
    const uint32_t sliceB = (uint32_t)nk * tileB;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kMaxStages], bar_empty[kMaxStages], bar_b, bar_acc, bar_done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ int eY_sh[2][NT];
    __shared__ uint32_t cm_sh[2][4][NT / 2];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t bbuf = base, stg = base + kYS * sliceB;
    uint8_t* bgen = smem_raw + (base - raw);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_b), 256);
        mbar_init(smem_u32(&bar_acc), 1);
        mbar_init(smem_u32(&bar_done), 1);
        abort_sh = 0;
        fence_barrier_init();
    }
    if (warp == 9) {
        tmem_alloc(smem_u32(&tmem_base_sh), TCOLS);
        tc_fence_before();
    }
    // rows of the Y slices beyond N (padding up to a 64-row chunk) stay zero
    for (uint32_t q = threadIdx.x; q < kYS * sliceB / 16; q += kThreads)
        reinterpret_cast<uint4*>(bgen)[q] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const int per_slice = nk * MT * kFS;
    int issued = 0;

    if (warp == 8) {
        // ---- TMA producer: F slice fs, rows mt*128.., K chunk kc, for every slice of the group ----
        if (lane == 0) {
            const int total = nsl * per_slice;
            for (int t = 0; t < total; ++t) {
                const int st = t % kStages;
                if (t >= kStages && !mbar_wait(smem_u32(&bar_empty[st]), ((t / kStages) - 1) & 1, err)) {
                    abort_sh = 1;
                    break;
                }
                if (abort_sh) break;
                const int u = t % per_slice, kc = u / (MT * kFS), mt = (u / kFS) % MT, fs = u % kFS;
                const uint32_t fb = smem_u32(&bar_full[st]);
                mbar_expect_tx(fb, kStageBytes);
                tma_load_3d(stg + st * kStageBytes, &tmF, kc * 64, mt * 128, fs, fb);
                issued = t + 1;
            }
            // teardown: copies in flight (bounded)
            for (int t = issued - 1; t >= 0 && t >= issued - kStages; --t)
                mbar_wait(smem_u32(&bar_full[t % kStages]), (t / kStages) & 1, err);
        }
    } else if (warp == 9) {
        // ---- MMA issuer ----
        if (lane == 0) {
            int t = 0;
            bool ok = true;
            for (int s = 0; s < nsl && ok; ++s) {
                if (!mbar_wait(smem_u32(&bar_b), s & 1, err) || abort_sh) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                uint32_t written = 0;
                for (int u = 0; u < per_slice && ok; ++u, ++t) {
                    const int st = t % kStages, kc = u / (MT * kFS), mt = (u / kFS) % MT, fs = u % kFS;
                    if (!mbar_wait(smem_u32(&bar_full[st]), (t / kStages) & 1, err) || abort_sh) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = stg + st * kStageBytes;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ad = smem_desc_sw128(a + ks * 32);
#pragma unroll
                        for (int j = 0; j < kYS; ++j) {
                            if (fs + j >= kLevels) continue;
                            const int bit = (fs + j) * MT + mt;
                            const uint64_t bd = smem_desc_sw128(bbuf + j * sliceB + kc * tileB + ks * 32);
                            mma_bf16(tmem + (uint32_t)(bit * NT), ad, bd, IDESC, (written >> bit) & 1u);
                            written |= 1u << bit;
                        }
                    }
                    mma_commit(smem_u32(&bar_empty[st]));
                }
                if (ok) mma_commit(smem_u32(&bar_acc));
            }
            if (!ok) abort_sh = 1;
            // every MMA issued above has completed once bar_done fires
            mma_commit(smem_u32(&bar_done));
            mbar_wait(smem_u32(&bar_done), 0, err);
        }
    } else {
        // ---- epilogue: warp w owns rows 32 (w % 4) + lane of every M tile, columns of half w / 4 ----
        constexpr int NH = NT / 2;
        const int q = warp & 3, h = warp >> 2, r = 32 * q + lane, jh = j0 + h * NH;
        float y[MT][NH];
        int eFr[MT];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const int i = mt * 128 + r;
            eFr[mt] = eF[i];
            const float* src = U32 + ((size_t)f * N + jh) * N + i;
#pragma unroll
            for (int c0 = 0; c0 < NH; c0 += 8) {
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    y[mt][c0 + c] = (i < N && jh + c0 + c < N) ? src[(size_t)(c0 + c) * N] : 0.f;
                asm volatile("" ::: "memory");  // bounded number of loads in flight per thread
            }
        }
        float sc[MT];
        // s = -1 publishes the group's input; slice s >= 0 combines the accumulators into y and
        // publishes y as the operand of slice s + 1 (the last slice stores y instead).
        for (int s = -1; s < nsl; ++s) {
            if (s >= 0) {
                // the slice's phonon scales, loaded before the wait so their latency is hidden
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    const int i = mt * 128 + r;
                    sc[mt] = i < N ? sc32[((size_t)f * L + l0 + s) * N + i] : 0.f;
                }
                const bool bad = !mbar_wait(smem_u32(&bar_acc), s & 1, err) || abort_sh;
                if (named_sync_or(3, 256, bad)) {  // one decision for all epilogue warps
                    abort_sh = 1;
                    break;
                }
                tc_fence_after();
                const int* ey = eY_sh[s & 1] + h * NH;
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
                    for (int c0 = 0; c0 < NH; c0 += 8) {
                        uint32_t a[kLevels][8];
                        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(h * NH + c0);
#pragma unroll
                        for (int lv = 0; lv < kLevels; ++lv) tmem_ld8(tl + (uint32_t)((lv * MT + mt) * NT), a[lv]);
                        tmem_ld_wait();
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            // levels smallest first; the scalings by powers of two are exact
                            float t = __fadd_rn(__fmul_rn(__uint_as_float(a[3][c]), 0x1p-21f),
                                                __fmul_rn(__uint_as_float(a[2][c]), 0x1p-14f));
                            t = __fadd_rn(t, __fmul_rn(__uint_as_float(a[1][c]), 0x1p-7f));
                            t = __fadd_rn(t, __uint_as_float(a[0][c]));
                            const float fy = __fmul_rn(t, pow2f(eFr[mt] + ey[c0 + c] - 2 * (kW - 1)));
                            y[mt][c0 + c] = __fmul_rn(__fadd_rn(y[mt][c0 + c], fy), sc[mt]);
                        }
                        asm volatile("" ::: "memory");
                    }
                }
                if (s == nsl - 1) {
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt) {
                        const int i = mt * 128 + r;
                        if (i >= N) continue;
                        double* dst = Yout + ((size_t)f * N + jh) * N + i;
#pragma unroll
                        for (int c0 = 0; c0 < NH; c0 += 8) {
#pragma unroll
                            for (int c = 0; c < 8; ++c)
                                if (jh + c0 + c < N) dst[(size_t)(c0 + c) * N] = (double)y[mt][c0 + c];
                            asm volatile("" ::: "memory");
                        }
                    }
                    break;
                }
            }
            // ---- publish: column exponents, then the three slices of y into the B buffer ----
            const int b = (s + 1) & 1;
#pragma unroll
            for (int c = 0; c < NH; ++c) {
                uint32_t m = 0u;
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) m = max(m, __float_as_uint(fabsf(y[mt][c])));
                m = __reduce_max_sync(0xffffffffu, m);
                if (lane == 0) cm_sh[h][q][c] = m;
            }
            named_sync(1 + h, 128);
            for (int c = r; c < NH; c += 128) {
                const uint32_t m = max(max(cm_sh[h][0][c], cm_sh[h][1][c]), max(cm_sh[h][2][c], cm_sh[h][3][c]));
                eY_sh[b][h * NH + c] = col_exponent(m);
            }
            named_sync(1 + h, 128);
            const int* eyn = eY_sh[b] + h * NH;
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const int i = mt * 128 + r;
                if (i >= Npad) continue;
                const uint32_t rowoff = (uint32_t)(i >> 6) * tileB + (uint32_t)(i & 7) * 2u;
                const int kchunk = (i & 63) >> 3;
#pragma unroll
                for (int c0 = 0; c0 < NH; c0 += 8) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float v = __fmul_rn(y[mt][c0 + c], pow2f(kW - 1 - eyn[c0 + c]));
                        const float q0 = rintf(v);
                        v = __fmul_rn(__fsub_rn(v, q0), 128.f);
                        const float q1 = rintf(v);
                        v = __fmul_rn(__fsub_rn(v, q1), 128.f);
                        const float q2 = rintf(v);
                        // K-major 128-byte swizzle: row (column of Y) h NH + c0 + c, 16-byte chunk kchunk ^ c
                        const uint32_t off =
                            rowoff + (uint32_t)(h * NH + c0 + c) * 128u + ((uint32_t)(kchunk ^ c) << 4);
                        *reinterpret_cast<__nv_bfloat16*>(bgen + off) = __float2bfloat16_rn(q0);
                        *reinterpret_cast<__nv_bfloat16*>(bgen + sliceB + off) = __float2bfloat16_rn(q1);
                        *reinterpret_cast<__nv_bfloat16*>(bgen + 2 * sliceB + off) = __float2bfloat16_rn(q2);
                    }
                    asm volatile("" ::: "memory");
                }
            }
            fence_async_shared();
            tc_fence_before();
            mbar_arrive(smem_u32(&bar_b));
        }
    }

    // ---- teardown: every copy and MMA of this CTA has completed; free tensor memory ----
    tc_fence_before();
    __syncthreads();
    if (warp == 9) tmem_dealloc(tmem, TCOLS);
}

// F = E - I (FP64) -> kFS fixed-point slices per row, BF16, [kFS][rows][Npad] (zero padded), the
// row exponents eF[rows] and, per slice, the largest row sum of |slice| (for the exactness bound).
__global__ void k_tcx_split_F(const double* __restrict__ E, __nv_bfloat16* __restrict__ Fs, int* __restrict__ eF,
                              unsigned long long* __restrict__ rowsum_max, int N, int Npad, int rows) {
    const int i = blockIdx.x;
    __shared__ double red[256];
    double m = 0.0;
    for (int k = threadIdx.x; k < N && i < N; k += blockDim.x)
        m = fmax(m, fabs(E[(size_t)i * N + k] - (i == k ? 1.0 : 0.0)));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    m = red[0];
    __syncthreads();
    int e = 0;
    if (m > 0.0) {
        frexp(m, &e);  // m = g 2^e, g in [0.5, 1): the power of two below m is 2^(e-1)
        e -= 1;
    }
    if (threadIdx.x == 0) eF[i] = e;
    double rs[kFS] = {0.0, 0.0, 0.0, 0.0};
    const size_t plane = (size_t)rows * Npad;
    for (int k = threadIdx.x; k < Npad; k += blockDim.x) {
        double v = (i < N && k < N) ? (E[(size_t)i * N + k] - (i == k ? 1.0 : 0.0)) : 0.0;
        v = ldexp(v, kW - 1 - e);
        for (int s = 0; s < kFS; ++s) {
            const double qv = rint(v);
            Fs[s * plane + (size_t)i * Npad + k] = __double2bfloat16(qv);
            rs[s] += fabs(qv);
            v = (v - qv) * 128.0;
        }
    }
    for (int s = 0; s < kFS; ++s) {
        red[threadIdx.x] = rs[s];
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) atomicMax(rowsum_max + s, (unsigned long long)red[0]);
        __syncthreads();
    }
}

// Shared memory of the Y slices and the ring (up to kMaxStages tiles within the 227 KB).
template <int MT, int NT>
cudaError_t launch_group(const slmc_ctx* c, int nf, int l0, int nsl, cudaStream_t s) {
    const int Npad = c->tcx_npad;
    const size_t fixed = 1024 + (size_t)kYS * (Npad / 64) * NT * 128;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_tcx_group<MT, NT>);
    if (e != cudaSuccess) return e;
    const size_t limit = 227 * 1024;  // dynamic + static shared memory of one CTA
    if (fa.sharedSizeBytes + fixed + 2 * kStageBytes > limit) return cudaErrorInvalidConfiguration;
    const int stages = (int)std::min<size_t>(kMaxStages, (limit - fa.sharedSizeBytes - fixed) / kStageBytes);
    const size_t smem = fixed + (size_t)stages * kStageBytes;
    e = cudaFuncSetAttribute(k_tcx_group<MT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((c->N + NT - 1) / NT, nf);
    k_tcx_group<MT, NT><<<grid, kThreads, smem, s>>>(c->tcx_mapF, c->tcx_eF, c->U32, c->Y, c->sc32, c->N, Npad,
                                                      c->L, l0, nsl, stages, c->err);
    return cudaGetLastError();
}

}  // namespace

namespace slmc {

// M tiles (128 rows) of the CTA and its column count NT: 4 accumulators x MT x NT <= 512
// tensor-memory columns.
void tcx_geometry(int N, int* mt, int* nt, int* npad) {
    *mt = (N + 127) / 128;
    *nt = *mt == 1 ? (N <= 64 ? 64 : 128) : (*mt == 2 ? 64 : (*mt <= 4 ? 32 : 16));
    *npad = (N + 63) / 64 * 64;
}

size_t tcx_F_bytes(int N) {
    int mt, nt, npad;
    tcx_geometry(N, &mt, &nt, &npad);
    return (size_t)kFS * mt * 128 * npad * sizeof(__nv_bfloat16);
}

// Slices of F, row exponents and the TMA descriptor; checks the exactness bound of every level:
// sum over its products (a, b) of max_i sum_k |f_a[i][k]| times the largest |y_b| (128, 64, 64).
cudaError_t tcx_init(slmc_ctx* c, cudaStream_t s) {
    int mt, nt, npad;
    tcx_geometry(c->N, &mt, &nt, &npad);
    c->tcx_npad = npad;
    const int rows = mt * 128;
    unsigned long long* rsum = nullptr;
    cudaError_t e = cudaMalloc(&rsum, kFS * sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(rsum, 0, kFS * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->tcx_F, 0, tcx_F_bytes(c->N), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->tcx_eF, 0, rows * sizeof(int), s);
    if (e == cudaSuccess) {
        k_tcx_split_F<<<rows, 256, 0, s>>>(c->E64, reinterpret_cast<__nv_bfloat16*>(c->tcx_F), c->tcx_eF, rsum, c->N,
                                           npad, rows);
        e = cudaGetLastError();
    }
    unsigned long long h[kFS] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, rsum, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(rsum);
    if (e != cudaSuccess) return e;
    const double ymax[kYS] = {128.0, 64.0, 64.0};
    for (int lv = 0; lv < kLevels; ++lv) {
        double b = 0.0;
        for (int a = 0; a < kFS; ++a)
            if (lv - a >= 0 && lv - a < kYS) b += (double)h[a] * ymax[lv - a];
        if (b > 16777216.0) return cudaErrorNotSupported;  // a partial sum could exceed 2^24
    }
    if (!make_map_sw128(&c->tcx_mapF, c->tcx_F, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, npad, rows, kFS, 128))
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t tcx_slice_group(slmc_ctx* c, int nf, int l0, int nsl, cudaStream_t s) {
    int mt, nt, npad;
    tcx_geometry(c->N, &mt, &nt, &npad);
    switch (mt) {
        case 1: return nt == 64 ? launch_group<1, 64>(c, nf, l0, nsl, s) : launch_group<1, 128>(c, nf, l0, nsl, s);
        case 2: return launch_group<2, 64>(c, nf, l0, nsl, s);
        case 3: return launch_group<3, 32>(c, nf, l0, nsl, s);
        case 4: return launch_group<4, 32>(c, nf, l0, nsl, s);
        case 5: return launch_group<5, 16>(c, nf, l0, nsl, s);
        case 6: return launch_group<6, 16>(c, nf, l0, nsl, s);
        case 7: return launch_group<7, 16>(c, nf, l0, nsl, s);
        default: return launch_group<8, 16>(c, nf, l0, nsl, s);
    }
}

}  // namespace slmc
