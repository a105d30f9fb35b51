// Tensor-core (tcgen05) slice products in split precision [Suppl. Eq. (S2)].
//
// One launch applies one slice to every column of every field of the batch:
//   Y' = D_l (Y + F Y),   F = E - I,   D_l = diag(exp(-dtau lambda x[:, l])),
// with F and Y each represented as a sum of reduced-precision pieces:
//   SLMC_PREC_TF32X3: two TF32 pieces each, products F0Y0 + F0Y1 + F1Y0   (kind::tf32)
//   SLMC_PREC_BF16X9: three BF16 pieces each, all nine products          (kind::f16, BF16)
// accumulated in FP32 in tensor memory. Multiplying by F rather than E keeps the rounding
// error of the operand that every slice reuses relative to |F| (diagonal ~0.01 instead of
// ~1), and the identity part is added exactly in the epilogue; with that, plain FP32
// accumulation meets |d ln det| <= 5e-5 (measured in the numerical model of both modes).
//
// CTA = 128 rows of F (MMA M) x NT columns of one field (MMA N), K = all N sites in chunks of
// one 128-byte swizzle atom. Thread 0 streams the F and Y pieces into shared memory with TMA
// (128B swizzle, K-major, 2 stages), thread 32 issues tcgen05.mma into one TMEM accumulator,
// and all four warps read it back with tcgen05.ld for the epilogue: add Y (FP32), scale the
// row by exp(-dtau lambda x_il), store FP32 Y' and its pieces for the next slice (or FP64 Y
// for the QR after the last slice of a group). Every mbarrier wait is bounded: on timeout the
// kernel flags SLMC_ERR_TIMEOUT, stops issuing, waits (bounded) for its own copies and always
// frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "slmc_internal.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kStages = 2;
constexpr uint32_t kAtom = 128;  // bytes of K per swizzle atom row
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

template <int MODE>
struct Cfg;
template <>
struct Cfg<0> {  // 3 x TF32
    static constexpr int NP = 2, KC = 32, NTMAX = 256, NPROD = 3;  // K per MMA: 8
    static constexpr uint32_t FMT = 2;  // TF32
    __device__ static int pa(int q) { return q == 2 ? 1 : 0; }
    __device__ static int pb(int q) { return q == 1 ? 1 : 0; }
};
template <>
struct Cfg<1> {  // 9 x BF16
    static constexpr int NP = 3, KC = 64, NTMAX = 128, NPROD = 9;  // K per MMA: 16
    static constexpr uint32_t FMT = 1;  // BF16
    __device__ static int pa(int q) { return q / 3; }
    __device__ static int pb(int q) { return q % 3; }
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false (and the error flag) after ~2 s.
__device__ bool mbar_wait(uint32_t addr, uint32_t parity, unsigned int* err) {
    const long long t0 = clock64();
    while (!mbar_try(addr, parity)) {
        if (clock64() - t0 > kWaitCycles) {
            atomicOr(err, SLMC_EBIT_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(mbar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle layout (8-row x
// 128-byte atoms stacked along M/N, 1024 bytes apart), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;        // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

template <int MODE>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if (MODE == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

// Stores the pieces of v at element offset `off` of each piece array (piece stride pstride).
template <int MODE>
__device__ __forceinline__ void store_pieces(void* P, size_t pstride, size_t off, float v) {
    if (MODE == 0) {
        uint32_t* q = reinterpret_cast<uint32_t*>(P);
        const uint32_t hi = to_tf32(v);
        q[off] = hi;
        q[pstride + off] = to_tf32(v - __uint_as_float(hi));
    } else {
        uint16_t* q = reinterpret_cast<uint16_t*>(P);
        const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
        const float r1 = v - __bfloat162float(b0);
        const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
        const __nv_bfloat16 b2 = __float2bfloat16_rn(r1 - __bfloat162float(b1));
        q[off] = __bfloat16_as_ushort(b0);
        q[pstride + off] = __bfloat16_as_ushort(b1);
        q[2 * pstride + off] = __bfloat16_as_ushort(b2);
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_slice(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const float* __restrict__ ycur, float* __restrict__ ynext, void* __restrict__ pnext,
               double* __restrict__ yout, const float* __restrict__ sc32, int N, int Npad, int L, int l, int NT,
               int nfmax, unsigned int* __restrict__ err) {
    using C = Cfg<MODE>;
    const int m0 = blockIdx.x * 128, j0 = blockIdx.y * NT, f = blockIdx.z;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t a_bytes = 128 * kAtom, b_bytes = (uint32_t)NT * kAtom;
    const uint32_t stage_bytes = C::NP * (a_bytes + b_bytes);
    const uint32_t tcols = NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256));
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages], bar_acc;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const int nk = Npad / C::KC;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_acc), 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    int issued = 0;  // chunks whose copies thread 0 has issued
    if (tid == 0) {
        // ---- TMA producer ----
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % kStages, use = kc / kStages;
            if (use > 0 && !mbar_wait(smem_u32(&bar_empty[s]), (use - 1) & 1, err)) {
                abort_sh = 1;
                break;
            }
            const uint32_t fb = smem_u32(&bar_full[s]);
            mbar_expect_tx(fb, stage_bytes);
            const uint32_t sA = base + s * stage_bytes, sB = sA + C::NP * a_bytes;
            for (int pc = 0; pc < C::NP; ++pc) {
                tma_load_3d(sA + pc * a_bytes, &tmA, kc * C::KC, m0, pc, fb);
                tma_load_3d(sB + pc * b_bytes, &tmB, kc * C::KC, f * N + j0, pc, fb);
            }
            issued = kc + 1;
        }
    } else if (tid == 32) {
        // ---- MMA issuer ----
        const uint32_t idesc = (1u << 4) | (C::FMT << 7) | (C::FMT << 10) | ((uint32_t)(NT >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % kStages, use = kc / kStages;
            if (!mbar_wait(smem_u32(&bar_full[s]), use & 1, err)) {
                abort_sh = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sA = base + s * stage_bytes, sB = sA + C::NP * a_bytes;
#pragma unroll
            for (int ks = 0; ks < (int)(kAtom / 32); ++ks) {
#pragma unroll
                for (int q = 0; q < C::NPROD; ++q) {
                    const uint64_t ad = smem_desc_sw128(sA + C::pa(q) * a_bytes + ks * 32);
                    const uint64_t bd = smem_desc_sw128(sB + C::pb(q) * b_bytes + ks * 32);
                    mma<MODE>(tmem, ad, bd, idesc, (kc | ks | q) != 0 ? 1u : 0u);
                }
            }
            mma_commit(smem_u32(&bar_empty[s]));
        }
        mma_commit(smem_u32(&bar_acc));
    }
    __syncwarp();

    // ---- epilogue: all four warps, warp w owns TMEM lanes (rows) 32w..32w+31 ----
    const bool ok = mbar_wait(smem_u32(&bar_acc), 0, err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int i = m0 + warp * 32 + lane;
    float scale = 0.f;
    if (i < N) scale = sc32[((size_t)f * L + l) * N + i];
    const size_t pstride = (size_t)nfmax * N * Npad;
    for (int c0 = 0; c0 < NT; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
              "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (i < N && ok && !abort_sh) {
#pragma unroll
            for (int cc = 0; cc < 32; ++cc) {
                const int j = j0 + c0 + cc;
                if (c0 + cc >= NT || j >= N) continue;
                const size_t col = (size_t)f * N + j;
                const float v = (__uint_as_float(r[cc]) + ycur[col * N + i]) * scale;
                if (yout) {
                    yout[col * N + i] = (double)v;
                } else {
                    ynext[col * N + i] = v;
                    store_pieces<MODE>(pnext, pstride, col * Npad + i, v);
                }
            }
        }
    }

    // ---- teardown: copies in flight (bounded), then free tensor memory ----
    if (tid == 0) {
        for (int kc = issued - 1; kc >= 0 && kc >= issued - kStages; --kc)
            mbar_wait(smem_u32(&bar_full[kc % kStages]), (kc / kStages) & 1, err);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
    }
}

// U (FP32, column-major per field) -> FP32 copy and pieces: the first slice's operand.
template <int MODE>
__global__ void k_tc_split_in(const float* __restrict__ U, float* __restrict__ y32, void* __restrict__ P, int N,
                              int Npad, int nfmax, size_t total) {
    const size_t pstride = (size_t)nfmax * N * Npad;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t col = idx / N;
        const int i = (int)(idx - col * N);
        const float v = U[idx];
        y32[idx] = v;
        store_pieces<MODE>(P, pstride, col * Npad + i, v);
    }
}

// F = E - I (FP64) -> padded pieces [p][Npad][Npad] (zeros outside N x N).
template <int MODE>
__global__ void k_tc_split_F(const double* __restrict__ E, void* __restrict__ P, int N, int Npad) {
    using C = Cfg<MODE>;
    const size_t tot = (size_t)Npad * Npad;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / Npad), c = (int)(idx - (size_t)r * Npad);
        double v = (r < N && c < N) ? E[(size_t)r * N + c] - (r == c ? 1.0 : 0.0) : 0.0;
        for (int p = 0; p < C::NP; ++p) {
            if (MODE == 0) {
                const uint32_t t = to_tf32((float)v);
                reinterpret_cast<uint32_t*>(P)[p * tot + idx] = t;
                v -= (double)__uint_as_float(t);
            } else {
                const __nv_bfloat16 b = __float2bfloat16_rn((float)v);
                reinterpret_cast<uint16_t*>(P)[p * tot + idx] = __bfloat16_as_ushort(b);
                v -= (double)__bfloat162float(b);
            }
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map(CUtensorMap* m, void* gaddr, int mode, uint64_t inner, uint64_t rows, uint64_t pieces, uint32_t box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const int es = mode == 0 ? 4 : 2;
    const cuuint64_t dims[3] = {inner, rows, pieces};
    const cuuint64_t strides[2] = {inner * es, inner * rows * es};
    const cuuint32_t box[3] = {kAtom / (cuuint32_t)es, box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(m, mode == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, gaddr,
                          dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int MODE>
cudaError_t run_group(slmc_ctx* c, const double* x, int nf, int l0, int nsl, cudaStream_t s) {
    using C = Cfg<MODE>;
    const int N = c->N, Npad = c->tc_npad, NT = c->tc_nt;
    const size_t total = (size_t)nf * N * N;
    k_tc_split_in<MODE><<<1024, 256, 0, s>>>(c->U32, c->tc_y32[0], c->tc_p[0], N, Npad, c->max_fields, total);
    const size_t smem = 1024 + (size_t)kStages * C::NP * (128 * kAtom + (size_t)NT * kAtom);
    cudaError_t e = cudaFuncSetAttribute(k_tc_slice<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((N + 127) / 128, (N + NT - 1) / NT, nf);
    (void)x;
    for (int q = 0; q < nsl; ++q) {
        const int cur = q & 1, nxt = cur ^ 1;
        const bool last = (q == nsl - 1);
        k_tc_slice<MODE><<<grid, kThreads, smem, s>>>(c->tc_mapF, c->tc_mapP[cur], c->tc_y32[cur], c->tc_y32[nxt],
                                                      c->tc_p[nxt], last ? c->Y : nullptr, c->sc32, N, Npad, c->L,
                                                      l0 + q, NT, c->max_fields, c->err);
    }
    return cudaGetLastError();
}

}  // namespace

namespace slmc {

int tc_launches(int nsl) { return 1 + nsl; }

// Workspace geometry of the tensor-core path: K padded to one swizzle atom, column tile NT.
void tc_geometry(int N, int precision, int* npad, int* nt, size_t* piece_bytes, int* npieces) {
    const int mode = precision == SLMC_PREC_TF32X3 ? 0 : 1;
    const int kc = mode == 0 ? Cfg<0>::KC : Cfg<1>::KC;
    const int ntmax = mode == 0 ? Cfg<0>::NTMAX : Cfg<1>::NTMAX;
    *npad = (N + kc - 1) / kc * kc;
    const int ntiles = (N + ntmax - 1) / ntmax;
    int t = (N + ntiles - 1) / ntiles;
    *nt = (t + 15) / 16 * 16;
    *piece_bytes = mode == 0 ? 4 : 2;
    *npieces = mode == 0 ? Cfg<0>::NP : Cfg<1>::NP;
}

cudaError_t tc_init(slmc_ctx* c, cudaStream_t s) {
    const int mode = c->p.precision == SLMC_PREC_TF32X3 ? 0 : 1;
    const int Npad = c->tc_npad;
    if (mode == 0) k_tc_split_F<0><<<256, 256, 0, s>>>(c->E64, c->tc_F, c->N, Npad);
    else k_tc_split_F<1><<<256, 256, 0, s>>>(c->E64, c->tc_F, c->N, Npad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int np = mode == 0 ? Cfg<0>::NP : Cfg<1>::NP;
    if (!make_map(&c->tc_mapF, c->tc_F, mode, Npad, Npad, np, 128)) return cudaErrorInvalidValue;
    for (int b = 0; b < 2; ++b)
        if (!make_map(&c->tc_mapP[b], c->tc_p[b], mode, Npad, (uint64_t)c->max_fields * c->N, np, c->tc_nt))
            return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t tc_slice_group(slmc_ctx* c, const double* x, int nf, int l0, int nsl, cudaStream_t s) {
    return c->p.precision == SLMC_PREC_TF32X3 ? run_group<0>(c, x, nf, l0, nsl, s) : run_group<1>(c, x, nf, l0, nsl, s);
}

}  // namespace slmc
