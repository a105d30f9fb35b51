// Tensor-core (tcgen05) slice products in split TF32 [Suppl. Eq. (S2)] (precision mode
// SLMC_PREC_TF32X3).
//
// One launch applies one slice to every column of every field of the batch:
//   Y' = D_l (Y + F Y),   F = E - I,   D_l = diag(exp(-dtau lambda x[:, l])),
// with F and Y each split into two TF32 pieces (hi = TF32(v), lo = TF32(v - hi)) and the three
// products F0Y0 + F0Y1 + F1Y0 accumulated in FP32 in tensor memory (kind::tf32). This is the
// 3xTF32 scheme of the literature. The tensor cores' FP32 accumulation truncates, and every
// accumulation step of the K sweep adds a one-sided error of up to an ulp of the running sum;
// over the slices of a chain these add up coherently, so this mode does not reach the
// accuracy of the FP32 SIMT kernel or of the exact sliced BF16 mode (k_tcx.cu). TF32 pieces
// cannot be made exact the same way: the remainders of a split are dense, and 11-bit dense
// pieces summed over a row overflow the 24 bits an FP32 accumulator holds exactly.
//
// CTA = 128 rows of F (MMA M) x NT columns of one field (MMA N), K = all N sites in chunks of
// one 128-byte swizzle atom. Thread 0 streams the F and Y pieces into shared memory with TMA
// (128B swizzle, K-major, 2 stages), thread 32 issues tcgen05.mma into one TMEM accumulator,
// and all four warps read it back with tcgen05.ld for the epilogue: add Y (FP32), scale the
// row by exp(-dtau lambda x_il), store FP32 Y' and its pieces for the next slice (or FP64 Y
// for the QR after the last slice of a group). Every mbarrier wait is bounded: on timeout the
// kernel flags SLMC_ERR_TIMEOUT, stops issuing, waits (bounded) for its own copies and always
// frees its tensor memory.
#include "tc_ptx.cuh"

namespace {

using namespace slmc::tc;

constexpr int kThreads = 128;
constexpr int kStages = 2;
constexpr int kNP = 2, kKC = 32, kNTMAX = 256, kNPROD = 3;  // pieces, K per atom, widest tile, products

__device__ __forceinline__ int piece_a(int q) { return q == 2 ? 1 : 0; }
__device__ __forceinline__ int piece_b(int q) { return q == 1 ? 1 : 0; }

__device__ __forceinline__ uint32_t to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

// Stores the two pieces of v at element offset `off` of each piece array (piece stride pstride).
__device__ __forceinline__ void store_pieces(uint32_t* q, size_t pstride, size_t off, float v) {
    const uint32_t hi = to_tf32(v);
    q[off] = hi;
    q[pstride + off] = to_tf32(v - __uint_as_float(hi));
}

__global__ void __launch_bounds__(kThreads, 1)
    k_tc_slice(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const float* __restrict__ ycur, float* __restrict__ ynext, uint32_t* __restrict__ pnext,
               double* __restrict__ yout, const float* __restrict__ sc32, int N, int Npad, int L, int l, int NT,
               int nfmax, unsigned int* __restrict__ err) {
    const int m0 = blockIdx.x * 128, j0 = blockIdx.y * NT, f = blockIdx.z;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t a_bytes = 128 * kAtom, b_bytes = (uint32_t)NT * kAtom;
    const uint32_t stage_bytes = kNP * (a_bytes + b_bytes);
    const uint32_t tcols = NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256));
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages], bar_acc;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const int nk = Npad / kKC;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_acc), 1);
        abort_sh = 0;
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(&tmem_base_sh), tcols);
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
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
            const uint32_t sA = base + s * stage_bytes, sB = sA + kNP * a_bytes;
            for (int pc = 0; pc < kNP; ++pc) {
                tma_load_3d(sA + pc * a_bytes, &tmA, kc * kKC, m0, pc, fb);
                tma_load_3d(sB + pc * b_bytes, &tmB, kc * kKC, f * N + j0, pc, fb);
            }
            issued = kc + 1;
        }
    } else if (tid == 32) {
        // ---- MMA issuer ----
        const uint32_t idesc = idesc_f32acc(2, 128, NT);
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % kStages, use = kc / kStages;
            if (!mbar_wait(smem_u32(&bar_full[s]), use & 1, err)) {
                abort_sh = 1;
                break;
            }
            tc_fence_after();
            const uint32_t sA = base + s * stage_bytes, sB = sA + kNP * a_bytes;
#pragma unroll
            for (int ks = 0; ks < (int)(kAtom / 32); ++ks) {
#pragma unroll
                for (int q = 0; q < kNPROD; ++q) {
                    const uint64_t ad = smem_desc_sw128(sA + piece_a(q) * a_bytes + ks * 32);
                    const uint64_t bd = smem_desc_sw128(sB + piece_b(q) * b_bytes + ks * 32);
                    mma_tf32(tmem, ad, bd, idesc, (kc | ks | q) != 0 ? 1u : 0u);
                }
            }
            mma_commit(smem_u32(&bar_empty[s]));
        }
        mma_commit(smem_u32(&bar_acc));
    }
    __syncwarp();

    // ---- epilogue: all four warps, warp w owns TMEM lanes (rows) 32w..32w+31 ----
    const bool ok = mbar_wait(smem_u32(&bar_acc), 0, err);
    tc_fence_after();
    const int i = m0 + warp * 32 + lane;
    float scale = 0.f;
    if (i < N) scale = sc32[((size_t)f * L + l) * N + i];
    const size_t pstride = (size_t)nfmax * N * Npad;
    for (int c0 = 0; c0 < NT; c0 += 8) {
        uint32_t r[8];
        tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
        tmem_ld_wait();
        if (i < N && ok && !abort_sh) {
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                const int j = j0 + c0 + cc;
                if (c0 + cc >= NT || j >= N) continue;
                const size_t col = (size_t)f * N + j;
                const float v = (__uint_as_float(r[cc]) + ycur[col * N + i]) * scale;
                if (yout) {
                    yout[col * N + i] = (double)v;
                } else {
                    ynext[col * N + i] = v;
                    store_pieces(pnext, pstride, col * Npad + i, v);
                }
            }
        }
    }

    // ---- teardown: copies in flight (bounded), then free tensor memory ----
    if (tid == 0) {
        for (int kc = issued - 1; kc >= 0 && kc >= issued - kStages; --kc)
            mbar_wait(smem_u32(&bar_full[kc % kStages]), (kc / kStages) & 1, err);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tcols);
}

// U (FP32, column-major per field) -> FP32 copy and pieces: the first slice's operand.
__global__ void k_tc_split_in(const float* __restrict__ U, float* __restrict__ y32, uint32_t* __restrict__ P, int N,
                              int Npad, int nfmax, size_t total) {
    const size_t pstride = (size_t)nfmax * N * Npad;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t col = idx / N;
        const int i = (int)(idx - col * N);
        const float v = U[idx];
        y32[idx] = v;
        store_pieces(P, pstride, col * Npad + i, v);
    }
}

// F = E - I (FP64) -> padded pieces [p][Npad][Npad] (zeros outside N x N).
__global__ void k_tc_split_F(const double* __restrict__ E, uint32_t* __restrict__ P, int N, int Npad) {
    const size_t tot = (size_t)Npad * Npad;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / Npad), c = (int)(idx - (size_t)r * Npad);
        double v = (r < N && c < N) ? E[(size_t)r * N + c] - (r == c ? 1.0 : 0.0) : 0.0;
        for (int p = 0; p < kNP; ++p) {
            const uint32_t t = to_tf32((float)v);
            P[p * tot + idx] = t;
            v -= (double)__uint_as_float(t);
        }
    }
}

}  // namespace

namespace slmc {

int tc_launches(int nsl) { return 1 + nsl; }

// Workspace geometry of the split-TF32 path: K padded to one swizzle atom, column tile NT.
void tc_geometry(int N, int* npad, int* nt, size_t* piece_bytes, int* npieces) {
    *npad = (N + kKC - 1) / kKC * kKC;
    const int ntiles = (N + kNTMAX - 1) / kNTMAX;
    const int t = (N + ntiles - 1) / ntiles;
    *nt = (t + 15) / 16 * 16;
    *piece_bytes = 4;
    *npieces = kNP;
}

cudaError_t tc_init(slmc_ctx* c, cudaStream_t s) {
    const int Npad = c->tc_npad;
    k_tc_split_F<<<256, 256, 0, s>>>(c->E64, reinterpret_cast<uint32_t*>(c->tc_F), c->N, Npad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (!make_map_sw128(&c->tc_mapF, c->tc_F, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Npad, Npad, kNP, 128))
        return cudaErrorInvalidValue;
    for (int b = 0; b < 2; ++b)
        if (!make_map_sw128(&c->tc_mapP[b], c->tc_p[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Npad,
                            (uint64_t)c->max_fields * c->N, kNP, c->tc_nt))
            return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t tc_slice_group(slmc_ctx* c, const double* x, int nf, int l0, int nsl, cudaStream_t s) {
    (void)x;
    const int N = c->N, Npad = c->tc_npad, NT = c->tc_nt;
    const size_t total = (size_t)nf * N * N;
    uint32_t* p0 = reinterpret_cast<uint32_t*>(c->tc_p[0]);
    k_tc_split_in<<<1024, 256, 0, s>>>(c->U32, c->tc_y32[0], p0, N, Npad, c->max_fields, total);
    const size_t smem = 1024 + (size_t)kStages * kNP * (128 * kAtom + (size_t)NT * kAtom);
    cudaError_t e = cudaFuncSetAttribute(k_tc_slice, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((N + 127) / 128, (N + NT - 1) / NT, nf);
    for (int q = 0; q < nsl; ++q) {
        const int cur = q & 1, nxt = cur ^ 1;
        const bool last = (q == nsl - 1);
        k_tc_slice<<<grid, kThreads, smem, s>>>(c->tc_mapF, c->tc_mapP[cur], c->tc_y32[cur], c->tc_y32[nxt],
                                                reinterpret_cast<uint32_t*>(c->tc_p[nxt]), last ? c->Y : nullptr,
                                                c->sc32, N, Npad, c->L, l0 + q, NT, c->max_fields, c->err);
    }
    return cudaGetLastError();
}

}  // namespace slmc
