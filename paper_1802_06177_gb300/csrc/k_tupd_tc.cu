// T update of the UDT chain on the tensor cores, FP64-accurate: T_new = Rt P^T T_old.
//
// Rt (upper triangular, from the packed QR) and B = P^T T_old are each cut into seven 7-bit
// fixed-point slices, exact in BF16:
//   Rt[i][k] = 2^(eA_i - 6) sum_a a_a[i][k] 2^(-7a),   B[k][j] = 2^(eB_j - 6) sum_b b_b[k][j] 2^(-7b),
// with a power of two per row of Rt and per column of B, |a_0|, |b_0| <= 128 and |a_a|, |b_b| <= 64
// (balanced base-128 digits of the entry rounded once at 2^-42 of the scale, found with integer
// arithmetic so that the slicing spends no FP64 issue slots). This is an error-free splitting of
// the product into partial products that the tensor cores compute exactly (after Ozaki, Ogita,
// Oishi, Rump 2012): the 28 products a_a b_b with a + b <= 6 are summed per level a + b into seven
// FP32 accumulators in tensor memory, and a level's sum of absolute values is bounded per row by
// sum_a rowsum(a_a) * max|b_(level - a)|; when that bound is at most 2^24 for every row of a tile,
// every partial sum is an integer the FP32 accumulator holds exactly. The epilogue combines
// levels 0-2 and 3-6 in two 64-bit integers (Horner in 2^7) and rounds their sum once to FP64 (one
// FMA), so each entry is the correctly rounded value of the sliced product; the dropped terms
// (levels 7-12 and the slicing remainders) are below 2^-48 of the row and column scales, at the
// level of the FP64 chain's own rounding. Rows whose bound exceeds 2^24 (never met at the benchmark's parameters; the bound is
// computed on the actual slices) send their 128-row tile to a plain FP64 loop in the same kernel.
//
// Kernels: k_tt_slice_B (columns of T_old gathered by the pivots, sliced per column, written
// K-major, and the tiles' flags cleared), k_tt_slice_A (rows of Rt sliced per row, the bound
// checked per row), k_tt_gemm (one CTA per 128 rows x 32 columns of one field: TMA streams the
// seven A slices of each 64-wide K chunk through a 3-tile ring and the seven B slices double-buffered,
// one thread issues the MMAs, eight warps drain the accumulators, stage the tile in shared memory
// and write T_new row-major with coalesced stores; 32 columns per CTA keep the accumulators at
// 7 x 32 tensor-memory columns and the shared memory near 105 KB, so two CTAs share an SM). Row-tile mt starts its K loop at row 128 mt
// (Rt is zero to the left of its diagonal). All waits are clock-bounded as in the other
// tensor-core kernels.
#include <cuda_bf16.h>

#include "slice7.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace slmc::tc;
using slmc::s7::abs_bits;
using slmc::s7::exponent_of_bits;
using slmc::s7::kS;
using slmc::s7::pow2d;
using slmc::s7::slice7;
using slmc::s7::warp_max_bits;

constexpr int kW = 7;
constexpr int kLevels = 7;   // a + b = 0..6
constexpr int kNT = 32;      // columns per CTA (7 x 32 accumulator columns: two CTAs per SM)
constexpr int kThreads = 320;
constexpr uint32_t kATile = 128 * 128;  // 128 rows x 64 BF16
constexpr uint32_t kBTile = kNT * 128;  // 32 rows (columns of T) x 64 BF16
constexpr uint32_t kBChunk = kS * kBTile;
constexpr uint32_t kTmemCols = 256;     // 7 x 32 = 224 used
constexpr int kRingA = 3;               // A slices in flight (tile a is released after its products)
constexpr uint32_t kIdesc = idesc_f32acc(1, 128, kNT);

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// B = P^T T_old: B[k][j] = T_old[perm[k]][j]. Block = CB columns of one field; the columns are read
// row by row (coalesced), sliced per column and written K-major (k contiguous). Also clears the
// field's exactness flags (the A slicer, launched after this kernel, sets them).
__global__ void __launch_bounds__(256) k_tt_slice_B(const double* __restrict__ Told, const int* __restrict__ perm_all,
                                                    __nv_bfloat16* __restrict__ Bs, int* __restrict__ eB,
                                                    int* __restrict__ flag, int N, int npad, int MT, int fbase,
                                                    size_t plane, int CB) {
    extern __shared__ double tile[];  // [N][CB + 1]
    int* perm_s = reinterpret_cast<int*>(tile + (size_t)N * (CB + 1));
    const int f = blockIdx.y, j0 = blockIdx.x * CB, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double* T = Told + (size_t)f * N * N;
    if (blockIdx.x == 0 && threadIdx.x < MT) flag[(size_t)(fbase + f) * MT + threadIdx.x] = 0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) perm_s[k] = perm_all[(size_t)f * N + k];
    for (int idx = threadIdx.x; idx < N * CB; idx += blockDim.x) {
        const int r = idx / CB, c = idx - r * CB;
        tile[(size_t)r * (CB + 1) + c] = (j0 + c < N) ? T[(size_t)r * N + j0 + c] : 0.0;
    }
    __syncthreads();
    for (int c = warp; c < CB; c += blockDim.x / 32) {
        const int j = j0 + c;
        if (j >= N) break;
        long long m = 0;
        for (int r = lane; r < N; r += 32) m = max(m, abs_bits(tile[(size_t)r * (CB + 1) + c]));
        const int e = exponent_of_bits(warp_max_bits(m));
        if (lane == 0) eB[(size_t)(fbase + f) * npad + j] = e;
        __nv_bfloat16* dst = Bs + ((size_t)(fbase + f) * npad + j) * npad;
        for (int k = lane; k < npad; k += 32) {
            __nv_bfloat16 q[kS];
            slice7(k < N ? tile[(size_t)perm_s[k] * (CB + 1) + c] : 0.0, e, q);
#pragma unroll
            for (int s = 0; s < kS; ++s) dst[(size_t)s * plane + k] = q[s];
        }
    }
}

// Rows of Rt (upper triangle of the packed QR, column-major) sliced per row and written K-major;
// the exactness bound of every level is checked per row and a failing row flags its tile.
__global__ void __launch_bounds__(256) k_tt_slice_A(const double* __restrict__ QRall, __nv_bfloat16* __restrict__ As,
                                                    int* __restrict__ eA, int* __restrict__ flag, int N, int npad,
                                                    int mpad, int MT, int fbase, size_t plane, int RB) {
    extern __shared__ double tile[];  // [RB][N + 1]
    const int f = blockIdx.y, i0 = blockIdx.x * RB, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double* QR = QRall + (size_t)f * N * N;
    for (int idx = threadIdx.x; idx < RB * N; idx += blockDim.x) {
        const int k = idx / RB, ii = idx - k * RB, i = i0 + ii;
        tile[(size_t)ii * (N + 1) + k] = (i < N && k >= i) ? QR[(size_t)k * N + i] : 0.0;
    }
    __syncthreads();
    for (int ii = warp; ii < RB; ii += blockDim.x / 32) {
        const int i = i0 + ii;
        if (i >= N) break;
        const double* row = tile + (size_t)ii * (N + 1);
        long long m = 0;
        for (int k = lane; k < N; k += 32) m = max(m, abs_bits(row[k]));
        const int e = exponent_of_bits(warp_max_bits(m));
        if (lane == 0) eA[(size_t)(fbase + f) * mpad + i] = e;
        __nv_bfloat16* dst = As + ((size_t)(fbase + f) * mpad + i) * npad;
        int rs[kS] = {0, 0, 0, 0, 0, 0, 0};
        for (int k = lane; k < npad; k += 32) {
            __nv_bfloat16 q[kS];
            slice7(k < N ? row[k] : 0.0, e, q);
#pragma unroll
            for (int s = 0; s < kS; ++s) {
                dst[(size_t)s * plane + k] = q[s];
                rs[s] += (int)fabsf(__bfloat162float(q[s]));
            }
        }
        bool bad = false;
#pragma unroll
        for (int s = 0; s < kS; ++s) rs[s] = warp_sum_int(rs[s]);
#pragma unroll
        for (int lv = 0; lv < kLevels; ++lv) {
            double b = 0.0;
#pragma unroll
            for (int a = 0; a <= lv; ++a) b += (double)rs[a] * (lv - a == 0 ? 128.0 : 64.0);
            bad = bad || b > 16777216.0;
        }
        if (bad && lane == 0) atomicOr(flag + (size_t)(fbase + f) * MT + i / 128, 1);
    }
}

__global__ void __launch_bounds__(kThreads, 2)
    k_tt_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const int* __restrict__ eA, const int* __restrict__ eB, const int* __restrict__ flag,
              const double* __restrict__ QRall, const double* __restrict__ Told, const int* __restrict__ perm_all,
              double* __restrict__ Tnew, int N, int npad, int mpad, int MT, int fbase, int force_fallback,
              unsigned int* __restrict__ err) {
    const int nt = blockIdx.x, mt = blockIdx.y, f = blockIdx.z, j0 = nt * kNT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = npad / 64, kc0 = (mt * 128) / 64, nkc = nk - kc0;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kRingA], bar_empty[kRingA], bar_bfull[2], bar_bempty[2], bar_acc, bar_done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ int eB_sh[kNT];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t bbuf = base, aring = base + 2 * kBChunk;
    double* stage_out = reinterpret_cast<double*>(smem_raw + (bbuf - raw));  // [128][kNT + 1] after the MMAs
    const bool fallback = force_fallback || flag[(size_t)(fbase + f) * MT + mt] != 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kRingA; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bar_bfull[b]), 1);
            mbar_init(smem_u32(&bar_bempty[b]), 1);
        }
        mbar_init(smem_u32(&bar_acc), 1);
        mbar_init(smem_u32(&bar_done), 1);
        abort_sh = 0;
        fence_barrier_init();
    }
    if (threadIdx.x < kNT) eB_sh[threadIdx.x] = j0 + threadIdx.x < N ? eB[(size_t)(fbase + f) * npad + j0 + threadIdx.x] : 0;
    if (warp == 9) {
        tmem_alloc(smem_u32(&tmem_base_sh), kTmemCols);
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (fallback) {
        // Plain FP64 loop for this tile: thread (row r, column half h) accumulates kNT / 2 columns.
        constexpr int HC = kNT / 2;
        if (warp < 8) {
            const int r = threadIdx.x & 127, h = threadIdx.x >> 7, i = mt * 128 + r;
            const double* QR = QRall + (size_t)f * N * N;
            const double* T = Told + (size_t)f * N * N;
            const int* perm = perm_all + (size_t)f * N;
            double acc[HC];
#pragma unroll
            for (int c = 0; c < HC; ++c) acc[c] = 0.0;
            for (int k = mt * 128; k < N; ++k) {
                const double a = (i < N && k >= i) ? QR[(size_t)k * N + i] : 0.0;
                const double* trow = T + (size_t)perm[k] * N + j0 + HC * h;
#pragma unroll
                for (int c = 0; c < HC; ++c)
                    if (j0 + HC * h + c < N) acc[c] = fma(a, trow[c], acc[c]);
            }
            if (i < N)
#pragma unroll
                for (int c = 0; c < HC; ++c)
                    if (j0 + HC * h + c < N) Tnew[((size_t)f * N + i) * N + j0 + HC * h + c] = acc[c];
        }
    } else if (warp == 8) {
        // ---- TMA producer: per K chunk the six B slices, then the six A slices ----
        if (lane == 0) {
            int issued_a = 0, issued_b = 0;
            for (int u = 0; u < nkc && !abort_sh; ++u) {
                const int kc = kc0 + u, bs = u & 1;
                if (u >= 2 && !mbar_wait(smem_u32(&bar_bempty[bs]), ((u >> 1) - 1) & 1, err)) {
                    abort_sh = 1;
                    break;
                }
                const uint32_t bb = smem_u32(&bar_bfull[bs]);
                mbar_expect_tx(bb, kBChunk);
                for (int b = 0; b < kS; ++b)
                    tma_load_3d(bbuf + bs * kBChunk + b * kBTile, &tmB, kc * 64, (fbase + f) * npad + j0, b, bb);
                issued_b = u + 1;
                for (int a = 0; a < kS; ++a) {
                    const int t = u * kS + a, slot = t % kRingA;
                    if (t >= kRingA && !mbar_wait(smem_u32(&bar_empty[slot]), ((t / kRingA) - 1) & 1, err)) {
                        abort_sh = 1;
                        break;
                    }
                    const uint32_t fb = smem_u32(&bar_full[slot]);
                    mbar_expect_tx(fb, kATile);
                    tma_load_3d(aring + slot * kATile, &tmA, kc * 64, (fbase + f) * mpad + mt * 128, a, fb);
                    issued_a = t + 1;
                }
                if (abort_sh) break;
            }
            // teardown: copies in flight (bounded)
            for (int t = issued_a - 1; t >= 0 && t >= issued_a - kRingA; --t)
                mbar_wait(smem_u32(&bar_full[t % kRingA]), (t / kRingA) & 1, err);
            for (int u = issued_b - 1; u >= 0 && u >= issued_b - 2; --u)
                mbar_wait(smem_u32(&bar_bfull[u & 1]), (u >> 1) & 1, err);
        }
    } else if (warp == 9) {
        // ---- MMA issuer: product (a, b) of a K chunk into the accumulator of level a + b ----
        if (lane == 0) {
            bool ok = true;
            uint32_t written = 0;
            for (int u = 0; u < nkc && ok; ++u) {
                const int bs = u & 1;
                if (!mbar_wait(smem_u32(&bar_bfull[bs]), (u >> 1) & 1, err) || abort_sh) {
                    ok = false;
                    break;
                }
                for (int a = 0; a < kS && ok; ++a) {
                    const int t = u * kS + a, slot = t % kRingA;
                    if (!mbar_wait(smem_u32(&bar_full[slot]), (t / kRingA) & 1, err) || abort_sh) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ad = smem_desc_sw128(aring + slot * kATile + ks * 32);
#pragma unroll
                        for (int b = 0; b < kS; ++b) {
                            if (a + b >= kLevels) continue;
                            const int lv = a + b;
                            const uint64_t bd = smem_desc_sw128(bbuf + bs * kBChunk + b * kBTile + ks * 32);
                            mma_bf16(tmem + (uint32_t)(lv * kNT), ad, bd, kIdesc, (written >> lv) & 1u);
                            written |= 1u << lv;
                        }
                    }
                    mma_commit(smem_u32(&bar_empty[slot]));
                }
                if (ok) mma_commit(smem_u32(&bar_bempty[bs]));
            }
            if (ok) mma_commit(smem_u32(&bar_acc));
            else abort_sh = 1;
            mma_commit(smem_u32(&bar_done));
            mbar_wait(smem_u32(&bar_done), 0, err);
        }
    } else {
        // ---- epilogue: warp w drains lanes 32 (w % 4).. (rows) for columns (kNT / 2) (w / 4).. ----
        const int q = warp & 3, h = warp >> 2, r = 32 * q + lane, i = mt * 128 + r;
        const bool bad = !mbar_wait(smem_u32(&bar_acc), 0, err) || abort_sh;
        if (!named_sync_or(1, 256, bad)) {
            tc_fence_after();
            const int ea = i < N ? eA[(size_t)(fbase + f) * mpad + i] : 0;
#pragma unroll
            for (int c0 = 0; c0 < kNT / 2; c0 += 8) {
                uint32_t v[kLevels][8];
                const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((kNT / 2) * h + c0);
#pragma unroll
                for (int lv = 0; lv < kLevels; ++lv) tmem_ld8(tl + (uint32_t)(lv * kNT), v[lv]);
                tmem_ld_wait();
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    // sum_l acc_l 2^(7 (6 - l)) = hi 2^28 + lo with hi (levels 0-2, < 2^39) and lo
                    // (levels 3-6, < 2^46) exact in 64-bit integers and in FP64; one FMA rounds the sum
                    long long hi = (long long)__float2int_rn(__uint_as_float(v[0][c]));
#pragma unroll
                    for (int lv = 1; lv < 3; ++lv) hi = hi * 128 + (long long)__float2int_rn(__uint_as_float(v[lv][c]));
                    long long lo = (long long)__float2int_rn(__uint_as_float(v[3][c]));
#pragma unroll
                    for (int lv = 4; lv < kLevels; ++lv) lo = lo * 128 + (long long)__float2int_rn(__uint_as_float(v[lv][c]));
                    const int col = (kNT / 2) * h + c0 + c;
                    stage_out[r * (kNT + 1) + col] = fma(__ll2double_rn(hi), 268435456.0, __ll2double_rn(lo)) *
                                                     pow2d(ea + eB_sh[col] - 2 * (kW - 1) - kW * (kLevels - 1));
                }
            }
        }
        named_sync(1, 256);
        if (!bad && !abort_sh) {
            // coalesced row-major stores: warp w writes rows w, w + 8, ..., one column per lane
            for (int rr = warp; rr < 128; rr += 8) {
                const int ii = mt * 128 + rr;
                if (ii >= N) break;
                double* dst = Tnew + ((size_t)f * N + ii) * N + j0;
#pragma unroll
                for (int cc = lane; cc < kNT; cc += 32)
                    if (j0 + cc < N) dst[cc] = stage_out[rr * (kNT + 1) + cc];
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 9) tmem_dealloc(tmem, kTmemCols);
}

int rows_per_block(int N) { return N <= 256 ? 32 : (N <= 512 ? 16 : 8); }

}  // namespace

namespace slmc {

size_t tt_slices() { return kS; }

// Buffers are allocated by slmc_init (tt_A, tt_B, tt_eA, tt_eB, tt_flag); zero the padding (never
// written afterwards) and encode the TMA descriptors.
cudaError_t tt_init(slmc_ctx* c) {
    const int N = c->N;
    c->tt_npad = (N + 63) / 64 * 64;
    c->tt_mpad = (N + 127) / 128 * 128;
    const size_t na = (size_t)kS * c->max_fields * c->tt_mpad * c->tt_npad, nb = (size_t)kS * c->max_fields * c->tt_npad * c->tt_npad;
    cudaError_t e = cudaMemset(c->tt_A, 0, na * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMemset(c->tt_B, 0, nb * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMemset(c->tt_flag, 0, (size_t)c->max_fields * (c->tt_mpad / 128) * sizeof(int));
    if (e != cudaSuccess) return e;
    if (!make_map_sw128(&c->tt_mapA, c->tt_A, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, c->tt_npad,
                        (uint64_t)c->max_fields * c->tt_mpad, kS, 128) ||
        !make_map_sw128(&c->tt_mapB, c->tt_B, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, c->tt_npad,
                        (uint64_t)c->max_fields * c->tt_npad, kS, kNT))
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

int t_update_launches(const slmc_ctx* c) { return (c->tt_A && c->tt_path != 1) ? 3 : 1; }

cudaError_t t_update(slmc_ctx* c, int nf, cudaStream_t s) {
    if (!c->tt_A || c->tt_path == 1) return t_update_tiled(c, nf, s);
    const int N = c->N, npad = c->tt_npad, mpad = c->tt_mpad, MT = mpad / 128;
    const size_t pa = (size_t)c->max_fields * mpad * npad, pb = (size_t)c->max_fields * npad * npad;
    __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(c->tt_A);
    __nv_bfloat16* B = reinterpret_cast<__nv_bfloat16*>(c->tt_B);
    const int CB = rows_per_block(N), RB = rows_per_block(N);
    const size_t smB = (size_t)N * (CB + 1) * sizeof(double) + (size_t)N * sizeof(int);
    const size_t smA = (size_t)RB * (N + 1) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_tt_slice_B, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smB);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tt_slice_A, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smA);
    if (e != cudaSuccess) return e;
    k_tt_slice_B<<<dim3((N + CB - 1) / CB, nf), 256, smB, s>>>(c->Ta, c->perm, B, c->tt_eB, c->tt_flag, N, npad, MT,
                                                               c->fbase, pb, CB);
    k_tt_slice_A<<<dim3((N + RB - 1) / RB, nf), 256, smA, s>>>(c->QR, A, c->tt_eA, c->tt_flag, N, npad, mpad, MT,
                                                               c->fbase, pa, RB);
    const size_t smem = 1024 + 2 * (size_t)kBChunk + (size_t)kRingA * kATile;
    e = cudaFuncSetAttribute(k_tt_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tt_gemm<<<dim3(npad / kNT, MT, nf), kThreads, smem, s>>>(c->tt_mapA, c->tt_mapB, c->tt_eA, c->tt_eB, c->tt_flag,
                                                               c->QR, c->Ta, c->perm, c->Tb, N, npad, mpad, MT,
                                                               c->fbase, c->tt_path == 2 ? 1 : 0, c->err);
    e = cudaGetLastError();
    double* t = c->Ta;
    c->Ta = c->Tb;
    c->Tb = t;
    return e;
}

}  // namespace slmc
