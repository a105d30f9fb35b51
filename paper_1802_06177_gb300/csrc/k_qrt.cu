// Blocked Householder QR of the UDT stabilisation with its trailing updates on the tensor cores,
// FP64-accurate.
//
// The pre-pivoted blocked QR (see k_qrb.cu) spends about half of its FP64 issue slots on the
// trailing updates C <- (I - V S^T V^T) C = C - V W', W' = S^T W, W = V^T C, after each panel of BP
// reflectors. Here the panels are factored as before (FP64, one CTA per field, k_qrt_panel), and the
// two products of each trailing update run on the tensor cores in exact fixed-point BF16 slices
// (the same Ozaki-style splitting as the T update): every operand row or column is cut into seven
// 7-bit digits (slice7.cuh) against its own power of two, the products of digit slices a, b with
// a + b <= 6 are summed per level a + b in FP32 accumulators in tensor memory -- exactly, because a
// level's sum of absolute terms stays below 2^24 by construction (at most 36864 per K index, and
// the K range of one accumulator is at most 448) -- and the epilogue combines the levels in two
// 64-bit integers and rounds once to FP64. Each product entry is then the correctly rounded value
// of the sliced operands' product; the slicing (rounding at 2^-48 of each row's / column's largest
// entry) and the dropped levels 7..12 leave an error below 2^-44 K max_k|a_ik| max_k|b_kj| per
// entry: normwise the size of the FP64 loop's own rounding, which is what the backward stability of
// the Householder update needs (errors relative to each column of C, each reflector, each row of
// W').
//
// Per panel t (p = t BP), on the caller's stream:
//   k_qrt_panel<BP>  factor the panel (shared panel_step); write its outputs; slice V twice: per
//                    reflector over the rows (B operand of W^T = C^T V) and per row over the
//                    reflectors (A operand of V W');
//   k_qrt_slice_C    slice the trailing columns of C (rows p..N-1), one exponent per column;
//   k_qrt_gemm1<BP>  W^T = C^T V on the tensor cores (M = trailing columns, N = BP, K = rows), then
//                    W'^T = W^T S and its slices, one exponent per trailing column;
//   k_qrt_gemm2<BP>  C -= V W' on the tensor cores (M = rows, N = 32 trailing columns, K = BP), the
//                    FP64 read-modify-write of C in the epilogue.
// Outputs are those of k_qrb (packed QR, tau, perm, new ln D, sgnU, the panels' S). All waits are
// clock-bounded and set SLMC_EBIT_TIMEOUT; a CTA that gives up drains its copies and frees its
// tensor memory.
#include <algorithm>

#include "qr_panel.cuh"
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

constexpr int kLv = 7;                       // levels a + b = 0..6
constexpr int kQT = 320;                     // GEMM threads: 8 epilogue warps, TMA warp, MMA warp
constexpr uint32_t kTileA = 128 * 128;       // 128 rows x 64 BF16 (one 128-byte swizzle row each)
constexpr int kSegChunks = 7;                // K chunks (64 rows) per accumulator set of W^T = C^T V
constexpr int kMaxN = 2 * kSegChunks * 64;   // 896: two accumulator sets
constexpr int kVRows = 32;                   // rows of the V1 slice buffer per field (BP <= 32)
// W^T = C^T V streams the seven C slices of a K chunk through a ring of three tiles (tile a is
// released once its products with the seven V slices are issued), so two CTAs fit on an SM: one's
// FP64 epilogue then overlaps the other's copies and products.
constexpr int kRing = 3;
// 2^-54: the digits' units 2^(e - 6) per operand and the level weights 2^(-7 level), 2^-42 at level 6
constexpr int kUnitShift = 2 * 6 + 7 * (kLv - 1);

// Level sums (FP32 integers) of one accumulator entry -> hi 2^28 + lo as 64-bit integers.
__device__ __forceinline__ void levels_to_int(const uint32_t (&v)[kLv], long long& hi, long long& lo) {
    hi = (long long)__float2int_rn(__uint_as_float(v[0]));
#pragma unroll
    for (int lv = 1; lv < 3; ++lv) hi = hi * 128 + (long long)__float2int_rn(__uint_as_float(v[lv]));
    lo = (long long)__float2int_rn(__uint_as_float(v[3]));
#pragma unroll
    for (int lv = 4; lv < kLv; ++lv) lo = lo * 128 + (long long)__float2int_rn(__uint_as_float(v[lv]));
}

// Compact-WY triangle S of BP reflectors from their Gram matrix G (row stride ldg) and tau, by the 256
// threads of the 8 epilogue warps (named barrier 1), in blocks: S is the inverse of the upper
// triangular T with T_cc = 1 / tau_c and T_qc = G_qc (q < c), so the four diagonal blocks of BP/4
// columns follow the column recurrence S_cc = tau_c, S[., c] = -tau_c S[., <c] G[<c, c] (one warp
// each), and blocks merge as S12 = -S11 T12 S22 (T12 = G of the two blocks; no division by tau, so a
// trivial reflector, tau = 0, gives its zero column as the recurrence does). The recurrence of one
// warp over all BP columns was a chain of BP dependent steps. tmp holds BP x BP doubles.
template <int BP>
__device__ __forceinline__ void wy_triangle_blocked(const double* G, int ldg, const double* tau, double* S, double* tmp,
                                                    int tid) {
    constexpr int B4 = BP / 4, B2 = BP / 2;
    const int warp = tid >> 5, lane = tid & 31;
    for (int idx = tid; idx < BP * BP; idx += 256) S[idx] = 0.0;
    slmc::tc::named_sync(1, 256);
    if (warp < 4) {  // diagonal block b = warp: rows and columns o .. o + B4 - 1
        const int o = warp * B4;
        for (int c = 0; c < B4; ++c) {
            double v = 0.0;
            if (lane < c) {
                for (int q = lane; q < c; ++q) v = fma(S[(o + lane) * BP + o + q], G[(o + q) * ldg + o + c], v);
                v = -tau[o + c] * v;
            } else if (lane == c) {
                v = tau[o + c];
            }
            if (lane <= c) S[(o + lane) * BP + o + c] = v;
            __syncwarp();
        }
    }
    slmc::tc::named_sync(1, 256);
    {  // two merges of block pairs (2m, 2m + 1) into B2 x B2 triangles: U = T12 S22, then S12 = -S11 U
        const int m = tid / (B4 * B4), e = tid % (B4 * B4), r = e / B4, c = e % B4;
        const int o1 = m * B2, o2 = o1 + B4;
        if (m < 2) {
            double u = 0.0;
            for (int k = 0; k <= c; ++k) u = fma(G[(o1 + r) * ldg + o2 + k], S[(o2 + k) * BP + o2 + c], u);
            tmp[m * B4 * B4 + e] = u;
        }
        slmc::tc::named_sync(1, 256);
        if (m < 2) {
            double v = 0.0;
            for (int k = r; k < B4; ++k) v = fma(S[(o1 + r) * BP + o1 + k], tmp[m * B4 * B4 + k * B4 + c], v);
            S[(o1 + r) * BP + o2 + c] = -v;
        }
        slmc::tc::named_sync(1, 256);
    }
    for (int e = tid; e < B2 * B2; e += 256) {  // the last merge: U = T12 S22 over the two halves
        const int r = e / B2, c = e % B2;
        double u = 0.0;
        for (int k = 0; k <= c; ++k) u = fma(G[r * ldg + B2 + k], S[(B2 + k) * BP + B2 + c], u);
        tmp[e] = u;
    }
    slmc::tc::named_sync(1, 256);
    for (int e = tid; e < B2 * B2; e += 256) {  // S12 = -S11 U
        const int r = e / B2, c = e % B2;
        double v = 0.0;
        for (int k = r; k < B2; ++k) v = fma(S[r * BP + k], tmp[k * B2 + c], v);
        S[r * BP + B2 + c] = -v;
    }
    slmc::tc::named_sync(1, 256);
}

// ---- panel ----------------------------------------------------------------------------------
// 16 warps per field: the panel is a chain of latency-bound column steps (dot products, warp
// reductions, a block barrier each) that leaves the FP64 pipe half idle with 8 warps.
constexpr int kPT = 512;
constexpr int kPW = kPT / 32;

template <int BP>
__global__ void __launch_bounds__(kPT, 2)
    k_qrt_panel(double* __restrict__ Yall, double* __restrict__ lnD_all, double* __restrict__ QRall,
                double* __restrict__ tau_all, int* __restrict__ perm_all, int* __restrict__ sgnU,
                double* __restrict__ Sall, unsigned int* __restrict__ err, int N, int t, double* __restrict__ lnDn_ws,
                int* __restrict__ ntriv_ws, __nv_bfloat16* __restrict__ V1, int* __restrict__ eV1,
                __nv_bfloat16* __restrict__ V2, int* __restrict__ eV2, int kpad, int mpad, size_t plane1,
                size_t plane2, int fbase) {
    constexpr int BPS = BP + 1;
    const int f = blockIdx.x, gf = fbase + f;
    const size_t NN = (size_t)N * N;
    double* __restrict__ Y = Yall + f * NN;
    double* __restrict__ QR = QRall + f * NN;
    extern __shared__ __align__(16) unsigned char smraw[];
    double* Vp = reinterpret_cast<double*>(smraw);
    double* Ssm = Vp + (size_t)N * BPS;
    double* Wsm = Ssm + BP * BP;
    double* s_key = Wsm + kWarps * BP * kCT;  // the layout of QrSmem<BP> (Wsm holds the Gram matrix here)
    double* s_lnd = s_key + N;
    double* s_lnDn = s_lnd + N;
    double* s_g = s_lnDn + N;
    double* s_tau = s_g + N;
    double* s_beta = s_tau + BP;
    int* s_perm = reinterpret_cast<int*>(s_beta + BP);
    __shared__ double s_mx;
    __shared__ int s_ntriv, s_wide;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int p = t * BP, nb = min(BP, N - p), npanels = (N + BP - 1) / BP;

    for (int j = tid; j < N; j += kPT) s_lnd[j] = lnD_all[(size_t)f * N + j];
    if (tid == 0) {
        s_ntriv = 0;
        s_wide = 0;
    }
    __syncthreads();
    if (t == 0) {  // scaled column norms and the pre-pivoting order, as in k_qrb
        if (warp == 0) {
            double mx = -DBL_MAX;
            for (int j = lane; j < N; j += 32) mx = fmax(mx, s_lnd[j]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) s_mx = mx;
        }
        __syncthreads();
        for (int j = warp; j < N; j += kPW) {
            double a = 0.0;
            for (int i = lane; i < N; i += 32) {
                const double y = Y[(size_t)j * N + i];
                a = fma(y, y, a);
            }
            a = slmc::warp_allsum(a);
            if (lane == 0) {
                const double key = a * exp(2.0 * (s_lnd[j] - s_mx));
                s_key[j] = (key >= 0.0) ? key : -1.0;
            }
        }
        __syncthreads();
        for (int j = tid; j < N; j += kPT) {
            // keys are >= +0 or -1: their bit patterns as 64-bit integers order as the values do, and
            // the integer compares leave the FP64 pipe to the factorisation
            const long long kj = __double_as_longlong(s_key[j]);
            int r = 0;
            for (int i = 0; i < N; ++i) {
                const long long ki = __double_as_longlong(s_key[i]);
                r += (ki > kj) || (ki == kj && i < j);
            }
            s_perm[r] = j;
        }
        __syncthreads();
        for (int j = tid; j < N; j += kPT) perm_all[(size_t)f * N + j] = s_perm[j];
    } else {
        for (int j = tid; j < N; j += kPT) s_perm[j] = perm_all[(size_t)f * N + j];
        for (int i = tid; i < p; i += kPT) {
            const double l = lnDn_ws[(size_t)gf * N + i];
            s_lnDn[i] = l;
            s_g[i] = exp(-l);
            if (fabs(l) > 600.0) s_wide = 1;
        }
    }
    for (int k = tid; k < N; k += kPT)
        if (fabs(s_lnd[k]) > 600.0) s_wide = 1;
    __syncthreads();

    // the Gram matrix and S of every panel but the last are formed on the tensor cores (k_qrt_gemm1)
    panel_step<BP, kPT>(Y, QR, tau_all + (size_t)f * N, Sall + (size_t)f * N * BP, Vp, Ssm, Wsm, s_lnd, s_lnDn, s_g, s_tau,
                        s_beta, s_perm, &s_ntriv, &s_wide, N, p, nb, t == npanels - 1);
    __syncthreads();
    if (tid < nb) lnDn_ws[(size_t)gf * N + p + tid] = s_lnDn[p + tid];
    if (tid == 0) {  // reflectors with tau != 0 so far (their parity is the sign of det U)
        const int ntriv = (t == 0 ? 0 : ntriv_ws[gf]) + s_ntriv;
        if (t == npanels - 1) sgnU[f] = (ntriv & 1) ? -1 : 1;
        else ntriv_ws[gf] = ntriv;
    }
    if (t == npanels - 1) {  // every scale is known: publish ln D'
        bool bad = false;
        for (int k = tid; k < N; k += kPT) {
            lnD_all[(size_t)f * N + k] = s_lnDn[k];
            bad |= !isfinite(s_lnDn[k]);
        }
        if (bad) atomicOr(err, SLMC_EBIT_NONFINITE);
        return;
    }
    // V1: reflector m over rows p..N-1 (K-major, K chunks from the one holding row p)
    const int kstart = (p / 64) * 64;
    for (int m = warp; m < BP; m += kPW) {
        long long mx = 0;
        for (int r = p + lane; r < N; r += 32) mx = max(mx, abs_bits(Vp[r * BPS + m]));
        const int e = exponent_of_bits(warp_max_bits(mx));
        if (lane == 0) eV1[(size_t)gf * kVRows + m] = e;
        __nv_bfloat16* dst = V1 + ((size_t)gf * kVRows + m) * kpad;
        for (int k = kstart + lane; k < kpad; k += 32) {
            __nv_bfloat16 q[kS];
            slice7((k >= p && k < N) ? Vp[k * BPS + m] : 0.0, e, q);
#pragma unroll
            for (int s = 0; s < kS; ++s) dst[(size_t)s * plane1 + k] = q[s];
        }
    }
    // V2: row r over the reflectors (K = the BP reflectors, padded to 64 with zeros set at init),
    // rows of the first row tile that holds row p onward
    for (int r = (p / 128) * 128 + warp; r < mpad; r += kPW) {
        const double v = (r >= p && r < N && lane < BP) ? Vp[r * BPS + lane] : 0.0;
        const int e = exponent_of_bits(warp_max_bits(abs_bits(v)));
        if (lane == 0) eV2[(size_t)gf * mpad + r] = e;
        if (lane < BP) {
            __nv_bfloat16 q[kS];
            slice7(v, e, q);
#pragma unroll
            for (int s = 0; s < kS; ++s) V2[(size_t)s * plane2 + ((size_t)gf * mpad + r) * 64 + lane] = q[s];
        }
    }
}

// ---- slices of the trailing columns ---------------------------------------------------------
// Warp w of block x slices trailing column jj = 8 x + w (logical column j0 + jj) over rows p..N-1.
__global__ void __launch_bounds__(256) k_qrt_slice_C(const double* __restrict__ Yall, const int* __restrict__ perm_all,
                                                     __nv_bfloat16* __restrict__ Cs, int* __restrict__ eC, int N,
                                                     int p, int j0, int kpad, int jpad, size_t plane, int fbase) {
    const int f = blockIdx.y, gf = fbase + f, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int jj = blockIdx.x * 8 + warp, j = j0 + jj;
    if (j >= N) return;
    const double* col = Yall + (size_t)f * N * N + (size_t)perm_all[(size_t)f * N + j] * N;
    long long mx = 0;
    for (int r = p + lane; r < N; r += 32) mx = max(mx, abs_bits(col[r]));
    const int e = exponent_of_bits(warp_max_bits(mx));
    if (lane == 0) eC[(size_t)gf * jpad + jj] = e;
    __nv_bfloat16* dst = Cs + ((size_t)gf * jpad + jj) * kpad;
    for (int k = (p / 64) * 64 + lane; k < kpad; k += 32) {
        __nv_bfloat16 q[kS];
        slice7((k >= p && k < N) ? col[k] : 0.0, e, q);
#pragma unroll
        for (int s = 0; s < kS; ++s) dst[(size_t)s * plane + k] = q[s];
    }
}

// ---- [G; W^T] = [V C]^T V, S from G, then W'^T = W^T S and its slices -----------------------
// CTA = the BP reflectors plus 128 - BP trailing columns of one field: each 128-row A tile holds the
// slices of V's columns (rows 0..BP-1, from the reflector slice buffer) above those of the CTA's
// trailing columns of C, so the product's first BP rows are the panel's Gram matrix G = V^T V. The
// epilogue forms the compact-WY triangle S from G (the panel kernel no longer does; CTA 0 writes it
// out for the formation of Q), then W' = S^T W. TMA streams per 64-row K chunk the seven A slices
// through a 3-tile ring and the seven V slices double-buffered; products (a, b), a + b <= 6, go to
// the accumulator of level a + b of the chunk's segment (seven chunks per segment).
template <int BP>
__global__ void __launch_bounds__(kQT, 2)
    k_qrt_gemm1(const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmV,
                const int* __restrict__ eC, const int* __restrict__ eV1, const double* __restrict__ tau_all,
                double* __restrict__ Sall, __nv_bfloat16* __restrict__ Ws, int* __restrict__ eW, int N, int p,
                int n_t, int kpad, int jpad, int wpad, size_t planeW, int fbase, unsigned int* __restrict__ err) {
    constexpr uint32_t kTileB = BP * 128;
    constexpr uint32_t kChunkB = kS * kTileB;
    constexpr uint32_t kIdesc = idesc_f32acc(1, 128, BP);
    constexpr int WS = BP + 1;
    constexpr int kMC = 128 - BP;  // trailing columns per CTA
    const int mt = blockIdx.x, f = blockIdx.y, gf = fbase + f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kc0 = p / 64, nkc = kpad / 64 - kc0;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kRing], bar_empty[kRing], bar_bfull[2], bar_bempty[2], bar_acc, bar_done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ int eV_sh[BP];
    __shared__ double tau_sh[BP];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t bbuf = base, aring = base + 2 * kChunkB;
    // after the MMAs: stage of [G; W] [128][WS], W' [128][WS] and S [BP][BP] over the B buffers and the ring
    double* stW = reinterpret_cast<double*>(smem_raw + (bbuf - raw));
    double* stWp = stW + 128 * WS;
    double* Ssh = stWp + 128 * WS;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kRing; ++s) {
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
    if (threadIdx.x < BP) {
        eV_sh[threadIdx.x] = eV1[(size_t)gf * kVRows + threadIdx.x];
        tau_sh[threadIdx.x] = tau_all[(size_t)f * N + p + threadIdx.x];
    }
    const int nseg = (nkc + kSegChunks - 1) / kSegChunks;
    const uint32_t tcols = nseg == 1 ? 256u : 512u;  // 7 levels x BP columns per accumulator set
    if (warp == 9) {
        tmem_alloc(smem_u32(&tmem_base_sh), tcols);
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 8) {
        if (lane == 0) {
            int issued_a = 0, issued_b = 0;
            for (int u = 0; u < nkc && !abort_sh; ++u) {
                const int kc = kc0 + u, bs = u & 1;
                if (u >= 2 && !mbar_wait(smem_u32(&bar_bempty[bs]), ((u >> 1) - 1) & 1, err)) {
                    abort_sh = 1;
                    break;
                }
                const uint32_t bb = smem_u32(&bar_bfull[bs]);
                mbar_expect_tx(bb, kChunkB);
                for (int b = 0; b < kS; ++b) tma_load_3d(bbuf + bs * kChunkB + b * kTileB, &tmV, kc * 64, gf * kVRows, b, bb);
                issued_b = u + 1;
                for (int a = 0; a < kS; ++a) {
                    const int q = u * kS + a, slot = q % kRing;
                    if (q >= kRing && !mbar_wait(smem_u32(&bar_empty[slot]), ((q / kRing) - 1) & 1, err)) {
                        abort_sh = 1;
                        break;
                    }
                    const uint32_t fb = smem_u32(&bar_full[slot]);
                    mbar_expect_tx(fb, kTileA);  // BP rows of V + kMC rows of C
                    tma_load_3d(aring + slot * kTileA, &tmV, kc * 64, gf * kVRows, a, fb);
                    tma_load_3d(aring + slot * kTileA + kTileB, &tmC, kc * 64, gf * jpad + mt * kMC, a, fb);
                    issued_a = q + 1;
                }
                if (abort_sh) break;
            }
            for (int q = issued_a - 1; q >= 0 && q >= issued_a - kRing; --q)
                mbar_wait(smem_u32(&bar_full[q % kRing]), (q / kRing) & 1, err);
            for (int u = issued_b - 1; u >= 0 && u >= issued_b - 2; --u)
                mbar_wait(smem_u32(&bar_bfull[u & 1]), (u >> 1) & 1, err);
        }
    } else if (warp == 9) {
        if (lane == 0) {
            bool ok = true;
            uint32_t written = 0;
            for (int u = 0; u < nkc && ok; ++u) {
                const int bs = u & 1, seg = u / kSegChunks;
                if (!mbar_wait(smem_u32(&bar_bfull[bs]), (u >> 1) & 1, err) || abort_sh) {
                    ok = false;
                    break;
                }
                for (int a = 0; a < kS && ok; ++a) {
                    const int q = u * kS + a, slot = q % kRing;
                    if (!mbar_wait(smem_u32(&bar_full[slot]), (q / kRing) & 1, err) || abort_sh) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ad = smem_desc_sw128(aring + slot * kTileA + ks * 32);
#pragma unroll
                        for (int b = 0; b < kS; ++b) {
                            if (a + b >= kLv) continue;
                            const int acc = seg * kLv + a + b;
                            const uint64_t bd = smem_desc_sw128(bbuf + bs * kChunkB + b * kTileB + ks * 32);
                            mma_bf16(tmem + (uint32_t)(acc * BP), ad, bd, kIdesc, (written >> acc) & 1u);
                            written |= 1u << acc;
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
        // ---- epilogue: warp w drains rows 32 (w % 4).. for reflectors (w / 4) BP/2 .. ----
        // row r < BP: G[r][.] (exponents of the reflectors); row r >= BP: W of trailing column
        // jj = mt kMC + r - BP
        constexpr int HC = BP / 2;
        const int q4 = warp & 3, h = warp >> 2, r = 32 * q4 + lane, jj = mt * kMC + r - BP;
        const bool bad = !mbar_wait(smem_u32(&bar_acc), 0, err) || abort_sh;
        if (!named_sync_or(1, 256, bad)) {
            tc_fence_after();
            const int er = r < BP ? eV_sh[r] : (jj < n_t ? eC[(size_t)gf * jpad + jj] : 0);
#pragma unroll
            for (int c0 = 0; c0 < HC; c0 += 8) {
                long long hi[8], lo[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) hi[c] = lo[c] = 0;
                for (int sg = 0; sg < nseg; ++sg) {
                    uint32_t v[kLv][8];
                    const uint32_t tl = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(sg * kLv * BP + h * HC + c0);
#pragma unroll
                    for (int lv = 0; lv < kLv; ++lv) tmem_ld8(tl + (uint32_t)(lv * BP), v[lv]);
                    tmem_ld_wait();
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        uint32_t w[kLv];
#pragma unroll
                        for (int lv = 0; lv < kLv; ++lv) w[lv] = v[lv][c];
                        long long a, b;
                        levels_to_int(w, a, b);
                        hi[c] += a;
                        lo[c] += b;
                    }
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int m = h * HC + c0 + c;
                    stW[r * WS + m] = fma(__ll2double_rn(hi[c]), 268435456.0, __ll2double_rn(lo[c])) *
                                      pow2d(er + eV_sh[m] - kUnitShift);
                }
            }
        }
        named_sync(1, 256);
        if (!bad) wy_triangle_blocked<BP>(stW, WS, tau_sh, Ssh, stWp, threadIdx.x);  // S from G = rows 0..BP-1
        if (!bad) {
            if (mt == 0)  // S of the panel for the formation of Q
                for (int idx = threadIdx.x; idx < BP * BP; idx += 256)
                    Sall[((size_t)f * N + p) * BP + idx] = Ssh[idx];
            // W'[m] = sum_{q <= m} S[q][m] W[q]  (S upper triangular); thread (row, half)
            const int rr = BP + (threadIdx.x & 127) % kMC, hh = threadIdx.x >> 7;
            if ((threadIdx.x & 127) < kMC)
                for (int m = hh * HC; m < hh * HC + HC; ++m) {
                    double a = 0.0;
                    for (int q = 0; q <= m; ++q) a = fma(Ssh[q * BP + m], stW[rr * WS + q], a);
                    stWp[rr * WS + m] = a;
                }
        }
        named_sync(1, 256);
        if (!bad) {
            // slices of W', one row (trailing column) per warp at a time, lane = reflector: the row's
            // exponent by a warp reduction, each plane's row one coalesced store
            for (int t = warp; t < kMC; t += 8) {
                const int rr = BP + t, j2 = mt * kMC + t;
                if (j2 >= n_t) break;
                const double v = lane < BP ? stWp[rr * WS + lane] : 0.0;
                const int e = exponent_of_bits(warp_max_bits(abs_bits(v)));
                if (lane == 0) eW[(size_t)gf * wpad + j2] = e;
                if (lane < BP) {
                    __nv_bfloat16 q[kS];
                    slice7(v, e, q);
                    __nv_bfloat16* dst = Ws + ((size_t)gf * wpad + j2) * 64 + lane;
#pragma unroll
                    for (int s = 0; s < kS; ++s) dst[(size_t)s * planeW] = q[s];
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 9) tmem_dealloc(tmem, tcols);
}

// ---- C -= V W' -----------------------------------------------------------------------------
// CTA = 128 rows (row tile p/128 + blockIdx.y) x kNC trailing columns of one field; one K chunk (BP
// reflectors): the seven W' slices resident, the seven V slices streamed through the 3-tile ring.
// 32 columns keep the accumulators at 7 x 32 tensor-memory columns, so two CTAs share an SM.
constexpr int kNC = 32;

template <int BP>
__global__ void __launch_bounds__(kQT, 2)
    k_qrt_gemm2(const __grid_constant__ CUtensorMap tmV, const __grid_constant__ CUtensorMap tmW,
                const int* __restrict__ eV2, const int* __restrict__ eW, const int* __restrict__ perm_all,
                double* __restrict__ Yall, int N, int p, int j0, int n_t, int mpad, int wpad, int fbase,
                unsigned int* __restrict__ err) {
    constexpr uint32_t kTileW = kNC * 128;
    constexpr uint32_t kIdesc = idesc_f32acc(1, 128, kNC);
    const int nt = blockIdx.x, mt = p / 128 + blockIdx.y, f = blockIdx.z, gf = fbase + f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kRing], bar_empty[kRing], bar_bfull, bar_acc, bar_done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ int eW_sh[kNC];
    __shared__ int col_sh[kNC];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t bbuf = base, aring = base + kS * kTileW;

    if (threadIdx.x == 0) {
        for (int q = 0; q < kRing; ++q) {
            mbar_init(smem_u32(&bar_full[q]), 1);
            mbar_init(smem_u32(&bar_empty[q]), 1);
        }
        mbar_init(smem_u32(&bar_bfull), 1);
        mbar_init(smem_u32(&bar_acc), 1);
        mbar_init(smem_u32(&bar_done), 1);
        abort_sh = 0;
        fence_barrier_init();
    }
    if (threadIdx.x < kNC) {
        const int jj = nt * kNC + threadIdx.x;
        eW_sh[threadIdx.x] = jj < n_t ? eW[(size_t)gf * wpad + jj] : 0;
        col_sh[threadIdx.x] = jj < n_t ? perm_all[(size_t)f * N + j0 + jj] : 0;
    }
    if (warp == 9) {
        tmem_alloc(smem_u32(&tmem_base_sh), 256);
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 8) {
        if (lane == 0) {
            const uint32_t bb = smem_u32(&bar_bfull);
            mbar_expect_tx(bb, kS * kTileW);
            for (int b = 0; b < kS; ++b) tma_load_3d(bbuf + b * kTileW, &tmW, 0, gf * wpad + nt * kNC, b, bb);
            int issued = 0;
            for (int a = 0; a < kS; ++a) {
                const int slot = a % kRing;
                if (a >= kRing && !mbar_wait(smem_u32(&bar_empty[slot]), ((a / kRing) - 1) & 1, err)) break;
                const uint32_t fb = smem_u32(&bar_full[slot]);
                mbar_expect_tx(fb, kTileA);
                tma_load_3d(aring + slot * kTileA, &tmV, 0, gf * mpad + mt * 128, a, fb);
                issued = a + 1;
            }
            // (bounded) the copies have landed before the CTA can exit
            mbar_wait(bb, 0, err);
            for (int a = issued - 1; a >= 0 && a >= issued - kRing; --a)
                mbar_wait(smem_u32(&bar_full[a % kRing]), (a / kRing) & 1, err);
        }
    } else if (warp == 9) {
        if (lane == 0) {
            bool ok = mbar_wait(smem_u32(&bar_bfull), 0, err);
            uint32_t written = 0;
            for (int a = 0; a < kS && ok; ++a) {
                const int slot = a % kRing;
                if (!mbar_wait(smem_u32(&bar_full[slot]), (a / kRing) & 1, err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int ks = 0; ks < BP / 16; ++ks) {
                    const uint64_t ad = smem_desc_sw128(aring + slot * kTileA + ks * 32);
#pragma unroll
                    for (int b = 0; b < kS; ++b) {
                        if (a + b >= kLv) continue;
                        const int lv = a + b;
                        const uint64_t bd = smem_desc_sw128(bbuf + b * kTileW + ks * 32);
                        mma_bf16(tmem + (uint32_t)(lv * kNC), ad, bd, kIdesc, (written >> lv) & 1u);
                        written |= 1u << lv;
                    }
                }
                mma_commit(smem_u32(&bar_empty[slot]));
            }
            if (ok) mma_commit(smem_u32(&bar_acc));
            else abort_sh = 1;
            mma_commit(smem_u32(&bar_done));
            mbar_wait(smem_u32(&bar_done), 0, err);
        }
    } else {
        // ---- epilogue: warp w: rows 32 (w % 4).. of the tile, columns 16 (w / 4)..; C -= V W' ----
        constexpr int HC = kNC / 2;
        const int q4 = warp & 3, h = warp >> 2, r = mt * 128 + 32 * q4 + lane;
        const bool bad = !mbar_wait(smem_u32(&bar_acc), 0, err) || abort_sh;
        if (!named_sync_or(1, 256, bad)) {
            tc_fence_after();
            const bool row_ok = r >= p && r < N;
            const int ev = row_ok ? eV2[(size_t)gf * mpad + r] : 0;
            double* Yf = Yall + (size_t)f * N * N;
#pragma unroll
            for (int c0 = 0; c0 < HC; c0 += 8) {
                uint32_t v[kLv][8];
                const uint32_t tl = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(HC * h + c0);
#pragma unroll
                for (int lv = 0; lv < kLv; ++lv) tmem_ld8(tl + (uint32_t)(lv * kNC), v[lv]);
                tmem_ld_wait();
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int cc = HC * h + c0 + c, jj = nt * kNC + cc;
                    if (!row_ok || jj >= n_t) continue;
                    uint32_t w[kLv];
#pragma unroll
                    for (int lv = 0; lv < kLv; ++lv) w[lv] = v[lv][c];
                    long long hi, lo;
                    levels_to_int(w, hi, lo);
                    const double t = fma(__ll2double_rn(hi), 268435456.0, __ll2double_rn(lo)) *
                                     pow2d(ev + eW_sh[cc] - kUnitShift);
                    double* y = Yf + (size_t)col_sh[cc] * N + r;
                    *y = *y - t;
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 9) tmem_dealloc(tmem, 256);
}

size_t gemm1_smem(int BP) { return 1024 + 2 * (size_t)kS * BP * 128 + (size_t)kRing * kTileA; }
size_t gemm2_smem() { return 1024 + (size_t)kS * kNC * 128 + (size_t)kRing * kTileA; }

struct QrtArgs {
    int N, kpad, mpad, wpad, jpad;
    size_t plane1, plane2, planeC, planeW;
    __nv_bfloat16 *V1, *V2, *Cs, *Ws;
};

QrtArgs qrt_args(const slmc_ctx* c) {
    QrtArgs a;
    a.N = c->N;
    a.kpad = c->qt_kpad;
    a.mpad = c->qt_mpad;
    a.wpad = c->qt_wpad;
    a.jpad = c->qt_mpad;
    const size_t F = c->max_fields;
    a.plane1 = F * kVRows * a.kpad;
    a.plane2 = F * a.mpad * 64;
    a.planeC = F * a.jpad * a.kpad;
    a.planeW = F * a.wpad * 64;
    a.V1 = reinterpret_cast<__nv_bfloat16*>(c->qt_V1);
    a.V2 = reinterpret_cast<__nv_bfloat16*>(c->qt_V2);
    a.Cs = reinterpret_cast<__nv_bfloat16*>(c->qt_C);
    a.Ws = reinterpret_cast<__nv_bfloat16*>(c->qt_W);
    return a;
}

template <int BP>
cudaError_t launch_panel(slmc_ctx* c, int nf, int t, cudaStream_t s) {
    const QrtArgs a = qrt_args(c);
    const size_t smP = QrSmem<BP>::bytes(a.N);
    cudaError_t e = cudaFuncSetAttribute(k_qrt_panel<BP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smP);
    if (e != cudaSuccess) return e;
    k_qrt_panel<BP><<<nf, kPT, smP, s>>>(c->Y, c->lnD, c->QR, c->tau, c->perm, c->sgnU, c->Sws, c->err, a.N, t,
                                              c->qt_lnDn, c->qt_ntriv, a.V1, c->qt_eV1, a.V2, c->qt_eV2, a.kpad,
                                              a.mpad, a.plane1, a.plane2, c->fbase);
    return cudaGetLastError();
}

// Trailing update of panel t (t < last panel): slices of C, W'^T = (C^T V) S, C -= V W'.
template <int BP>
cudaError_t launch_trailing(slmc_ctx* c, int nf, int t, cudaStream_t s) {
    const QrtArgs a = qrt_args(c);
    const size_t sm1 = gemm1_smem(BP), sm2 = gemm2_smem();
    cudaError_t e = cudaFuncSetAttribute(k_qrt_gemm1<BP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_qrt_gemm2<BP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
    if (e != cudaSuccess) return e;
    const CUtensorMap& mapV1 = BP == 32 ? c->qt_mapV1_32 : c->qt_mapV1_16;
    const int N = a.N, p = t * BP, j0 = p + BP, n_t = N - j0;
    k_qrt_slice_C<<<dim3((n_t + 7) / 8, nf), 256, 0, s>>>(c->Y, c->perm, a.Cs, c->qt_eC, N, p, j0, a.kpad, a.jpad,
                                                          a.planeC, c->fbase);
    const CUtensorMap& mapC = BP == 32 ? c->qt_mapC96 : c->qt_mapC112;
    k_qrt_gemm1<BP><<<dim3((n_t + 127 - BP) / (128 - BP), nf), kQT, sm1, s>>>(
        mapC, mapV1, c->qt_eC, c->qt_eV1, c->tau, c->Sws, a.Ws, c->qt_eW, N, p, n_t, a.kpad, a.jpad, a.wpad, a.planeW,
        c->fbase, c->err);
    k_qrt_gemm2<BP><<<dim3((n_t + kNC - 1) / kNC, a.mpad / 128 - p / 128, nf), kQT, sm2, s>>>(
        c->qt_mapV2, c->qt_mapW, c->qt_eV2, c->qt_eW, c->perm, c->Y, N, p, j0, n_t, a.mpad, a.wpad, c->fbase, c->err);
    return cudaGetLastError();
}

}  // namespace

namespace slmc {

bool qrt_supported(int N) { return N >= 2 && N <= kMaxN; }

// Sizes of the slice buffers (BF16 elements) and exponent arrays of a context with F fields.
void qrt_sizes(int N, int F, size_t* bf16_elems, size_t* int_elems) {
    const size_t kpad = (N + 63) / 64 * 64, mpad = (N + 127) / 128 * 128, wpad = kpad;
    *bf16_elems = (size_t)kS * F * (mpad * kpad + kVRows * kpad + mpad * 64 + wpad * 64);
    *int_elems = (size_t)F * (mpad + kVRows + mpad + wpad + 1);
}

// Carves the buffers allocated by slmc_init, zeroes them (the padding is never written again) and
// encodes the TMA descriptors.
cudaError_t qrt_init(slmc_ctx* c, void* bf16_base, int* int_base) {
    const int N = c->N;
    const size_t F = c->max_fields;
    c->qt_kpad = (N + 63) / 64 * 64;
    c->qt_mpad = (N + 127) / 128 * 128;
    c->qt_wpad = c->qt_kpad;
    const size_t kpad = c->qt_kpad, mpad = c->qt_mpad, wpad = c->qt_wpad;
    __nv_bfloat16* b = reinterpret_cast<__nv_bfloat16*>(bf16_base);
    c->qt_C = b;
    b += (size_t)kS * F * mpad * kpad;
    c->qt_V1 = b;
    b += (size_t)kS * F * kVRows * kpad;
    c->qt_V2 = b;
    b += (size_t)kS * F * mpad * 64;
    c->qt_W = b;
    b += (size_t)kS * F * wpad * 64;
    c->qt_eC = int_base;
    c->qt_eV1 = c->qt_eC + F * mpad;
    c->qt_eV2 = c->qt_eV1 + F * kVRows;
    c->qt_eW = c->qt_eV2 + F * mpad;
    c->qt_ntriv = c->qt_eW + F * wpad;
    size_t nb16 = 0, nint = 0;
    qrt_sizes(N, (int)F, &nb16, &nint);
    cudaError_t e = cudaMemset(bf16_base, 0, nb16 * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMemset(int_base, 0, nint * sizeof(int));
    if (e != cudaSuccess) return e;
    if (!make_map_sw128(&c->qt_mapC96, c->qt_C, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, kpad, F * mpad, kS, 96) ||
        !make_map_sw128(&c->qt_mapC112, c->qt_C, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, kpad, F * mpad, kS, 112) ||
        !make_map_sw128(&c->qt_mapV1_32, c->qt_V1, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, kpad, F * kVRows, kS, 32) ||
        !make_map_sw128(&c->qt_mapV1_16, c->qt_V1, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, kpad, F * kVRows, kS, 16) ||
        !make_map_sw128(&c->qt_mapV2, c->qt_V2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 64, F * mpad, kS, 128) ||
        !make_map_sw128(&c->qt_mapW, c->qt_W, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 64, F * wpad, kS, kNC))
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

bool qrt_active(const slmc_ctx* c) { return c->qt_C && c->qr_path == 0 && qrt_supported(c->N); }

int qrt_panels(const slmc_ctx* c) {
    const int BP = qr_panel_width(c);
    return (c->N + BP - 1) / BP;
}

cudaError_t qrt_panel(slmc_ctx* c, int nf, int t, cudaStream_t s) {
    return qr_panel_width(c) == 32 ? launch_panel<32>(c, nf, t, s) : launch_panel<16>(c, nf, t, s);
}

cudaError_t qrt_trailing(slmc_ctx* c, int nf, int t, cudaStream_t s) {
    return qr_panel_width(c) == 32 ? launch_trailing<32>(c, nf, t, s) : launch_trailing<16>(c, nf, t, s);
}

}  // namespace slmc
