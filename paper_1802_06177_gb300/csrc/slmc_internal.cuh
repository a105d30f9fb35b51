// Internal declarations shared by the libslmc translation units (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/slmc.h"

// Device-side sticky error bits (ctx->err).
#define SLMC_EBIT_NONFINITE 1u
#define SLMC_EBIT_SINGULAR 2u
#define SLMC_EBIT_TIMEOUT 4u

#define SLMC_MAX_N 1024

namespace slmc {
constexpr int kKronMaxLine = 32;             // longest lattice side of the circulant factors
constexpr int kKronTab = 2 * kKronMaxLine;   // doubles per stored factor
}  // namespace slmc

struct slmc_ctx {
    slmc_params p;
    int N, L, max_fields, device;
    // exp(-dtau K), built on the device from the plane-wave eigenbasis of K.
    double* E64;
    double* Einv64;  // exp(+dtau K), for carrying G between slices in the DQMC updates
    // One-dimensional circulant factors of exp(-+dtau K) = e^{-+dtau mu} E_x kron E_y (site
    // i = ix + Lx iy), each stored twice over: [E_x | E_x^-1 | E_y | E_y^-1], kKronTab
    // doubles apiece. Null when a lattice side exceeds kKronMaxLine (dense products then).
    double* kron;
    double* dq_stack;     // DQMC: [groups][max_fields] (U | T | lnD) of the transposed left products
    int dq_groups;        // groups the stack holds
    int dense_slices;  // 1: FP64 slice products by the dense exp(-dtau K) even where kron exists
    float* F32;      // F = E - I rounded to FP32 (reduced-precision slices use Y + F Y)
    int* lo_kidx;    // FP32 modes: [S][N] column of the S-th stencil entry of row i, then sel[S]
    float* lo_val;   // [S] FP32 rounding residual of F on the S largest-|F| displacements
    int lo_S;        // stencil size min(kLoStencil, N)
    float* sc32;     // [max_fields][L][N] slice scales exp(-dtau lambda x), FP64-computed, rounded to FP32
    // Per-field workspace, [max_fields][N][N] column-major unless stated.
    double* Y;       // slice-group product; reused for M in the final step
    double* QR;      // packed pivoted-QR output; reused for G in the cumulative update
    double* U;       // orthogonal factor
    float* U32;      // FP32 orthogonal factor feeding reduced-precision slice groups (mixed modes)
    double* Ta;      // T factor (ping), row-major
    double* Tb;      // T factor (pong), row-major
    double* lnD;     // [max_fields][N] ln of the D scales
    double* tau;     // [max_fields][N] Householder coefficients
    int* perm;       // [max_fields][N] column permutation of the last QR
    int* piv;        // [max_fields][N] LU row pivots
    int* sgnU;       // [max_fields] det(U) = +-1
    double* Sws;     // [max_fields][N][32] WY triangles of the blocked QR panels
    // Chain workspace.
    double* x_old;   // [max_fields][N][L]
    double* scal;    // [max_fields][8] scratch scalars per chain
    int* iscal;      // [max_fields][4] scratch ints per chain
    // Regression workspace.
    double* feat;    // [max_fields][8]
    double* fitR;    // [64] Givens-QR state of the regression
    unsigned int* err;
    unsigned long long* dctr;  // device-side cumulative-update counter (Philox stream position)
    int nwolff;                        // Wolff cluster updates between the half-sweeps of a sweep
    unsigned long long* wolff_sites;   // device total of reflected columns
    int tune_qr_panel;          // 0: by N; else 16 or 32 (blocked QR panel width)
    int tune_slice_cols;
    int tune_slice_groups;
    int tune_qr_cluster;    // CTAs per field of the QR / formation of Q (0 = by field count)
    int num_sms;            // multiprocessors of the device
    // Exact sliced tensor-core slice path (SLMC_PREC_BF16X9): fixed-point BF16 slices of F
    // [4][128 MT][tcx_npad], their row exponents and the TMA descriptor of the slices.
    void* tcx_F;
    int* tcx_eF;
    int tcx_npad;
    CUtensorMap tcx_mapF;
    // T update on the tensor cores (k_tupd_tc.cu): 7-bit BF16 slices of Rt [6][fields * tt_mpad][tt_npad]
    // and of P^T T [6][fields * tt_npad][tt_npad] (K-major), their row / column exponents, one
    // exactness flag per field and 128-row tile, and the TMA descriptors. tt_path: 0 tensor cores,
    // 1 the FP64 tiled kernel, 2 the tensor kernel with every tile on its FP64 fallback (tests).
    void* tt_A;
    void* tt_B;
    int* tt_eA;
    int* tt_eB;
    int* tt_flag;
    int tt_mpad, tt_npad, tt_path;
    CUtensorMap tt_mapA, tt_mapB;
    // Blocked QR with its trailing updates on the tensor cores (k_qrt.cu): one allocation (qt_buf) of
    // BF16 slices of the trailing columns C [7][fields * qt_mpad][qt_kpad], of the panel reflectors
    // for W = V^T C [7][fields * 32][qt_kpad] and for V W' [7][fields * qt_mpad][64], of W'
    // [7][fields * qt_wpad][64]; one of int exponents (qt_ibuf) and a [fields][N] array of the
    // panels' new scales. qr_path: 0 tensor-core trailing updates, 1 the one-kernel FP64 QR.
    void* qt_buf;
    int* qt_ibuf;
    void* qt_C;
    void* qt_V1;
    void* qt_V2;
    void* qt_W;
    int* qt_eC;
    int* qt_eV1;
    int* qt_eV2;
    int* qt_eW;
    int* qt_ntriv;
    double* qt_lnDn;
    int qt_kpad, qt_mpad, qt_wpad, qr_path;
    CUtensorMap qt_mapC96, qt_mapC112, qt_mapV1_16, qt_mapV1_32, qt_mapV2, qt_mapW;
    int fbase;  // first field of this context's workspace within the owner's (views of sub-batches)
    // Split-TF32 slice path (SLMC_PREC_TF32X3): operand pieces of F and of the running slice
    // product (ping/pong), FP32 copies of it, and their TMA descriptors.
    int tc_npad, tc_nt;
    void* tc_F;         // [pieces][Npad][Npad]
    void* tc_p[2];      // [pieces][max_fields * N][Npad]
    float* tc_y32[2];   // [max_fields][N][N]
    CUtensorMap tc_mapF;
    CUtensorMap tc_mapP[2];
    // Sub-batches: a large logdet batch is split over nsub forked streams so that the
    // kernels of one sub-batch fill the tails of the other's. A view is a shallow copy of the
    // context with the per-field workspace pointers offset; parent points to the owner.
    static constexpr int kMaxSub = 4;
    int nsub;       // sub-batches used for large batches (1 = no split)
    int nsub_avail; // forked streams created at init (0 or kMaxSub)
    cudaStream_t sub_stream[kMaxSub];
    cudaStream_t sub_stream_prio[kMaxSub];  // same, with descending scheduling priorities
    int sub_prio;                           // 1: sub-batches use the prioritised streams
    cudaEvent_t sub_fork, sub_join[kMaxSub];
    slmc_ctx* parent;
    // Launch accounting and optional per-class event timing (host side).
    long long launches;
    bool prof_on;
    std::vector<cudaEvent_t> ev_pool;            // free events
    std::vector<int> ev_cls;                      // class of each recorded pair
    std::vector<cudaEvent_t> ev_rec;             // recorded begin/end pairs
    std::vector<int> ev_units;                    // fields processed by each recorded call
    cudaEvent_t prof_base;                        // time origin of the recorded intervals
    int cur_units;                                // fields of the calls being enqueued
    double prof_ms[SLMC_PROF_NCLASS];
    long long prof_calls[SLMC_PROF_NCLASS];
    double prof_busy[SLMC_PROF_NCLASS];           // union of the class's call intervals (ms)
    long long prof_units[SLMC_PROF_NCLASS];
};

namespace slmc {

// ---- launch helpers ---------------------------------------------------------------
// Stencil size of the FP32 rounding residual of F in the FP32 slice products.
constexpr int kLoStencil = 32;

inline int rows_per_lane_class(int N) {
    const int r = (N + 31) / 32;
    if (r <= 1) return 1;
    if (r <= 2) return 2;
    if (r <= 4) return 4;
    if (r <= 5) return 5;
    if (r <= 8) return 8;
    if (r <= 12) return 12;
    if (r <= 18) return 18;
    return 32;
}

// ---- Philox-4x32-10 (Salmon et al., SC'11), written from the published definition ----
// One in-place circulant line transform of a strided vector v[m] = g[base + m stride],
// m < Ld: out[d] = sum_m tab[(d - m) mod Ld] v[m] (kLeft: a circulant applied from the left)
// or sum_m v[m] tab[(m - d) mod Ld] (from the right), with optional input scales
// in_sc[m in_st] and output scales out_sc[d out_st] * out_mul. tab holds the factor twice
// over so that the index needs no modulo. The outputs stay in registers until the whole line
// has been read.
template <int LMAX, bool kLeft>
__device__ __forceinline__ void circ_line(double* g, int base, int stride, int Ld, const double* __restrict__ tab,
                                          const double* in_sc, int in_st, const double* out_sc, int out_st,
                                          double out_mul) {
    double acc[LMAX];
#pragma unroll
    for (int d = 0; d < LMAX; ++d) acc[d] = 0.0;
#pragma unroll 2
    for (int m = 0; m < Ld; ++m) {
        const double v = in_sc ? g[base + m * stride] * in_sc[m * in_st] : g[base + m * stride];
#pragma unroll
        for (int d = 0; d < LMAX; ++d)
            if (d < Ld) acc[d] = fma(v, tab[kLeft ? d - m + Ld : m - d + Ld], acc[d]);
    }
#pragma unroll
    for (int d = 0; d < LMAX; ++d)
        if (d < Ld) g[base + d * stride] = out_sc ? acc[d] * (out_sc[d * out_st] * out_mul) : acc[d];
}

struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    }
    return c;
}

// 53-bit uniform double in [0, 1) from two words (top 27 bits of hi, top 26 of lo).
__device__ __forceinline__ double uniform53(uint32_t hi, uint32_t lo) {
    return ((double)(hi >> 5) * 67108864.0 + (double)(lo >> 6)) * (1.0 / 9007199254740992.0);
}

// ---- warp reductions ----------------------------------------------------------------
__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace slmc

// ---- kernel launchers (defined in the .cu files) ---------------------------------------
namespace slmc {
cudaError_t build_hopping_exp(slmc_ctx* c, cudaStream_t s);
cudaError_t slice_group(slmc_ctx* c, const double* x, int nf, int l0, int nsl, cudaStream_t s);
cudaError_t tc_slice_group(slmc_ctx* c, const double* x, int nf, int l0, int nsl, cudaStream_t s);
cudaError_t tc_init(slmc_ctx* c, cudaStream_t s);
void tcx_geometry(int N, int* mt, int* nt, int* npad);
size_t tcx_F_bytes(int N);
cudaError_t tcx_init(slmc_ctx* c, cudaStream_t s);
cudaError_t tcx_slice_group(slmc_ctx* c, int nf, int l0, int nsl, cudaStream_t s);
cudaError_t slice_scales(slmc_ctx* c, const double* x, int nf, cudaStream_t s);
void tc_geometry(int N, int* npad, int* nt, size_t* piece_bytes, int* npieces);
int tc_launches(int nsl);
cudaError_t t_update_tiled(slmc_ctx* c, int nf, cudaStream_t s);
// T <- Rt P^T T by the context's path (tensor cores where set up, else t_update_tiled), and the
// number of kernels that enqueues.
cudaError_t t_update(slmc_ctx* c, int nf, cudaStream_t s);
int t_update_launches(const slmc_ctx* c);
size_t tt_slices();  // BF16 slices per operand of the tensor-core T update
// QR with tensor-core trailing updates (k_qrt.cu)
bool qrt_supported(int N);
void qrt_sizes(int N, int F, size_t* bf16_elems, size_t* int_elems);
cudaError_t qrt_init(slmc_ctx* c, void* bf16_base, int* int_base);
bool qrt_active(const slmc_ctx* c);
int qrt_panels(const slmc_ctx* c);
cudaError_t qrt_panel(slmc_ctx* c, int nf, int t, cudaStream_t s);     // factor panel t (1 launch)
cudaError_t qrt_trailing(slmc_ctx* c, int nf, int t, cudaStream_t s);  // its trailing update (3 launches)
cudaError_t tt_init(slmc_ctx* c);
cudaError_t qr_blocked(slmc_ctx* c, int nf, cudaStream_t s);
cudaError_t form_q_blocked(slmc_ctx* c, int nf, bool fp32, cudaStream_t s);
int qr_panel_width(const slmc_ctx* c);
cudaError_t qr_pivoted(slmc_ctx* c, int nf, cudaStream_t s);
cudaError_t form_q(slmc_ctx* c, int nf, cudaStream_t s);
cudaError_t set_identity(slmc_ctx* c, int nf, cudaStream_t s);
cudaError_t u_to_f32(slmc_ctx* c, int nf, cudaStream_t s);
cudaError_t final_logdet(slmc_ctx* c, int nf, double* lndet, int* sign, cudaStream_t s);
// LU of the matrix already in c->Y (the step of final_logdet after assembling M)
cudaError_t final_lu(slmc_ctx* c, int nf, double* lndet, int* sign, cudaStream_t s);
cudaError_t final_greens(slmc_ctx* c, int nf, double* G, cudaStream_t s);
cudaError_t bose_log_weight(slmc_ctx* c, const double* x, int nf, const double* lndet, double* lnw,
                            cudaStream_t s);
cudaError_t eff_features(slmc_ctx* c, const double* x, int nf, const double* J, double* F, int ldF,
                         double* lnw_eff, cudaStream_t s);
cudaError_t eff_half_sweep(slmc_ctx* c, double* x, int nf, int chain0, const double* J, uint64_t sweep,
                           int colour, const int* colour_per_chain, int colour_xor, long long* n_acc,
                           cudaStream_t s, const unsigned long long* dctr = nullptr, int nsweeps = 0);
cudaError_t eff_wolff(slmc_ctx* c, double* x, int nf, int chain0, const double* J, uint64_t sweep, int k,
                      cudaStream_t s, const unsigned long long* dctr = nullptr, int nsweeps = 0);
cudaError_t slice_group_kron(slmc_ctx* c, const double* x, int nf, int l0, int nsl, bool transposed, cudaStream_t s);
// G(g0) = [I + B(g0,0) B(L,g0)]^-1 into G (row-major) from the running product in (U, lnD, Ta)
// and the transposed left product (Ul column-major, lnDl, Tl row-major); uses Y, Tb, Sws, piv.
cudaError_t dqmc_combine(slmc_ctx* c, const double* Ul, const double* lnDl, const double* Tl, int nf, double* G,
                         double* lndet_scratch, int* sign_scratch, cudaStream_t s);
bool dqmc_ok(const slmc_ctx* c);  // L >= 2 and both lattice sides <= 32
cudaError_t dqmc_slices(slmc_ctx* c, double* x, double* G, int nf, int chain0, int l0, int nsl, uint64_t sweep,
                        long long* n_acc, cudaStream_t s);
cudaError_t dqmc_block_propose(slmc_ctx* c, double* x, int nf, int chain0, uint64_t sweep, int k, double* u,
                               cudaStream_t s);
cudaError_t update_draws(slmc_ctx* c, int nf, int chain0, uint64_t u_off, int* first_colour, double* u_acc,
                         cudaStream_t s);
cudaError_t counter_op(slmc_ctx* c, uint64_t v, bool add, cudaStream_t s);
cudaError_t accept_update(slmc_ctx* c, int nf, double* x, const double* x_old, const double* lnw_new,
                          const double* lnweff_old, const double* lnweff_new, const double* u_acc,
                          double* lnw, int* accepted, long long* n_acc, cudaStream_t s);
cudaError_t cdw_measure(slmc_ctx* c, const double* G, int nf, double* S, const int* only_if,
                        double* obs, cudaStream_t s);
cudaError_t fit_begin(slmc_ctx* c, double* R, cudaStream_t s);
cudaError_t fit_accumulate(slmc_ctx* c, double* R, const double* feat, const double* lnw, int nconf,
                           cudaStream_t s);
cudaError_t fit_merge(slmc_ctx* c, const double* states, int nparts, cudaStream_t s);
cudaError_t fit_finish(slmc_ctx* c, int nconf, double* J_out, double* resid, cudaStream_t s);
int validate_params(const slmc_params* p);
int logdet_fields(slmc_ctx* c, const double* x, int nf, double* lndet, int* sign, cudaStream_t s);

// Phases of one cumulative update (slmc_cumulative_update runs all three, update by update).
constexpr int kPhasePre = 1, kPhaseSweeps = 2, kPhasePost = 4, kPhaseAll = 7;
int cumulative_phases(slmc_ctx* c, double* x, int n, const double* J, int nsweeps, int u0, int u1, int phases,
                      double* lnw, double* s_cdw, long long* n_acc, long long* n_sweep_acc, double* obs,
                      cudaStream_t s);
const int* first_colours(slmc_ctx* c);

// Persistent E_eff sweep queue over the chains of several lattice classes. One lattice class:
struct QueueClass {
    double* x;                           // chains [nchains][N][L]
    const double* J;                     // couplings of E_eff (6)
    const int* first_colour;             // per chain: colour of the first half-sweep of this update
    unsigned long long* n_acc;           // per chain accepted site moves, or null
    unsigned long long* wolff_sites;     // class total of flipped sites, or null
    const unsigned long long* dctr;      // device update counter of the class
    unsigned int* err;                   // error word of the class's context
    int Lx, Ly, L, nsweeps, nwolff;
    int done0;                           // index of chain 0's completion counter
    double dtau, a2, delta;
    uint32_t key0, key1;
};
// An item of the queue (int4): x = class << 24 | chain, y = sweep << 8 | kind << 7 | (colour step
// h or Wolff index k), z = slab of kQueueSlab sites of the half-sweep, w = number of the chain's
// earlier items of this update that must be complete before it starts.
constexpr int kQueueSlab = 1024;
constexpr int kQueueWolff = 1;
int sweep_queue_grid();  // CTAs of the persistent launch on the current device
cudaError_t sweep_queue(const QueueClass* classes, int ncls, const int4* items, int nitems, unsigned int* done,
                        unsigned int* ctl, int max_N, uint32_t u, long long wait_cycles, int grid, cudaStream_t s);
}  // namespace slmc
