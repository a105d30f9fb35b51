/*
 * slmc.h -- C ABI of libslmc, the GB300 (sm_103a) hot path of symmetry-enforced
 * self-learning Monte Carlo for the 2D Holstein model (arXiv:1802.06177).
 *
 * What the library computes (paper passages in brackets):
 *   - ln|det(I + B_L ... B_1)|, its sign and the equal-time Green's function
 *     G = (I + B_L ... B_1)^-1 for phonon fields x[N, L], with
 *     B_l = diag(exp(-dtau lambda x[:, l])) exp(-dtau K)      [Suppl. Eq. (S2), (S3)];
 *   - the full log-weight ln w(x) = 2 ln|det| + dtau lambda sum x - dtau S_Bose
 *                                                              [Sec. "Model", Eq. (S2)];
 *   - the symmetric effective model E_eff, its features and local Metropolis sweeps
 *                                                              [Eq. (4) / (S7)];
 *   - the cumulative update with exact acceptance              [Eq. (6)];
 *   - the multi-linear regression of E_eff on ln w             [Eq. (5)];
 *   - the CDW structure factor S(pi, pi) from G                [Sec. "Results"].
 *
 * Conventions shared by every entry point
 *   - All array arguments are DEVICE pointers owned by the caller (for example the
 *     data pointers of torch tensors); the library never frees or retains them. The
 *     library owns only the context and the workspace it allocates in slmc_init.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*, NULL = legacy default
 *     stream); no call synchronises the host, so outputs are valid once the stream has
 *     reached that point. A context may be used by one stream at a time.
 *   - Site index i = ix + Lx * iy on the periodic Lx x Ly square lattice, N = Lx * Ly.
 *     Phonon fields are row-major double x[n][N][L] (x[f*N*L + i*L + l]); column l
 *     (0-based) belongs to slice matrix B_{l+1}. Matrices returned to the caller (G) are
 *     row-major double [n][N][N].
 *   - The coupling is the particle-hole symmetric lambda * x_i * (n_i - 1); the paper's
 *     field X is x shifted by its mirror axis alpha = -g/Omega^2, and a = lambda/omega0^2
 *     is the distance of the double-well minima from that axis.
 *   - Effective-model couplings are a device array J[6] = {E0, J_k, J_p, J_p', J_nn,
 *     J_nn'} with ln w_eff(x) = -dtau (E0 + J_k F_k + J_p F_p + J_p' F_p' + J_nn F_nn
 *     + J_nn' F_nn').
 *   - Every call returns a status code. Argument errors are detected on the host before
 *     anything is enqueued. Errors that only the GPU can see (non-finite input or result,
 *     a singular matrix) set a sticky flag in the context and make the affected outputs
 *     NaN (sign 0); slmc_get_error synchronises the stream and reports them.
 */
#ifndef SLMC_H
#define SLMC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SLMC_API __attribute__((visibility("default")))
#else
#define SLMC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SLMC_OK 0
#define SLMC_ERR_ARG 1          /* bad argument (NULL pointer, size out of range) */
#define SLMC_ERR_NONFINITE 2    /* NaN/Inf in an input field or a result */
#define SLMC_ERR_CUDA 3         /* a CUDA runtime call failed */
#define SLMC_ERR_TIMEOUT 4      /* a bounded device-side wait gave up */
#define SLMC_ERR_UNSUPPORTED 5  /* valid but unsupported shape (odd side for checkerboard, N > 1024) */
#define SLMC_ERR_NOMEM 6        /* workspace allocation failed in slmc_init */
#define SLMC_ERR_SINGULAR 7     /* exactly singular matrix met in the final LU */

/* Arithmetic of the slice products B_l ... B_{l+n_s-1} U between two stabilisations.
 * The pivoted QR, the D scales, the final LU / log-det / G and every Metropolis
 * log-ratio are FP64 in all modes. */
#define SLMC_PREC_FP64 0    /* FP64 FMA */
#define SLMC_PREC_FP32 1    /* FP32 FMA (SIMT) */
/* Tensor cores (tcgen05), the literature's split TF32: two TF32 pieces per operand, three
 * products accumulated in FP32. The tensor cores' FP32 accumulation truncates and its error
 * adds up over the slices of a chain: this mode misses |d ln w| <= 1e-4 (about 2e-3 in ln det
 * at 16x16, beta = 16). */
#define SLMC_PREC_TF32X3 2
/* Tensor cores (tcgen05), exact sliced BF16: F = E - I in four and Y in three 7-bit fixed-point
 * BF16 slices (per-row / per-column powers of two), the nine products with a + b <= 3 summed
 * per level a + b into FP32 accumulators whose every partial sum is an integer below 2^24
 * (bound checked at slmc_init), so the accumulation is exact; |d ln det| ~ 5e-6 at 16x16,
 * beta = 16. A whole stabilisation group runs in one launch with Y resident on chip. */
#define SLMC_PREC_BF16X9 3

/* Model, discretisation and algorithm parameters. */
typedef struct slmc_params {
    int Lx, Ly;          /* periodic lattice sides, >= 2 each; N = Lx * Ly <= 1024 */
    int L;               /* imaginary-time slices, >= 1; beta = L * dtau */
    double dtau;         /* Trotter step (> 0) */
    double t;            /* nearest-neighbour hopping */
    double mu;           /* chemical potential (0 = half filling) */
    double omega0;       /* phonon frequency Omega (M = 1), > 0 */
    double lambda;       /* electron-phonon coupling g */
    int n_s;             /* slices multiplied between two QR stabilisations, >= 1 */
    int precision;       /* SLMC_PREC_* */
    double sweep_delta;  /* half-width of the uniform local proposal x -> x + U[-d, d] */
    uint64_t seed;       /* Philox-4x32-10 key for sweeps and acceptance draws */
    int qr_mode;         /* SLMC_QR_* column ordering of the stabilising QR */
} slmc_params;

/* Column ordering of the stabilising QR (both FP64, both order columns by ||y_j|| D_j). */
#define SLMC_QR_PREPIVOT 0  /* sort once per QR, then blocked Householder with WY updates (default) */
#define SLMC_QR_PIVOTED 1   /* re-pivot on downdated norms at every column (column-by-column) */

typedef struct slmc_ctx slmc_ctx;

/* Returns a static, human-readable name for a status code. */
SLMC_API const char* slmc_status_string(int status);

/* Creates a context on the current CUDA device: validates *p, builds exp(-dtau K) on the
 * device [Eq. (2), (S2)] and allocates the workspace for up to max_fields fields per
 * internal batch (calls with more fields are processed in batches of max_fields).
 * Workspace is about (6 N^2 + 4 N L) * 8 bytes per field. On success *out owns it.
 * Errors: SLMC_ERR_ARG (p or out NULL, sizes out of range), SLMC_ERR_UNSUPPORTED
 * (N > 1024; in SLMC_PREC_BF16X9, slices of exp(-dtau K) - I that could let a tensor-core partial
 * sum exceed 2^24; the worst case allows that only for N > 819), SLMC_ERR_NOMEM, SLMC_ERR_CUDA. */
SLMC_API int slmc_init(const slmc_params* p, int max_fields, slmc_ctx** out);

/* Frees the context and its workspace (synchronises the device first). NULL is a no-op. */
SLMC_API int slmc_destroy(slmc_ctx* ctx);

/* Synchronises `stream`, returns and clears the sticky device-side error of the context
 * (SLMC_OK, SLMC_ERR_NONFINITE, SLMC_ERR_SINGULAR, or SLMC_ERR_TIMEOUT if a bounded wait of the
 * tensor-core pipeline gave up), or SLMC_ERR_CUDA if a kernel failed. */
SLMC_API int slmc_get_error(slmc_ctx* ctx, void* stream);

/* ln|det(I + B_L ... B_1)| and its sign for n fields, one spin species
 * [Suppl. Eq. (S2)]. The product is stabilised every n_s slices by a pivoted
 * Householder QR (UDT form); the last group may hold fewer than n_s slices.
 *   x      [n][N][L] input fields (read only)
 *   lndet  [n] output, ln|det|
 *   sign   [n] output, +1 / -1 (0 if the result is not finite)
 * n = 0 is a no-op. */
SLMC_API int slmc_logdet(slmc_ctx* ctx, const double* x, int n, double* lndet, int* sign, void* stream);

/* As slmc_logdet, and also the equal-time Green's function G = (I + B_L ... B_1)^-1
 * (the paper's G(L) of Suppl. Eq. (S3)), written row-major to G[n][N][N]. */
SLMC_API int slmc_greens(slmc_ctx* ctx, const double* x, int n, double* G, double* lndet, int* sign,
                void* stream);

/* Full log-weight of n configurations [Sec. "Model", Eq. (S2)]:
 *   ln w = 2 ln|det| + dtau lambda sum_{i,l} x - dtau sum_{i,l} [omega0^2 x^2 / 2
 *          + (x_{i,l+1} - x_{i,l})^2 / (2 dtau^2)]   (l periodic).
 * lnw [n] output; lndet [n] and sign [n] optional outputs (may be NULL). */
SLMC_API int slmc_log_weight(slmc_ctx* ctx, const double* x, int n, double* lnw, double* lndet, int* sign,
                    void* stream);

/* The five features of the symmetric effective model [Eq. (4) / (S7)] for n fields:
 * F[n][5] = {F_k, F_p, F_p', F_nn, F_nn'} with
 *   F_k = sum (x_{i,l+1} - x_{i,l})^2,  F_p = sum (x^4/4 - a^2 x^2/2),
 *   F_p' = sum (x^6/6 - a^2 x^4/4),     F_nn = sum over bonds (+x, +y from each site) x_i x_j,
 *   F_nn' = sum x_{i,l} x_{i,l+1}      (all sums over sites and slices, l periodic). */
SLMC_API int slmc_eff_features(slmc_ctx* ctx, const double* x, int n, double* F, void* stream);

/* ln w_eff(x) = -dtau (E0 + J . F(x)) for n fields into lnw_eff[n]; J is a device [6]. */
SLMC_API int slmc_eff_log_weight(slmc_ctx* ctx, const double* x, int n, const double* J, double* lnw_eff,
                        void* stream);

/* Modified Wolff cluster updates of the effective model [Sec. "Wolff update of the effective
 * Hamiltonian", Eq. (S9)], inserted by slmc_eff_sweep and slmc_cumulative_update between the
 * two colours of every sweep (nwolff per sweep, 0..64; default 0 = local sweeps only). Each
 * update builds a cluster in the spatial plane out of whole temporal columns: bond term
 * (i, j) of J_nn F_nn (each site's +x and +y bonds) is activated with probability
 * max(0, 1 - exp(2 dtau J_nn sum_l x_il x_jl)) (uniform of Philox counter (b, ctr, chain, 2),
 * b = 2 i for +x, 2 i + 1 for +y, ctr = (sweep counter) * nwolff + k), the seed site is drawn
 * uniformly (counter (2N, ctr, chain, 2)), and the columns of the seed's connected component
 * are reflected, x -> -x. The other terms of E_eff are invariant under reflecting whole columns,
 * so the move needs no acceptance step. Placed between the colours, the Wolff updates keep the
 * composite proposal of a cumulative update reversible (its reverse is the sequence with the
 * other starting colour), so Eq. (6) stays exact. */
SLMC_API int slmc_set_wolff(slmc_ctx* ctx, int nwolff);

/* Total number of columns reflected by Wolff updates since the context was created or last
 * reset (synchronises `stream`; reset != 0 clears the total). */
SLMC_API int slmc_get_wolff_sites(slmc_ctx* ctx, long long* total, int reset, void* stream);

/* Metropolis sweeps of the effective model on n independent chains, in place
 * [Sec. "SLMC": local updates are O(1) on the bosonic model]. One sweep visits the
 * checkerboard colours (ix + iy + l) mod 2 in the order first_colour, 1 - first_colour;
 * each site proposes x + U[-sweep_delta, sweep_delta] and accepts with probability
 * min(1, exp(-dtau dE_eff)). Sweep s of this call uses the Philox counter
 * (i*L + l, sweep0 + s, chain, 0) with key = seed. Requires even Lx, Ly and L
 * (else SLMC_ERR_UNSUPPORTED).
 *   x       [n][N][L] in/out
 *   J       [6] device couplings
 *   n_acc   [n] int64 in/out: accepted local moves are added (may be NULL)
 * With slmc_set_wolff(ctx, k > 0), k Wolff cluster updates run between the two colours
 * of every sweep. */
SLMC_API int slmc_eff_sweep(slmc_ctx* ctx, double* x, int n, const double* J, int nsweeps, uint64_t sweep0,
                   int first_colour, long long* n_acc, void* stream);

/* Conventional DQMC updates of n independent chains, in place [Supplemental Material,
 * Eqs. (S3)-(S6), and the block update described after them]: the baseline the self-learning
 * method is compared with. Each of nsweeps sweeps visits the slices l = 1..L and, at each, the
 * sites i = 0..N-1: the field of B_l at site i proposes x + U[-sweep_delta, sweep_delta]
 * (Philox counter (i L + l - 1, sweep, chain, 3), words 0-1; acceptance uniform words 2-3),
 * accepted with probability min(1, R^2 exp(d ln w_bose)), R = 1 + (1 - G_ii(l)) Delta_ii,
 * Delta_ii = exp(-dtau lambda d) - 1 (fast ratio of Eq. (S5); both spin species); accepted
 * moves update G(l) by Sherman-Morrison (Eq. (S6)); G is carried to the next slice by
 * G(l) = B_l G(l-1) B_l^-1 and recomputed at the start of every group of n_s slices.
 * Then nblock block updates
 * reflect the whole column of one site (x -> -x, the paper's X -> -X - 2g/Omega^2), site and
 * acceptance uniform from Philox counter (k, sweep, chain, 4), accepted with the ratio of the
 * full weights. Sweep s uses counter sweep0 + s.
 *   x            [n][N][L] in/out
 *   n_acc_local  [n] int64 in/out: accepted local moves are added (may be NULL)
 *   n_acc_block  [n] int64 in/out: accepted block updates are added (may be NULL)
 * G(g0) comes from two stabilised FP64 products (whatever the context's precision): the
 * transposed products B(L, g0)^T of the slices still to come, built at the start of each
 * sweep and kept on a stack of ceil(L / n_s) x max_fields x (2 N^2 + N) doubles allocated on
 * the first call, and the running product B(g0, 0) of the slices already updated.
 * Requires L >= 2 and Lx, Ly <= 32 (else SLMC_ERR_UNSUPPORTED); SLMC_ERR_NOMEM if the stack
 * cannot be allocated. */
SLMC_API int slmc_dqmc_sweep(slmc_ctx* ctx, double* x, int n, int nsweeps, uint64_t sweep0, int nblock,
                             long long* n_acc_local, long long* n_acc_block, void* stream);

/* Prepares chain state for slmc_cumulative_update: lnw[n] = ln w(x) and, if s_cdw is not
 * NULL, s_cdw[n] = S(pi,pi) of each configuration. */
SLMC_API int slmc_chain_init(slmc_ctx* ctx, const double* x, int n, double* lnw, double* s_cdw, void* stream);

/* Passing this as update0 continues from the context's device-side update counter. */
#define SLMC_UPDATE_CONTINUE UINT64_MAX

/* nupdates cumulative updates of n independent chains [Eq. (6)]. The context keeps a
 * device-side update counter U: unless update0 is SLMC_UPDATE_CONTINUE it is first set to
 * update0, and it advances by nupdates at the end (so a call captured into a CUDA graph
 * draws fresh random numbers on every replay). Update u of chain c (global index U + u)
 * draws Philox block (U + u, 0, c, 1): bit 0 of word 0 is the first colour, words 2-3 the
 * acceptance uniform. It then runs nsweeps effective-model sweeps with sweep counters
 * (U + u) * nsweeps + s, evaluates the exact ln w(x') and accepts with
 * min{1, [w(x')/w(x)] [w_eff(x)/w_eff(x')]}; on rejection x is restored. The random starting
 * colour makes the proposal reversible w.r.t. w_eff.
 *   x            [n][N][L] in/out chain states
 *   J            [6] device couplings of E_eff
 *   lnw          [n] in/out cached exact ln w of the current states
 *   s_cdw        [n] in/out cached S(pi,pi) of the current states (may be NULL)
 *   n_acc        [n] int64 in/out, accepted cumulative updates are added (may be NULL)
 *   n_sweep_acc  [n] int64 in/out, accepted local moves are added (may be NULL)
 *   obs          [nupdates][n] out, S(pi,pi) of the state after each update (may be NULL;
 *                requires s_cdw) */
SLMC_API int slmc_cumulative_update(slmc_ctx* ctx, double* x, int n, const double* J, int nsweeps,
                           int nupdates, uint64_t update0, double* lnw, double* s_cdw,
                           long long* n_acc, long long* n_sweep_acc, double* obs, void* stream);

/* Sets the device-side cumulative-update counter to `value` (enqueued on `stream`); with
 * slmc_get_update_counter and the chain state it is all a checkpoint needs to resume the
 * identical random stream. */
SLMC_API int slmc_set_update_counter(slmc_ctx* ctx, uint64_t value, void* stream);

/* Synchronises `stream` and returns the device-side cumulative-update counter. */
SLMC_API int slmc_get_update_counter(slmc_ctx* ctx, uint64_t* value, void* stream);

/* Kernel tile choices (found by slmc_autotune): qr_panel = width of the blocked-QR panels
 * (0 = by N, 16 or 32); slice_cols = columns per thread of the FP32 slice kernel (0 = by N,
 * 8 or 16; 16 is used only for N <= 256). Results do not depend on them beyond rounding. */
SLMC_API int slmc_set_tuning(slmc_ctx* ctx, int qr_panel, int slice_cols);

/* Number of sub-batches (1..4) a determinant batch of at least 32 fields per sub-batch is
 * split into; each runs on its own forked stream so that the kernels of one fill the SMs
 * the others leave idle (default 3; 1 = no split). Results do not depend on it. Contexts
 * created with max_fields < 64 have no forked streams (SLMC_ERR_UNSUPPORTED for n > 1). */
SLMC_API int slmc_set_sub_batches(slmc_ctx* ctx, int n);

/* on = 1: sub-batch k runs on a stream of scheduling priority (highest - k), so the first
 * sub-batch runs ahead and the others fill the SMs it leaves idle; on = 0: equal priorities.
 * Results do not depend on it. SLMC_ERR_UNSUPPORTED for contexts without forked streams. */
SLMC_API int slmc_set_sub_batch_priorities(slmc_ctx* ctx, int on);

/* CTAs per field for the stabilising QR and the formation of Q: 1, 2 or 4 (0 = automatic:
 * 4 when there are at most a quarter as many fields as SMs, 2 up to half, else 1). With more
 * than one, the QR of a field runs on a thread-block cluster (panels round-robin over the
 * CTAs, the panel's reflectors shared through distributed shared memory) and Q's columns are
 * split over the CTAs. Results are bit-identical for every value. */
SLMC_API int slmc_set_qr_cluster(slmc_ctx* ctx, int ctas);

/* FP64 mode. dense = 0 (default): the slice products go through the separable
 * exp(-dtau K) = e^{dtau mu} E_x kron E_y of the periodic lattice [Suppl. Eq. (S2); the x and
 * y hoppings commute], N (Lx + Ly) FMAs per column and slice; dense = 1: dense N^2 products
 * with exp(-dtau K). Both agree to rounding; lattices with a side above 32 always take the
 * dense products. The reduced-precision modes always use their dense F = E - I kernels and
 * the DQMC updates always use the separable factors. SLMC_ERR_ARG for values other than 0
 * and 1. */
SLMC_API int slmc_set_dense_slices(slmc_ctx* ctx, int dense);

/* How the stabilisation updates T <- (D^-1 R) P^T T after each pivoted QR (the T factor of the
 * UDT chain; the paper defers stabilisation to the DQMC literature), in every precision mode:
 *   path = 0 (default): on the tensor cores, FP64-accurate. D^-1 R and P^T T are cut into seven
 *            7-bit fixed-point BF16 slices (a power of two per row and per column), the 28 slice
 *            products with a + b <= 6 are summed per level in FP32 accumulators that provably
 *            hold every partial sum exactly (the bound is checked per row on the actual slices;
 *            a 128-row tile whose bound could exceed 2^24 is computed with FP64 FMAs instead),
 *            and each entry is rounded once to FP64. Entries differ from the FP64 product by
 *            below 2^-48 of their row and column scales.
 *   path = 1: FP64 FMAs (tiled triangular GEMM).
 *   path = 2: the tensor-core kernel with every tile on its FP64 fallback (for tests).
 * The DQMC updates always use path 1. Errors: SLMC_ERR_ARG for other values. */
SLMC_API int slmc_set_tupdate_path(slmc_ctx* ctx, int path);

/* How the pre-pivoted blocked QR (qr_mode SLMC_QR_PREPIVOT) applies each panel's block of BP
 * Householder reflectors to the trailing columns, C <- C - V S^T V^T C (compact WY form), in every
 * precision mode:
 *   path = 0 (default where available, N <= 896): the panels are factored in FP64 as before and
 *            the two products of each trailing update, W = V^T C and C - V W' (W' = S^T W), run on
 *            the tensor cores, FP64-accurate: C, V and W' are cut into seven 7-bit fixed-point
 *            BF16 slices (a power of two per column of C, per reflector, per row of V, per column
 *            of W'), the slice products with a + b <= 6 are summed per level in FP32 accumulators
 *            that hold every partial sum exactly by construction (at most 448 rows per
 *            accumulator), and each entry is rounded once to FP64. Each product entry then differs
 *            from the exact product of the operands by below 2^-44 K max|a_row| max|b_column| (K
 *            the inner dimension): normwise the size of the FP64 loop's own rounding. 4 launches
 *            per panel on the caller's stream.
 *   path = 1: the one-kernel FP64 QR (trailing updates with FP64 FMAs).
 * The DQMC updates and qr_mode SLMC_QR_PIVOTED are unaffected. Errors: SLMC_ERR_ARG for other
 * values, SLMC_ERR_UNSUPPORTED for path 0 when N > 896. */
SLMC_API int slmc_set_qr_path(slmc_ctx* ctx, int path);

/* Thread layout of the FP32 slice kernel: 1: one column group of 256 row threads; 2: two such
 * groups (512 threads); 4 (N <= 256): four column groups of 64 row threads, each thread up to
 * 4 rows x 8 columns. 0 (default) selects 4 for N <= 256 and 1 above. The 256-thread layouts (about 104 KB of shared memory
 * at N = 256) leave room on the SM for a CTA of another sub-batch's FP64 stabilisation, so the
 * FP32 and FP64 pipes work at the same time. Results do not depend on it. */
SLMC_API int slmc_set_slice_groups(slmc_ctx* ctx, int groups);

/* Multi-linear regression of the effective model [Eq. (5)]: least squares of
 * lnw[c] on [1, F(xs[c])] over nconf configurations (Givens-rotation QR in FP64), then
 * (E0, J) = -coefficients / dtau.
 *   xs     [nconf][N][L] configurations, lnw [nconf] their exact log-weights
 *   J_out  [6] device output {E0, J_k, J_p, J_p', J_nn, J_nn'}
 *   resid  [1] device output, RMS residual of ln w (may be NULL)
 * nconf must be >= 6. */
SLMC_API int slmc_fit_eff(slmc_ctx* ctx, const double* xs, const double* lnw, int nconf, double* J_out,
                 double* resid, void* stream);

/* The regression of Eq. (5) split over several processes (each holding its own chains):
 * every process reduces its configurations to a fixed-size state, the states are exchanged
 * (an all-gather of SLMC_FIT_STATE_DOUBLES doubles per process, done by the caller), and every
 * process merges all states into the same couplings.
 * State layout (FP64): [0..48] the 7x7 triangular factor R (row-major) of the rows
 * [1, (F - F_ref)/(N L), lnw - lnw_ref]; [49..54] F_ref[5], lnw_ref (the first configuration
 * of the call); [55] 1 if the state holds data, else 0; [56] number of configurations;
 * [57..63] zero. Configurations are centred for conditioning only: the merge shifts every
 * state to one reference exactly (a unit upper-triangular change of columns), so the merged
 * fit equals the fit of all configurations at once up to rounding.
 *   slmc_fit_eff_state: xs [nconf][N][L], lnw [nconf]; nconf >= 0 (0 gives an empty state);
 *                       state [SLMC_FIT_STATE_DOUBLES] device output.
 *   slmc_fit_eff_merge: states [nparts][SLMC_FIT_STATE_DOUBLES] device input (nparts >= 1;
 *                       empty states are skipped), J_out [6] and resid [1] (may be NULL) as in
 *                       slmc_fit_eff. Fewer than 6 configurations in total, or linearly
 *                       dependent features, set the SINGULAR flag (slmc_get_error). */
#define SLMC_FIT_STATE_DOUBLES 64
SLMC_API int slmc_fit_eff_state(slmc_ctx* ctx, const double* xs, const double* lnw, int nconf, double* state,
                                void* stream);
SLMC_API int slmc_fit_eff_merge(slmc_ctx* ctx, const double* states, int nparts, double* J_out, double* resid,
                                void* stream);

/* CDW structure factor per configuration [Sec. "Results"] from G [n][N][N] (row-major):
 * S = (1/N) sum_ij s_i s_j [4 (1 - G_ii)(1 - G_jj) + 2 (delta_ij - G_ji) G_ij],
 * s_i = (-1)^(ix+iy). Output S[n]. */
SLMC_API int slmc_measure_cdw(slmc_ctx* ctx, const double* G, int n, double* S, void* stream);

/* Kernel classes reported by slmc_profile_read (index into its arrays). */
#define SLMC_PROF_SLICE 0     /* slice-group products B ... B U */
#define SLMC_PROF_QR 1        /* pivoted Householder QR (with SLMC_PROF_QRTC: its panels only) */
#define SLMC_PROF_FORMQ 2     /* formation of Q */
#define SLMC_PROF_TUPDATE 3   /* T <- Rt P^T T */
#define SLMC_PROF_FINAL 4     /* identity init, M assembly, LU and log-det */
#define SLMC_PROF_GREENS 5    /* G solve */
#define SLMC_PROF_SWEEP 6     /* effective-model half-sweeps */
#define SLMC_PROF_EFF 7       /* effective-model features / ln w_eff */
#define SLMC_PROF_BOSE 8      /* bosonic part of ln w */
#define SLMC_PROF_ACCEPT 9    /* acceptance draws, accept/restore */
#define SLMC_PROF_FIT 10      /* regression */
#define SLMC_PROF_CDW 11      /* S(pi,pi) */
#define SLMC_PROF_WOLFF 12    /* Wolff cluster updates of the effective model */
#define SLMC_PROF_DQMC 13     /* DQMC local updates (fast ratio, Sherman-Morrison, wrapping) */
#define SLMC_PROF_QRTC 14     /* QR trailing updates on the tensor cores (slmc_set_qr_path 0) */
#define SLMC_PROF_NCLASS 15

/* Total number of CUDA kernels this context has enqueued since slmc_init (host counter,
 * no synchronisation). */
SLMC_API long long slmc_launch_count(slmc_ctx* ctx);

/* on != 0: from now on every kernel enqueued by the context is bracketed by a pair of
 * CUDA events on its stream (a few microseconds per launch); on = 0 stops recording.
 * Enabling clears the accumulated totals. */
SLMC_API int slmc_profile_enable(slmc_ctx* ctx, int on);

/* Synchronises `stream`, then writes per kernel class the summed device time in ms[c]
 * and the number of timed launch calls in calls[c] (arrays of SLMC_PROF_NCLASS entries;
 * calls may be NULL). A call covers the kernels of one class enqueued together. */
SLMC_API int slmc_profile_read(slmc_ctx* ctx, double* ms, long long* calls, void* stream);

/* As slmc_profile_read, plus per class: busy_ms[c], the union of the class's call intervals
 * (the wall time during which at least one call of the class was running; calls of one class
 * on concurrent sub-batch streams overlap, so busy_ms <= ms), and units[c], the number of
 * fields (or chains) the timed calls processed in total. busy_ms and units may be NULL. */
SLMC_API int slmc_profile_read_detail(slmc_ctx* ctx, double* ms, long long* calls, double* busy_ms,
                                      long long* units, void* stream);

/* ---- Batches of chains of uneven size in one CUDA graph ----------------------------------
 * A batch owns one context per lattice class (nclasses parameter sets, nchains[c] chains
 * each) and one non-blocking stream per class. After the chain buffers of every class are
 * bound, slmc_batch_capture records one round -- nupdates cumulative updates of every class
 * [Eq. (6)] -- into a CUDA graph; slmc_batch_launch replays it. Each update of the round runs
 * (1) the classes' draws and F(x) as concurrent branches forked from and joined back to `stream`,
 * (2) ONE persistent launch for the E_eff Markov chain of every chain of every class: the CTAs
 * pull half-sweep slabs and Wolff updates from a device work queue that lists, phase after
 * phase, the chains in order of decreasing N L; an item waits (bounded, about 2 s) until its
 * chain's earlier items are done, and a wait that gives up sets SLMC_ERR_TIMEOUT in every
 * class's context (slmc_get_error) and stops the queue; and (3) the classes' ln w with G,
 * acceptances and S(pi, pi) as concurrent branches. Each round continues every class's
 * device-side update counter, so replays reproduce bit for bit the random streams and results
 * of successive direct calls to slmc_cumulative_update with SLMC_UPDATE_CONTINUE (the queue
 * runs the same site and Wolff arithmetic). `stream` must be a created stream (not the legacy
 * default stream). Buffer layouts and ownership are those of slmc_cumulative_update. The queue
 * table (16 bytes per item; an item is 1024 sites of a half-sweep or one Wolff update of one
 * chain) is allocated at capture. */
typedef struct slmc_batch slmc_batch;
SLMC_API int slmc_batch_create(const slmc_params* classes, const int* nchains, int nclasses, slmc_batch** out);
SLMC_API int slmc_batch_destroy(slmc_batch* batch);
/* The context of class cls (owned by the batch), for slmc_chain_init, counters, tuning. */
SLMC_API slmc_ctx* slmc_batch_context(slmc_batch* batch, int cls);
SLMC_API int slmc_batch_bind(slmc_batch* batch, int cls, double* x, const double* J, double* lnw, double* s_cdw,
                             long long* n_acc, long long* n_sweep_acc);
SLMC_API int slmc_batch_capture(slmc_batch* batch, int nsweeps, int nupdates, void* stream);
/* on = 1 (default): step (2) above is the persistent queue launch; on = 0: each class runs its
 * own kernel-per-half-sweep sequence on its branch. Takes effect at the next capture. */
SLMC_API int slmc_batch_set_sweep_queue(slmc_batch* batch, int on);
/* Test hook of the bounded waits: with wait_cycles > 0 the next capture's first queue item
 * waits for a completion count that no item reaches, and every queue wait gives up after
 * wait_cycles clock cycles, so the replay ends with SLMC_ERR_TIMEOUT in every class's context
 * and the device stays usable. 0 restores the normal queue at the next capture. */
SLMC_API int slmc_batch_inject_stall(slmc_batch* batch, long long wait_cycles);
SLMC_API int slmc_batch_launch(slmc_batch* batch, int nrounds, void* stream);

/* ---- Autotuner ------------------------------------------------------------------------------
 * For the class described by *p (its precision and qr_mode), times slmc_logdet on ntune
 * synthetic Gaussian fields for every candidate stabilisation interval n_s in
 * {4, 6, 8, 10, 12, 16, 20, 24, 32} (<= L), blocked-QR panel width {16, 32} and FP32 slice
 * tile {8, 16}, and returns the fastest candidate whose max |d ln det| against the library's
 * FP64 path (n_s = 4) on the same fields is <= tol. Allocates and frees its own buffers and
 * synchronises the device (an initialisation-time call). SLMC_ERR_UNSUPPORTED if no candidate
 * meets tol. */
typedef struct slmc_tune_result {
    int n_s;
    int qr_panel;          /* pass to slmc_set_tuning */
    int slice_cols;        /* pass to slmc_set_tuning */
    double sec_per_eval;   /* measured seconds per field evaluation */
    double max_abs_dlndet; /* against the FP64 path */
    int candidates;        /* candidates timed */
} slmc_tune_result;
SLMC_API int slmc_autotune(const slmc_params* p, int ntune, double tol, slmc_tune_result* out);

/* Allocation-free ln|det(I + B_L ... B_1)| (the paper has no counterpart; this is a library
 * service). For callers that cannot allocate device memory where they need the result:
 * code running during CUDA-graph stream capture, latency-critical loops that must avoid
 * the allocator and the device synchronisation cudaMalloc may imply, and hosts whose own
 * allocator owns the device memory budget. No context is needed and nothing is allocated
 * (no cudaMalloc/cudaFree, no allocating library call): E and the whole UDT workspace live
 * in one file-scope device array of slmc_logdet_noalloc_scratch_bytes() = 16 MiB that every
 * GPU loading the library holds until process exit.
 *   p       model parameters as for slmc_init; precision SLMC_PREC_FP64 or SLMC_PREC_FP32
 *   x, n, lndet, sign  as for slmc_logdet (device pointers, results on `stream`)
 * Size limit: the 16 MiB must hold E, F and at least one field's workspace, about
 * 52 N^2 + 300 N bytes (+ 2 KB), so N <= 560 (a 16x16 or 20x20 lattice, not 24x24); larger N returns
 * SLMC_ERR_UNSUPPORTED before anything is enqueued. Fields beyond the array's capacity are
 * processed in consecutive batches.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 * and caches it; make that first call before any stream capture. A device reset
 * (cudaDeviceReset) or a new primary context on that device invalidates the cached address:
 * do not use this entry point on that device afterwards in the same process. The arithmetic
 * is that of slmc_logdet with slmc_set_tupdate_path(1) and slmc_set_qr_path(1): the T update and
 * the QR trailing updates with FP64 FMAs (there is no room for their tensor-core slices); FP64
 * slices through the separable factors for sides <= 32. All calls share the array
 * and it keeps the last call's contents; each call clears the error word it uses on the
 * stream. Calls that overlap on the GPU race on the array: serialise them. Device-side
 * failures are reported only through the outputs (lndet NaN, sign 0). */
SLMC_API int slmc_logdet_noalloc(const slmc_params* p, const double* x, int n, double* lndet, int* sign,
                                 void* stream);

/* Size in bytes of the device array used by slmc_logdet_noalloc. */
SLMC_API size_t slmc_logdet_noalloc_scratch_bytes(void);

#ifdef __cplusplus
}
#endif

#endif /* SLMC_H */
