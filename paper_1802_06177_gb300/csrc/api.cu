// C ABI of libslmc: argument validation, workspace ownership and the enqueue order of the
// kernels that make up each entry point. No entry point synchronises the host except
// slmc_init, slmc_destroy and slmc_get_error.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <new>

#include "slmc_internal.cuh"

namespace {

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

#define SLMC_CK(expr)                                    \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess) return SLMC_ERR_CUDA;     \
    } while (0)

#define SLMC_TRY(expr)                 \
    do {                               \
        int st_ = (expr);              \
        if (st_ != SLMC_OK) return st_; \
    } while (0)

constexpr int kMaxGridY = 65535;

int validate(const slmc_params* p) {
    if (!p) return SLMC_ERR_ARG;
    if (p->Lx < 2 || p->Ly < 2 || p->L < 1 || p->n_s < 1) return SLMC_ERR_ARG;
    if (!(p->dtau > 0.0) || !(p->omega0 > 0.0) || !std::isfinite(p->t) || !std::isfinite(p->mu) ||
        !std::isfinite(p->lambda) || !std::isfinite(p->dtau) || !std::isfinite(p->omega0) ||
        !std::isfinite(p->sweep_delta) || p->sweep_delta < 0.0)
        return SLMC_ERR_ARG;
    if (p->precision < SLMC_PREC_FP64 || p->precision > SLMC_PREC_BF16X9) return SLMC_ERR_ARG;
    if (p->qr_mode != SLMC_QR_PREPIVOT && p->qr_mode != SLMC_QR_PIVOTED) return SLMC_ERR_ARG;
    if ((long long)p->Lx * p->Ly > SLMC_MAX_N) return SLMC_ERR_UNSUPPORTED;
    if ((long long)p->Lx * p->Ly * p->L >= (1ll << 31)) return SLMC_ERR_UNSUPPORTED;
    return SLMC_OK;
}


// ---- launch accounting and optional event timing ------------------------------------
cudaEvent_t take_event(slmc_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
}

// Drains the recorded event pairs into the per-class totals: summed call durations, and the
// union of the call intervals (calls of one class on concurrent streams overlap in time; the
// union is the wall time during which at least one call of the class was running).
int flush_profile(slmc_ctx* c) {
    std::vector<std::pair<float, float>> iv[SLMC_PROF_NCLASS];
    for (size_t q = 0; q < c->ev_cls.size(); ++q) {
        cudaEvent_t b = c->ev_rec[2 * q], e = c->ev_rec[2 * q + 1];
        float ms = 0.f, t0 = 0.f, t1 = 0.f;
        if (cudaEventSynchronize(e) != cudaSuccess || cudaEventElapsedTime(&ms, b, e) != cudaSuccess ||
            cudaEventElapsedTime(&t0, c->prof_base, b) != cudaSuccess ||
            cudaEventElapsedTime(&t1, c->prof_base, e) != cudaSuccess)
            return SLMC_ERR_CUDA;
        const int cls = c->ev_cls[q];
        c->prof_ms[cls] += ms;
        c->prof_calls[cls] += 1;
        c->prof_units[cls] += c->ev_units[q];
        iv[cls].emplace_back(t0, t1);
        c->ev_pool.push_back(b);
        c->ev_pool.push_back(e);
    }
    for (int cls = 0; cls < SLMC_PROF_NCLASS; ++cls) {
        auto& v = iv[cls];
        std::sort(v.begin(), v.end());
        double busy = 0.0, lo = 0.0, hi = -1.0;
        for (const auto& w : v) {
            if (w.first > hi) {
                if (hi > lo) busy += hi - lo;
                lo = w.first;
                hi = w.second;
            } else if (w.second > hi) {
                hi = w.second;
            }
        }
        if (hi > lo) busy += hi - lo;
        c->prof_busy[cls] += busy;
    }
    c->ev_cls.clear();
    c->ev_rec.clear();
    c->ev_units.clear();
    return SLMC_OK;
}

// Enqueues fn() (which launches nkernels kernels of class cls on s) with accounting.
template <typename Fn>
int launch(slmc_ctx* c, int cls, int nkernels, cudaStream_t s, Fn&& fn) {
    cudaEvent_t b = nullptr;
    if (c->prof_on) {
        b = take_event(c);
        if (!b || cudaEventRecord(b, s) != cudaSuccess) return SLMC_ERR_CUDA;
    }
    if (fn() != cudaSuccess) return SLMC_ERR_CUDA;
    c->launches += nkernels;
    if (c->prof_on) {
        cudaEvent_t e = take_event(c);
        if (!e || cudaEventRecord(e, s) != cudaSuccess) return SLMC_ERR_CUDA;
        c->ev_rec.push_back(b);
        c->ev_rec.push_back(e);
        c->ev_cls.push_back(cls);
        c->ev_units.push_back(c->cur_units);
        // bounded pool: drains the recorded pairs (a device synchronisation) every 65536 calls,
        // well beyond a profiled region of a few steps
        if (c->ev_cls.size() >= 65536) return flush_profile(c);
    }
    return SLMC_OK;
}

#define SLMC_LAUNCH(cls, nk, s, expr) SLMC_TRY(launch(c, (cls), (nk), (s), [&]() { return (expr); }))

bool checkerboard_ok(const slmc_ctx* c) { return c->p.Lx % 2 == 0 && c->p.Ly % 2 == 0 && c->L % 2 == 0; }

// Scratch columns of ctx->scal ([8][max_fields]) and ctx->iscal ([4][max_fields]).
double* scal(slmc_ctx* c, int col) { return c->scal + (size_t)col * c->max_fields; }
int* iscal(slmc_ctx* c, int col) { return c->iscal + (size_t)col * c->max_fields; }

// Stabilised UDT chain + final LU for fields [0, nf) of the context (or view) v; launches are
// accounted on `c` (the owning context).
int logdet_run(slmc_ctx* c, slmc_ctx* v, const double* x, int nf, double* lndet, int* sign, double* G,
               cudaStream_t s) {
    c->cur_units = nf;
    SLMC_LAUNCH(SLMC_PROF_FINAL, 1, s, slmc::set_identity(v, nf, s));
    if (v->p.precision != SLMC_PREC_FP64) SLMC_LAUNCH(SLMC_PROF_SLICE, 1, s, slmc::slice_scales(v, x, nf, s));
    for (int l0 = 0; l0 < v->L; l0 += v->p.n_s) {
        const int nsl = std::min(v->p.n_s, v->L - l0);
        if (v->p.precision == SLMC_PREC_TF32X3)
            SLMC_LAUNCH(SLMC_PROF_SLICE, slmc::tc_launches(nsl), s, slmc::tc_slice_group(v, x, nf, l0, nsl, s));
        else if (v->p.precision == SLMC_PREC_BF16X9)
            SLMC_LAUNCH(SLMC_PROF_SLICE, 1, s, slmc::tcx_slice_group(v, nf, l0, nsl, s));
        else
            SLMC_LAUNCH(SLMC_PROF_SLICE, 1, s, slmc::slice_group(v, x, nf, l0, nsl, s));
        if (v->p.qr_mode == SLMC_QR_PIVOTED) {
            SLMC_LAUNCH(SLMC_PROF_QR, 1, s, slmc::qr_pivoted(v, nf, s));
            SLMC_LAUNCH(SLMC_PROF_FORMQ, 1, s, slmc::form_q(v, nf, s));
            if (v->p.precision != SLMC_PREC_FP64 && l0 + nsl < v->L)
                SLMC_LAUNCH(SLMC_PROF_FORMQ, 1, s, slmc::u_to_f32(v, nf, s));
        } else {
            if (slmc::qrt_active(v)) {  // panels in FP64, trailing updates on the tensor cores
                const int np = slmc::qrt_panels(v);
                for (int t = 0; t < np; ++t) {
                    SLMC_LAUNCH(SLMC_PROF_QR, 1, s, slmc::qrt_panel(v, nf, t, s));
                    if (t + 1 < np) SLMC_LAUNCH(SLMC_PROF_QRTC, 3, s, slmc::qrt_trailing(v, nf, t, s));
                }
            } else {
                SLMC_LAUNCH(SLMC_PROF_QR, 1, s, slmc::qr_blocked(v, nf, s));
            }
            // Q enters the next reduced-precision slice group (rounded to FP32 there anyway) except
            // after the last group, where it enters the FP64 final step.
            const bool q32 = v->p.precision != SLMC_PREC_FP64 && l0 + nsl < v->L;
            SLMC_LAUNCH(SLMC_PROF_FORMQ, 1, s, slmc::form_q_blocked(v, nf, q32, s));
        }
        SLMC_LAUNCH(SLMC_PROF_TUPDATE, slmc::t_update_launches(v), s, slmc::t_update(v, nf, s));
    }
    SLMC_LAUNCH(SLMC_PROF_FINAL, 2, s, slmc::final_logdet(v, nf, lndet, sign, s));
    if (G) SLMC_LAUNCH(SLMC_PROF_GREENS, 1, s, slmc::final_greens(v, nf, G, s));
    return SLMC_OK;
}


constexpr int kMinSubFields = 32;

// A view of context c for fields [f0, ...): per-field workspace pointers offset by f0.
slmc_ctx make_view(slmc_ctx* c, int f0) {
    slmc_ctx v{};
    v.p = c->p;
    v.N = c->N;
    v.L = c->L;
    v.max_fields = c->max_fields;
    v.device = c->device;
    const size_t N = c->N, NN = N * N, F0 = (size_t)f0;
    v.E64 = c->E64;
    v.Einv64 = c->Einv64;
    v.kron = c->kron;
    v.dense_slices = c->dense_slices;
    v.F32 = c->F32;
    v.lo_kidx = c->lo_kidx;
    v.lo_val = c->lo_val;
    v.lo_S = c->lo_S;
    v.tcx_F = c->tcx_F;
    v.tcx_eF = c->tcx_eF;
    v.tcx_npad = c->tcx_npad;
    v.tcx_mapF = c->tcx_mapF;
    v.tt_A = c->tt_A;
    v.tt_B = c->tt_B;
    v.tt_eA = c->tt_eA;
    v.tt_eB = c->tt_eB;
    v.tt_flag = c->tt_flag;
    v.tt_mpad = c->tt_mpad;
    v.tt_npad = c->tt_npad;
    v.tt_path = c->tt_path;
    v.tt_mapA = c->tt_mapA;
    v.tt_mapB = c->tt_mapB;
    v.qt_buf = c->qt_buf;
    v.qt_ibuf = c->qt_ibuf;
    v.qt_C = c->qt_C;
    v.qt_V1 = c->qt_V1;
    v.qt_V2 = c->qt_V2;
    v.qt_W = c->qt_W;
    v.qt_eC = c->qt_eC;
    v.qt_eV1 = c->qt_eV1;
    v.qt_eV2 = c->qt_eV2;
    v.qt_eW = c->qt_eW;
    v.qt_ntriv = c->qt_ntriv;
    v.qt_lnDn = c->qt_lnDn;
    v.qt_kpad = c->qt_kpad;
    v.qt_mpad = c->qt_mpad;
    v.qt_wpad = c->qt_wpad;
    v.qr_path = c->qr_path;
    v.qt_mapC96 = c->qt_mapC96;
    v.qt_mapC112 = c->qt_mapC112;
    v.qt_mapV1_16 = c->qt_mapV1_16;
    v.qt_mapV1_32 = c->qt_mapV1_32;
    v.qt_mapV2 = c->qt_mapV2;
    v.qt_mapW = c->qt_mapW;
    v.fbase = c->fbase + f0;
    v.sc32 = c->sc32 ? c->sc32 + F0 * c->L * N : nullptr;
    v.Y = c->Y + F0 * NN;
    v.QR = c->QR + F0 * NN;
    v.U = c->U + F0 * NN;
    v.U32 = c->U32 ? c->U32 + F0 * NN : nullptr;
    v.Ta = c->Ta + F0 * NN;
    v.Tb = c->Tb + F0 * NN;
    v.lnD = c->lnD + F0 * N;
    v.tau = c->tau + F0 * N;
    v.perm = c->perm + F0 * N;
    v.piv = c->piv + F0 * N;
    v.sgnU = c->sgnU + F0;
    v.Sws = c->Sws + F0 * N * 32;
    v.err = c->err;
    v.dctr = c->dctr;
    v.nwolff = c->nwolff;
    v.wolff_sites = c->wolff_sites;
    v.tune_qr_panel = c->tune_qr_panel;
    v.tune_slice_cols = c->tune_slice_cols;
    v.tune_slice_groups = c->tune_slice_groups;
    v.tune_qr_cluster = c->tune_qr_cluster;
    v.num_sms = c->num_sms;
    v.nsub = 0;
    v.parent = c;
    return v;
}

int logdet_batch(slmc_ctx* c, const double* x, int nf, double* lndet, int* sign, double* G, cudaStream_t s) {
    const bool tc = c->p.precision == SLMC_PREC_TF32X3;  // per-slice workspace not split into views
    const int nsub = std::min(c->nsub, nf / kMinSubFields);
    if (nsub < 2 || tc) return logdet_run(c, c, x, nf, lndet, sign, G, s);
    const size_t NL = (size_t)c->N * c->L, NN = (size_t)c->N * c->N;
    SLMC_CK(cudaEventRecord(c->sub_fork, s));
    for (int k = 0; k < nsub; ++k) {
        const int f0 = (int)((long long)k * nf / nsub), f1 = (int)((long long)(k + 1) * nf / nsub);
        cudaStream_t sk = c->sub_prio ? c->sub_stream_prio[k] : c->sub_stream[k];
        SLMC_CK(cudaStreamWaitEvent(sk, c->sub_fork, 0));
        slmc_ctx v = make_view(c, f0);
        SLMC_TRY(logdet_run(c, &v, x + f0 * NL, f1 - f0, lndet + f0, sign + f0, G ? G + f0 * NN : nullptr, sk));
        SLMC_CK(cudaEventRecord(c->sub_join[k], sk));
        SLMC_CK(cudaStreamWaitEvent(s, c->sub_join[k], 0));
    }
    return SLMC_OK;
}

template <typename F>
int for_batches(slmc_ctx* c, int n, F&& fn) {
    for (int f0 = 0; f0 < n; f0 += c->max_fields) {
        const int nf = std::min(c->max_fields, n - f0);
        c->cur_units = nf;
        SLMC_TRY(fn(f0, nf));
    }
    return SLMC_OK;
}

void free_ctx(slmc_ctx* c) {
    for (int k = 0; k < slmc_ctx::kMaxSub; ++k) {
        if (c->sub_stream[k]) cudaStreamDestroy(c->sub_stream[k]);
        if (c->sub_stream_prio[k]) cudaStreamDestroy(c->sub_stream_prio[k]);
        if (c->sub_join[k]) cudaEventDestroy(c->sub_join[k]);
    }
    if (c->sub_fork) cudaEventDestroy(c->sub_fork);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_rec) cudaEventDestroy(e);
    if (c->prof_base) cudaEventDestroy(c->prof_base);
    void* bufs[] = {c->E64, c->Einv64, c->kron, c->F32, c->lo_kidx, c->lo_val, c->sc32, c->tcx_F, c->tcx_eF,
                    c->tt_A, c->tt_B, c->tt_eA, c->tt_eB, c->tt_flag, c->qt_buf, c->qt_ibuf, c->qt_lnDn,
                    c->Y, c->QR, c->U, c->U32, c->Ta, c->Tb, c->lnD, c->tau,
                    c->perm, c->piv, c->sgnU, c->Sws, c->x_old, c->scal, c->iscal, c->feat, c->fitR, c->err, c->dctr,
                    c->wolff_sites, c->dq_stack,
                    c->tc_F, c->tc_p[0], c->tc_p[1], c->tc_y32[0], c->tc_y32[1]};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete c;
}

}  // namespace

namespace slmc {
// Shared with the allocation-free entry point (k_noalloc.cu): parameter validation and the
// stabilised UDT chain + LU of slmc_logdet for one batch of fields.
int validate_params(const slmc_params* p) { return validate(p); }
int logdet_fields(slmc_ctx* c, const double* x, int nf, double* lndet, int* sign, cudaStream_t s) {
    return logdet_batch(c, x, nf, lndet, sign, nullptr, s);
}

// Updates [u0, u1) of the cumulative-update cycle [Eq. (6)] of chains [0, n), restricted to the
// phases in the mask: kPhasePre (the update's draws, the saved field, F(x) of E_eff), kPhaseSweeps
// (the E_eff Markov chain: nsweeps checkerboard sweeps with the Wolff updates between their two
// colours) and kPhasePost (F(x') of E_eff, ln w with G, the acceptance and S). Chains are
// independent: a batch is split into sub-batches (as for slmc_logdet), each running its updates on
// its own forked stream, so the sweeps of one sub-batch overlap the determinants of another. The
// arithmetic of a chain does not depend on the split or on the phases being run apart.
int cumulative_phases(slmc_ctx* c, double* x, int n, const double* J, int nsweeps, int u0, int u1, int phases,
                      double* lnw, double* s_cdw, long long* n_acc, long long* n_sweep_acc, double* obs,
                      cudaStream_t s) {
    const size_t NL = (size_t)c->N * c->L;
    return for_batches(c, n, [&](int f0, int nf) {
        const bool tc = c->p.precision == SLMC_PREC_TF32X3;
        int nsub = std::min(c->nsub, nf / kMinSubFields);
        if (nsub < 2 || tc || !(phases & kPhasePost)) nsub = 1;
        if (nsub > 1) SLMC_CK(cudaEventRecord(c->sub_fork, s));
        for (int k = 0; k < nsub; ++k) {
            const int a = (int)((long long)k * nf / nsub), b = (int)((long long)(k + 1) * nf / nsub), m = b - a;
            cudaStream_t sk = nsub == 1 ? s : (c->sub_prio ? c->sub_stream_prio[k] : c->sub_stream[k]);
            if (nsub > 1) SLMC_CK(cudaStreamWaitEvent(sk, c->sub_fork, 0));
            slmc_ctx view = make_view(c, a);
            slmc_ctx* v = nsub == 1 ? c : &view;
            const int g0 = f0 + a;  // first chain of the sub-batch
            double* xc = x + (size_t)g0 * NL;
            double* xo = c->x_old + (size_t)a * NL;
            auto sc = [&](int col) { return scal(c, col) + a; };
            auto isc = [&](int col) { return iscal(c, col) + a; };
            for (int u = u0; u < u1; ++u) {
                c->cur_units = m;
                if (phases & kPhasePre) {
                    SLMC_LAUNCH(SLMC_PROF_ACCEPT, 1, sk, update_draws(c, m, g0, (uint64_t)u, isc(1), sc(4), sk));
                    SLMC_CK(cudaMemcpyAsync(xo, xc, m * NL * sizeof(double), cudaMemcpyDeviceToDevice, sk));
                    SLMC_LAUNCH(SLMC_PROF_EFF, 1, sk, eff_features(c, xc, m, J, nullptr, 0, sc(1), sk));
                }
                if (phases & kPhaseSweeps)
                    for (int sw = 0; sw < nsweeps; ++sw)
                        for (int h = 0; h < 2; ++h) {
                            if (h == 1)  // Wolff cluster updates between the two colours of the sweep
                                for (int k = 0; k < c->nwolff; ++k)
                                    SLMC_LAUNCH(SLMC_PROF_WOLFF, 1, sk,
                                                eff_wolff(c, xc, m, g0, J, (uint64_t)u * nsweeps + sw, k, sk, c->dctr,
                                                          nsweeps));
                            SLMC_LAUNCH(SLMC_PROF_SWEEP, 1, sk,
                                        eff_half_sweep(c, xc, m, g0, J, (uint64_t)u * nsweeps + sw, 0, isc(1), h,
                                                       n_sweep_acc ? n_sweep_acc + g0 : nullptr, sk, c->dctr,
                                                       nsweeps));
                        }
                if (phases & kPhasePost) {
                    SLMC_LAUNCH(SLMC_PROF_EFF, 1, sk, eff_features(c, xc, m, J, nullptr, 0, sc(2), sk));
                    SLMC_TRY(logdet_run(c, v, xc, m, sc(0), isc(0), s_cdw ? v->QR : nullptr, sk));
                    c->cur_units = m;
                    SLMC_LAUNCH(SLMC_PROF_BOSE, 1, sk, bose_log_weight(c, xc, m, sc(0), sc(3), sk));
                    SLMC_LAUNCH(SLMC_PROF_ACCEPT, 2, sk,
                                accept_update(c, m, xc, xo, sc(3), sc(1), sc(2), sc(4), lnw + g0, isc(2),
                                              n_acc ? n_acc + g0 : nullptr, sk));
                    if (s_cdw)
                        SLMC_LAUNCH(SLMC_PROF_CDW, 1, sk,
                                    cdw_measure(c, v->QR, m, s_cdw + g0, isc(2),
                                                obs ? obs + (size_t)u * n + g0 : nullptr, sk));
                }
            }
            if (nsub > 1) {
                SLMC_CK(cudaEventRecord(c->sub_join[k], sk));
                SLMC_CK(cudaStreamWaitEvent(s, c->sub_join[k], 0));
            }
        }
        return SLMC_OK;
    });
}

// Device pointers of a class's per-chain draws (first colour of each chain's sweeps).
const int* first_colours(slmc_ctx* c) { return iscal(c, 1); }
}  // namespace slmc

extern "C" {

const char* slmc_status_string(int status) {
    switch (status) {
        case SLMC_OK: return "ok";
        case SLMC_ERR_ARG: return "invalid argument";
        case SLMC_ERR_NONFINITE: return "non-finite input or result";
        case SLMC_ERR_CUDA: return "CUDA runtime error";
        case SLMC_ERR_TIMEOUT: return "bounded device wait timed out";
        case SLMC_ERR_UNSUPPORTED: return "unsupported shape or mode";
        case SLMC_ERR_NOMEM: return "out of device memory";
        case SLMC_ERR_SINGULAR: return "singular matrix";
        default: return "unknown status";
    }
}

int slmc_init(const slmc_params* p, int max_fields, slmc_ctx** out) {
    if (!out) return SLMC_ERR_ARG;
    *out = nullptr;
    SLMC_TRY(validate(p));
    if (max_fields < 1 || max_fields > kMaxGridY) return SLMC_ERR_ARG;
    slmc_ctx* c = new (std::nothrow) slmc_ctx();
    if (!c) return SLMC_ERR_NOMEM;
    c->p = *p;
    c->N = p->Lx * p->Ly;
    c->L = p->L;
    c->max_fields = max_fields;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        delete c;
        return SLMC_ERR_CUDA;
    }
    const size_t N = c->N, L = c->L, F = max_fields, NN = N * N;
    bool ok = true;
    auto alloc = [&](auto** ptr, size_t bytes) {
        if (!ok) return;
        if (cudaMalloc(reinterpret_cast<void**>(ptr), bytes) != cudaSuccess) ok = false;
    };
    alloc(&c->E64, NN * sizeof(double));
    alloc(&c->Einv64, NN * sizeof(double));
    if (c->p.Lx <= slmc::kKronMaxLine && c->p.Ly <= slmc::kKronMaxLine) alloc(&c->kron, 4 * slmc::kKronTab * sizeof(double));
    alloc(&c->F32, NN * sizeof(float));
    if (p->precision == SLMC_PREC_FP32) {
        c->lo_S = std::min(slmc::kLoStencil, (int)N);
        alloc(&c->lo_kidx, ((size_t)c->lo_S * N + c->lo_S) * sizeof(int));
        alloc(&c->lo_val, (size_t)c->lo_S * sizeof(float));
    }
    if (p->precision != SLMC_PREC_FP64) alloc(&c->sc32, F * L * N * sizeof(float));
    if (p->precision == SLMC_PREC_BF16X9) {
        int mt = 0, nt = 0, npad = 0;
        slmc::tcx_geometry(c->N, &mt, &nt, &npad);
        alloc(&c->tcx_F, slmc::tcx_F_bytes(c->N));
        alloc(&c->tcx_eF, (size_t)mt * 128 * sizeof(int));
    }
    {  // tensor-core T update: slices of Rt and P^T T, exponents, exactness flags
        const size_t npad = (N + 63) / 64 * 64, mpad = (N + 127) / 128 * 128;
        alloc(&c->tt_A, slmc::tt_slices() * F * mpad * npad * 2);
        alloc(&c->tt_B, slmc::tt_slices() * F * npad * npad * 2);
        alloc(&c->tt_eA, F * mpad * sizeof(int));
        alloc(&c->tt_eB, F * npad * sizeof(int));
        alloc(&c->tt_flag, F * (mpad / 128) * sizeof(int));
    }
    if (slmc::qrt_supported((int)N)) {  // QR with tensor-core trailing updates
        size_t nb16 = 0, nint = 0;
        slmc::qrt_sizes((int)N, (int)F, &nb16, &nint);
        alloc(&c->qt_buf, nb16 * 2);
        alloc(reinterpret_cast<void**>(&c->qt_ibuf), nint * sizeof(int));
        alloc(reinterpret_cast<void**>(&c->qt_lnDn), F * N * sizeof(double));
    }
    alloc(&c->Y, F * NN * sizeof(double));
    alloc(&c->QR, F * NN * sizeof(double));
    alloc(&c->U, F * NN * sizeof(double));
    if (p->precision != SLMC_PREC_FP64) alloc(&c->U32, F * NN * sizeof(float));
    alloc(&c->Ta, F * NN * sizeof(double));
    alloc(&c->Tb, F * NN * sizeof(double));
    alloc(&c->lnD, F * N * sizeof(double));
    alloc(&c->tau, F * N * sizeof(double));
    alloc(&c->perm, F * N * sizeof(int));
    alloc(&c->piv, F * N * sizeof(int));
    alloc(&c->sgnU, F * sizeof(int));
    alloc(&c->Sws, F * N * 32 * sizeof(double));
    alloc(&c->x_old, F * N * L * sizeof(double));
    alloc(&c->scal, 8 * F * sizeof(double));
    alloc(&c->iscal, 4 * F * sizeof(int));
    alloc(&c->feat, 8 * F * sizeof(double));
    alloc(&c->fitR, 64 * sizeof(double));
    alloc(&c->err, sizeof(unsigned int));
    alloc(&c->dctr, sizeof(unsigned long long));
    if (ok && cudaMemset(c->dctr, 0, sizeof(unsigned long long)) != cudaSuccess) ok = false;
    alloc(&c->wolff_sites, sizeof(unsigned long long));
    if (ok && cudaMemset(c->wolff_sites, 0, sizeof(unsigned long long)) != cudaSuccess) ok = false;
    const bool tc = p->precision == SLMC_PREC_TF32X3;
    if (tc) {
        size_t es = 0;
        int np = 0;
        slmc::tc_geometry(c->N, &c->tc_npad, &c->tc_nt, &es, &np);
        const size_t Np = c->tc_npad;
        alloc(&c->tc_F, np * Np * Np * es);
        for (int b = 0; b < 2; ++b) {
            alloc(&c->tc_p[b], np * F * N * Np * es);
            alloc(&c->tc_y32[b], F * NN * sizeof(float));
            if (ok && cudaMemset(c->tc_p[b], 0, np * F * N * Np * es) != cudaSuccess) ok = false;
        }
    }
    if (!ok) {
        cudaGetLastError();
        free_ctx(c);
        return SLMC_ERR_NOMEM;
    }
    c->nsub = 0;
    if (max_fields >= 2 * kMinSubFields) {
        bool sok = cudaEventCreateWithFlags(&c->sub_fork, cudaEventDisableTiming) == cudaSuccess;
        int prio_least = 0, prio_greatest = 0;
        sok = sok && cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) == cudaSuccess;
        for (int k = 0; k < slmc_ctx::kMaxSub && sok; ++k) {
            // sub-batch k on priority greatest + k: the first sub-batch runs ahead and the others fill
            // the SMs it leaves idle, so the sub-batches drift out of phase (FP32 slice products of one
            // beside FP64 stabilisation of another)
            const int prio = std::min(prio_greatest + k, prio_least);
            sok = cudaStreamCreateWithFlags(&c->sub_stream[k], cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithPriority(&c->sub_stream_prio[k], cudaStreamNonBlocking, prio) == cudaSuccess &&
                  cudaEventCreateWithFlags(&c->sub_join[k], cudaEventDisableTiming) == cudaSuccess;
        }
        if (sok) {
            c->nsub_avail = slmc_ctx::kMaxSub;
            c->nsub = 3;
        } else {
            cudaGetLastError();
        }
    }
    if (cudaMemset(c->err, 0, sizeof(unsigned int)) != cudaSuccess ||
        slmc::build_hopping_exp(c, nullptr) != cudaSuccess || (tc && slmc::tc_init(c, nullptr) != cudaSuccess) ||
        slmc::tt_init(c) != cudaSuccess || (c->qt_buf && slmc::qrt_init(c, c->qt_buf, c->qt_ibuf) != cudaSuccess) ||
        cudaDeviceSynchronize() != cudaSuccess) {
        free_ctx(c);
        return SLMC_ERR_CUDA;
    }
    if (p->precision == SLMC_PREC_BF16X9) {
        const cudaError_t e = slmc::tcx_init(c, nullptr);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_ctx(c);
            return e == cudaErrorNotSupported ? SLMC_ERR_UNSUPPORTED : SLMC_ERR_CUDA;
        }
    }
    *out = c;
    return SLMC_OK;
}

int slmc_destroy(slmc_ctx* c) {
    if (!c) return SLMC_OK;
    const cudaError_t e = cudaDeviceSynchronize();
    free_ctx(c);
    return e == cudaSuccess ? SLMC_OK : SLMC_ERR_CUDA;
}

int slmc_get_error(slmc_ctx* c, void* stream) {
    if (!c) return SLMC_ERR_ARG;
    if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return SLMC_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return SLMC_ERR_CUDA;
    unsigned int bits = 0;
    if (cudaMemcpy(&bits, c->err, sizeof(bits), cudaMemcpyDeviceToHost) != cudaSuccess) return SLMC_ERR_CUDA;
    if (bits && cudaMemset(c->err, 0, sizeof(bits)) != cudaSuccess) return SLMC_ERR_CUDA;
    if (bits & SLMC_EBIT_TIMEOUT) return SLMC_ERR_TIMEOUT;
    if (bits & SLMC_EBIT_SINGULAR) return SLMC_ERR_SINGULAR;
    if (bits & SLMC_EBIT_NONFINITE) return SLMC_ERR_NONFINITE;
    return SLMC_OK;
}

int slmc_logdet(slmc_ctx* c, const double* x, int n, double* lndet, int* sign, void* stream) {
    if (!c || n < 0 || (n > 0 && (!x || !lndet || !sign))) return SLMC_ERR_ARG;
    const size_t NL = (size_t)c->N * c->L;
    return for_batches(c, n, [&](int f0, int nf) {
        return logdet_batch(c, x + f0 * NL, nf, lndet + f0, sign + f0, nullptr, as_stream(stream));
    });
}

int slmc_greens(slmc_ctx* c, const double* x, int n, double* G, double* lndet, int* sign, void* stream) {
    if (!c || n < 0 || (n > 0 && (!x || !G || !lndet || !sign))) return SLMC_ERR_ARG;
    const size_t NL = (size_t)c->N * c->L, NN = (size_t)c->N * c->N;
    return for_batches(c, n, [&](int f0, int nf) {
        return logdet_batch(c, x + f0 * NL, nf, lndet + f0, sign + f0, G + f0 * NN, as_stream(stream));
    });
}

int slmc_log_weight(slmc_ctx* c, const double* x, int n, double* lnw, double* lndet, int* sign, void* stream) {
    if (!c || n < 0 || (n > 0 && (!x || !lnw))) return SLMC_ERR_ARG;
    const size_t NL = (size_t)c->N * c->L;
    cudaStream_t s = as_stream(stream);
    return for_batches(c, n, [&](int f0, int nf) {
        double* ld = lndet ? lndet + f0 : scal(c, 0);
        int* sg = sign ? sign + f0 : iscal(c, 0);
        SLMC_TRY(logdet_batch(c, x + f0 * NL, nf, ld, sg, nullptr, s));
        SLMC_LAUNCH(SLMC_PROF_BOSE, 1, s, slmc::bose_log_weight(c, x + f0 * NL, nf, ld, lnw + f0, s));
        return SLMC_OK;
    });
}

int slmc_eff_features(slmc_ctx* c, const double* x, int n, double* F, void* stream) {
    if (!c || n < 0 || (n > 0 && (!x || !F))) return SLMC_ERR_ARG;
    if (n == 0) return SLMC_OK;
    cudaStream_t s = as_stream(stream);
    SLMC_LAUNCH(SLMC_PROF_EFF, 1, s, slmc::eff_features(c, x, n, nullptr, F, 5, nullptr, s));
    return SLMC_OK;
}

int slmc_eff_log_weight(slmc_ctx* c, const double* x, int n, const double* J, double* lnw_eff, void* stream) {
    if (!c || n < 0 || (n > 0 && (!x || !J || !lnw_eff))) return SLMC_ERR_ARG;
    if (n == 0) return SLMC_OK;
    cudaStream_t s = as_stream(stream);
    SLMC_LAUNCH(SLMC_PROF_EFF, 1, s, slmc::eff_features(c, x, n, J, nullptr, 0, lnw_eff, s));
    return SLMC_OK;
}

int slmc_eff_sweep(slmc_ctx* c, double* x, int n, const double* J, int nsweeps, uint64_t sweep0, int first_colour,
                   long long* n_acc, void* stream) {
    if (!c || n < 0 || n > kMaxGridY || nsweeps < 0 || (first_colour != 0 && first_colour != 1) ||
        (n > 0 && (!x || !J)))
        return SLMC_ERR_ARG;
    if (!checkerboard_ok(c)) return SLMC_ERR_UNSUPPORTED;
    cudaStream_t s = as_stream(stream);
    c->cur_units = n;
    for (int sw = 0; sw < nsweeps && n > 0; ++sw)
        for (int h = 0; h < 2; ++h) {
            if (h == 1)  // Wolff cluster updates between the two colours of the sweep
                for (int k = 0; k < c->nwolff; ++k)
                    SLMC_LAUNCH(SLMC_PROF_WOLFF, 1, s, slmc::eff_wolff(c, x, n, 0, J, sweep0 + sw, k, s));
            SLMC_LAUNCH(SLMC_PROF_SWEEP, 1, s,
                        slmc::eff_half_sweep(c, x, n, 0, J, sweep0 + sw, first_colour ^ h, nullptr, 0, n_acc, s));
        }
    return SLMC_OK;
}

int slmc_chain_init(slmc_ctx* c, const double* x, int n, double* lnw, double* s_cdw, void* stream) {
    if (!c || n < 0 || (n > 0 && (!x || !lnw))) return SLMC_ERR_ARG;
    const size_t NL = (size_t)c->N * c->L;
    cudaStream_t s = as_stream(stream);
    return for_batches(c, n, [&](int f0, int nf) {
        SLMC_TRY(logdet_batch(c, x + f0 * NL, nf, scal(c, 0), iscal(c, 0), s_cdw ? c->QR : nullptr, s));
        SLMC_LAUNCH(SLMC_PROF_BOSE, 1, s, slmc::bose_log_weight(c, x + f0 * NL, nf, scal(c, 0), lnw + f0, s));
        if (s_cdw) SLMC_LAUNCH(SLMC_PROF_CDW, 1, s, slmc::cdw_measure(c, c->QR, nf, s_cdw + f0, nullptr, nullptr, s));
        return SLMC_OK;
    });
}

int slmc_cumulative_update(slmc_ctx* c, double* x, int n, const double* J, int nsweeps, int nupdates,
                           uint64_t update0, double* lnw, double* s_cdw, long long* n_acc, long long* n_sweep_acc,
                           double* obs, void* stream) {
    if (!c || n < 0 || nsweeps < 0 || nupdates < 0 || (n > 0 && (!x || !J || !lnw)) || (obs && !s_cdw))
        return SLMC_ERR_ARG;
    if (!checkerboard_ok(c)) return SLMC_ERR_UNSUPPORTED;
    cudaStream_t s = as_stream(stream);
    if (update0 != SLMC_UPDATE_CONTINUE) SLMC_LAUNCH(SLMC_PROF_ACCEPT, 1, s, slmc::counter_op(c, update0, false, s));
    SLMC_TRY(slmc::cumulative_phases(c, x, n, J, nsweeps, 0, nupdates, slmc::kPhaseAll, lnw, s_cdw, n_acc,
                                     n_sweep_acc, obs, s));
    if (nupdates > 0) SLMC_LAUNCH(SLMC_PROF_ACCEPT, 1, s, slmc::counter_op(c, (uint64_t)nupdates, true, s));
    return SLMC_OK;
}

namespace {
// One FP64 step of the stabilised chain on the product already in Y: pivoted QR, Q, T.
int chain_step64(slmc_ctx* c, int nf, cudaStream_t s) {
    c->cur_units = nf;
    if (c->p.qr_mode == SLMC_QR_PIVOTED) {
        SLMC_LAUNCH(SLMC_PROF_QR, 1, s, slmc::qr_pivoted(c, nf, s));
        SLMC_LAUNCH(SLMC_PROF_FORMQ, 1, s, slmc::form_q(c, nf, s));
    } else {
        SLMC_LAUNCH(SLMC_PROF_QR, 1, s, slmc::qr_blocked(c, nf, s));
        SLMC_LAUNCH(SLMC_PROF_FORMQ, 1, s, slmc::form_q_blocked(c, nf, false, s));
    }
    SLMC_LAUNCH(SLMC_PROF_TUPDATE, 1, s, slmc::t_update_tiled(c, nf, s));
    return SLMC_OK;
}

// chain state (U, T, lnD) of fields [0, nf) into stack slot k
int stack_store(slmc_ctx* c, int k, int nf, cudaStream_t s) {
    const size_t NN = (size_t)c->N * c->N, F = c->max_fields;
    double* slot = c->dq_stack + (size_t)k * F * (2 * NN + c->N);
    SLMC_CK(cudaMemcpyAsync(slot, c->U, nf * NN * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SLMC_CK(cudaMemcpyAsync(slot + F * NN, c->Ta, nf * NN * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SLMC_CK(cudaMemcpyAsync(slot + 2 * F * NN, c->lnD, nf * c->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return SLMC_OK;
}
}  // namespace

int slmc_dqmc_sweep(slmc_ctx* c, double* x, int n, int nsweeps, uint64_t sweep0, int nblock, long long* n_acc_local,
                    long long* n_acc_block, void* stream) {
    if (!c || n < 0 || nsweeps < 0 || nblock < 0 || (n > 0 && !x)) return SLMC_ERR_ARG;
    if (!slmc::dqmc_ok(c)) return SLMC_ERR_UNSUPPORTED;
    const int ngroups = (c->L + c->p.n_s - 1) / c->p.n_s;
    if (!c->dq_stack) {  // the left-product stack, allocated on first use
        const size_t NN = (size_t)c->N * c->N;
        const size_t bytes = (size_t)ngroups * c->max_fields * (2 * NN + c->N) * sizeof(double);
        if (cudaMalloc(reinterpret_cast<void**>(&c->dq_stack), bytes) != cudaSuccess) {
            cudaGetLastError();
            c->dq_stack = nullptr;
            return SLMC_ERR_NOMEM;
        }
        c->dq_groups = ngroups;
    }
    const size_t NL = (size_t)c->N * c->L;
    cudaStream_t s = as_stream(stream);
    return for_batches(c, n, [&](int f0, int nf) {
        double* xc = x + (size_t)f0 * NL;
        for (int sw = 0; sw < nsweeps; ++sw) {
            const uint64_t sweep = sweep0 + (uint64_t)sw;
            // transposed left products B(L, g0)^T, g0 = k n_s, from the top group down
            const int ng = (c->L + c->p.n_s - 1) / c->p.n_s;
            c->cur_units = nf;
            SLMC_LAUNCH(SLMC_PROF_FINAL, 1, s, slmc::set_identity(c, nf, s));
            for (int k = ng - 1; k >= 0; --k) {
                const int l0 = k * c->p.n_s, nsl = std::min(c->p.n_s, c->L - l0);
                SLMC_LAUNCH(SLMC_PROF_SLICE, 1, s, slmc::slice_group_kron(c, xc, nf, l0, nsl, true, s));
                SLMC_TRY(chain_step64(c, nf, s));
                SLMC_TRY(stack_store(c, k, nf, s));
            }
            // upward pass: G(g0) from the running product B(g0, 0) and the stored B(L, g0), local
            // updates of the group's slices (G carried between them), then the group joins B(g0, 0)
            SLMC_LAUNCH(SLMC_PROF_FINAL, 1, s, slmc::set_identity(c, nf, s));
            for (int k = 0; k < ng; ++k) {
                const int l0 = k * c->p.n_s, nsl = std::min(c->p.n_s, c->L - l0);
                const size_t NN = (size_t)c->N * c->N, slot = (size_t)k * c->max_fields * (2 * NN + c->N);
                const double* Ul = c->dq_stack + slot;
                const double* Tl = Ul + (size_t)c->max_fields * NN;
                const double* lnDl = Tl + (size_t)c->max_fields * NN;
                SLMC_LAUNCH(SLMC_PROF_GREENS, 5, s,
                            slmc::dqmc_combine(c, Ul, lnDl, Tl, nf, c->QR, scal(c, 6), iscal(c, 3), s));
                SLMC_LAUNCH(SLMC_PROF_DQMC, 1, s,
                            slmc::dqmc_slices(c, xc, c->QR, nf, f0, l0, nsl, sweep,
                                              n_acc_local ? n_acc_local + f0 : nullptr, s));
                if (k + 1 == ng) break;
                SLMC_LAUNCH(SLMC_PROF_SLICE, 1, s, slmc::slice_group_kron(c, xc, nf, l0, nsl, false, s));
                SLMC_TRY(chain_step64(c, nf, s));
            }
            if (nblock == 0) continue;
            // block updates: reflect one column, accept with the ratio of the full weights
            SLMC_TRY(logdet_batch(c, xc, nf, scal(c, 0), iscal(c, 0), nullptr, s));
            SLMC_LAUNCH(SLMC_PROF_BOSE, 1, s, slmc::bose_log_weight(c, xc, nf, scal(c, 0), scal(c, 5), s));
            SLMC_CK(cudaMemsetAsync(scal(c, 1), 0, nf * sizeof(double), s));  // no effective-model terms
            SLMC_CK(cudaMemsetAsync(scal(c, 2), 0, nf * sizeof(double), s));
            for (int k = 0; k < nblock; ++k) {
                SLMC_CK(cudaMemcpyAsync(c->x_old, xc, nf * NL * sizeof(double), cudaMemcpyDeviceToDevice, s));
                c->cur_units = nf;
                SLMC_LAUNCH(SLMC_PROF_DQMC, 1, s, slmc::dqmc_block_propose(c, xc, nf, f0, sweep, k, scal(c, 4), s));
                SLMC_TRY(logdet_batch(c, xc, nf, scal(c, 0), iscal(c, 0), nullptr, s));
                SLMC_LAUNCH(SLMC_PROF_BOSE, 1, s, slmc::bose_log_weight(c, xc, nf, scal(c, 0), scal(c, 3), s));
                SLMC_LAUNCH(SLMC_PROF_ACCEPT, 2, s,
                            slmc::accept_update(c, nf, xc, c->x_old, scal(c, 3), scal(c, 1), scal(c, 2), scal(c, 4),
                                                scal(c, 5), iscal(c, 2), n_acc_block ? n_acc_block + f0 : nullptr, s));
            }
        }
        return SLMC_OK;
    });
}

int slmc_set_update_counter(slmc_ctx* c, uint64_t value, void* stream) {
    if (!c) return SLMC_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    SLMC_LAUNCH(SLMC_PROF_ACCEPT, 1, s, slmc::counter_op(c, value, false, s));
    return SLMC_OK;
}

int slmc_get_update_counter(slmc_ctx* c, uint64_t* value, void* stream) {
    if (!c || !value) return SLMC_ERR_ARG;
    unsigned long long v = 0;
    if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess ||
        cudaMemcpy(&v, c->dctr, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SLMC_ERR_CUDA;
    *value = v;
    return SLMC_OK;
}

int slmc_set_tuning(slmc_ctx* c, int qr_panel, int slice_cols) {
    if (!c || (qr_panel != 0 && qr_panel != 16 && qr_panel != 32) ||
        (slice_cols != 0 && slice_cols != 8 && slice_cols != 16))
        return SLMC_ERR_ARG;
    c->tune_qr_panel = qr_panel;
    c->tune_slice_cols = slice_cols;
    return SLMC_OK;
}

int slmc_set_slice_groups(slmc_ctx* c, int groups) {
    if (!c || groups < 0 || groups > 4 || groups == 3) return SLMC_ERR_ARG;
    c->tune_slice_groups = groups;
    return SLMC_OK;
}

int slmc_set_wolff(slmc_ctx* c, int nwolff) {
    if (!c || nwolff < 0 || nwolff > 64) return SLMC_ERR_ARG;
    c->nwolff = nwolff;
    return SLMC_OK;
}

int slmc_get_wolff_sites(slmc_ctx* c, long long* total, int reset, void* stream) {
    if (!c || !total) return SLMC_ERR_ARG;
    unsigned long long v = 0;
    if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess ||
        cudaMemcpy(&v, c->wolff_sites, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SLMC_ERR_CUDA;
    if (reset && cudaMemset(c->wolff_sites, 0, sizeof(v)) != cudaSuccess) return SLMC_ERR_CUDA;
    *total = (long long)v;
    return SLMC_OK;
}

int slmc_set_qr_cluster(slmc_ctx* c, int ctas) {
    if (!c || (ctas != 0 && ctas != 1 && ctas != 2 && ctas != 4)) return SLMC_ERR_ARG;
    c->tune_qr_cluster = ctas;
    return SLMC_OK;
}

int slmc_set_dense_slices(slmc_ctx* c, int dense) {
    if (!c || dense < 0 || dense > 1) return SLMC_ERR_ARG;
    c->dense_slices = dense;
    return SLMC_OK;
}

int slmc_set_tupdate_path(slmc_ctx* c, int path) {
    if (!c || path < 0 || path > 2) return SLMC_ERR_ARG;
    if (path != 1 && !c->tt_A) return SLMC_ERR_UNSUPPORTED;
    c->tt_path = path;
    return SLMC_OK;
}

int slmc_set_qr_path(slmc_ctx* c, int path) {
    if (!c || path < 0 || path > 1) return SLMC_ERR_ARG;
    if (path == 0 && !c->qt_buf) return SLMC_ERR_UNSUPPORTED;
    c->qr_path = path;
    return SLMC_OK;
}

int slmc_set_sub_batch_priorities(slmc_ctx* c, int on) {
    if (!c || on < 0 || on > 1) return SLMC_ERR_ARG;
    if (on && c->nsub_avail == 0) return SLMC_ERR_UNSUPPORTED;
    c->sub_prio = on;
    return SLMC_OK;
}

int slmc_set_sub_batches(slmc_ctx* c, int n) {
    if (!c || n < 1 || n > slmc_ctx::kMaxSub) return SLMC_ERR_ARG;
    if (n > 1 && c->nsub_avail < n) return SLMC_ERR_UNSUPPORTED;
    c->nsub = n;
    return SLMC_OK;
}

int slmc_fit_eff(slmc_ctx* c, const double* xs, const double* lnw, int nconf, double* J_out, double* resid,
                 void* stream) {
    if (!c || nconf < 6 || !xs || !lnw || !J_out) return SLMC_ERR_ARG;
    const size_t NL = (size_t)c->N * c->L;
    cudaStream_t s = as_stream(stream);
    SLMC_LAUNCH(SLMC_PROF_FIT, 1, s, slmc::fit_begin(c, c->fitR, s));
    SLMC_TRY(for_batches(c, nconf, [&](int f0, int nf) {
        SLMC_LAUNCH(SLMC_PROF_EFF, 1, s, slmc::eff_features(c, xs + f0 * NL, nf, nullptr, c->feat, 8, nullptr, s));
        SLMC_LAUNCH(SLMC_PROF_FIT, 1, s, slmc::fit_accumulate(c, c->fitR, c->feat, lnw + f0, nf, s));
        return SLMC_OK;
    }));
    SLMC_LAUNCH(SLMC_PROF_FIT, 1, s, slmc::fit_finish(c, nconf, J_out, resid, s));
    return SLMC_OK;
}

int slmc_fit_eff_state(slmc_ctx* c, const double* xs, const double* lnw, int nconf, double* state, void* stream) {
    if (!c || nconf < 0 || !state || (nconf > 0 && (!xs || !lnw))) return SLMC_ERR_ARG;
    const size_t NL = (size_t)c->N * c->L;
    cudaStream_t s = as_stream(stream);
    SLMC_LAUNCH(SLMC_PROF_FIT, 1, s, slmc::fit_begin(c, state, s));
    SLMC_TRY(for_batches(c, nconf, [&](int f0, int nf) {
        SLMC_LAUNCH(SLMC_PROF_EFF, 1, s, slmc::eff_features(c, xs + f0 * NL, nf, nullptr, c->feat, 8, nullptr, s));
        SLMC_LAUNCH(SLMC_PROF_FIT, 1, s, slmc::fit_accumulate(c, state, c->feat, lnw + f0, nf, s));
        return SLMC_OK;
    }));
    return SLMC_OK;
}

int slmc_fit_eff_merge(slmc_ctx* c, const double* states, int nparts, double* J_out, double* resid, void* stream) {
    if (!c || !states || nparts < 1 || !J_out) return SLMC_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    SLMC_LAUNCH(SLMC_PROF_FIT, 1, s, slmc::fit_merge(c, states, nparts, s));
    SLMC_LAUNCH(SLMC_PROF_FIT, 1, s, slmc::fit_finish(c, 0, J_out, resid, s));
    return SLMC_OK;
}

int slmc_measure_cdw(slmc_ctx* c, const double* G, int n, double* S, void* stream) {
    if (!c || n < 0 || (n > 0 && (!G || !S))) return SLMC_ERR_ARG;
    if (n == 0) return SLMC_OK;
    cudaStream_t s = as_stream(stream);
    SLMC_LAUNCH(SLMC_PROF_CDW, 1, s, slmc::cdw_measure(c, G, n, S, nullptr, nullptr, s));
    return SLMC_OK;
}

long long slmc_launch_count(slmc_ctx* c) { return c ? c->launches : 0; }

int slmc_profile_enable(slmc_ctx* c, int on) {
    if (!c) return SLMC_ERR_ARG;
    if (on) {
        SLMC_TRY(flush_profile(c));
        for (int q = 0; q < SLMC_PROF_NCLASS; ++q) {
            c->prof_ms[q] = 0.0;
            c->prof_calls[q] = 0;
            c->prof_busy[q] = 0.0;
            c->prof_units[q] = 0;
        }
        // time origin: recorded and completed before any call timed from now on
        if (!c->prof_base && cudaEventCreate(&c->prof_base) != cudaSuccess) return SLMC_ERR_CUDA;
        if (cudaEventRecord(c->prof_base, 0) != cudaSuccess || cudaEventSynchronize(c->prof_base) != cudaSuccess)
            return SLMC_ERR_CUDA;
    }
    c->prof_on = on != 0;
    return SLMC_OK;
}

int slmc_profile_read(slmc_ctx* c, double* ms, long long* calls, void* stream) {
    return slmc_profile_read_detail(c, ms, calls, nullptr, nullptr, stream);
}

int slmc_profile_read_detail(slmc_ctx* c, double* ms, long long* calls, double* busy_ms, long long* units,
                             void* stream) {
    if (!c || !ms) return SLMC_ERR_ARG;
    if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return SLMC_ERR_CUDA;
    SLMC_TRY(flush_profile(c));
    for (int q = 0; q < SLMC_PROF_NCLASS; ++q) {
        ms[q] = c->prof_ms[q];
        if (calls) calls[q] = c->prof_calls[q];
        if (busy_ms) busy_ms[q] = c->prof_busy[q];
        if (units) units[q] = c->prof_units[q];
    }
    return SLMC_OK;
}

}  // extern "C"
