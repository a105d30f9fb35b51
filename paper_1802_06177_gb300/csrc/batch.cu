// Batches of independent chains of uneven lattice size and slice count, advanced together
// through one captured CUDA graph, and the autotuner of the stabilisation interval and
// kernel tiles.
//
// A batch holds one context per lattice class (its own workspace and exp(-dtau K)) and one
// stream per class. slmc_batch_capture records a round (nupdates cumulative updates of every
// class) into a graph replayed by one launch per round; because each context draws its random
// numbers from a device-side update counter that the round advances, replays continue the
// Philox streams exactly as successive direct calls would. Each update of the round is
//   (1) per class, on its own branch: the update's draws, the saved field, F(x) of E_eff;
//   (2) one persistent launch (k_sweep_queue) that runs the E_eff Markov chain of every chain of
//       every class: half-sweep slabs and Wolff updates pulled from a device work queue in which
//       the chains stand in order of decreasing N L (longest first), phase after phase;
//   (3) per class, on its own branch: F(x'), ln w with G, the acceptance [Eq. (6)] and S.
// With the queue switched off, (2) is the kernel-per-half-sweep sequence of each class on its
// branch, as in slmc_cumulative_update.
//
// slmc_autotune picks, for one class, the stabilisation interval n_s (and the blocked-QR panel
// width and FP32 slice tile) that evaluates ln det fastest while agreeing with the library's
// FP64 path on synthetic fields within a tolerance.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "slmc_internal.cuh"

struct slmc_batch {
    struct Bind {
        double* x = nullptr;
        const double* J = nullptr;
        double* lnw = nullptr;
        double* s_cdw = nullptr;
        long long* n_acc = nullptr;
        long long* n_sweep_acc = nullptr;
    };
    std::vector<slmc_ctx*> ctx;
    std::vector<int> nchains;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    std::vector<Bind> bind;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // persistent sweep queue
    bool queue = true;
    long long stall_cycles = 0;  // > 0: the first item waits for a count nothing reaches (test hook)
    slmc::QueueClass* d_cls = nullptr;
    int4* d_items = nullptr;
    unsigned int* d_done = nullptr;  // per-chain completion counters
    unsigned int* d_ctl = nullptr;   // [0] queue head, [1] abort
};

namespace {

void free_queue(slmc_batch* b) {
    cudaFree(b->d_cls);
    cudaFree(b->d_items);
    cudaFree(b->d_done);
    cudaFree(b->d_ctl);
    b->d_cls = nullptr;
    b->d_items = nullptr;
    b->d_done = nullptr;
    b->d_ctl = nullptr;
}

void release(slmc_batch* b) {
    free_queue(b);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (slmc_ctx* c : b->ctx) slmc_destroy(c);
    delete b;
}

// Gaussian fields x ~ N(0, 1) from Philox-4x32-10 by the Box-Muller transform (tuning input).
__global__ void k_gauss(double* __restrict__ x, size_t total, uint32_t key0, uint32_t key1) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const slmc::u32x4 w = slmc::philox4x32_10(slmc::u32x4{(uint32_t)i, (uint32_t)(i >> 32), 0u, 2u}, key0, key1);
        const double u1 = 1.0 - slmc::uniform53(w.x, w.y);  // (0, 1]
        const double u2 = slmc::uniform53(w.z, w.w);
        x[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
}


constexpr long long kQueueWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

// Host-built item table of one update of the sweep queue and its class descriptors (see
// k_sweep_queue): for every sweep, the phases colour 0, Wolff update 0 .. W-1, colour 1; within a
// phase the chains in order of decreasing N L, each with its slabs of kQueueSlab sites (or its one
// Wolff item), all carrying the count of the chain's items in earlier phases.
struct QueuePlan {
    std::vector<slmc::QueueClass> cls;
    std::vector<int4> items;
    int nchains = 0;
    int max_N = 0;
};

QueuePlan plan_queue(slmc_batch* b, int nsweeps) {
    QueuePlan P;
    const int ncls = (int)b->ctx.size();
    std::vector<int> order(ncls);
    int maxw = 0;
    for (int q = 0; q < ncls; ++q) {
        slmc_ctx* c = b->ctx[q];
        const auto& bd = b->bind[q];
        slmc::QueueClass C{};
        C.x = bd.x;
        C.J = bd.J;
        C.first_colour = slmc::first_colours(c);
        C.n_acc = reinterpret_cast<unsigned long long*>(bd.n_sweep_acc);
        C.wolff_sites = c->wolff_sites;
        C.dctr = c->dctr;
        C.err = c->err;
        C.Lx = c->p.Lx;
        C.Ly = c->p.Ly;
        C.L = c->L;
        C.nsweeps = nsweeps;
        C.nwolff = c->nwolff;
        C.done0 = P.nchains;
        const double a = c->p.lambda / (c->p.omega0 * c->p.omega0);
        C.dtau = c->p.dtau;
        C.a2 = a * a;
        C.delta = c->p.sweep_delta;
        C.key0 = (uint32_t)(c->p.seed & 0xffffffffu);
        C.key1 = (uint32_t)(c->p.seed >> 32);
        P.cls.push_back(C);
        P.nchains += b->nchains[q];
        P.max_N = std::max(P.max_N, c->N);
        maxw = std::max(maxw, c->nwolff);
        order[q] = q;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (long long)b->ctx[a]->N * b->ctx[a]->L > (long long)b->ctx[c]->N * b->ctx[c]->L;
    });
    std::vector<int> need(P.nchains, 0);
    for (int sw = 0; sw < nsweeps; ++sw)
        for (int ph = 0; ph < maxw + 2; ++ph) {  // 0: colour 0, 1..maxw: Wolff ph-1, maxw+1: colour 1
            const bool wolff = ph > 0 && ph <= maxw;
            for (int q : order) {
                const slmc::QueueClass& C = P.cls[q];
                if (wolff && ph - 1 >= C.nwolff) continue;
                const int sites = C.Lx * C.Ly * (C.L / 2);
                const int nslab = wolff ? 1 : (sites + slmc::kQueueSlab - 1) / slmc::kQueueSlab;
                const int y = (sw << 8) | (wolff ? (0x80 | (ph - 1)) : (ph == 0 ? 0 : 1));
                for (int f = 0; f < b->nchains[q]; ++f) {
                    const int g = C.done0 + f;
                    for (int z = 0; z < nslab; ++z) P.items.push_back(make_int4((q << 24) | f, y, z, need[g]));
                    need[g] += nslab;
                }
            }
        }
    return P;
}

// Uploads the plan for captured rounds; the launch itself is recorded by the caller.
int upload_queue(slmc_batch* b, const QueuePlan& P) {
    free_queue(b);
    const size_t ni = std::max<size_t>(P.items.size(), 1);
    if (cudaMalloc(&b->d_cls, P.cls.size() * sizeof(slmc::QueueClass)) != cudaSuccess ||
        cudaMalloc(&b->d_items, ni * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(&b->d_done, std::max(P.nchains, 1) * sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&b->d_ctl, 2 * sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        free_queue(b);
        return SLMC_ERR_NOMEM;
    }
    std::vector<int4> items = P.items;
    if (b->stall_cycles > 0 && !items.empty()) items[0].w = 0x7fffffff;
    if (cudaMemcpy(b->d_cls, P.cls.data(), P.cls.size() * sizeof(slmc::QueueClass), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        (!items.empty() &&
         cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemset(b->d_ctl, 0, 2 * sizeof(unsigned int)) != cudaSuccess)
        return SLMC_ERR_CUDA;
    return SLMC_OK;
}

}  // namespace

extern "C" {

int slmc_batch_create(const slmc_params* classes, const int* nchains, int nclasses, slmc_batch** out) {
    if (!out || !classes || !nchains || nclasses < 1) return SLMC_ERR_ARG;
    *out = nullptr;
    slmc_batch* b = new (std::nothrow) slmc_batch();
    if (!b) return SLMC_ERR_NOMEM;
    for (int c = 0; c < nclasses; ++c) {
        slmc_ctx* ctx = nullptr;
        const int st = nchains[c] < 1 ? SLMC_ERR_ARG : slmc_init(&classes[c], nchains[c], &ctx);
        if (st != SLMC_OK) {
            release(b);
            return st;
        }
        b->ctx.push_back(ctx);
        b->nchains.push_back(nchains[c]);
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            if (s) cudaStreamDestroy(s);
            release(b);
            return SLMC_ERR_CUDA;
        }
        b->streams.push_back(s);
        b->join.push_back(e);
    }
    b->bind.resize(nclasses);
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        release(b);
        return SLMC_ERR_CUDA;
    }
    *out = b;
    return SLMC_OK;
}

int slmc_batch_destroy(slmc_batch* b) {
    if (!b) return SLMC_OK;
    const cudaError_t e = cudaDeviceSynchronize();
    release(b);
    return e == cudaSuccess ? SLMC_OK : SLMC_ERR_CUDA;
}

slmc_ctx* slmc_batch_context(slmc_batch* b, int cls) {
    if (!b || cls < 0 || cls >= (int)b->ctx.size()) return nullptr;
    return b->ctx[cls];
}

int slmc_batch_bind(slmc_batch* b, int cls, double* x, const double* J, double* lnw, double* s_cdw, long long* n_acc,
                    long long* n_sweep_acc) {
    if (!b || cls < 0 || cls >= (int)b->ctx.size() || !x || !J || !lnw) return SLMC_ERR_ARG;
    b->bind[cls] = slmc_batch::Bind{x, J, lnw, s_cdw, n_acc, n_sweep_acc};
    return SLMC_OK;
}

int slmc_batch_capture(slmc_batch* b, int nsweeps, int nupdates, void* stream) {
    if (!b || !stream || nsweeps < 0 || nupdates < 1) return SLMC_ERR_ARG;
    for (const auto& bd : b->bind)
        if (!bd.x) return SLMC_ERR_ARG;
    cudaStream_t main = reinterpret_cast<cudaStream_t>(stream);
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    const int ncls = (int)b->ctx.size();
    QueuePlan plan;
    int grid = 0;
    if (b->queue) {
        plan = plan_queue(b, nsweeps);
        grid = slmc::sweep_queue_grid();
        if (grid < 1) return SLMC_ERR_CUDA;
        const int st = upload_queue(b, plan);
        if (st != SLMC_OK) return st;
    }
    const long long wait = b->stall_cycles > 0 ? b->stall_cycles : kQueueWaitCycles;
    // runs `phases` of update u of every class as concurrent branches forked from and joined to main
    auto branches = [&](int u, int phases) -> int {
        if (cudaEventRecord(b->fork, main) != cudaSuccess) return SLMC_ERR_CUDA;
        for (int c = 0; c < ncls; ++c) {
            const auto& bd = b->bind[c];
            if (cudaStreamWaitEvent(b->streams[c], b->fork, 0) != cudaSuccess) return SLMC_ERR_CUDA;
            const int st = slmc::cumulative_phases(b->ctx[c], bd.x, b->nchains[c], bd.J, nsweeps, u, u + 1, phases,
                                                   bd.lnw, bd.s_cdw, bd.n_acc, bd.n_sweep_acc, nullptr, b->streams[c]);
            if (st != SLMC_OK) return st;
            if (cudaEventRecord(b->join[c], b->streams[c]) != cudaSuccess ||
                cudaStreamWaitEvent(main, b->join[c], 0) != cudaSuccess)
                return SLMC_ERR_CUDA;
        }
        return SLMC_OK;
    };
    if (cudaStreamBeginCapture(main, cudaStreamCaptureModeRelaxed) != cudaSuccess) return SLMC_ERR_CUDA;
    int st = SLMC_OK;
    for (int u = 0; u < nupdates && st == SLMC_OK; ++u) {
        if (!b->queue) {
            st = branches(u, slmc::kPhaseAll);
            continue;
        }
        st = branches(u, slmc::kPhasePre);
        if (st == SLMC_OK && (cudaMemsetAsync(b->d_done, 0, std::max(plan.nchains, 1) * sizeof(unsigned int), main) !=
                                  cudaSuccess ||
                              cudaMemsetAsync(b->d_ctl, 0, sizeof(unsigned int), main) != cudaSuccess))
            st = SLMC_ERR_CUDA;
        if (st == SLMC_OK && slmc::sweep_queue(b->d_cls, ncls, b->d_items, (int)plan.items.size(), b->d_done, b->d_ctl,
                                               plan.max_N, (uint32_t)u, wait, grid, main) != cudaSuccess)
            st = SLMC_ERR_CUDA;
        if (st == SLMC_OK) st = branches(u, slmc::kPhasePost);
    }
    for (int c = 0; c < ncls && st == SLMC_OK; ++c)
        if (slmc::counter_op(b->ctx[c], (uint64_t)nupdates, true, main) != cudaSuccess) st = SLMC_ERR_CUDA;
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(main, &g);
    if (st == SLMC_OK && ec != cudaSuccess) st = SLMC_ERR_CUDA;
    if (st == SLMC_OK && cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) st = SLMC_ERR_CUDA;
    if (st == SLMC_OK) b->graph = g;
    else if (g) cudaGraphDestroy(g);
    return st;
}

int slmc_batch_set_sweep_queue(slmc_batch* b, int on) {
    if (!b || (on != 0 && on != 1)) return SLMC_ERR_ARG;
    b->queue = on != 0;
    return SLMC_OK;
}

int slmc_batch_inject_stall(slmc_batch* b, long long wait_cycles) {
    if (!b || wait_cycles < 0) return SLMC_ERR_ARG;
    b->stall_cycles = wait_cycles;
    return SLMC_OK;
}

int slmc_batch_launch(slmc_batch* b, int nrounds, void* stream) {
    if (!b || !b->exec || nrounds < 0) return SLMC_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int r = 0; r < nrounds; ++r)
        if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return SLMC_ERR_CUDA;
    return SLMC_OK;
}

int slmc_autotune(const slmc_params* p, int ntune, double tol, slmc_tune_result* out) {
    if (!p || !out || ntune < 1 || !(tol > 0.0)) return SLMC_ERR_ARG;
    const size_t N = (size_t)p->Lx * p->Ly, L = (size_t)p->L, total = (size_t)ntune * N * L;
    double* x = nullptr;
    double* lnd = nullptr;
    int* sg = nullptr;
    if (cudaMalloc(&x, total * sizeof(double)) != cudaSuccess || cudaMalloc(&lnd, 2 * ntune * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&sg, ntune * sizeof(int)) != cudaSuccess) {
        cudaFree(x);
        cudaFree(lnd);
        return SLMC_ERR_NOMEM;
    }
    int st = SLMC_OK;
    std::vector<double> ref(ntune), got(ntune);
    slmc_tune_result best{};
    best.sec_per_eval = -1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_gauss<<<256, 256>>>(x, total, (uint32_t)(p->seed & 0xffffffffu) ^ 0x7a11u, (uint32_t)(p->seed >> 32));
    {  // FP64 reference at a short stabilisation interval
        slmc_params q = *p;
        q.precision = SLMC_PREC_FP64;
        q.n_s = (int)std::min<size_t>(4, L);
        slmc_ctx* c = nullptr;
        st = slmc_init(&q, ntune, &c);
        if (st == SLMC_OK) st = slmc_logdet(c, x, ntune, lnd, sg, nullptr);
        if (st == SLMC_OK && cudaMemcpy(ref.data(), lnd, ntune * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = SLMC_ERR_CUDA;
        slmc_destroy(c);
    }
    const int ns_cand[] = {4, 6, 8, 10, 12, 16, 20, 24, 32};
    const bool fp32 = p->precision == SLMC_PREC_FP32 && N <= 256;
    const bool blocked = p->qr_mode == SLMC_QR_PREPIVOT;
    for (int ns : ns_cand) {
        if (st != SLMC_OK || (size_t)ns > L) break;
        slmc_params q = *p;
        q.n_s = ns;
        slmc_ctx* c = nullptr;
        st = slmc_init(&q, ntune, &c);
        for (int panel : {16, 32}) {
            if (st != SLMC_OK || (!blocked && panel == 32)) break;
            for (int cols : {8, 16}) {
                if (st != SLMC_OK || (!fp32 && cols == 16)) break;
                st = slmc_set_tuning(c, blocked ? panel : 0, fp32 ? cols : 0);
                if (st == SLMC_OK) st = slmc_logdet(c, x, ntune, lnd + ntune, sg, nullptr);  // warm-up
                float ms = 0.f;
                if (st == SLMC_OK) {
                    cudaEventRecord(e0);
                    for (int r = 0; r < 2 && st == SLMC_OK; ++r) st = slmc_logdet(c, x, ntune, lnd + ntune, sg, nullptr);
                    cudaEventRecord(e1);
                    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                        st = SLMC_ERR_CUDA;
                }
                if (st == SLMC_OK &&
                    cudaMemcpy(got.data(), lnd + ntune, ntune * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
                    st = SLMC_ERR_CUDA;
                if (st != SLMC_OK) break;
                double err = 0.0;
                for (int f = 0; f < ntune; ++f) err = std::max(err, std::fabs(got[f] - ref[f]));
                if (!std::isfinite(err)) err = INFINITY;
                const double sec = ms / 1e3 / (2.0 * ntune);
                best.candidates += 1;
                if (err <= tol && (best.sec_per_eval < 0.0 || sec < best.sec_per_eval)) {
                    best.n_s = ns;
                    best.qr_panel = blocked ? panel : 0;
                    best.slice_cols = fp32 ? cols : 0;
                    best.sec_per_eval = sec;
                    best.max_abs_dlndet = err;
                }
            }
        }
        slmc_destroy(c);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(lnd);
    cudaFree(sg);
    if (st != SLMC_OK) return st;
    if (best.sec_per_eval < 0.0) return SLMC_ERR_UNSUPPORTED;  // no candidate met the tolerance
    *out = best;
    return SLMC_OK;
}

}  // extern "C"
