// Allocation-free variant of slmc_logdet (see slmc_logdet_noalloc in include/slmc.h).
//
// Some callers cannot allocate device memory at the point where they need a determinant:
// code that runs while a stream is being captured into a CUDA graph (cudaMalloc is not a
// stream operation and may synchronise the device), latency-critical loops that must not
// hit the allocator or an implicit device synchronisation, and hosts that own the whole
// device memory budget through their own allocator and forbid foreign allocations. For them
// this entry point keeps all of its workspace in one fixed, file-scope device array.
//
// The array lives in every GPU that loads the library until the process exits. Its device
// address is looked up once per device (cudaGetSymbolAddress on the first call with that
// device current) and cached, so a device reset (cudaDeviceReset) or a new primary context on
// that device invalidates it for the rest of the process; in host code the symbol itself is only a host-side stand-in
// and must never be passed to a kernel. The first call on a device should therefore happen
// before any stream capture. Every call reuses the same array: the parts that must start
// at zero (the error word) are cleared on the stream at the start of each call, everything
// else is fully written before it is read. Calls that overlap on the GPU (different
// streams, or different threads) race on the array and must be serialised by the caller.
#include <mutex>

#include "slmc_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // 16 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

unsigned char* g_scratch_addr[kMaxDevices];
int g_num_sms[kMaxDevices];
std::mutex g_scratch_mutex;

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes of the per-context part (E, F, the circulant factors, error word) and of one field's workspace.
size_t fixed_bytes(size_t N) {
    const size_t S = N < (size_t)slmc::kLoStencil ? N : (size_t)slmc::kLoStencil;
    return align256(N * N * sizeof(double)) + align256(N * N * sizeof(float)) +
           align256((S * N + S) * sizeof(int)) + align256(S * sizeof(float)) +
           align256(4 * slmc::kKronTab * sizeof(double)) + 256;
}
// L > 0 (FP32 mode): also the FP32 slice scales and the FP32 orthogonal factor.
size_t field_bytes(size_t N, size_t L) {
    return 5 * N * N * sizeof(double) + 32 * N * sizeof(double) + 2 * N * sizeof(double) + 2 * N * sizeof(int) +
           sizeof(int) + L * N * sizeof(float) + (L ? N * N * sizeof(float) : 0);
}

// Device address of the array and the multiprocessor count of the current device, looked up
// once per device (with that device current) and cached.
int scratch_address(int device, unsigned char** out, int* num_sms) {
    if (device < 0 || device >= kMaxDevices) return SLMC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void* ptr = nullptr;
        int sms = 0;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
            return SLMC_ERR_CUDA;
        g_scratch_addr[device] = static_cast<unsigned char*>(ptr);
        g_num_sms[device] = sms;
    }
    *out = g_scratch_addr[device];
    *num_sms = g_num_sms[device];
    return SLMC_OK;
}

}  // namespace

extern "C" {

size_t slmc_logdet_noalloc_scratch_bytes(void) { return kScratchBytes; }

int slmc_logdet_noalloc(const slmc_params* p, const double* x, int n, double* lndet, int* sign, void* stream) {
    int st = slmc::validate_params(p);
    if (st != SLMC_OK) return st;
    if (n < 0 || (n > 0 && (!x || !lndet || !sign))) return SLMC_ERR_ARG;
    if (p->precision != SLMC_PREC_FP64 && p->precision != SLMC_PREC_FP32) return SLMC_ERR_UNSUPPORTED;
    const size_t N = (size_t)p->Lx * p->Ly;
    const size_t Lz = p->precision == SLMC_PREC_FP32 ? (size_t)p->L : 0;  // slice scales (FP32 mode only)
    if (fixed_bytes(N) + field_bytes(N, Lz) > kScratchBytes) return SLMC_ERR_UNSUPPORTED;  // one field must fit
    if (n == 0) return SLMC_OK;
    const int capacity = (int)((kScratchBytes - fixed_bytes(N)) / field_bytes(N, Lz));

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return SLMC_ERR_CUDA;
    unsigned char* base = nullptr;
    int num_sms = 0;
    st = scratch_address(device, &base, &num_sms);
    if (st != SLMC_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    // Context view over the static array: no member owns memory.
    slmc_ctx c{};
    c.p = *p;
    c.N = (int)N;
    c.L = p->L;
    c.max_fields = capacity < n ? capacity : n;
    c.device = device;
    c.num_sms = num_sms;  // lets few fields spread their QR over clusters of CTAs, as in slmc_logdet
    const size_t NN = N * N, F = (size_t)c.max_fields;
    unsigned char* q = base;
    auto take = [&](size_t bytes) { unsigned char* r = q; q += align256(bytes); return r; };
    c.E64 = reinterpret_cast<double*>(take(NN * sizeof(double)));
    c.F32 = reinterpret_cast<float*>(take(NN * sizeof(float)));
    if (Lz) {  // stencil of F's FP32 rounding residual (FP32 mode)
        c.lo_S = (int)(N < (size_t)slmc::kLoStencil ? N : (size_t)slmc::kLoStencil);
        c.lo_kidx = reinterpret_cast<int*>(take(((size_t)c.lo_S * N + c.lo_S) * sizeof(int)));
        c.lo_val = reinterpret_cast<float*>(take((size_t)c.lo_S * sizeof(float)));
    }
    // the circulant factors of exp(-dtau K): FP64 slice products through them, as in slmc_logdet
    if (p->Lx <= slmc::kKronMaxLine && p->Ly <= slmc::kKronMaxLine)
        c.kron = reinterpret_cast<double*>(take(4 * slmc::kKronTab * sizeof(double)));
    c.err = reinterpret_cast<unsigned int*>(take(sizeof(unsigned int)));
    c.Y = reinterpret_cast<double*>(q);
    c.QR = c.Y + F * NN;
    c.U = c.QR + F * NN;
    c.Ta = c.U + F * NN;
    c.Tb = c.Ta + F * NN;
    c.Sws = c.Tb + F * NN;
    c.lnD = c.Sws + F * N * 32;
    c.tau = c.lnD + F * N;
    c.perm = reinterpret_cast<int*>(c.tau + F * N);
    c.piv = c.perm + F * N;
    c.sgnU = c.piv + F * N;
    c.sc32 = Lz ? reinterpret_cast<float*>(c.sgnU + F) : nullptr;
    c.U32 = Lz ? c.sc32 + F * Lz * N : nullptr;

    if (cudaMemsetAsync(c.err, 0, sizeof(unsigned int), s) != cudaSuccess) return SLMC_ERR_CUDA;
    if (slmc::build_hopping_exp(&c, s) != cudaSuccess) return SLMC_ERR_CUDA;
    const size_t NL = N * (size_t)p->L;
    for (int f0 = 0; f0 < n; f0 += c.max_fields) {
        const int nf = (n - f0) < c.max_fields ? (n - f0) : c.max_fields;
        st = slmc::logdet_fields(&c, x + f0 * NL, nf, lndet + f0, sign + f0, s);
        if (st != SLMC_OK) return st;
    }
    return SLMC_OK;
}

}  // extern "C"
