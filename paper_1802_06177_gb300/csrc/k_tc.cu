// Tensor-core (tcgen05) slice-group products in split precision: placeholder until the
// kernels land; slmc_init rejects SLMC_PREC_TF32X3 / SLMC_PREC_BF16X9 meanwhile.
#include "slmc_internal.cuh"

namespace slmc {

cudaError_t tc_slice_group(slmc_ctx*, const double*, int, int, int, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace slmc
