// tcgen05 BF16 GEMM for the dense backflow layers (placeholder until the tensor-core kernel
// lands: every shape is declined and the SIMT kernel runs).
#include "ansatz.cuh"

int gemm_bf16_tc(const GemmArgs& g, bool out_bf16, cudaStream_t s) {
    (void)g;
    (void)out_bf16;
    (void)s;
    return NQS_ERR_UNSUPPORTED;
}
