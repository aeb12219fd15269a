// Instantiates the ragged persistent kernel for 4-byte words with RED_BARRETT.
#include "ragged_kernel.cuh"

namespace nttgb {
template cudaError_t ragged_kernel_launch<RED_BARRETT, uint32_t>(const RaggedArgs &, unsigned, cudaStream_t);
template cudaError_t ragged_kernel_config<RED_BARRETT, uint32_t>(size_t *, int *);
}
