// Instantiates the ragged persistent kernel for 8-byte words with RED_MONTGOMERY.
#include "ragged_kernel.cuh"

namespace nttgb {
template cudaError_t ragged_kernel_launch<RED_MONTGOMERY, uint64_t>(const RaggedArgs &, unsigned, cudaStream_t);
template cudaError_t ragged_kernel_config<RED_MONTGOMERY, uint64_t>(size_t *, int *);
}
