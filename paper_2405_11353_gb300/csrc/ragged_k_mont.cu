// Instantiates the ragged persistent kernel with RED_MONTGOMERY.
#include "ragged_kernel.cuh"

namespace nttgb {
template cudaError_t ragged_kernel_launch<RED_MONTGOMERY>(const RaggedArgs &, unsigned, cudaStream_t);
template cudaError_t ragged_kernel_config<RED_MONTGOMERY>(size_t *, int *);
}
