// Instantiates the ragged persistent kernel with RED_SHOUP.
#include "ragged_kernel.cuh"

namespace nttgb {
template cudaError_t ragged_kernel_launch<RED_SHOUP>(const RaggedArgs &, unsigned, cudaStream_t);
template cudaError_t ragged_kernel_config<RED_SHOUP>(size_t *, int *);
}
