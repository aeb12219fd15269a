// Instantiates the ragged persistent kernel with RED_BARRETT.
#include "ragged_kernel.cuh"

namespace nttgb {
template cudaError_t ragged_kernel_launch<RED_BARRETT>(const RaggedArgs &, unsigned, cudaStream_t);
template cudaError_t ragged_kernel_config<RED_BARRETT>(size_t *, int *);
}
