// Instantiates the fused path for uint64_t words with RED_BARRETT.
#include "fused_launch.cuh"

namespace nttgb {
template cudaError_t run_fused_t<uint64_t, RED_BARRETT>(ntt_plan_s &, void *, uint32_t, bool, cudaStream_t);
template cudaError_t run_fused_pwinv_t<uint64_t, RED_BARRETT>(ntt_plan_s &, void *, const void *, const void *, uint32_t,
                                                      cudaStream_t);
}
