// Instantiates the chunk passes of the shuffle forms for uint32_t words
// with RED_SHOUP (exchanges between rounds by warp shuffles).
#define NTTGB_SHFL_UNIT
#include "fused_launch.cuh"

namespace nttgb {
template cudaError_t run_chunk_pass_shfl<uint32_t, RED_SHOUP, false, 64>(ntt_plan_s &, int, uint32_t *, const void *,
                                                                 uint64_t, bool, cudaStream_t, uint32_t *,
                                                                 const uint32_t *);
template cudaError_t run_chunk_pass_shfl<uint32_t, RED_SHOUP, true, 64>(ntt_plan_s &, int, uint32_t *, const void *,
                                                                uint64_t, bool, cudaStream_t, uint32_t *,
                                                                const uint32_t *);
template cudaError_t run_chunk_pass_shfl<uint32_t, RED_SHOUP, false, 80>(ntt_plan_s &, int, uint32_t *, const void *,
                                                                 uint64_t, bool, cudaStream_t, uint32_t *,
                                                                 const uint32_t *);
template cudaError_t run_chunk_pass_shfl<uint32_t, RED_SHOUP, true, 80>(ntt_plan_s &, int, uint32_t *, const void *,
                                                                uint64_t, bool, cudaStream_t, uint32_t *,
                                                                const uint32_t *);
}
