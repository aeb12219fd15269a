// Instantiates the cluster form (cluster.cuh) with RED_SHOUP.
#include "cluster.cuh"

namespace nttgb {
template <> cudaError_t run_cluster<RED_SHOUP>(ntt_plan_s &p, void *data, uint32_t batch, bool inverse, cudaStream_t st) {
    return run_cluster_t<RED_SHOUP>(p, data, batch, inverse, st);
}
}  // namespace nttgb
