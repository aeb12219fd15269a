// Instantiates the cluster form (cluster.cuh) with RED_BARRETT.
#include "cluster.cuh"

namespace nttgb {
template <> cudaError_t run_cluster<RED_BARRETT>(ntt_plan_s &p, void *data, uint32_t batch, bool inverse, cudaStream_t st) {
    return run_cluster_t<RED_BARRETT>(p, data, batch, inverse, st);
}
}  // namespace nttgb
