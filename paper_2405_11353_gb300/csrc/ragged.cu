// ragged.cu -- heterogeneous batches in one persistent launch (placeholder
// until the persistent kernel lands; every entry point reports
// NTT_ERR_UNSUPPORTED).
#include "plan.hpp"

struct ntt_ragged_s { int unused; };

extern "C" {
ntt_status ntt_ragged_create(ntt_ragged_t *out, const ntt_job *, uint32_t, uint32_t) {
    if (out) *out = nullptr;
    return NTT_ERR_UNSUPPORTED;
}
ntt_status ntt_ragged_launch(ntt_ragged_t, ntt_stream_t) { return NTT_ERR_UNSUPPORTED; }
ntt_status ntt_ragged_status(ntt_ragged_t, ntt_stream_t) { return NTT_ERR_UNSUPPORTED; }
void ntt_ragged_destroy(ntt_ragged_t) {}
}
