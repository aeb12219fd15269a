// peak.cu -- microbenchmark of the 32-bit integer multiply-add rate, the
// denominator of the integer roofline the butterfly kernels are reported
// against (each Shoup butterfly issues three 32-bit multiplies).
//
// Every thread runs eight independent chains x <- x * m + c (mad.lo.u32 or
// mad.hi.u32 in inline PTX, m and c run-time values so nothing folds) for
// `iters` rounds; the grid covers every SM several times over.  The result
// words depend on every step, so no step can be dropped.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/ntt.h"

namespace nttgb {
namespace {

template <bool HI>
__global__ void __launch_bounds__(256) k_imad_rate(uint32_t *out, uint32_t m, uint32_t c, uint32_t iters) {
    uint32_t x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 8u + (uint32_t)i + blockIdx.x;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (HI) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[i]) : "r"(m), "r"(c));
            else asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[i]) : "r"(m), "r"(c));
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) r ^= x[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

}  // namespace
}  // namespace nttgb

extern "C" {

ntt_status ntt_measure_int_mad_rate(int high, uint32_t iters, void *d_scratch, size_t scratch_bytes,
                                    uint32_t *blocks_out, ntt_stream_t stream) {
    if (!d_scratch || !blocks_out || iters == 0) return NTT_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return NTT_ERR_CUDA;
    }
    const uint32_t blocks = (uint32_t)sms * 8u;
    if (scratch_bytes < (size_t)blocks * 256 * sizeof(uint32_t)) return NTT_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint32_t *out = reinterpret_cast<uint32_t *>(d_scratch);
    if (high) nttgb::k_imad_rate<true><<<blocks, 256, 0, st>>>(out, 0x9E3779B1u, 12345u, iters);
    else nttgb::k_imad_rate<false><<<blocks, 256, 0, st>>>(out, 0x9E3779B1u, 12345u, iters);
    if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
    *blocks_out = blocks;
    return NTT_OK;
}

}  // extern "C"
