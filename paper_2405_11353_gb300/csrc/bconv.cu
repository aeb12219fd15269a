// bconv.cu -- fast RNS base conversion on the integer pipes.
//
// The step after the inverse transform in RNS homomorphic schemes (Sec. I
// motivates the NTT with them; the paper defines no conversion): residues
// x_i = x mod q_i (i < L) of every coefficient become residues modulo a
// second basis p_j (j < K),
//     y_i = x_i qhat_i^-1 mod q_i,   z_j = sum_i y_i (qhat_i mod p_j) mod p_j,
// qhat_i = prod_{k != i} q_k.  z_j = (x + alpha Q) mod p_j for one integer
// 0 <= alpha < L.  Per coefficient it is an L-by-K matrix-vector product
// mod p_j: a thread owns one coefficient at a time (persistent grid, the
// next coefficient's words loaded while this one is converted), keeps its L
// values y_i in registers (L up to the template bucket LB) and runs the K
// rows, four at a time, against the matrix (qhat_i mod p_j) broadcast from
// shared memory.
// Products y_i m_ij < 2^60 accumulate in 64 bits, reduced (Barrett, 2^64 /
// p_j) every 12 terms so the sum never wraps.  Words are 4 bytes (primes
// below 2^30); reads and writes coalesce along the coefficients.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ntt.h"
#include "host_nt.hpp"
#include "modarith.cuh"

struct ntt_bconv_s {
    uint32_t L = 0, K = 0, N = 0;
    int device = 0;
    // device: [K][LB] matrix (qhat_i mod p_j, zero-padded), [L] Shoup pairs
    // of qhat_i^-1 mod q_i, [L] q_i, [K] p_j, [K] floor(2^64 / p_j)
    void *d_tab = nullptr;
    uint32_t lb = 0;              // padded row length of the matrix
    uint32_t last_launches = 0;
};

namespace nttgb {
namespace {

constexpr uint32_t kBcThreads = 256;
constexpr uint32_t kBcMaxL = 64, kBcMaxK = 64;

struct BcTab {
    const uint32_t *m;            // [K][LB]
    const uint32_t *qinv;         // [L][2]: value, Shoup companion
    const uint32_t *q;            // [L]
    const uint32_t *p;            // [K]
    const uint64_t *mu;           // [K]
};

__device__ __forceinline__ uint32_t bc_reduce64(uint64_t z, uint32_t p, uint64_t mu) {
    // floor(z / p) - 1 <= hi(z mu) <= floor(z / p): remainder in [0, 2p)
    const uint64_t qh = __umul64hi(z, mu);
    uint32_t r = (uint32_t)(z - qh * p);
    return r >= p ? r - p : r;
}

template <uint32_t LB>
__global__ void __launch_bounds__(kBcThreads, 2) k_bconv(const uint32_t *__restrict__ x, uint32_t *__restrict__ z,
                                                          BcTab t, uint32_t L, uint32_t K, uint32_t N,
                                                          uint64_t total) {
    // the matrix rows (K x LB words) in shared memory, read as broadcasts
    extern __shared__ __align__(16) uint32_t bc_smem[];
    uint32_t *sm = bc_smem;
    for (uint32_t e = threadIdx.x; e < K * LB; e += blockDim.x) sm[e] = t.m[e];
    __syncthreads();
    // persistent: a thread takes coefficients c, c + stride, ...; the words
    // of the next one are loaded while the current one is converted
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t xn[LB];
    auto load = [&](uint64_t cc) {
        const uint64_t b = cc / N, n = cc % N;
        const uint32_t *xc = x + b * L * N + n;
#pragma unroll
        for (uint32_t i = 0; i < LB; ++i) xn[i] = i < L ? __ldg(xc + (size_t)i * N) : 0u;
    };
    if (c < total) load(c);
    for (; c < total; c += stride) {
        uint32_t y[LB];
#pragma unroll
        for (uint32_t i = 0; i < LB; ++i) {
            y[i] = 0;
            if (i < L) {
                const uint32_t xi = xn[i];
                const uint32_t w = __ldg(t.qinv + 2 * i), wc = __ldg(t.qinv + 2 * i + 1), q = __ldg(t.q + i);
                uint32_t r = xi * w - __umulhi(xi, wc) * q;      // Shoup, in [0, 2q)
                y[i] = r >= q ? r - q : r;
            }
        }
        if (c + stride < total) load(c + stride);
        const uint64_t b = c / N, n = c % N;
        uint32_t *zc = z + b * K * N + n;
        for (uint32_t j0 = 0; j0 < K; j0 += 4) {
            uint64_t acc[4] = {0, 0, 0, 0};
            uint32_t pj[4];
            uint64_t muj[4];
#pragma unroll
            for (uint32_t r = 0; r < 4; ++r) {
                const uint32_t j = j0 + r < K ? j0 + r : K - 1;
                pj[r] = __ldg(t.p + j);
                muj[r] = __ldg(t.mu + j);
            }
#pragma unroll
            for (uint32_t i0 = 0; i0 < LB; i0 += 4) {
                if (i0 >= L) break;
#pragma unroll
                for (uint32_t r = 0; r < 4; ++r) {
                    const uint32_t j = j0 + r < K ? j0 + r : K - 1;
                    const uint4 mv = *reinterpret_cast<const uint4 *>(sm + j * LB + i0);
                    acc[r] += (uint64_t)y[i0] * mv.x + (uint64_t)y[i0 + 1] * mv.y + (uint64_t)y[i0 + 2] * mv.z +
                              (uint64_t)y[i0 + 3] * mv.w;
                }
                // at most 12 products (< 2^60 each) since the last reduction,
                // plus a remainder < 2^30: no wrap before the next one
                if ((i0 / 4) % 3 == 2) {
#pragma unroll
                    for (uint32_t r = 0; r < 4; ++r) acc[r] = bc_reduce64(acc[r], pj[r], muj[r]);
                }
            }
#pragma unroll
            for (uint32_t r = 0; r < 4; ++r)
                if (j0 + r < K) zc[(size_t)(j0 + r) * N] = bc_reduce64(acc[r], pj[r], muj[r]);
        }
    }
}

template <uint32_t LB> cudaError_t bc_launch(const ntt_bconv_s &p, const uint32_t *x, uint32_t *z, uint64_t total,
                                             cudaStream_t st) {
    BcTab t;
    const uint32_t *base = reinterpret_cast<const uint32_t *>(p.d_tab);
    t.m = base;
    t.qinv = base + (size_t)p.K * LB;
    t.q = t.qinv + 2 * p.L;
    t.p = t.q + p.L;
    t.mu = reinterpret_cast<const uint64_t *>(t.p + p.K + ((3 * p.L + p.K) & 1u));   // 8-byte aligned
    const size_t smem = (size_t)p.K * LB * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_bconv<LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // persistent grid: the CTAs that fit at once (or fewer, for small calls)
    static int resident = 0;
    if (!resident) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bconv<LB>, kBcThreads,
                                                                      (size_t)kBcMaxK * LB * sizeof(uint32_t));
        if (e != cudaSuccess) return e;
        resident = sms * (per_sm > 0 ? per_sm : 1);
    }
    uint64_t blocks = (total + kBcThreads - 1) / kBcThreads;
    if (blocks > (uint64_t)resident) blocks = (uint64_t)resident;
    k_bconv<LB><<<(unsigned)blocks, kBcThreads, smem, st>>>(x, z, t, p.L, p.K, p.N, total);
    return cudaGetLastError();
}

}  // namespace
}  // namespace nttgb

namespace H = nttgb::host;

extern "C" {

ntt_status ntt_bconv_create(ntt_bconv_t *out, const uint64_t *q, uint32_t L, const uint64_t *p, uint32_t K,
                            uint32_t N) {
    if (!out) return NTT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!q || !p || L == 0 || K == 0 || N == 0 || L > nttgb::kBcMaxL || K > nttgb::kBcMaxK)
        return NTT_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < L + K; ++i) {
        const uint64_t v = i < L ? q[i] : p[i - L];
        if (v < 3 || v >= (1ull << 30)) return NTT_ERR_Q_WIDTH;
        if (!H::is_prime(v)) return NTT_ERR_Q_NOT_PRIME;
    }
    for (uint32_t i = 0; i < L; ++i)
        for (uint32_t k = i + 1; k < L; ++k)
            if (q[i] == q[k]) return NTT_ERR_INVALID_ARG;       // a basis has distinct primes
    ntt_bconv_s *b = new (std::nothrow) ntt_bconv_s();
    if (!b) return NTT_ERR_OOM;
    b->L = L;
    b->K = K;
    b->N = N;
    b->lb = L <= 8 ? 8 : L <= 16 ? 16 : L <= 32 ? 32 : 64;
    cudaGetDevice(&b->device);
    // host tables
    const uint32_t LB = b->lb;
    const uint32_t pad = (3 * L + K) & 1u;     // the 64-bit constants start 8-byte aligned
    const size_t words = (size_t)K * LB + 2 * L + L + K + pad + 2 * (size_t)K;
    std::vector<uint32_t> h(words, 0);
    auto qhat_mod = [&](uint32_t i, uint64_t m) {
        uint64_t r = 1 % m;
        for (uint32_t k = 0; k < L; ++k)
            if (k != i) r = H::mulm(r, q[k] % m, m);
        return r;
    };
    for (uint32_t j = 0; j < K; ++j)
        for (uint32_t i = 0; i < L; ++i) h[(size_t)j * LB + i] = (uint32_t)qhat_mod(i, p[j]);
    uint32_t *qinv = h.data() + (size_t)K * LB;
    for (uint32_t i = 0; i < L; ++i) {
        const uint64_t v = H::invm(qhat_mod(i, q[i]), q[i]);
        qinv[2 * i] = (uint32_t)v;
        qinv[2 * i + 1] = (uint32_t)(((unsigned __int128)v << 32) / q[i]);
    }
    uint32_t *qv = qinv + 2 * L, *pv = qv + L;
    for (uint32_t i = 0; i < L; ++i) qv[i] = (uint32_t)q[i];
    for (uint32_t j = 0; j < K; ++j) pv[j] = (uint32_t)p[j];
    uint64_t *mu = reinterpret_cast<uint64_t *>(pv + K + pad);
    for (uint32_t j = 0; j < K; ++j) mu[j] = (uint64_t)(((unsigned __int128)1 << 64) / p[j]);
    if (cudaMalloc(&b->d_tab, words * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return NTT_ERR_OOM;
    }
    if (cudaMemcpy(b->d_tab, h.data(), words * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b->d_tab);
        delete b;
        return NTT_ERR_CUDA;
    }
    *out = b;
    return NTT_OK;
}

ntt_status ntt_bconv(ntt_bconv_t plan, void *d_out, const void *d_in, uint32_t batch, ntt_stream_t stream) {
    if (!plan || !d_out || !d_in || batch == 0) return NTT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_out) & 3u) || (reinterpret_cast<uintptr_t>(d_in) & 3u))
        return NTT_ERR_ALIGNMENT;
    const uint64_t total = (uint64_t)batch * plan->N;
    const uint32_t *x = reinterpret_cast<const uint32_t *>(d_in);
    uint32_t *z = reinterpret_cast<uint32_t *>(d_out);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (plan->lb) {
    case 8: e = nttgb::bc_launch<8>(*plan, x, z, total, st); break;
    case 16: e = nttgb::bc_launch<16>(*plan, x, z, total, st); break;
    case 32: e = nttgb::bc_launch<32>(*plan, x, z, total, st); break;
    default: e = nttgb::bc_launch<64>(*plan, x, z, total, st); break;
    }
    plan->last_launches = 1;
    if (e != cudaSuccess) { cudaGetLastError(); return NTT_ERR_CUDA; }
    return NTT_OK;
}

void ntt_bconv_destroy(ntt_bconv_t plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    if (plan->d_tab) cudaFree(plan->d_tab);
    delete plan;
}

}  // extern "C"
