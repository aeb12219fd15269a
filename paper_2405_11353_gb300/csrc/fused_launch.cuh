// fused_launch.cuh -- host launcher of the fused path for one (word,
// reduction) pair; each fused_<w>_<red>.cu instantiates it once so the
// kernels compile in parallel.
#pragma once
#include "fused.cuh"
#include "plan.hpp"

namespace nttgb {

template <class W, int RED, bool INV, int LOGS, int KIND>
cudaError_t launch_pass(FArgs<W> a, uint32_t threads, size_t smem, cudaStream_t st) {
    auto kern = k_fused<W, RED, INV, LOGS, KIND>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    unsigned grid = a.ntiles > 0x7fffffffull ? 0x7fffffffu : (unsigned)a.ntiles;
    kern<<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <class W, int RED, bool INV, int KIND, int LOGS = 4>
cudaError_t pass_dispatch(int logS, FArgs<W> a, uint32_t threads, size_t smem, cudaStream_t st) {
    constexpr int MAXS = KIND == TK_SINGLE ? (sizeof(W) == 4 ? kSingleMaxLog32 : kSingleMaxLog64)
                                           : (KIND == TK_COLS ? 9 : kChunkLog);
    constexpr int MINS = KIND == TK_SINGLE ? 4 : (KIND == TK_COLS ? 5 : kChunkLog);
    if constexpr (LOGS > MAXS) {
        return cudaErrorInvalidValue;
    } else {
        if constexpr (LOGS >= MINS) {
            if (logS == LOGS) return launch_pass<W, RED, INV, LOGS, KIND>(a, threads, smem, st);
        }
        return pass_dispatch<W, RED, INV, KIND, LOGS + 1>(logS, a, threads, smem, st);
    }
}

template <class W, int KIND> size_t smem_for(int logS, uint32_t K) {
    switch (logS) {
#define NTTGB_CASE(s) case s: return fused_smem_bytes<W, s, KIND>(K);
        NTTGB_CASE(4) NTTGB_CASE(5) NTTGB_CASE(6) NTTGB_CASE(7) NTTGB_CASE(8) NTTGB_CASE(9)
        NTTGB_CASE(10) NTTGB_CASE(11) NTTGB_CASE(12) NTTGB_CASE(13) NTTGB_CASE(14)
#undef NTTGB_CASE
    }
    return 0;
}

// Tile geometry: K sub-transforms of 2^logS words per CTA, 2^logS / 16
// threads each.
inline uint32_t ilog2(uint32_t x) { uint32_t r = 0; while ((1u << r) < x) ++r; return r; }

template <class W, int RED, bool INV, int KIND>
cudaError_t run_pass(ntt_plan_s &p, W *data, const void *tw, uint64_t ntrans, int logS, bool final_pass,
                     cudaStream_t st) {
    FArgs<W> a;
    a.data = data;
    a.tw = reinterpret_cast<const Tw<W> *>(tw);
    a.lc = p.d_limb;
    a.ntrans = ntrans;
    a.logN = p.logN;
    a.L = p.L;
    a.s2 = p.s2;
    a.final_pass = final_pass ? 1u : 0u;
    const uint32_t T = (1u << logS) / 16;
    uint32_t K;
    if (KIND == TK_SINGLE) {
        K = (1u << logS) >= 4096 ? 1u : 4096u >> logS;
        a.ntiles = (ntrans + K - 1) / K;
    } else if (KIND == TK_COLS) {
        K = 256 / T;
        uint32_t kmin = sizeof(W) == 4 ? 16 : 8;
        if (K < kmin) K = kmin;
        a.ntiles = ntrans * ((1u << p.s2) / K);
    } else {
        K = 16;
        a.ntiles = ntrans * ((1u << (p.logN - p.s2)) / K);
    }
    a.logK = ilog2(K);
    size_t smem = smem_for<W, KIND>(logS, K);
    ++p.last_launches;
    return pass_dispatch<W, RED, INV, KIND>(logS, a, K * T, smem, st);
}

template <class W, int RED>
cudaError_t run_fused_t(ntt_plan_s &p, void *data_v, uint32_t batch, bool inverse, cudaStream_t st) {
    W *data = reinterpret_cast<W *>(data_v);
    const uint64_t ntrans = (uint64_t)batch * p.L;
    cudaError_t e;
    if (p.fused_mode == FUSED_SINGLE) {
        if (!inverse) return run_pass<W, RED, false, TK_SINGLE>(p, data, p.d_main_fwd, ntrans, p.logN, true, st);
        return run_pass<W, RED, true, TK_SINGLE>(p, data, p.d_main_inv, ntrans, p.logN, true, st);
    }
    if (!inverse) {
        e = run_pass<W, RED, false, TK_COLS>(p, data, p.d_main_fwd, ntrans, p.s1, false, st);
        if (e != cudaSuccess) return e;
        return run_pass<W, RED, false, TK_CHUNKS>(p, data, p.d_chunk_fwd, ntrans, p.s2, true, st);
    }
    e = run_pass<W, RED, true, TK_CHUNKS>(p, data, p.d_chunk_inv, ntrans, p.s2, false, st);
    if (e != cudaSuccess) return e;
    return run_pass<W, RED, true, TK_COLS>(p, data, p.d_main_inv, ntrans, p.s1, true, st);
}

}  // namespace nttgb
