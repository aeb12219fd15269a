// ragged_kernel.cuh -- the persistent kernel of a ragged batch (instantiated
// once per reduction in ragged_k_<reduction>.cu).
#pragma once
#include "fused.cuh"
#include "ragged.hpp"

namespace nttgb {

// Largest shared-memory footprint over the item kinds (P = 1 tiles).
template <class W, bool INV> __host__ __device__ constexpr size_t ragged_data_bytes_w() {
    size_t m = 0;
#define NTTGB_MAX(x) m = (x) > m ? (x) : m
    NTTGB_MAX((fused_smem_bytes<W, 12, TK_SINGLE, INV, 1>()));
    NTTGB_MAX((fused_smem_bytes<W, 5, TK_COLS, INV, 1>()));
    NTTGB_MAX((fused_smem_bytes<W, 6, TK_COLS, INV, 1>()));
    NTTGB_MAX((fused_smem_bytes<W, 7, TK_COLS, INV, 1>()));
    NTTGB_MAX((fused_smem_bytes<W, 8, TK_COLS, INV, 1>()));
    NTTGB_MAX((fused_smem_bytes<W, 9, TK_COLS, INV, 1>()));
    NTTGB_MAX((fused_smem_bytes<W, 8, TK_CHUNKS, INV, 1>()));
#undef NTTGB_MAX
    return m;
}
// Dynamic shared memory of the kernel for one word size (+ barriers).
template <class W> __host__ __device__ constexpr size_t ragged_smem_bytes() {
    size_t a = ragged_data_bytes_w<W, false>(), b = ragged_data_bytes_w<W, true>();
    return (a > b ? a : b) + 64;
}
// barriers live at a fixed offset past the largest data footprint
template <class W> __host__ __device__ constexpr size_t ragged_bar_offset() {
    return ((ragged_smem_bytes<W>() - 64 - 1024) + 15) & ~size_t(15);
}
// CTAs of 256 threads per SM the kernel is built for: three with 4-byte
// words (73.8 KB of shared memory and at most 80 registers a thread), two
// with 8-byte words (78.9 KB; the 64-bit butterflies take more registers).
template <class W> __host__ __device__ constexpr int ragged_min_blocks() { return sizeof(W) == 4 ? 3 : 2; }

// Grid-wide barrier of a cooperative launch: the last CTA to arrive resets
// the count and bumps the generation; the others wait for the bump, giving
// up after about 2^32 SM cycles (the caller then reports a timeout).
__device__ __forceinline__ bool grid_barrier(uint32_t *count, uint32_t *gen, uint32_t *abort_flag) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile uint32_t *vg = gen;
        const uint32_t g = *vg;
        __threadfence();
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vg == g) {
                if (*(volatile uint32_t *)abort_flag) { ok = 0; break; }
                if (clock64() - t0 > (1ll << 32)) { ok = 0; break; }
                __nanosleep(256);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class W, int RED, bool INV, int LOGS, int KIND>
__device__ __forceinline__ bool ragged_item(const RaggedArgs &ra, const RItem &it, unsigned char *base, uint64_t *bar,
                                            PipeState &ps) {
    const RJob &J = ra.jobs[it.job];
    FArgs<W> a;
    a.data = reinterpret_cast<W *>(J.data);
    a.out = a.data;
    a.pw_b = nullptr;
    const int which = KIND == TK_CHUNKS ? (INV ? 3 : 2) : (INV ? 1 : 0);
    a.tw = reinterpret_cast<const Tw<W> *>(J.tw[which]);
    a.lc = J.lc;
    a.status = ra.status;
    a.ntrans = J.ntrans;
    a.ntiles = 0;
    a.stall_tx = 0;
    a.logN = J.logN;
    a.L = J.L;
    a.logK = 0;
    a.s2 = kN2Log;
    a.final_pass = KIND == TK_SINGLE ? 1u : (KIND == TK_CHUNKS ? (INV ? 0u : 1u) : (INV ? 1u : 0u));
    const CUtensorMap *tmap = ra.tmaps + 2 * (size_t)it.job + (KIND == TK_CHUNKS ? 1 : 0);
    return run_tiles<W, RED, INV, LOGS, KIND, 1>(a, tmap, it.t0, it.t1, base, bar, ps);
}

template <class W, int RED, bool INV>
__device__ __forceinline__ bool ragged_dispatch_w(const RaggedArgs &ra, const RItem &it, uint32_t kind,
                                                  unsigned char *base, uint64_t *bar, PipeState &ps) {
    switch (kind) {
    case RK_SINGLE12: return ragged_item<W, RED, INV, 12, TK_SINGLE>(ra, it, base, bar, ps);
    case RK_COLS5 + 0: return ragged_item<W, RED, INV, 5, TK_COLS>(ra, it, base, bar, ps);
    case RK_COLS5 + 1: return ragged_item<W, RED, INV, 6, TK_COLS>(ra, it, base, bar, ps);
    case RK_COLS5 + 2: return ragged_item<W, RED, INV, 7, TK_COLS>(ra, it, base, bar, ps);
    case RK_COLS5 + 3: return ragged_item<W, RED, INV, 8, TK_COLS>(ra, it, base, bar, ps);
    case RK_COLS5 + 4: return ragged_item<W, RED, INV, 9, TK_COLS>(ra, it, base, bar, ps);
    default: return ragged_item<W, RED, INV, 8, TK_CHUNKS>(ra, it, base, bar, ps);
    }
}

// The persistent kernel of the items of one word size W.
template <int RED, class W>
__global__ void __launch_bounds__(256, ragged_min_blocks<W>()) k_ragged(const __grid_constant__ RaggedArgs ra) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint32_t s_item;
    unsigned char *base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + ragged_bar_offset<W>());
    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < 3; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    PipeState ps{{0, 0, 0}, 0};
    for (int phase = 0; phase < 4; ++phase) {
        // thread 0 takes each item one ahead (the atomic's round trip runs
        // under the current item); a CTA leaves a phase holding one index
        // past its end, which the launch's counter reset makes harmless
        uint32_t next = 0;
        if (threadIdx.x == 0) next = ra.phase_begin[phase] + atomicAdd(&ra.counters[phase], 1u);
        for (;;) {
            if (threadIdx.x == 0) s_item = next;
            __syncthreads();
            const uint32_t item = s_item;
            __syncthreads();
            if (item >= ra.phase_begin[phase + 1] || *(volatile uint32_t *)ra.abort_flag) break;
            if (threadIdx.x == 0) next = ra.phase_begin[phase] + atomicAdd(&ra.counters[phase], 1u);
            const RItem it = ra.items[item];
            const uint32_t kind = it.code % RK_KINDS;
            const bool inv = (it.code / RK_KINDS) & 1u;
            // (the host gives this kernel the items of its word size only)
            const bool ok = inv ? ragged_dispatch_w<W, RED, true>(ra, it, kind, base, bar, ps)
                                : ragged_dispatch_w<W, RED, false>(ra, it, kind, base, bar, ps);
            if (!ok) {
                if (threadIdx.x == 0) atomicExch(ra.abort_flag, 1u);
                break;
            }
        }
        // test hook: CTA 0 (its copies all landed: run_tiles drains its
        // pipeline) leaves without arriving, so the others' bounded wait
        // at the barrier runs out
        if (ra.stall && phase == 0 && blockIdx.x == 0) return;
        if (!grid_barrier(ra.bar_count, ra.bar_gen, ra.abort_flag)) {
            if (threadIdx.x == 0) atomicOr(ra.status, 2u);
            return;
        }
    }
}

template <int RED, class W> cudaError_t ragged_kernel_config(size_t *smem, int *blocks_per_sm) {
    *smem = ragged_smem_bytes<W>();
    cudaError_t e = cudaFuncSetAttribute(k_ragged<RED, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_ragged<RED, W>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_ragged<RED, W>, 256, *smem);
}

// Cooperative launch: every CTA is resident, so the grid barrier cannot
// wait on a CTA that has not started.
template <int RED, class W> cudaError_t ragged_kernel_launch(const RaggedArgs &a, unsigned grid, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = ragged_smem_bytes<W>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_ragged<RED, W>, a);
}

}  // namespace nttgb
