// stream.cuh -- both passes of a two-pass transform in one persistent launch.
//
// The two-pass split (four-step idea of Sec. II: sub-transforms small enough
// for on-chip memory) writes every word after the first pass and reads it
// back in the second.  Run as two launches, the whole batch sits between the
// passes and the intermediate goes to HBM and back.  Here one launch streams
// the passes limb by limb: CTAs take work items (runs of tiles of one pass of
// one limb) from an atomic queue whose order interleaves the first pass of
// limb r with the second pass of limb r - lag, so the second pass reads a
// limb's intermediate while it is still in L2.  A second-pass item waits
// (bounded) until every first-pass tile of its limb has been stored; items
// only ever wait on items earlier in the queue, which CTAs already hold and
// finish without waiting on later ones, so no launch shape can deadlock.
//
// Tiles are those of the per-pass kernels (fused.cuh) in their 256-thread
// configuration (P = 1).
//
// Per call the kernel uses one counter set of the plan (a ring of
// kStreamRing sets, so that up to that many calls of one plan may overlap):
// [0, L) first-pass tiles stored per limb, then the queue head, the exit
// count and an abort flag.  The last CTA to leave puts the set back to zero.
#pragma once
#include "fused.cuh"

namespace nttgb {

// Tile configuration of the stream kernel: 256-thread CTAs, three per SM
// (512-thread CTAs with 32-chunk tiles fit only one per SM and ran slower).
template <class W> __host__ __device__ constexpr int stream_p() { return 1; }
template <class W> __host__ __device__ constexpr uint32_t stream_threads() { return 256u; }
template <class W> __host__ __device__ constexpr int stream_min_blocks() { return 3; }

template <class W> struct StreamArgs {
    FArgs<W> pass[2];           // in run order: [0] first pass, [1] second pass
    uint32_t *ctr;              // this call's counter set
    uint32_t L;
    uint32_t tiles_per_limb[2]; // tiles of each pass per limb
    uint32_t tiles_per_item[2];
    uint32_t items_per_limb[2];
    uint32_t lag;               // rounds between a limb's first and second pass (>= 1)
};

// Shared-memory bytes a tile kind uses in the stream kernel.
template <class W, int LOGS, int KIND, bool INV> __host__ __device__ constexpr size_t stream_kind_bytes() {
    return (size_t)n_stages<W, LOGS, KIND>() * buf_words<W, LOGS, KIND, INV, stream_p<W>()>() * sizeof(W) +
           (size_t)tw_pairs<W, LOGS, KIND, stream_p<W>()>() * 2 * sizeof(W);
}
template <class W, int S1, bool INV> __host__ __device__ constexpr size_t stream_bar_offset() {
    constexpr size_t a = stream_kind_bytes<W, S1, TK_COLS, INV>();
    constexpr size_t b = stream_kind_bytes<W, kN2Log, TK_CHUNKS, INV>();
    return ((a > b ? a : b) + 15) & ~size_t(15);
}
template <class W, int S1, bool INV> __host__ __device__ constexpr size_t stream_smem_bytes() {
    return stream_bar_offset<W, S1, INV>() + 64 + 1024;   // barriers, alignment slack
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Thread 0: wait until *c >= target (first-pass tiles of a limb stored),
// giving up when the call is aborted or after about 2^31 SM cycles.
__device__ __forceinline__ bool wait_count(const uint32_t *c, uint32_t target, const uint32_t *abort_flag) {
    if (ld_acquire(c) < target) {
        const long long t0 = clock64();
        while (ld_acquire(c) < target) {
            if (*(volatile const uint32_t *)abort_flag) return false;
            if (clock64() - t0 > (1ll << 31)) return false;
            __nanosleep(64);
        }
    }
    // the tiles are read next by TMA (the async proxy)
    fence_proxy_async_global();
    return true;
}

template <class W, int RED, bool INV, int S1>
__global__ void __launch_bounds__(stream_threads<W>(), stream_min_blocks<W>())
k_stream(const __grid_constant__ StreamArgs<W> sa) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint32_t s_item;
    __shared__ int s_go;
    constexpr int KIND0 = INV ? TK_CHUNKS : TK_COLS;   // first pass
    constexpr int KIND1 = INV ? TK_COLS : TK_CHUNKS;   // second pass
    constexpr int LOGS0 = INV ? (int)kN2Log : S1;
    constexpr int LOGS1 = INV ? S1 : (int)kN2Log;
    unsigned char *base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + stream_bar_offset<W, S1, INV>());
    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        for (uint32_t s = 0; s < 3; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint32_t L = sa.L;
    uint32_t *ctr = sa.ctr;
    uint32_t *head = ctr + L, *exit_count = ctr + L + 1, *abort_flag = ctr + L + 2;
    const uint32_t n0 = sa.items_per_limb[0], n1 = sa.items_per_limb[1];
    const uint32_t slots = n0 + n1;                       // items per round
    const uint64_t total = (uint64_t)(L + sa.lag) * slots;
    PipeState ps{{0, 0, 0}, 0};
    bool ok = true;
    // thread 0 takes the next item while this one runs (its atomic's
    // latency hides behind the work); holding one item ahead cannot
    // deadlock: the earliest unfinished item is always one a CTA is running
    uint32_t ahead = 0;
    if (tid == 0) ahead = atomicAdd(head, 1u);
    for (;;) {
        if (tid == 0) {
            s_item = *(volatile uint32_t *)abort_flag ? 0xffffffffu : ahead;
            if (s_item < total) ahead = atomicAdd(head, 1u);
        }
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= total) break;
        // round r, slot s: first-pass items spread evenly among the slots
        const uint32_t r = item / slots, s = item % slots;
        const uint32_t f = (uint32_t)((uint64_t)s * n0 / slots);
        const bool first = (uint32_t)((uint64_t)(s + 1) * n0 / slots) > f;
        const uint32_t j = first ? f : s - f;
        const int which = first ? 0 : 1;
        if (!first && r < sa.lag) continue;
        const uint32_t limb = first ? r : r - sa.lag;
        if (limb >= L) continue;
        const uint32_t tpl = sa.tiles_per_limb[which], tpi = sa.tiles_per_item[which];
        const uint32_t t0 = limb * tpl + j * tpi;
        const uint32_t t1 = t0 + tpi < (limb + 1) * tpl ? t0 + tpi : (limb + 1) * tpl;
        if (first) {
            ok = run_tiles<W, RED, INV, LOGS0, KIND0, stream_p<W>()>(sa.pass[0], &sa.pass[0].tmap, t0, t1, base, bar,
                                                                    ps);
            if (!ok) break;
            // every thread's stores of this item, then the count
            fence_proxy_async_global();
            __threadfence();
            __syncthreads();
            if (tid == 0) atomicAdd(&ctr[limb], t1 - t0);
        } else {
            if (tid == 0) {
                const bool got = wait_count(&ctr[limb], sa.tiles_per_limb[0], abort_flag);
                if (!got) atomicOr(sa.pass[1].status, 2u);
                s_go = got ? 1 : 0;
            }
            __syncthreads();
            if (!s_go) { ok = false; break; }
            ok = run_tiles<W, RED, INV, LOGS1, KIND1, stream_p<W>()>(sa.pass[1], &sa.pass[1].tmap, t0, t1, base, bar,
                                                                    ps);
            if (!ok) break;
        }
    }
    if (!ok && tid == 0) atomicExch(abort_flag, 1u);
    // the last CTA out puts the counter set back to zero for a later call
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(exit_count, 1u) == gridDim.x - 1) {
            for (uint32_t l = 0; l < L + 3; ++l) ctr[l] = 0u;
            __threadfence();
        }
    }
}

template <class W, int RED, bool INV, int S1> cudaError_t stream_config(size_t *smem, int *per_sm) {
    auto kern = k_stream<W, RED, INV, S1>;
    *smem = stream_smem_bytes<W, S1, INV>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, (int)stream_threads<W>(), *smem);
}

// Grid of the stream kernel: every CTA that fits on the GPU at once.
template <class W, int RED, bool INV, int S1> cudaError_t stream_resident_s1(int *resident, size_t *smem_out) {
    static int res = 0;
    static size_t smem = 0;
    if (!res) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaError_t e = stream_config<W, RED, INV, S1>(&smem, &per_sm);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        res = sms * (per_sm > 0 ? per_sm : 1);
    }
    *resident = res;
    *smem_out = smem;
    return cudaSuccess;
}

template <class W, int RED, bool INV> cudaError_t stream_resident(int s1, int *resident) {
    size_t smem = 0;
    switch (s1) {
    case 6: return stream_resident_s1<W, RED, INV, 6>(resident, &smem);
    case 7: return stream_resident_s1<W, RED, INV, 7>(resident, &smem);
    case 8: return stream_resident_s1<W, RED, INV, 8>(resident, &smem);
    case 9: return stream_resident_s1<W, RED, INV, 9>(resident, &smem);
    }
    return cudaErrorInvalidValue;
}

template <class W, int RED, bool INV, int S1>
cudaError_t stream_launch(const StreamArgs<W> &sa, cudaStream_t st) {
    int resident = 0;
    size_t smem = 0;
    cudaError_t e = stream_resident_s1<W, RED, INV, S1>(&resident, &smem);
    if (e != cudaSuccess) return e;
    k_stream<W, RED, INV, S1><<<resident, stream_threads<W>(), smem, st>>>(sa);
    return cudaGetLastError();
}

}  // namespace nttgb
