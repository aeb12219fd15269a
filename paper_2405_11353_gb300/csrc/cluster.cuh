// cluster.cuh -- one-pass fused transform of N = 2^16 four-byte words on a
// cluster of eight CTAs (instantiated once per reduction in cluster_<red>.cu).
//
// The two-pass split moves every word through DRAM twice.  Here the eight
// CTAs of a thread-block cluster share one transform and each word is read
// from and written to DRAM once.  The merged-twist Cooley-Tukey recursion
// (Eq. 4-5 with the table psi^bitrev(i) of Sec. II) splits the transform into
// independent blocks after every stage; write a word index as
// g = 8192 k + 1024 r + j (k, r < 8, j < 1024).  Forward, CTA c:
//   round A  stages m = 1, 2, 4 (they pair the eight k) on the words with
//            r = c, loaded by TMA as eight 4 KiB pieces into slots k of the
//            stage buffer; output k is stored into slot c of CTA k's stage
//            buffer (distributed shared memory);
//   round X  stages m = 8, 16, 32 (they pair the eight r) on the eight slots
//            CTA c received: the words with k = c;
//   rounds   after six stages the words 8192 c + 1024 r + (0..1023) form
//            eight independent 1024-point blocks: stages m = 64 .. 32768
//            run as the rounds of a 1024-point fused tile (fused.cuh), the
//            last one writing 16 consecutive words per thread.
// The inverse runs the same steps backwards (Gentleman-Sande, Eq. 6) with
// N^-1 folded into its last stage.  Round A and round X are the four-step
// split of Sec. II applied twice, with the exchange between them on chip.
//
// Two cluster barriers per transform order the exchange: the first (its
// arrive after a CTA has read its slots, its wait before it stores into the
// others', with the round's arithmetic in between) frees the slots, the
// second publishes the stores.  Each CTA keeps its eighth of the limb's
// twiddles (8 blocks x 1024 pairs, plus the 14 of rounds A and X) in shared
// memory and runs a contiguous range of transforms polynomial-fastest, so
// the table is loaded once per limb.  With 512 threads and about 100 KiB of
// shared memory, two CTAs share an SM.
#pragma once
#include "fused.cuh"
#include "plan.hpp"

namespace nttgb {

constexpr int kCluLog = 3;                       // 8 CTAs per transform
constexpr uint32_t kCluC = 1u << kCluLog;
constexpr int kCluBlkLog = 10;                   // 1024-point blocks after round X
constexpr uint32_t kCluBlk = 1u << kCluBlkLog;
constexpr uint32_t kCluWords = kCluC * kCluBlk;  // 8192 words per CTA
constexpr uint32_t kCluThreads = kCluWords / 16; // 512
// Twiddle pairs per (limb, CTA): the eight block tables, then round A's
// entries 1..7 at kCluWords + e and round X's at kCluWords + 8 + e.
constexpr uint32_t kCluTwPairs = kCluWords + 16;

struct CArgs {
    uint32_t *data;
    const Tw<uint32_t> *tw;     // [L][8 c][kCluTwPairs]: block tables (level_pos layout), heads
    const LimbConst *lc;
    uint32_t *status;           // bit 1: a bounded wait gave up
    uint64_t ntrans;            // batch * L
    uint32_t L;
    uint32_t stall_tx;          // test hook: extra bytes CTA 0 expects on its first tile
};

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Cluster barrier in two halves (every thread of the eight CTAs): memory
// accesses before a CTA's arrive are ordered before the others' accesses
// after their wait.
__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
// Two words into the shared memory of CTA `rank` of the cluster, at the
// address `local` has in this CTA.
__device__ __forceinline__ void st_cluster_v2(const void *local, uint32_t rank, uint32_t a, uint32_t b) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_addr(local)), "r"(rank));
    asm volatile("st.shared::cluster.v2.u32 [%0], {%1, %2};" ::"r"(remote), "r"(a), "r"(b) : "memory");
}

// Stages m = 1, 2, 4 of an 8-point block of the recursion (forward), or
// m = 4, 2, 1 (inverse, N^-1 folded into m = 1 when FOLD), on v[0..7] of
// two columns; twiddle of stage 2^a, sub-block b at t[2^a + b] (shared
// memory, read stage by stage).
template <int RED, bool INV, bool FOLD>
__device__ __forceinline__ void radix8(uint32_t (&v)[8][2], const Tw<uint32_t> *t, Tw<uint32_t> tn,
                                       Tw<uint32_t> twn, const Lc<uint32_t> &kk) {
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) {
        const int a = INV ? 2 - aa : aa;
        const int half = 4 >> a;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            if (r & half) continue;
            const Tw<uint32_t> w = (FOLD && a == 0) ? tn : t[(1 << a) + (r >> (3 - a))];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (!INV) ct_bfly<RED, uint32_t>(v[r][c], v[r + half][c], w, kk);
                else if (FOLD && a == 0) gs_bfly_last<RED, uint32_t>(v[r][c], v[r + half][c], tn, twn, kk);
                else gs_bfly<RED, uint32_t>(v[r][c], v[r + half][c], w, kk);
            }
        }
    }
}

// Stage buffer: the TMA tile (8192 words), then the eight blocks in the
// padded exchange layout of fused.cuh (sm_off, rows_pitch apart).
template <bool INV> __host__ __device__ constexpr uint32_t cluster_stage_words() {
    return ((kCluC * rows_pitch<uint32_t, kCluBlkLog>() > kCluWords ? kCluC * rows_pitch<uint32_t, kCluBlkLog>()
                                                                     : kCluWords) + 255) & ~255u;
}
template <bool INV> __host__ __device__ constexpr size_t cluster_smem_bytes() {
    return (size_t)cluster_stage_words<INV>() * 4 + (size_t)kCluTwPairs * 8 + 64 + 1024;
}
static_assert(kCluTwPairs * 8 % 16 == 0, "twiddle slices are copied in 16-byte units");

template <int RED, bool INV>
__global__ void __cluster_dims__(kCluC, 1, 1) __launch_bounds__(kCluThreads, 2)
k_cluster(const __grid_constant__ CArgs a) {
    using W = uint32_t;
    constexpr int LB = kCluBlkLog;
    constexpr uint32_t BLK = kCluBlk, C = kCluC, SUB = kCluWords, N = SUB * C;
    constexpr uint32_t SW = cluster_stage_words<INV>();
    constexpr uint32_t TB = BLK / 16;   // threads per block in the block rounds
    using R0 = RoundOf<LB, INV, 0>;
    using RL = RoundOf<LB, INV, R0::NR - 1>;
    static_assert(INV || (RL::RR == 4 && RL::LO == 0), "the last forward round holds 16 consecutive words");
    static_assert(!INV || (R0::RR == 4 && R0::LO == 0), "the first inverse round holds 16 consecutive words");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    W *sb = reinterpret_cast<W *>(base);
    Tw<W> *tws = reinterpret_cast<Tw<W> *>(base + (size_t)SW * 4);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + (size_t)SW * 4 + (size_t)kCluTwPairs * 8);
    const uint32_t tid = threadIdx.x;
    const uint32_t c = cluster_ctarank();
    const uint32_t ncl = gridDim.x / C, cid = blockIdx.x / C;
    const uint64_t i_begin = cid * a.ntrans / ncl, i_end = (cid + 1) * a.ntrans / ncl;
    const uint32_t L = a.L;
    const uint64_t B = a.ntrans / L;
    // block rounds: block kb = tid / TB, thread tb within it
    const uint32_t kb = tid / TB, tb = tid % TB;
    const uint32_t smb = sm_off<W, LB, TK_SINGLE, 0>(kb, 0);
    if (tid == 0) {
        mbar_init(&bar[0], 1);   // tile
        mbar_init(&bar[1], 1);   // twiddles
        fence_mbar_init();
    }
    __syncthreads();
    if (i_begin >= i_end) return;   // (the whole cluster: same range)

    auto t_of = [&](uint64_t i) -> uint64_t { return (i % B) * L + i / B; };   // polynomial-fastest
    auto issue = [&](uint64_t i) {
        const W *src = a.data + t_of(i) * N;
        mbar_expect_tx(&bar[0], SUB * (uint32_t)sizeof(W));
        if (!INV) {
            for (uint32_t k = 0; k < C; ++k) bulk_g2s(sb + k * BLK, src + k * SUB + c * BLK, BLK * sizeof(W), &bar[0]);
        } else {
            bulk_g2s(sb, src + c * SUB, SUB * sizeof(W), &bar[0]);
        }
    };
    auto prefetch = [&](uint64_t i) {
        const W *src = a.data + t_of(i) * N;
        if (!INV) {
            for (uint32_t k = 0; k < C; ++k) prefetch_l2(src + k * SUB + c * BLK, BLK * sizeof(W));
        } else {
            prefetch_l2(src + c * SUB, SUB * sizeof(W));
        }
    };

    uint64_t issued = i_begin;   // (thread 0) next position to load
    if (tid == 0) {
        if (a.stall_tx && blockIdx.x == 0) mbar_add_tx(&bar[0], a.stall_tx);
        issue(issued++);
        if (issued < i_end) prefetch(issued);
    }
    bool ok = true;              // uniform in the CTA
    bool tile_pending = true;    // (thread 0) a tile copy not yet waited for
    uint32_t tile_phase = 0;     // tile copies waited for
    uint32_t tw_limb = 0xffffffffu, tw_phase = 0;
    bool tw_pending = false;
    const Tw<W> tz{};
    uint32_t it = 0;
    for (uint64_t i = i_begin; i < i_end; ++i, ++it) {
        const uint64_t t = t_of(i);
        const uint32_t l = (uint32_t)(t % L);
        Lc<W> kk;
        kk.load(a.lc + l);
        W *g = a.data + t * N;
        const Tw<W> *hA = tws + SUB, *hX = tws + SUB + 8;   // heads of rounds A and X
        // restage this CTA's twiddle blocks when the limb changes (every
        // thread finished with the old ones at the end of the last tile)
        if (ok && l != tw_limb) {
            if (tid == 0) {
                fence_proxy_async();
                mbar_expect_tx(&bar[1], kCluTwPairs * (uint32_t)sizeof(Tw<W>));
                bulk_g2s(tws, a.tw + ((size_t)l * C + c) * kCluTwPairs, kCluTwPairs * sizeof(Tw<W>), &bar[1]);
            }
            tw_pending = true;
            const bool got = mbar_wait_bounded(&bar[1], tw_phase & 1u);
            ++tw_phase;
            tw_limb = l;
            if (got) tw_pending = false;
            if (__syncthreads_or(!got)) {
                if (tid == 0) atomicOr(a.status, 2u);
                ok = false;
            }
        }
        // a CTA whose wait gave up stops computing but keeps meeting the
        // cluster barriers, so its partners finish
        if (ok) {
            const bool got = mbar_wait_bounded(&bar[0], tile_phase & 1u);
            if (got) { tile_pending = false; ++tile_phase; }
            if (__syncthreads_or(!got)) {
                if (tid == 0) atomicOr(a.status, 2u);
                ok = false;
            }
        }
        // columns j = 2 tid, 2 tid + 1 of the eight slots (rounds A and X)
        const uint32_t j0 = 2 * tid;
        W v[8][2];
        if (!INV) {
            // ---- round A: stages 1, 2, 4 across k
            if (ok) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    uint2 w2 = *reinterpret_cast<const uint2 *>(sb + k * BLK + j0);
                    v[k][0] = w2.x; v[k][1] = w2.y;
                }
            }
            cluster_arrive();   // this CTA's slots are read
            if (ok) {
                radix8<RED, false, false>(v, hA, tz, tz, kk);
            }
            cluster_wait();     // every CTA's slots are read: store into them
            if (ok) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if ((uint32_t)k == c)
                        *reinterpret_cast<uint2 *>(sb + c * BLK + j0) = make_uint2(v[k][0], v[k][1]);
                    else
                        st_cluster_v2(sb + c * BLK + j0, k, v[k][0], v[k][1]);
                }
            }
            cluster_arrive();
            cluster_wait();     // the eight slots of this CTA hold its words k = c
            if (ok) {
                // ---- round X: stages 8, 16, 32 across r, into the block layout
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    uint2 w2 = *reinterpret_cast<const uint2 *>(sb + r * BLK + j0);
                    v[r][0] = w2.x; v[r][1] = w2.y;
                }
                radix8<RED, false, false>(v, hX, tz, tz, kk);
                __syncthreads();   // the slots are read: the block layout overwrites them
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    *reinterpret_cast<uint2 *>(sb + sm_off<W, LB, TK_SINGLE, 0>(r, j0)) = make_uint2(v[r][0], v[r][1]);
                __syncthreads();
                // ---- the eight 1024-point blocks
                W x[16];
                const uint32_t A0 = R0::A(tb);
#pragma unroll
                for (int e = 0; e < 16; ++e) x[e] = sb[smb + sm_off<W, LB, TK_SINGLE, 0>(0, A0 | R0::E(e))];
                __syncthreads();
                const Tw<W> *twb = tws + kb * BLK;
                round_bfly<W, RED, false, LB, 0, true>(x, tb, twb, kk, false, tz, tz);
                later_rounds<W, RED, false, LB, TK_SINGLE, false, true, 1, 0>(x, sb, smb, tb, twb, kk, false, tz, tz);
                __syncthreads();   // the stage buffer is free
                if (tid == 0 && issued < i_end) {
                    fence_proxy_async();
                    issue(issued++);
                    tile_pending = true;
                    if (issued < i_end) prefetch(issued);
                }
                W *q = g + c * SUB + kb * BLK + RL::A(tb);
#pragma unroll
                for (int v4 = 0; v4 < 4; ++v4) {
                    W y[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) y[e] = csub<W>(csub<W>(x[4 * v4 + e], kk.two_q), kk.q);
                    *reinterpret_cast<uint4 *>(q + 4 * v4) = make_uint4(y[0], y[1], y[2], y[3]);
                }
            }
        } else {
            if (ok) {
                // ---- the eight 1024-point blocks, bottom stages first
                W x[16];
                {
                    const W *q = sb + kb * BLK + R0::A(tb);
#pragma unroll
                    for (int v4 = 0; v4 < 4; ++v4) {
                        uint4 w4 = reinterpret_cast<const uint4 *>(q)[v4];
                        x[4 * v4] = w4.x; x[4 * v4 + 1] = w4.y; x[4 * v4 + 2] = w4.z; x[4 * v4 + 3] = w4.w;
                    }
                }
                __syncthreads();   // every staged word read: the buffer serves the exchanges
                const Tw<W> *twb = tws + kb * BLK;
                round_bfly<W, RED, true, LB, 0, true>(x, tb, twb, kk, false, tz, tz);
                later_rounds<W, RED, true, LB, TK_SINGLE, false, true, 1, 0>(x, sb, smb, tb, twb, kk, false, tz, tz);
                __syncthreads();
                {
                    const uint32_t AL = RL::A(tb);
#pragma unroll
                    for (int e = 0; e < 16; ++e) sb[smb + sm_off<W, LB, TK_SINGLE, 0>(0, AL | RL::E(e))] = x[e];
                }
                __syncthreads();
                // ---- round X backwards: stages 32, 16, 8 across r
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    uint2 w2 = *reinterpret_cast<const uint2 *>(sb + sm_off<W, LB, TK_SINGLE, 0>(r, j0));
                    v[r][0] = w2.x; v[r][1] = w2.y;
                }
            }
            cluster_arrive();   // this CTA's buffer is read
            if (ok) {
                radix8<RED, true, false>(v, hX, tz, tz, kk);
            }
            cluster_wait();     // every CTA's buffer is read: store into its slots
            if (ok) {
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    if ((uint32_t)r == c)
                        *reinterpret_cast<uint2 *>(sb + c * BLK + j0) = make_uint2(v[r][0], v[r][1]);
                    else
                        st_cluster_v2(sb + c * BLK + j0, r, v[r][0], v[r][1]);
                }
            }
            cluster_arrive();
            cluster_wait();     // slot k holds word 8192 k + 1024 c + j
            if (ok) {
                // ---- round A backwards: stages 4, 2, 1 across k, N^-1 folded
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    uint2 w2 = *reinterpret_cast<const uint2 *>(sb + k * BLK + j0);
                    v[k][0] = w2.x; v[k][1] = w2.y;
                }
                Tw<W> th[8];
#pragma unroll
                for (int e = 1; e < 8; ++e) th[e] = hA[e];
                __syncthreads();   // the stage buffer and the twiddles are free
                if (tid == 0 && issued < i_end) {
                    fence_proxy_async();
                    issue(issued++);
                    tile_pending = true;
                    if (issued < i_end) prefetch(issued);
                }
                const LimbConst *lcp = a.lc + l;
                const Tw<W> tn{(W)lcp->ninv_w, (W)lcp->ninv_c}, twn{(W)lcp->ninv_w1_w, (W)lcp->ninv_w1_c};
                radix8<RED, true, true>(v, th, tn, twn, kk);   // (registers: th is a copy)
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    *reinterpret_cast<uint2 *>(g + k * SUB + c * BLK + j0) =
                        make_uint2(csub<W>(v[k][0], kk.q), csub<W>(v[k][1], kk.q));
            }
        }
    }
    // no CTA leaves while another may still store into its shared memory
    cluster_arrive();
    cluster_wait();
    if (tid == 0 && (tile_pending || tw_pending)) {
        // a wait gave up: let the copies still in flight land before the
        // CTA exits, again with a time limit
        const long long t0 = clock64();
        while (tile_pending && !mbar_try_wait(&bar[0], tile_phase & 1u))
            if (clock64() - t0 > (1ll << 30)) break;
        const long long t1 = clock64();
        while (tw_pending && !mbar_try_wait(&bar[1], (tw_phase - 1) & 1u))
            if (clock64() - t1 > (1ll << 30)) break;
    }
}

// Host side: a persistent grid of as many clusters as fit at once.
template <int RED, bool INV> cudaError_t launch_cluster_t(const CArgs &a, cudaStream_t st) {
    auto kern = k_cluster<RED, INV>;
    constexpr size_t smem = cluster_smem_bytes<INV>();
    static int clusters = 0;
    if (!clusters) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kCluC * (unsigned)(sms / kCluC));
        cfg.blockDim = dim3(kCluThreads);
        cfg.dynamicSmemBytes = smem;
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, (void *)kern, &cfg);
        if (e != cudaSuccess) return e;
        clusters = n > 0 ? n : 1;
    }
    uint64_t ncl = a.ntrans < (uint64_t)clusters ? a.ntrans : (uint64_t)clusters;
    if (ncl == 0) ncl = 1;
    kern<<<(unsigned)(kCluC * ncl), kCluThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int RED>
cudaError_t run_cluster_t(ntt_plan_s &p, void *data, uint32_t batch, bool inverse, cudaStream_t st) {
    CArgs a;
    a.data = reinterpret_cast<uint32_t *>(data);
    a.tw = reinterpret_cast<const Tw<uint32_t> *>(inverse ? p.d_clu_inv : p.d_clu_fwd);
    a.lc = p.d_limb;
    a.status = p.d_status;
    a.ntrans = (uint64_t)batch * p.L;
    a.L = p.L;
    a.stall_tx = (p.flags & NTT_TEST_STALL) && !inverse ? 16u : 0u;
    ++p.last_launches;
    return inverse ? launch_cluster_t<RED, true>(a, st) : launch_cluster_t<RED, false>(a, st);
}

}  // namespace nttgb
