// fused.cuh -- the fused fast path: radix-2^4 rounds in registers.
//
// The transform is the merged-twist Cooley-Tukey recursion of Eq. 4-5 with
// the precomputed twiddle table of Sec. II (psi^bitrev(i), i < N, so the psi
// twist costs no extra multiplies): for m = 1, 2, 4, ..., N/2 and t = N/(2m)
// the butterfly (x[j], x[j+t]) uses psi^bitrev(m + j/(2t)).  Output is in
// bit-reversed order.  The inverse is the Gentleman-Sande recursion of Eq. 6
// run backwards with psi^-bitrev(i) and N^-1 folded into its last stage.
//
// A CTA owns a tile of K independent sub-transforms of S = 2^LOGS points.
// Each thread holds 16 words in registers and applies up to four stages to
// them (one "round"); rounds exchange data through shared memory.  Three
// tile kinds cover every N:
//   single  sub-transform = one whole transform (N <= 2^14 / 2^13 words);
//   cols    (pass A of two) sub-transform = one column of the N1 x N2 view,
//           stages m = 1 .. N1/2, table entries 1 .. N1-1;
//   chunks  (pass B of two) sub-transform = 256 contiguous words, stages
//           m = N1 .. N/2, per-chunk table tw2[r][2^s + i] =
//           psi^bitrev(2^s (N1 + r) + i).
// The two-pass split is the four-step / six-step idea of Sec. II ("splits a
// large NTT into several smaller ones ... fit into a cache") with the
// inter-step twiddles absorbed by the merged table.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "modarith.cuh"

namespace nttgb {

enum TileKind : int { TK_SINGLE = 0, TK_COLS = 1, TK_CHUNKS = 2 };

template <class W> struct FArgs {
    W *data;
    const Tw<W> *tw;          // [L][N] table of this pass
    const LimbConst *lc;
    uint64_t ntrans;          // batch * L
    uint64_t ntiles;
    uint32_t logN, L, logK, s2;   // N2 = 2^s2 (cols / chunks)
    uint32_t final_pass;      // fully reduce output; inverse: fold N^-1
};

// ---------------------------------------------------- shared-memory layout
// Padding keeps every round's accesses free of bank conflicts for the
// thread <-> word maps below: 16 bytes after every 128 bytes and 64 bytes
// after every 1 KiB (4-byte words); 16 bytes after every 128 bytes and 64
// bytes after every 2 KiB (8-byte words).  Groups of 16 bytes stay contiguous
// so tiles move as 128-bit vectors.
template <class W> __host__ __device__ constexpr uint32_t pu(uint32_t u) {
    return sizeof(W) == 4 ? u + 4 * (u >> 5) + 16 * (u >> 8) : u + 2 * (u >> 4) + 8 * (u >> 8);
}
// pitch between the sub-transforms of a rows tile: >= pu(S), and an odd
// multiple of half the bank width so neighbouring subs use the other half
template <class W, int LOGS> __host__ __device__ constexpr uint32_t rows_pitch() {
    constexpr uint32_t span = pu<W>(1u << LOGS);
    constexpr uint32_t half = sizeof(W) == 4 ? 16 : 8;
    return ((span + half) / (2 * half)) * (2 * half) + half;
}
template <class W> __host__ __device__ constexpr uint32_t cols_phys(uint32_t k, uint32_t u, uint32_t K) {
    return k + K * (u + (u >> 4));
}

template <class W, int LOGS, int KIND> __host__ constexpr size_t fused_smem_bytes(uint32_t K) {
    return KIND == TK_COLS ? (size_t)K * ((1u << LOGS) + (1u << LOGS) / 16) * sizeof(W)
                           : (size_t)K * rows_pitch<W, LOGS>() * sizeof(W);
}

// word index u of slot e for a round covering bits [LO, LO+RR) of the
// sub-transform index, thread tau of the sub-transform
template <int LOGS, int LO, int RR> __device__ __forceinline__ uint32_t slot_u(uint32_t tau, int e) {
    if (RR == 4) {
        return (tau & ((1u << LO) - 1)) | ((uint32_t)e << LO) | ((tau >> LO) << (LO + 4));
    } else {
        // short round, always the top bits: LO = LOGS - RR
        uint32_t o = (tau << (4 - RR)) | ((uint32_t)e >> RR);
        return o | (((uint32_t)e & ((1u << RR) - 1)) << LO);
    }
}

template <class W, int RED, bool INV, int LOGS, int LO, int RR>
__device__ __forceinline__ void round_bfly(W (&x)[16], uint32_t tau, const Tw<W> *__restrict__ tw, const Lc<W> &k,
                                           bool last_pass, Tw<W> tn, Tw<W> twn) {
    constexpr uint32_t S = 1u << LOGS;
    if (!INV) {
#pragma unroll
        for (int d = RR - 1; d >= 0; --d) {
            const int b = LO + d;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                if (e & (1 << d)) continue;
                uint32_t u = slot_u<LOGS, LO, RR>(tau, e);
                uint32_t idx = (S >> (b + 1)) + (u >> (b + 1));
                ct_bfly<RED, W>(x[e], x[e | (1 << d)], ldtw(tw + idx), k);
            }
        }
    } else {
#pragma unroll
        for (int d = 0; d < RR; ++d) {
            const int b = LO + d;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                if (e & (1 << d)) continue;
                uint32_t u = slot_u<LOGS, LO, RR>(tau, e);
                if (b == LOGS - 1 && last_pass) {
                    gs_bfly_last<RED, W>(x[e], x[e | (1 << d)], tn, twn, k);
                } else {
                    uint32_t idx = (S >> (b + 1)) + (u >> (b + 1));
                    gs_bfly<RED, W>(x[e], x[e | (1 << d)], ldtw(tw + idx), k);
                }
            }
        }
    }
}

template <class W, int LOGS, int KIND> __device__ __forceinline__ uint32_t sm_addr(uint32_t k, uint32_t u, uint32_t K) {
    if (KIND == TK_COLS) return cols_phys<W>(k, u, K);
    return k * rows_pitch<W, LOGS>() + pu<W>(u);
}

// One round: load 16 slots from shared memory, apply the stages, store back.
template <class W, int RED, bool INV, int LOGS, int KIND, int LO, int RR>
__device__ __forceinline__ void do_round(W *sm, uint32_t k, uint32_t tau, uint32_t K, const Tw<W> *__restrict__ tw,
                                         const Lc<W> &kk, bool last_pass, Tw<W> tn, Tw<W> twn) {
    W x[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) x[e] = sm[sm_addr<W, LOGS, KIND>(k, slot_u<LOGS, LO, RR>(tau, e), K)];
    round_bfly<W, RED, INV, LOGS, LO, RR>(x, tau, tw, kk, last_pass, tn, twn);
#pragma unroll
    for (int e = 0; e < 16; ++e) sm[sm_addr<W, LOGS, KIND>(k, slot_u<LOGS, LO, RR>(tau, e), K)] = x[e];
}

// Rounds of a sub-transform.  Forward: bits from the top down, the short
// round (LOGS mod 4 bits) first; inverse: from the bottom up, short last.
template <class W, int RED, bool INV, int LOGS, int KIND, int J>
__device__ __forceinline__ void all_rounds(W *sm, uint32_t k, uint32_t tau, uint32_t K, const Tw<W> *__restrict__ tw,
                                           const Lc<W> &kk, bool last_pass, Tw<W> tn, Tw<W> twn) {
    constexpr int NR = (LOGS + 3) / 4;
    if constexpr (J < NR) {
        constexpr int SHORT = LOGS % 4;
        constexpr int RR = INV ? ((LOGS - 4 * J) < 4 ? (LOGS - 4 * J) : 4) : ((SHORT && J == 0) ? SHORT : 4);
        constexpr int LO = INV ? 4 * J
                               : ((SHORT && J == 0) ? LOGS - SHORT : LOGS - SHORT - 4 * J - (SHORT ? 0 : 4));
        do_round<W, RED, INV, LOGS, KIND, LO, RR>(sm, k, tau, K, tw, kk, last_pass, tn, twn);
        __syncthreads();
        all_rounds<W, RED, INV, LOGS, KIND, J + 1>(sm, k, tau, K, tw, kk, last_pass, tn, twn);
    }
}

template <class W, int RED, bool INV, int LOGS, int KIND>
__global__ void __launch_bounds__(sizeof(W) == 4 ? 1024 : 512)
k_fused(FArgs<W> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    W *sm = reinterpret_cast<W *>(smem_raw);
    constexpr uint32_t S = 1u << LOGS;
    constexpr uint32_t T = S / 16;
    constexpr int V = 16 / sizeof(W);
    using Vec = typename std::conditional<sizeof(W) == 4, uint4, ulonglong2>::type;
    const uint32_t K = 1u << a.logK;
    const uint32_t N = 1u << a.logN;
    const uint32_t tid = threadIdx.x;
    const uint32_t nthr = K * T;

    for (uint64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        // ---------------------------------------------------- tile decode
        uint64_t t;            // transform of sub 0 (single) / of the tile
        uint32_t pos0 = 0;     // first column (cols) or chunk (chunks)
        if (KIND == TK_SINGLE) {
            t = tile << a.logK;
        } else {
            const uint32_t per = (KIND == TK_COLS ? (N >> (a.logN - a.s2)) : (N >> a.s2)) >> a.logK;
            t = tile / per;
            pos0 = (uint32_t)(tile % per) << a.logK;
        }
        // ---------------------------------------------------- load tile
        if (KIND == TK_COLS) {
            const W *g = a.data + t * N + pos0;
            const uint32_t vpr = K / V;   // vectors per row of the strip
            for (uint32_t i = tid; i < S * vpr; i += nthr) {
                uint32_t u = i / vpr, kv = (i % vpr) * V;
                Vec v = *reinterpret_cast<const Vec *>(g + ((size_t)u << a.s2) + kv);
                *reinterpret_cast<Vec *>(sm + cols_phys<W>(kv, u, K)) = v;
            }
        } else {
            const uint32_t vps = S / V;
            for (uint32_t i = tid; i < K * vps; i += nthr) {
                uint32_t k = i / vps, u = (i % vps) * V;
                const W *g;
                if (KIND == TK_SINGLE) {
                    if (t + k >= a.ntrans) continue;
                    g = a.data + (t + k) * N;
                } else {
                    g = a.data + t * N + ((size_t)(pos0 + k) << a.s2);
                }
                Vec v = *reinterpret_cast<const Vec *>(g + u);
                *reinterpret_cast<Vec *>(sm + sm_addr<W, LOGS, KIND>(k, u, K)) = v;
            }
        }
        __syncthreads();
        // ---------------------------------------------------- compute
        uint32_t k, tau;
        if (KIND == TK_COLS) { k = tid % K; tau = tid / K; }
        else { tau = tid % T; k = tid / T; }
        const uint64_t tk = KIND == TK_SINGLE ? t + k : t;
        const uint32_t l = (uint32_t)((tk < a.ntrans ? tk : 0) % a.L);
        Lc<W> kk;
        kk.load(a.lc + l);
        const Tw<W> *twb = a.tw + (size_t)l * N + (KIND == TK_CHUNKS ? ((size_t)(pos0 + k) << a.s2) : 0);
        Tw<W> tn{}, twn{};
        if (INV && a.final_pass) {
            tn.w = (W)a.lc[l].ninv_w; tn.c = (W)a.lc[l].ninv_c;
            twn.w = (W)a.lc[l].ninv_w1_w; twn.c = (W)a.lc[l].ninv_w1_c;
        }
        all_rounds<W, RED, INV, LOGS, KIND, 0>(sm, k, tau, K, twb, kk, INV && a.final_pass, tn, twn);
        // ---------------------------------------------------- store tile
        if (KIND == TK_COLS) {
            W *g = a.data + t * N + pos0;
            const uint32_t vpr = K / V;
            for (uint32_t i = tid; i < S * vpr; i += nthr) {
                uint32_t u = i / vpr, kv = (i % vpr) * V;
                Vec v = *reinterpret_cast<const Vec *>(sm + cols_phys<W>(kv, u, K));
                if (a.final_pass) {
                    // the column pass is last only for the inverse
                    W *pv = reinterpret_cast<W *>(&v);
#pragma unroll
                    for (int j = 0; j < V; ++j) pv[j] = csub<W>(pv[j], kk.q);
                }
                *reinterpret_cast<Vec *>(g + ((size_t)u << a.s2) + kv) = v;
            }
        } else {
            const uint32_t vps = S / V;
            for (uint32_t i = tid; i < K * vps; i += nthr) {
                uint32_t k2 = i / vps, u = (i % vps) * V;
                W *g;
                Lc<W> k2c = kk;
                if (KIND == TK_SINGLE) {
                    if (t + k2 >= a.ntrans) continue;
                    g = a.data + (t + k2) * N;
                    k2c.load(a.lc + (uint32_t)((t + k2) % a.L));
                } else {
                    g = a.data + t * N + ((size_t)(pos0 + k2) << a.s2);
                }
                Vec v = *reinterpret_cast<const Vec *>(sm + sm_addr<W, LOGS, KIND>(k2, u, K));
                if (a.final_pass) {
                    W *pv = reinterpret_cast<W *>(&v);
#pragma unroll
                    for (int j = 0; j < V; ++j) {
                        W y = pv[j];
                        if (!INV) y = csub<W>(y, k2c.two_q);
                        pv[j] = csub<W>(y, k2c.q);
                    }
                }
                *reinterpret_cast<Vec *>(g + u) = v;
            }
        }
        __syncthreads();
    }
}

}  // namespace nttgb
