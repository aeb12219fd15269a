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
#include <cuda.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "modarith.cuh"

namespace nttgb {

enum TileKind : int { TK_SINGLE = 0, TK_COLS = 1, TK_CHUNKS = 2 };

// Two-pass split: N = N1 * N2 with N2 = 2^s2 (chunks of 2^s2 words; the
// per-plan passes take s2 = 7, 8 or 9, the item kernels of the ragged and
// streamed forms s2 = kN2Log).
constexpr uint32_t kN2Log = 8;

template <class W> struct FArgs {
    W *data;                  // the tiles are read from here ...
    W *out;                   // ... and written here (the same buffer but in
                              // the fused pointwise + inverse first pass)
    const W *pw_b;            // inverse chunk pass: multiply each word by this
                              // operand's word first (Eq. 3), or null
    const Tw<W> *tw;          // table of this pass: [L][2^LOGS] pairs (single
                              // and column passes), [L][N1][pitch] (chunks)
    const W *tw_seed;         // chunk passes with twiddles made on the fly
    const Tw<W> *tw_root;     // (4-byte words, Shoup): [L][N1][8] stage
                              // seeds, [L][256] root pairs; else null
    const LimbConst *lc;
    uint32_t *status;         // plan status word (bit 1: timeout)
    uint64_t ntrans;          // batch * L
    uint64_t ntiles;
    uint32_t logN, L, logK, s2;   // N2 = 2^s2 (cols / chunks)
    uint32_t final_pass;      // fully reduce output; inverse: fold N^-1
    uint32_t stall_tx;        // test hook: extra bytes the first tile of a call waits for
    CUtensorMap tmap;         // column passes: the data as rows of N2 words
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
    return span + ((half + 2 * half - span % (2 * half)) % (2 * half));
}
template <class W> __host__ __device__ constexpr uint32_t cols_phys(uint32_t k, uint32_t u, uint32_t K) {
    return k + K * (u + (u >> 4));
}


// Sub-transforms per CTA (compile-time, so every shared-memory address is
// a per-round base plus an immediate offset): single-pass tiles hold 4096
// words (or one transform above that), column strips 16 (4-byte) or 8
// (8-byte) columns and at least 256 threads, chunk tiles 16 chunks, or 2
// chunks in the per-pass chunk kernels with P = 0: one warp per CTA, so the
// per-tile barriers are warp barriers and the many small CTAs of an SM run
// independently.  With P = 3 the per-pass chunk kernels keep 16-chunk
// tiles (256 threads); which one a plan uses per direction is its form
// (default: 2-chunk tiles forward, 16-chunk tiles inverse, whose copies
// land through the 128-byte swizzle and need 1 KiB alignment; the
// autotuner can choose otherwise).
// P = 0: per-plan passes; column strips have 128-byte rows (32 four-byte or
// 16 eight-byte columns).  P = 1: the ragged kernel and the streamed
// two-pass launch, whose CTAs always have 256 threads (4096-word column
// tiles).  P = 3: per-pass chunk kernels with 16-chunk tiles (as P = 0
// otherwise).  Bit 3 of P (P = 8, 11) pairs polynomials in chunk tiles
// (paired_chunks).  Bit 4 of P (per-plan column and chunk passes): rounds
// of three stages on 8 words a thread instead of four stages on 16
// (radix_log).  Bit 5 (column passes): rows of the plan's 2^s2 words
// instead of 256.  Bit 6 (per-plan chunk passes, 4-byte words): the
// exchanges between rounds go through warp shuffles instead of shared
// memory, where a chunk's threads are lanes of one warp (shfl_exchange).
template <int P> __host__ __device__ constexpr int radix_log() { return (P & 16) ? 3 : 4; }
template <class W, int LOGS, int KIND, int P = 0> __host__ __device__ constexpr uint32_t tile_k() {
    // threads per sub-transform: 2^(LOGS - LR).  Chunks: one warp per CTA
    // (at least one chunk), or 256 threads.  Columns: 128-byte rows (or
    // more columns for short columns), at most 1024 threads (512 with
    // 8-byte words, the kernels' launch bound).
    constexpr int LR = radix_log<P>();
    constexpr uint32_t T = 1u << (LOGS > LR ? LOGS - LR : 0);
    constexpr uint32_t KC = (256u >> (LOGS - LR)) > (128u / sizeof(W)) ? (256u >> (LOGS - LR))
                                                                        : (128u / (uint32_t)sizeof(W));
    constexpr uint32_t TMAX = sizeof(W) == 4 ? 1024u : 512u;
    return KIND == TK_SINGLE ? (LOGS >= 12 ? 1u : (4096u >> LOGS))
         : KIND == TK_CHUNKS ? ((P & 3) == 0 ? (T >= 32 ? 1u : 32u / T) : (T >= 256 ? 1u : 256u / T))
         : (P & 3) == 1 ? (4096u >> LOGS)
         : (KC * T > TMAX ? TMAX / T : KC);
}

// Round J of a sub-transform covers bits [LO, LO+RR) of the index u, in
// rounds of LR = 4 (or 3) stages on 2^LR words a thread.  Forward: from the
// top down with the short round (LOGS mod LR bits) first; inverse: from
// the bottom up with the short round last.  Thread tau holds the 2^LR
// words u = A(tau) | E(e), e < 2^LR, where E places e's bits on the
// round's bits (and, in a short round, the spare bits of e just above
// tau's share) and A places tau's bits elsewhere; A and E are disjoint bit
// fields, so every layout below maps u to A's address plus a constant for
// E.
template <int LOGS, bool INV, int J, int LR = 4> struct RoundOf {
    static constexpr int SHORT = LOGS % LR;
    static constexpr int NR = (LOGS + LR - 1) / LR;
    static constexpr int RR = INV ? ((LOGS - LR * J) < LR ? (LOGS - LR * J) : LR) : ((SHORT && J == 0) ? SHORT : LR);
    static constexpr int LO = INV ? LR * J
                                  : ((SHORT && J == 0) ? LOGS - SHORT : LOGS - SHORT - LR * J - (SHORT ? 0 : LR));
    __host__ __device__ static constexpr uint32_t E(int e) {
        return RR == LR ? ((uint32_t)e << LO)
                        : (((uint32_t)e >> RR) | (((uint32_t)e & ((1u << RR) - 1)) << LO));
    }
    __host__ __device__ static constexpr uint32_t A(uint32_t tau) {
        return RR == LR ? ((tau & ((1u << LO) - 1)) | ((tau >> LO) << (LO + LR))) : (tau << (LR - RR));
    }
};

// ------------------------------------------------ warp-shuffle exchange
// Where index bit p of u sits in round J's layout: at bit i of the thread
// index tau (loc = i), or at bit i of the word index e (loc = LB + i, LB =
// LOGS - LR bits of tau).  Both RoundOf maps place single bits, so a round's
// layout is a bijection from u's LOGS bits onto tau's and e's.
template <int LOGS, bool INV, int J, int LR> struct XLayout {
    static constexpr int LB = LOGS - LR;
    int loc[16];
    static constexpr int bit_of(uint32_t v) {
        int b = 0;
        while (b < 31 && (v >> b) != 1u) ++b;
        return b;
    }
    constexpr XLayout() : loc() {
        using R = RoundOf<LOGS, INV, J, LR>;
        for (int i = 0; i < LR; ++i) loc[bit_of(R::E(1 << i))] = LB + i;
        for (int i = 0; i < LB; ++i) loc[bit_of(R::A(1u << i))] = i;
    }
};

// The move from round J - 1's layout to round J's as: swaps of a tau bit
// with an e bit (one shuffle per pair of words, with the partner lane
// across that tau bit), then a permutation of the tau bits (one indexed
// shuffle per word) and one of the e bits (register renaming, free).  Each
// u bit that goes from e to tau is swapped with one that goes from tau to
// e, the one at its target tau bit when there is such a bit; the tau bits
// left out of place (radix 8, and 512-word chunks in radix 16) take the
// indexed shuffles.
template <int LOGS, bool INV, int J, int LR> struct XPlan {
    static constexpr int LB = LOGS - LR;
    int nsw;
    int sw_tau[8], sw_e[8];       // swap s exchanges tau bit sw_tau[s] with e bit sw_e[s]
    int tau_src[8];               // after the swaps, tau bit b comes from tau bit tau_src[b]
    int e_src[8];                 // e bit b comes from e bit e_src[b]
    bool tau_perm;
    constexpr XPlan() : nsw(0), sw_tau(), sw_e(), tau_src(), e_src(), tau_perm(false) {
        const XLayout<LOGS, INV, J - 1, LR> from{};
        const XLayout<LOGS, INV, J, LR> to{};
        int cur[16] = {};
        for (int b = 0; b < LOGS; ++b) cur[b] = from.loc[b];
        for (int b = 0; b < LOGS; ++b) {
            if (cur[b] < LB || to.loc[b] >= LB) continue;       // not an e -> tau bit
            int q = -1;
            for (int c = 0; c < LOGS; ++c)
                if (q < 0 && cur[c] == to.loc[b] && to.loc[c] >= LB) q = c;
            for (int c = 0; c < LOGS; ++c)
                if (q < 0 && cur[c] < LB && to.loc[c] >= LB) q = c;
            sw_tau[nsw] = cur[q];
            sw_e[nsw] = cur[b] - LB;
            ++nsw;
            const int t = cur[b];
            cur[b] = cur[q];
            cur[q] = t;
        }
        for (int b = 0; b < LOGS; ++b) {
            if (to.loc[b] < LB) {
                tau_src[to.loc[b]] = cur[b];
                if (cur[b] != to.loc[b]) tau_perm = true;
            } else {
                e_src[to.loc[b] - LB] = cur[b] - LB;
            }
        }
    }
};
template <int LOGS, bool INV, int J, int LR> struct XPlanOf {
    static constexpr XPlan<LOGS, INV, J, LR> value{};
};

// The plan run on every lane's word indices at compile time (the swaps,
// the tau permutation and the e permutation as shfl_exchange performs
// them): true when each lane ends with round J's words.
template <int LOGS, bool INV, int J, int LR> constexpr bool xplan_reaches_round() {
    constexpr int LB = LOGS - LR, T = 1 << LB, NW = 1 << LR;
    using RP = RoundOf<LOGS, INV, J - 1, LR>;
    using R = RoundOf<LOGS, INV, J, LR>;
    const XPlan<LOGS, INV, J, LR> pl{};
    uint32_t x[32][16] = {}, y[32][16] = {};
    for (int t = 0; t < T; ++t)
        for (int e = 0; e < NW; ++e) x[t][e] = RP::A((uint32_t)t) | RP::E(e);
    for (int s = 0; s < pl.nsw; ++s) {
        const int i = pl.sw_tau[s], j = pl.sw_e[s];
        for (int t = 0; t < T; ++t)
            for (int e = 0; e < NW; ++e) y[t][e] = x[t][e];
        for (int t = 0; t < T; ++t) {
            const bool up = (t >> i) & 1;
            const int partner = t ^ (1 << i);
            for (int r0 = 0; r0 < NW; ++r0) {
                if (r0 & (1 << j)) continue;
                const int r1 = r0 | (1 << j);
                const uint32_t got = !up ? x[partner][r0] : x[partner][r1];   // the partner's hand-over
                if (up) y[t][r0] = got;
                else y[t][r1] = got;
            }
        }
        for (int t = 0; t < T; ++t)
            for (int e = 0; e < NW; ++e) x[t][e] = y[t][e];
    }
    for (int t = 0; t < T; ++t) {
        int src = 0, lane_src = 0;
        for (int b = 0; b < LB; ++b) lane_src |= ((t >> b) & 1) << (pl.tau_perm ? pl.tau_src[b] : b);
        for (int e = 0; e < NW; ++e) {
            src = 0;
            for (int b = 0; b < LR; ++b) src |= ((e >> b) & 1) << pl.e_src[b];
            y[t][e] = x[lane_src][src];
        }
    }
    for (int t = 0; t < T; ++t)
        for (int e = 0; e < NW; ++e)
            if (y[t][e] != (R::A((uint32_t)t) | R::E(e))) return false;
    return true;
}

// Swap S of the plan: word pairs (r0, r1 = r0 | 2^j) and lanes across tau
// bit i.  After it, word e of lane tau is the word (e with bit j := tau's
// bit i) of lane (tau with bit i := e's bit j): lanes whose bit i is set
// hand over r0 and take the partner's r1 in its place, the others hand over
// r1 and take the partner's r0.
template <class W, int LOGS, bool INV, int J, int LR, int S>
__device__ __forceinline__ void shfl_swaps(W (&x)[1 << LR], uint32_t tau) {
    using PL = XPlanOf<LOGS, INV, J, LR>;
    if constexpr (S < PL::value.nsw) {
        constexpr int i = PL::value.sw_tau[S], j = PL::value.sw_e[S];
        const bool up = (tau >> i) & 1u;
#pragma unroll
        for (int r0 = 0; r0 < (1 << LR); ++r0) {
            if (r0 & (1 << j)) continue;
            const int r1 = r0 | (1 << j);
            const W mine = up ? x[r0] : x[r1];
            const W got = __shfl_xor_sync(0xffffffffu, mine, 1 << i);
            if (up) x[r0] = got;
            else x[r1] = got;
        }
        shfl_swaps<W, LOGS, INV, J, LR, S + 1>(x, tau);
    }
}

// Round J - 1's words of a thread to round J's through shuffles, for a
// sub-transform whose 2^(LOGS - LR) threads are consecutive lanes of one
// warp (tau = lane mod 2^(LOGS - LR)); every lane of the warp takes part.
template <class W, int LOGS, bool INV, int J, int LR>
__device__ __forceinline__ void shfl_exchange(W (&x)[1 << LR], uint32_t tau) {
    using PL = XPlanOf<LOGS, INV, J, LR>;
    constexpr int NW = 1 << LR, LB = LOGS - LR;
    static_assert(LB <= 5, "a sub-transform's threads must fit one warp");
    static_assert(xplan_reaches_round<LOGS, INV, J, LR>(), "the shuffle plan must give round J's layout");
    shfl_swaps<W, LOGS, INV, J, LR, 0>(x, tau);
    // the two permutations as 4-bit fields of integer constants
    constexpr uint32_t TSRC = PL::value.tau_src[0] | (PL::value.tau_src[1] << 4) | (PL::value.tau_src[2] << 8) |
                              (PL::value.tau_src[3] << 12) | (PL::value.tau_src[4] << 16);
    constexpr uint32_t ESRC = PL::value.e_src[0] | (PL::value.e_src[1] << 4) | (PL::value.e_src[2] << 8) |
                              (PL::value.e_src[3] << 12);
    if constexpr (PL::value.tau_perm) {
        uint32_t src = 0;
#pragma unroll
        for (int b = 0; b < LB; ++b) src |= ((tau >> b) & 1u) << ((TSRC >> (4 * b)) & 15u);
#pragma unroll
        for (int e = 0; e < NW; ++e) x[e] = __shfl_sync(0xffffffffu, x[e], (int)src, 1 << LB);
    }
    W y[NW];
#pragma unroll
    for (int e = 0; e < NW; ++e) {
        uint32_t s = 0;
#pragma unroll
        for (int b = 0; b < LR; ++b) s |= (((uint32_t)e >> b) & 1u) << ((ESRC >> (4 * b)) & 15u);
        y[e] = x[s];
    }
#pragma unroll
    for (int e = 0; e < NW; ++e) x[e] = y[e];
}

// shared-memory word offset of u in sub-transform k (linear in u's bits)
template <class W, int LOGS, int KIND, int P = 0> __host__ __device__ constexpr uint32_t sm_off(uint32_t k, uint32_t u) {
    return KIND == TK_COLS ? cols_phys<W>(k, u, tile_k<W, LOGS, KIND, P>()) : k * rows_pitch<W, LOGS>() + pu<W>(u);
}

// Twiddles of one stage for this thread: CNT pairs, pair j at p[j * STRIDE]
// (level-transposed table, see level_pos); contiguous runs move as 16-byte
// vectors.  SMEM: the table is staged in shared memory (plain loads), else
// it is read through the read-only cache.
template <class W, int CNT, int STRIDE, bool SMEM>
__device__ __forceinline__ void load_tw(Tw<W> (&t)[8], const Tw<W> *__restrict__ p) {
    if (STRIDE == 1 && CNT >= 2 && sizeof(W) == 4) {
#pragma unroll
        for (int i = 0; i < CNT / 2; ++i) {
            uint4 v = SMEM ? reinterpret_cast<const uint4 *>(p)[i] : __ldg(reinterpret_cast<const uint4 *>(p) + i);
            t[2 * i].w = (W)v.x; t[2 * i].c = (W)v.y;
            t[2 * i + 1].w = (W)v.z; t[2 * i + 1].c = (W)v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < CNT; ++i) {
            if (sizeof(W) == 4) {
                uint2 v = SMEM ? reinterpret_cast<const uint2 *>(p)[i * STRIDE]
                               : __ldg(reinterpret_cast<const uint2 *>(p) + i * STRIDE);
                t[i].w = (W)v.x; t[i].c = (W)v.y;
            } else {
                ulonglong2 v = SMEM ? reinterpret_cast<const ulonglong2 *>(p)[i * STRIDE]
                                    : __ldg(reinterpret_cast<const ulonglong2 *>(p) + i * STRIDE);
                t[i].w = (W)v.x; t[i].c = (W)v.y;
            }
        }
    }
}

template <class W, int RED, bool INV, int LOGS, int J, bool SMEM, int LR = 4>
__device__ __forceinline__ void round_bfly(W (&x)[1 << LR], uint32_t tau, const Tw<W> *__restrict__ tw,
                                           const Lc<W> &k, bool last_pass, Tw<W> tn, Tw<W> twn) {
    using R = RoundOf<LOGS, INV, J, LR>;
    constexpr int RR = R::RR, LO = R::LO;
#pragma unroll
    for (int dd = 0; dd < RR; ++dd) {
        const int d = INV ? dd : RR - 1 - dd;
        const int b = LO + d;                  // index bit of this stage
        const int lvl = LOGS - 1 - b;          // table level: entries [2^lvl, 2^(lvl+1))
        Tw<W> t[8];
        const bool fold = INV && b == LOGS - 1 && last_pass;
        if (!fold) {
            if constexpr (RR == LR) {
                // full round: pair j of thread tau at 2^lvl + j * ntau + (tau >> LO)
                constexpr int NTAU_LOG = LOGS - LR - LO >= 0 ? LOGS - LR - LO : 0;
                const Tw<W> *p = tw + (1u << lvl) + (tau >> LO);
                switch (LR - 1 - d) {
                case 0: load_tw<W, 1, (1 << NTAU_LOG), SMEM>(t, p); break;
                case 1: load_tw<W, 2, (1 << NTAU_LOG), SMEM>(t, p); break;
                case 2: load_tw<W, 4, (1 << NTAU_LOG), SMEM>(t, p); break;
                default: load_tw<W, 8, (1 << NTAU_LOG), SMEM>(t, p); break;
                }
            } else {
                // short round: the stage's entries, shared by every thread
                const Tw<W> *p = tw + (1u << lvl);
                switch (RR - 1 - d) {
                case 0: load_tw<W, 1, 1, SMEM>(t, p); break;
                case 1: load_tw<W, 2, 1, SMEM>(t, p); break;
                default: load_tw<W, 4, 1, SMEM>(t, p); break;
                }
            }
        }
#pragma unroll
        for (int e = 0; e < (1 << LR); ++e) {
            if (e & (1 << d)) continue;
            const int j = (e & ((1 << RR) - 1)) >> (d + 1);
            if (!INV) {
                ct_bfly<RED, W>(x[e], x[e | (1 << d)], t[j], k);
            } else if (fold) {
                gs_bfly_last<RED, W>(x[e], x[e | (1 << d)], tn, twn, k);
            } else {
                gs_bfly<RED, W>(x[e], x[e | (1 << d)], t[j], k);
            }
        }
    }
}

template <class W, bool WARP_SYNC> __device__ __forceinline__ void tile_sync() {
    if (WARP_SYNC) __syncwarp();
    else __syncthreads();
}

// ------------------------------------------------ TMA / mbarrier helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// Raise the bytes the current phase waits for, without arriving.
__device__ __forceinline__ void mbar_add_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of the barrier, giving up after about 2^31 SM
// cycles (about a second): returns false then, and the caller reports
// NTT_ERR_TIMEOUT instead of hanging the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}
// 1-D bulk copy global -> shared, completing on `bar` (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// 2-D tiled tensor copy global -> shared of the box at (x, y).
__device__ __forceinline__ void tma_2d_g2s(void *dst, const void *tmap, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Pull global data into L2 ahead of its TMA load (no shared memory used).
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void prefetch_tensor_2d(const void *tmap, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(tmap), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Programmatic dependent launch: let the next launch on the stream be
// scheduled once every CTA of this grid has started (its CTAs then take
// the SM slots this grid frees and run their set-up), and wait until the
// previous grid on the stream has completed and its writes are visible.
// Without the launch attribute both are no-ops.
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Rounds J = 1 .. NR-1 of one sub-transform (round 0 is done by the caller
// on the words read from the staged tile); rounds exchange through the
// padded layout sm_off in `xs` (the tile's own stage buffer, whose staged
// words have all been read by then).
template <class W, int RED, bool INV, int LOGS, int KIND, bool WS, bool SMEM, int J, int P>
__device__ __forceinline__ void later_rounds(W (&x)[1 << radix_log<P>()], W *xs, uint32_t smb_k, uint32_t tau,
                                             const Tw<W> *__restrict__ tw, const Lc<W> &kk, bool last_pass,
                                             Tw<W> tn, Tw<W> twn) {
    constexpr int LR = radix_log<P>();
    constexpr int NW = 1 << LR;
    using R = RoundOf<LOGS, INV, J, LR>;
    // bit 6 of P: exchanges by warp shuffles where a chunk's threads are
    // lanes of one warp (not for 512-word chunks in rounds of three stages,
    // whose 64 threads span two warps)
    constexpr bool SHFL = (P & 64) != 0 && KIND == TK_CHUNKS && LOGS - LR <= 5;
    if constexpr (J < R::NR && SHFL) {
        shfl_exchange<W, LOGS, INV, J, LR>(x, tau);
        round_bfly<W, RED, INV, LOGS, J, SMEM, LR>(x, tau, tw, kk, last_pass, tn, twn);
        later_rounds<W, RED, INV, LOGS, KIND, WS, SMEM, J + 1, P>(x, xs, smb_k, tau, tw, kk, last_pass, tn, twn);
    } else if constexpr (J < R::NR) {
        using RP = RoundOf<LOGS, INV, J - 1, LR>;
        // a thread's words are consecutive (round at bit 0) in the rows
        // layout: move them as 16-byte vectors
        constexpr bool VST = KIND != TK_COLS && RP::LO == 0 && RP::RR == LR;
        constexpr bool VLD = KIND != TK_COLS && R::LO == 0 && R::RR == LR;
        constexpr int V = 16 / sizeof(W);
        {
            const uint32_t base = smb_k + sm_off<W, LOGS, KIND, P>(0, RP::A(tau));
            if (J > 1) tile_sync<W, WS>();   // readers of the previous exchange are done
            if constexpr (VST) {
#pragma unroll
                for (int v = 0; v < NW / V; ++v) {
                    W *q = xs + base + sm_off<W, LOGS, KIND, P>(0, (uint32_t)(v * V));
                    if (sizeof(W) == 4)
                        *reinterpret_cast<uint4 *>(q) = make_uint4((uint32_t)x[4 * v], (uint32_t)x[4 * v + 1],
                                                                   (uint32_t)x[4 * v + 2], (uint32_t)x[4 * v + 3]);
                    else
                        *reinterpret_cast<ulonglong2 *>(q) =
                            make_ulonglong2((unsigned long long)x[2 * v], (unsigned long long)x[2 * v + 1]);
                }
            } else {
#pragma unroll
                for (int e = 0; e < NW; ++e) xs[base + sm_off<W, LOGS, KIND, P>(0, RP::E(e))] = x[e];
            }
        }
        tile_sync<W, WS>();
        {
            const uint32_t base = smb_k + sm_off<W, LOGS, KIND, P>(0, R::A(tau));
            if constexpr (VLD) {
#pragma unroll
                for (int v = 0; v < NW / V; ++v) {
                    const W *q = xs + base + sm_off<W, LOGS, KIND, P>(0, (uint32_t)(v * V));
                    if (sizeof(W) == 4) {
                        uint4 w4 = *reinterpret_cast<const uint4 *>(q);
                        x[4 * v] = (W)w4.x; x[4 * v + 1] = (W)w4.y; x[4 * v + 2] = (W)w4.z; x[4 * v + 3] = (W)w4.w;
                    } else {
                        ulonglong2 w2 = *reinterpret_cast<const ulonglong2 *>(q);
                        x[2 * v] = (W)w2.x; x[2 * v + 1] = (W)w2.y;
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < NW; ++e) x[e] = xs[base + sm_off<W, LOGS, KIND, P>(0, R::E(e))];
            }
        }
        round_bfly<W, RED, INV, LOGS, J, SMEM, LR>(x, tau, tw, kk, last_pass, tn, twn);
        later_rounds<W, RED, INV, LOGS, KIND, WS, SMEM, J + 1, P>(x, xs, smb_k, tau, tw, kk, last_pass, tn, twn);
    }
}

// Staged tile layouts (where TMA puts a tile in shared memory):
//   cols             [S][K] dense (2-D box of K columns x S rows);
//   chunks, forward  [K][S + pad]: one bulk copy per chunk, the pad puts the
//                    two chunks of a warp on different bank halves for the
//                    first round's word-per-thread reads;
//   chunks, inverse  [K * S / R][R] rows of 128 bytes (R words) written by a
//                    2-D copy with the 128-byte swizzle (16-byte unit j of row
//                    r lands at unit j ^ (r mod 8)), so the first round's
//                    16-byte reads of 64 consecutive bytes per thread are
//                    conflict-free;
//   single           [K][S] dense (one bulk copy of K whole transforms).
// After the first round has read a tile, the same buffer holds the round
// exchanges (layout sm_off), so a buffer is sized for the larger of the two.
template <class W, int LOGS, int KIND, bool INV> __host__ __device__ constexpr bool stage_swizzled() {
    return KIND == TK_CHUNKS && INV;
}
template <class W, int LOGS, int KIND, bool INV> __host__ __device__ constexpr uint32_t stage_pitch() {
    return (KIND == TK_CHUNKS && !INV) ? (1u << LOGS) + (sizeof(W) == 4 ? 16u : 8u) : (1u << LOGS);
}
template <class W, int LOGS, int KIND, int P = 0> __host__ __device__ constexpr size_t xchg_words() {
    return KIND == TK_COLS ? (size_t)tile_k<W, LOGS, KIND, P>() * ((1u << LOGS) + (1u << LOGS) / 16)
                           : (size_t)tile_k<W, LOGS, KIND, P>() * rows_pitch<W, LOGS>();
}
template <class W, int LOGS, int KIND, bool INV, int P = 0> __host__ __device__ constexpr uint32_t tile_words() {
    return KIND == TK_COLS ? (tile_k<W, LOGS, KIND, P>() << LOGS)
                           : tile_k<W, LOGS, KIND, P>() * stage_pitch<W, LOGS, KIND, INV>();
}
// Alignment of the stage buffers: 1 KiB where a 128-byte-swizzled tensor
// copy lands in them (and in the item kernels, which mix tile kinds), else
// 128 bytes (tensor copies without swizzle, bulk copies).
template <class W, int LOGS, int KIND, bool INV, int P = 0> __host__ __device__ constexpr uint32_t stage_align() {
    return ((P & 3) != 0 || (KIND == TK_CHUNKS && INV)) ? 1024u : 128u;
}
template <class W, int LOGS, int KIND, bool INV, int P = 0> __host__ __device__ constexpr uint32_t buf_words() {
    constexpr size_t A = stage_align<W, LOGS, KIND, INV, P>() / sizeof(W);
    return (uint32_t)(((tile_words<W, LOGS, KIND, INV, P>() > xchg_words<W, LOGS, KIND, P>()
                            ? tile_words<W, LOGS, KIND, INV, P>()
                            : xchg_words<W, LOGS, KIND, P>()) +
                       A - 1) & ~(A - 1));
}
// Two buffers per CTA: the next tile lands while the current one computes.
// (A third, with two tiles in flight, measured no faster on GB300.)
template <class W, int LOGS, int KIND, int P = 0> __host__ __device__ constexpr uint32_t n_stages() { return 2u; }
// Twiddles staged in shared memory: the column table (2^LOGS pairs per limb)
// and, for 4-byte words, the chunk tables of a tile (K chunk tables).
template <class W, int LOGS, int KIND> __host__ __device__ constexpr bool tw_staged() {
    return KIND == TK_COLS || (KIND == TK_CHUNKS && sizeof(W) == 4);
}
// Bit 3 of P (chunk passes): the K sub-transforms of a tile are the same
// chunk of K consecutive polynomials (one chunk table per tile) instead of
// K consecutive chunks of one polynomial (K tables); with bit 7 as well,
// the same 2 consecutive chunks of K / 2 consecutive polynomials (two
// tables), for batches that K / 2 divides but K does not.
template <int KIND, int P> __host__ __device__ constexpr bool paired_chunks() {
    return KIND == TK_CHUNKS && (P & 8) != 0;
}
// chunk positions per paired tile (its twiddle tables)
template <int KIND, int P> __host__ __device__ constexpr uint32_t pair_positions() {
    return (P & 128) ? 2u : 1u;
}
template <class W, int LOGS, int KIND, int P = 0> __host__ __device__ constexpr uint32_t tw_pairs() {
    return !tw_staged<W, LOGS, KIND>() ? 0u
           : KIND == TK_COLS ? (1u << LOGS)
           : (paired_chunks<KIND, P>() ? pair_positions<KIND, P>() : tile_k<W, LOGS, KIND, P>()) *
                 chunk_tab_pitch<W, LOGS>();
}

// Pipeline state carried across run_tiles calls of one CTA: how often each
// stage buffer and the twiddle buffer have completed a phase.
struct PipeState {
    uint32_t uses[3];
    uint32_t tw_phase;
    // uses[s] with a run-time s, without indexing (which would put the
    // state in local memory)
    __device__ __forceinline__ uint32_t use(uint32_t s) const { return s == 0 ? uses[0] : (s == 1 ? uses[1] : uses[2]); }
};

// Process tiles [t_begin, t_end) of one pass.  One thread keeps the next
// tile in flight with TMA copies into shared memory (1-D bulk copies of
// contiguous rows tiles, 2-D tensor copies of column strips), completing on
// one mbarrier per buffer, and prefetches the tile after it into L2.  Tiles
// of the two-pass kinds run polynomial-fastest, so a CTA reuses one set of
// twiddles (staged in shared memory) for many consecutive tiles.  `bar`
// holds NS tile barriers and one twiddle barrier, initialised by the caller.
// Returns false if a wait ran out of time (the abort has been recorded).
template <class W, int RED, bool INV, int LOGS, int KIND, int P, bool OTF_K = false, bool DEP = false>
__device__ __forceinline__ bool run_tiles(const FArgs<W> &a, const CUtensorMap *tmap, uint32_t t_begin,
                                          uint32_t t_end, unsigned char *base, uint64_t *bar, PipeState &ps) {
    constexpr int LR = radix_log<P>();          // 2^LR words a thread
    constexpr int NW = 1 << LR;
    constexpr uint32_t S = 1u << LOGS;
    constexpr uint32_t T = S >> LR;
    constexpr uint32_t K = tile_k<W, LOGS, KIND, P>();
    constexpr uint32_t NS = n_stages<W, LOGS, KIND, P>();
    constexpr uint32_t BW = buf_words<W, LOGS, KIND, INV, P>();
    constexpr uint32_t SP = stage_pitch<W, LOGS, KIND, INV>();
    constexpr bool SWZ = stage_swizzled<W, LOGS, KIND, INV>();
    constexpr bool TWS = tw_staged<W, LOGS, KIND>();
    constexpr uint32_t TWP = tw_pairs<W, LOGS, KIND, P>();
    constexpr uint32_t CP = chunk_tab_pitch<W, KIND == TK_CHUNKS ? LOGS : 8>();
    constexpr uint32_t RW = 128 / sizeof(W);     // words per 128-byte row
    constexpr bool WS = KIND != TK_COLS && T <= 32;
    using R0 = RoundOf<LOGS, INV, 0, LR>;
    using RL = RoundOf<LOGS, INV, R0::NR - 1, LR>;
    // Per-plan passes (long runs of tiles per CTA, registers to spare):
    // refill a buffer right after the next tile's first barrier, which saves
    // a barrier per tile; keep the limb constants in registers across tiles;
    // load the fused product's second operand before the tile wait.  The
    // 256-thread item kernels (short runs, three CTAs per SM, one kernel for
    // every tile kind under a 128-register cap) refill at the end of each
    // tile and load constants per tile, which keeps them free of spills.
    constexpr bool LATE_REFILL = (P & 3) == 0 || (P & 3) == 3;
    // chunk tables made on the fly from the plan's seeds (OTF_K: the
    // per-plan chunk kernels of NTT_TW_OTF plans, 4-byte words, Shoup)
    constexpr bool OTF = OTF_K && KIND == TK_CHUNKS && LOGS == 8 && sizeof(W) == 4 && RED == RED_SHOUP && (P & 3) != 1 && TWS;
    static_assert(!OTF_K || OTF, "twiddles made on the fly: 4-byte-word Shoup chunk kernels only");
    W *stage = reinterpret_cast<W *>(base);
    Tw<W> *tws = reinterpret_cast<Tw<W> *>(stage + (size_t)NS * BW);
    if (t_begin >= t_end) return true;

    const uint32_t N = 1u << a.logN;
    const uint32_t tid = threadIdx.x;
    uint32_t k, tau;
    if (KIND == TK_COLS) { k = tid % K; tau = tid / K; }
    else { tau = tid % T; k = tid / T; }
    const bool active = tid < K * T;       // (all threads of the block take part in barriers)
    const uint32_t smb_k = sm_off<W, LOGS, KIND, P>(k, 0);
    const uint32_t L = a.L;
    const uint32_t B = (uint32_t)(a.ntrans / L);
    // log2 of the row length N2 (two-pass kinds): the chunk size, or, for
    // the column pass, 256 (a compile-time constant, so the strided stores
    // take immediate offsets) unless bit 5 of P asks for the plan's split
    const uint32_t S2 = KIND == TK_CHUNKS ? (uint32_t)LOGS : ((P & 32) ? a.s2 : kN2Log);
    const uint32_t N1 = KIND == TK_SINGLE ? 1u : (N >> S2);
    // paired chunk tiles: sub k is chunk position pos0 + k % KG of
    // polynomial p + k / KG (the launcher makes
    // sure K divides the batch); else sub k is position pos0 + k
    constexpr bool PAIR = paired_chunks<KIND, P>();
    constexpr uint32_t KG = PAIR ? pair_positions<KIND, P>() : K;   // positions (chunks, columns) per tile
    constexpr uint32_t KP = K / KG;                                 // polynomials per tile
    static_assert(!PAIR || (K % KG == 0 && KG * KP == K), "a paired tile is KP polynomials x KG chunks");
    const uint32_t per = KIND == TK_SINGLE ? 1u : (KIND == TK_COLS ? (1u << S2) : N1) / KG;
    const uint32_t BP = B / KP;               // polynomial steps per position group
    // Tile cursor: single tiles are K consecutive transforms; two-pass tiles
    // run polynomial-fastest, then position group, then limb.  It is decoded
    // once and then stepped, so the loop does no division.
    struct Cur {
        uint32_t p, g, l;
    };
    auto cur_at = [&](uint32_t tile) {
        Cur c;
        if (KIND == TK_SINGLE) { c.p = tile * K; c.g = 0; c.l = 0; }
        else { c.p = (tile % BP) * KP; const uint32_t r = tile / BP; c.g = r % per; c.l = r / per; }
        return c;
    };
    auto cur_next = [&](Cur &c) {
        if (KIND == TK_SINGLE) { c.p += K; return; }
        c.p += KP;
        if (c.p == B) { c.p = 0; if (++c.g == per) { c.g = 0; ++c.l; } }
    };
    auto cur_t = [&](const Cur &c) -> uint64_t {
        return KIND == TK_SINGLE ? (uint64_t)c.p : (uint64_t)c.p * L + c.l;
    };
    // twiddle table of limb l (column pass: [L][N1] tables) or of the
    // chunks of group g
    auto tw_src = [&](uint32_t l, uint32_t g) -> const Tw<W> * {
        if (KIND == TK_CHUNKS) return a.tw + (size_t)l * N1 * CP + (size_t)g * KG * CP;
        return a.tw + (size_t)l * S;
    };
    auto issue = [&](const Cur &c, uint32_t s) {
        const uint64_t t = cur_t(c);
        const uint32_t pos0 = c.g * KG;
        W *dst = stage + (size_t)s * BW;
        if (KIND == TK_COLS) {
            const uint32_t rows = S < 256 ? S : 256u;
            mbar_expect_tx(&bar[s], (K << LOGS) * (uint32_t)sizeof(W));
            for (uint32_t r0 = 0; r0 < S; r0 += rows)
                tma_2d_g2s(dst + r0 * K, tmap, (int)pos0, (int)(t * N1 + r0), &bar[s]);
        } else if (SWZ) {
            mbar_expect_tx(&bar[s], K * S * (uint32_t)sizeof(W));
            if constexpr (PAIR) {
                // one box of KG S / RW rows per polynomial (1 KiB-aligned
                // blocks, so the swizzle phase is the smem row's)
                for (uint32_t c2 = 0; c2 < KP; ++c2) {
                    const uint64_t row0 = ((t + (uint64_t)c2 * L) * N + ((size_t)pos0 << S2)) / RW;
                    tma_2d_g2s(dst + c2 * KG * S, tmap, 0, (int)row0, &bar[s]);
                    if (a.pw_b) prefetch_l2(a.pw_b + (t + (uint64_t)c2 * L) * N + ((size_t)pos0 << S2),
                                            KG * S * (uint32_t)sizeof(W));
                }
            } else {
                const uint64_t row0 = (t * N + ((size_t)pos0 << S2)) / RW;
                tma_2d_g2s(dst, tmap, 0, (int)row0, &bar[s]);
                // the fused product's second operand (read by plain loads)
                // into L2 while this tile's copy is in flight
                if (a.pw_b) prefetch_l2(a.pw_b + t * N + ((size_t)pos0 << S2), K * S * (uint32_t)sizeof(W));
            }
        } else if (KIND == TK_CHUNKS) {
            mbar_expect_tx(&bar[s], K * S * (uint32_t)sizeof(W));
            const W *src = a.data + t * N + ((size_t)pos0 << S2);
            // sub c2: chunk pos0 + c2 % KG of polynomial t + c2 / KG (the
            // next chunk of the polynomial, or, paired, of the next one)
            for (uint32_t c2 = 0; c2 < K; ++c2)
                bulk_g2s(dst + c2 * SP, src + (size_t)(c2 / KG) * L * N + (size_t)(c2 % KG) * S, S * sizeof(W),
                         &bar[s]);
        } else {
            const uint64_t nval = a.ntrans - t < K ? a.ntrans - t : K;
            const uint32_t bytes = (uint32_t)(nval * S * sizeof(W));
            mbar_expect_tx(&bar[s], bytes);
            bulk_g2s(dst, a.data + t * N, bytes, &bar[s]);
        }
    };

    // L2 prefetch of a tile (one beyond the ones staged in shared memory)
    auto prefetch = [&](const Cur &c) {
        const uint64_t t = cur_t(c);
        const uint32_t pos0 = c.g * KG;
        if (KIND == TK_COLS) {
            const uint32_t rows = S < 256 ? S : 256u;
            for (uint32_t r0 = 0; r0 < S; r0 += rows) prefetch_tensor_2d(tmap, (int)pos0, (int)(t * N1 + r0));
        } else if (KIND == TK_CHUNKS) {
            if constexpr (PAIR) {
                for (uint32_t c2 = 0; c2 < KP; ++c2)
                    prefetch_l2(a.data + (t + (uint64_t)c2 * L) * N + ((size_t)pos0 << S2),
                                KG * S * (uint32_t)sizeof(W));
            } else {
                prefetch_l2(a.data + t * N + ((size_t)pos0 << S2), K * S * (uint32_t)sizeof(W));
            }
        } else {
            const uint64_t nval = a.ntrans - t < K ? a.ntrans - t : K;
            prefetch_l2(a.data + t * N, (uint32_t)(nval * S * sizeof(W)));
        }
    };

    Cur ahead = cur_at(t_begin);   // next tile to issue (thread 0)
    Cur cur = ahead;               // tile being processed
    uint32_t tw_key = 0xffffffffu;  // (limb, group) of the staged twiddles
    bool tw_pending = false;        // the first table was requested early
    // limb constants, reloaded only when the limb changes (tiles run
    // polynomial-fastest, so rarely)
    uint32_t kk_l = 0xffffffffu;
    Lc<W> kk;
    Tw<W> tn{}, twn{};
    auto load_limb = [&](uint32_t l) {
        kk.load(a.lc + l);
        if (INV && a.final_pass) {
            tn.w = (W)a.lc[l].ninv_w; tn.c = (W)a.lc[l].ninv_c;
            twn.w = (W)a.lc[l].ninv_w1_w; twn.c = (W)a.lc[l].ninv_w1_c;
        }
        kk_l = l;
    };
    if constexpr (DEP) {
        // launched as a dependent of the previous launch on the stream:
        // request the first tile's twiddle table (no data) before waiting
        // for that launch to end
        if constexpr (TWS && !OTF) {
            if (tid == 0) {
                fence_proxy_async();
                mbar_expect_tx(&bar[NS], TWP * (uint32_t)sizeof(Tw<W>));
                bulk_g2s(tws, tw_src(cur.l, cur.g), TWP * (uint32_t)sizeof(Tw<W>), &bar[NS]);
            }
            tw_key = KIND == TK_CHUNKS ? cur.l * per + cur.g : cur.l;
            tw_pending = true;
        }
        // and the first tile's limb constants and tensor map
        if constexpr (KIND != TK_SINGLE && LATE_REFILL) load_limb(cur.l);
        if constexpr (KIND == TK_COLS || SWZ) {
            if (tid == 0) asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
        }
        griddep_wait();
    }
    if (tid == 0) {
        fence_proxy_async();   // the buffers may have been read by a previous call
        // (test hook: the first barrier waits for bytes no copy delivers)
        // (per-plan launches: CTA 0; one-launch two-pass form: the item
        // holding the first tile)
        if (a.stall_tx && ((P & 3) == 0 ? blockIdx.x == 0 : t_begin == 0)) mbar_add_tx(&bar[0], a.stall_tx);
        for (uint32_t s = 0; s < NS && t_begin + s < t_end; ++s) { issue(ahead, s); cur_next(ahead); }
        if (t_begin + NS < t_end) prefetch(ahead);
    }
    uint32_t n_issued = t_end - t_begin < NS ? t_end - t_begin : NS;   // local tiles issued so far
    uint32_t &tw_phase = ps.tw_phase;
    bool ok = true;

    uint32_t i = 0;
    for (uint32_t tile = t_begin; tile < t_end; ++tile, ++i, cur_next(cur)) {
        const uint32_t s = i % NS;
        const uint32_t parity = (ps.use(s) + i / NS) & 1u;
        const uint32_t pos0 = cur.g * KG;
        // this thread's sub-transform: transform t, chunk / column position pk
        const uint64_t t = KIND == TK_SINGLE ? cur_t(cur) + k : (PAIR ? cur_t(cur) + (uint64_t)(k / KG) * L : cur_t(cur));
        const uint32_t pk = PAIR ? pos0 + k % KG : pos0 + k;
        const bool valid = t < a.ntrans;
        const uint32_t l = KIND == TK_SINGLE ? (uint32_t)((valid ? t : 0) % L) : cur.l;
        if (!LATE_REFILL || l != kk_l) load_limb(l);
        const Tw<W> *twb;
        if (TWS) {
            // restage the twiddles when the tile needs another table (every
            // thread finished with the old one before the previous refill barrier)
            const uint32_t key = KIND == TK_CHUNKS ? cur.l * per + cur.g : cur.l;
            if (tw_pending) {
                // the first tile's table, requested before the dependency wait
                ok = ok && mbar_wait_bounded(&bar[NS], tw_phase & 1u);
                ++tw_phase;
                tw_pending = false;
            } else if (key != tw_key) {
                // inside a run of tiles, the previous tile may still be
                // reading the old table (without LATE_REFILL the end-of-tile
                // barrier has already waited for it)
                if (LATE_REFILL && i > 0) __syncthreads();
                if constexpr (OTF) {
                    // (the launcher checks that the plan supplies seeds)
                    // the K chunk tables of this tile from their seeds:
                    // entry j of chunk r at stage level lv = floor(log2 j)
                    // is A_lv(r) * B[j] (see the plan's table builder)
                    // (thread tid makes entries j = tid + NT m of every
                    // chunk of the tile: one root pair and one stage level
                    // per j serve the K chunks; the loads of MB values of j
                    // are all issued before their products, so their
                    // latencies overlap)
                    constexpr uint32_t NT = K * T, JPT = S / NT, MB = JPT < 4 ? JPT : 4;
                    constexpr uint32_t KT = KG;     // tables in the tile
                    static_assert(NT <= S && S % NT == 0 && JPT % MB == 0, "threads per chunk table");
                    const W *sd = a.tw_seed + ((size_t)cur.l * N1 + pos0) * 8;
                    const Tw<W> *rt = a.tw_root + (size_t)cur.l * S;
#pragma unroll 1
                    for (uint32_t m0 = 0; m0 < JPT; m0 += MB) {
                        Tw<W> rb[MB];
                        W sa[MB][KT];
#pragma unroll
                        for (uint32_t m = 0; m < MB; ++m) {
                            const uint32_t j = tid + (m0 + m) * NT;
                            const uint32_t lv = j ? 31 - __clz(j) : 0;
                            rb[m] = ldtw(rt + j);
#pragma unroll
                            for (uint32_t c2 = 0; c2 < KT; ++c2) sa[m][c2] = __ldg(sd + c2 * 8 + lv);
                        }
#pragma unroll
                        for (uint32_t m = 0; m < MB; ++m) {
                            const uint32_t j = tid + (m0 + m) * NT;
#pragma unroll
                            for (uint32_t c2 = 0; c2 < KT; ++c2) {
                                Tw<W> tv{0, 0};
                                if (j != 0) {
                                    tv.w = mul_full<RED_SHOUP, W>(sa[m][c2], rb[m], kk);
                                    tv.c = shoup_quotient(tv.w, kk);
                                }
                                tws[c2 * CP + j] = tv;
                            }
                        }
                    }
                    __syncthreads();
                } else {
                    if (tid == 0) {
                        fence_proxy_async();
                        mbar_expect_tx(&bar[NS], TWP * (uint32_t)sizeof(Tw<W>));
                        bulk_g2s(tws, tw_src(cur.l, cur.g), TWP * (uint32_t)sizeof(Tw<W>), &bar[NS]);
                    }
                    ok = ok && mbar_wait_bounded(&bar[NS], tw_phase & 1u);
                    ++tw_phase;
                }
                tw_key = key;
            }
            twb = tws + (KIND == TK_CHUNKS ? (k % KG) * CP : 0);
        } else {
            twb = KIND == TK_CHUNKS ? tw_src(l, 0) + (size_t)pk * CP : a.tw + (size_t)l * N;
        }
        // fused pointwise product (inverse chunk pass): b's 16 words at this
        // thread's positions, loaded before the tile wait so they overlap it
        constexpr bool PW = KIND == TK_CHUNKS && INV && R0::RR == LR && R0::LO == 0;
        constexpr int NV = NW / (16 / (int)sizeof(W));
        using V16 = typename std::conditional<sizeof(W) == 4, uint4, ulonglong2>::type;
        V16 bv[PW ? NV : 1];
        const bool use_pw = PW && a.pw_b && valid;
        const V16 *bq = use_pw ? reinterpret_cast<const V16 *>(a.pw_b + t * N + ((size_t)pk << S2) +
                                                              R0::A(tau))
                               : nullptr;
        if constexpr (PW && LATE_REFILL) {
            if (use_pw) {
#pragma unroll
                for (int v = 0; v < NV; ++v) bv[v] = __ldg(bq + v);
            }
        }
        // ---- round 0 from the staged tile
        ok = ok && mbar_wait_bounded(&bar[s], parity);
        W *sb = stage + (size_t)s * BW;
        W x[NW];
        {
            const uint32_t A0 = R0::A(tau);
            if (KIND == TK_COLS) {
#pragma unroll
                for (int e = 0; e < NW; ++e) x[e] = sb[(A0 | R0::E(e)) * K + k];
            } else if (SWZ && R0::RR == LR && R0::LO == 0) {
                // 2^LR consecutive words of chunk k from swizzled 128-byte rows
                constexpr int V = 16 / sizeof(W);            // words per 16-byte unit
#pragma unroll
                for (int v = 0; v < NW / V; ++v) {
                    const uint32_t u = A0 + v * V;            // first word of the unit
                    const uint32_t row = k * (S / RW) + u / RW;
                    const uint32_t unit = ((u % RW) / V) ^ (row & 7u);
                    const W *q = sb + row * RW + unit * V;
                    if (sizeof(W) == 4) {
                        uint4 w4 = *reinterpret_cast<const uint4 *>(q);
                        x[4 * v] = (W)w4.x; x[4 * v + 1] = (W)w4.y; x[4 * v + 2] = (W)w4.z; x[4 * v + 3] = (W)w4.w;
                    } else {
                        ulonglong2 w2 = *reinterpret_cast<const ulonglong2 *>(q);
                        x[2 * v] = (W)w2.x; x[2 * v + 1] = (W)w2.y;
                    }
                }
            } else if (R0::RR == LR && R0::LO == 0) {
                // 2^LR consecutive words: 16-byte loads
                const W *q = sb + k * SP + A0;
#pragma unroll
                for (int v = 0; v < NW / (16 / (int)sizeof(W)); ++v) {
                    if (sizeof(W) == 4) {
                        uint4 w4 = reinterpret_cast<const uint4 *>(q)[v];
                        x[4 * v] = (W)w4.x; x[4 * v + 1] = (W)w4.y; x[4 * v + 2] = (W)w4.z; x[4 * v + 3] = (W)w4.w;
                    } else {
                        ulonglong2 w2 = reinterpret_cast<const ulonglong2 *>(q)[v];
                        x[2 * v] = (W)w2.x; x[2 * v + 1] = (W)w2.y;
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < NW; ++e) x[e] = sb[k * SP + (A0 | R0::E(e))];
            }
        }
        if constexpr (PW) {
            // the inverse of a (.) b: multiply by b's words first
            if (use_pw) {
                if constexpr (!LATE_REFILL) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) bv[v] = __ldg(bq + v);
                }
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if constexpr (sizeof(W) == 4) {
                        x[4 * v] = mul_var<RED>(x[4 * v], (W)bv[v].x, kk);
                        x[4 * v + 1] = mul_var<RED>(x[4 * v + 1], (W)bv[v].y, kk);
                        x[4 * v + 2] = mul_var<RED>(x[4 * v + 2], (W)bv[v].z, kk);
                        x[4 * v + 3] = mul_var<RED>(x[4 * v + 3], (W)bv[v].w, kk);
                    } else {
                        x[2 * v] = mul_var<RED>(x[2 * v], (W)bv[v].x, kk);
                        x[2 * v + 1] = mul_var<RED>(x[2 * v + 1], (W)bv[v].y, kk);
                    }
                }
            }
        }
        // every thread has its words (the buffer now serves the exchanges),
        // and every thread is done with the previous tile: with LATE_REFILL
        // its buffer takes the tile NS - 1 ahead of this one here
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(a.status, 2u);
            ok = false;
            break;
        }
        if (LATE_REFILL && tid == 0 && i > 0 && tile + NS - 1 < t_end) {
            fence_proxy_async();
            issue(ahead, (i + NS - 1) % NS);
            cur_next(ahead);
            ++n_issued;
            if (tile + NS < t_end) prefetch(ahead);
        }
        round_bfly<W, RED, INV, LOGS, 0, TWS, LR>(x, tau, twb, kk, INV && a.final_pass, tn, twn);
        later_rounds<W, RED, INV, LOGS, KIND, WS, TWS, 1, P>(x, sb, smb_k, tau, twb, kk, INV && a.final_pass, tn, twn);
        if (!LATE_REFILL) {
            // the buffer and the twiddles are free: refill with the tile NS ahead
            __syncthreads();
            if (tid == 0 && tile + NS < t_end) {
                fence_proxy_async();
                issue(ahead, s);
                cur_next(ahead);
                ++n_issued;
                if (tile + NS + 1 < t_end) prefetch(ahead);
            }
        }
        if (a.final_pass) {
#pragma unroll
            for (int e = 0; e < NW; ++e) {
                W y = x[e];
                if (!INV) y = csub<W>(y, kk.two_q);
                x[e] = csub<W>(y, kk.q);
            }
        }
        // ---- last round straight to global memory
        if (valid && active) {
            const uint32_t AL = RL::A(tau);
            if (KIND == TK_COLS) {
                W *g = a.out + t * N + pos0 + k;
#pragma unroll
                for (int e = 0; e < NW; ++e) g[(size_t)(AL | RL::E(e)) << S2] = x[e];
            } else {
                W *g = KIND == TK_SINGLE ? a.out + t * N : a.out + t * N + ((size_t)pk << S2);
                if (RL::RR == LR && RL::LO == 0) {
                    W *q = g + AL;
#pragma unroll
                    for (int v = 0; v < NW / (16 / (int)sizeof(W)); ++v) {
                        if (sizeof(W) == 4)
                            reinterpret_cast<uint4 *>(q)[v] = make_uint4((uint32_t)x[4 * v], (uint32_t)x[4 * v + 1],
                                                                         (uint32_t)x[4 * v + 2], (uint32_t)x[4 * v + 3]);
                        else
                            reinterpret_cast<ulonglong2 *>(q)[v] = make_ulonglong2((unsigned long long)x[2 * v],
                                                                                   (unsigned long long)x[2 * v + 1]);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < NW; ++e) g[AL | RL::E(e)] = x[e];
                }
            }
        }
    }
    const uint32_t n_local = t_end - t_begin;
    if (!ok) {
        // an aborted wait: let the copies already in flight (local tiles
        // i .. i+NS-1 and the twiddle table) land before the CTA goes on,
        // again with a time limit
        if (tid == 0) {
            for (uint32_t j = i; j < n_issued; ++j) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&bar[j % NS], (ps.use(j % NS) + j / NS) & 1u))
                    if (clock64() - t0 > (1ll << 30)) break;
            }
            if (TWS && tw_phase > 0) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&bar[NS], (tw_phase - 1) & 1u))
                    if (clock64() - t0 > (1ll << 30)) break;
            }
        }
        return false;
    }
    for (uint32_t s = 0; s < NS; ++s) ps.uses[s] += (n_local + NS - 1 - s) / NS;
    return true;
}

// Per-plan fused pass: CTA c processes tiles [c T / G, (c+1) T / G).
// PP: the tile configuration (see tile_k): 0, or 3 for 16-chunk tiles.
// Launch bounds: column passes of up to 256 points with 4-byte words (512
// threads), radix 16 and Shoup or Montgomery twiddles are held to the
// registers that let three CTAs share an SM, as their shared memory allows
// (40 a thread, no spills; forward call at N = 2^16, 32 limbs, 16
// polynomials 0.1214 -> 0.1195 ms with the forward pass held too);
// 512-point column passes take 1024 threads.
template <class W, int RED, int LOGS, int KIND, bool INV, int P> __host__ __device__ constexpr bool fused_cols3() {
    return KIND == TK_COLS && sizeof(W) == 4 && RED != RED_BARRETT && LOGS <= 8 && radix_log<P>() == 4;
}
template <class W, int RED, int LOGS, int KIND, bool INV, int P> __host__ __device__ constexpr int fused_max_threads() {
    return fused_cols3<W, RED, LOGS, KIND, INV, P>() ? 512 : (sizeof(W) == 4 ? 1024 : 512);
}
template <class W, int RED, int LOGS, int KIND, bool INV, int P> __host__ __device__ constexpr int fused_min_blocks() {
    return fused_cols3<W, RED, LOGS, KIND, INV, P>() ? 3 : 1;
}
template <class W, int RED, bool INV, int LOGS, int KIND, int PP, bool OTF_K = false>
__global__ void __launch_bounds__(fused_max_threads<W, RED, LOGS, KIND, INV, PP>(),
                                  fused_min_blocks<W, RED, LOGS, KIND, INV, PP>())
k_fused(const __grid_constant__ FArgs<W> a) {
    static_assert(tile_k<W, LOGS, KIND, PP>() * ((1u << LOGS) >> radix_log<PP>()) <=
                      (uint32_t)fused_max_threads<W, RED, LOGS, KIND, INV, PP>(),
                  "a tile's threads must fit the launch bound");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr uint32_t NS = n_stages<W, LOGS, KIND, PP>();
    constexpr uint32_t BW = buf_words<W, LOGS, KIND, INV, PP>();
    constexpr uint32_t TWP = tw_pairs<W, LOGS, KIND, PP>();
    constexpr uint32_t AL = stage_align<W, LOGS, KIND, INV, PP>();
    unsigned char *base = smem_raw + ((AL - (smem_addr(smem_raw) & (AL - 1))) & (AL - 1));
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + (size_t)NS * BW * sizeof(W) + (size_t)TWP * 2 * sizeof(W));
    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s <= NS; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    // the next launch may be scheduled now; run_tiles waits for the
    // previous one before its first data access
    griddep_launch_dependents();
    __syncthreads();
    PipeState ps{{0, 0, 0}, 0};
    const uint32_t t_begin = (uint32_t)((uint64_t)blockIdx.x * a.ntiles / gridDim.x);
    const uint32_t t_end = (uint32_t)((uint64_t)(blockIdx.x + 1) * a.ntiles / gridDim.x);
    run_tiles<W, RED, INV, LOGS, KIND, PP, OTF_K, true>(a, &a.tmap, t_begin, t_end, base, bar, ps);
}

template <class W, int LOGS, int KIND, bool INV, int P = 0> __host__ __device__ constexpr size_t fused_smem_bytes() {
    return (size_t)n_stages<W, LOGS, KIND, P>() * buf_words<W, LOGS, KIND, INV, P>() * sizeof(W) +
           (size_t)tw_pairs<W, LOGS, KIND, P>() * 2 * sizeof(W) + 8 * 4 + 16 + stage_align<W, LOGS, KIND, INV, P>();
}

}  // namespace nttgb
