// tc5.cu -- the tensor-core four-step form on the fifth-generation tensor
// cores (tcgen05.mma, accumulators in tensor memory).
//
// Same split as tc.cu (Sec. II "Six-step": the N = 2^16 transform as 256-point
// sub-transforms, each a dense 256 x 256 matrix product mod q, with the
// inter-step twiddles in an epilogue), same tables of matrices and output
// order.  What differs is how a product mod q is made exact on hardware whose
// only 8-bit-class tcgen05 kinds are floating point on this target:
//
//   * Both operands are split into four BALANCED 8-bit digits,
//     x = sum_i d_i 256^i with d_i in [-128, 128): the digits of a data word
//     are the bytes of x + 0x80808080 minus 128, those of a matrix entry are
//     precomputed.  Every digit is an fp16 integer (exact).
//   * The 16 digit products are accumulated by diagonal s = i + j into seven
//     fp32 accumulators in tensor memory: one M = 128, N = 256 product per
//     data digit i against the four matrix digit planes at once (they are
//     contiguous rows of one operand) lands A_i B_j in diagonal i + j.  A
//     tile's first product (digit 0, first K step) overwrites diagonals
//     0-3; diagonals 4-6 are zeroed at the start and by each epilogue
//     after reading.  A diagonal sums at most 4 x 256
//     products of magnitude <= 128 * 128 = 2^14, so every partial sum is an
//     integer of magnitude <= 2^24: exactly representable, so fp32
//     accumulation loses nothing, in any order -- ASSUMING the tensor core
//     adds with a full 24-bit fp32 significand.  The instruction set does not
//     state the internal precision of the accumulation; bit-exact results on
//     data words whose digits sit at the ends of their range (-128 and +127),
//     against the matrices of many primes, are the evidence for it.
//   * The epilogue reads the diagonals back (tcgen05.ld), recombines
//     sum_s D_s (2^(8 s) mod q) plus 7 2^24 q (which makes it positive) in
//     64-bit integers (< 2^58: one signed 32 x 32 -> 64-bit multiply-add
//     per diagonal) and reduces mod q (Barrett), then applies
//     the inter-step twiddle (Shoup) where the pass has one.
//
// GEMM view, D[m][n] = sum_k A[m][k] B[n][k], both operands K-major in shared
// memory (64-byte swizzle, tile M = 128, N = 64, K chunks of 32); A is 128
// data rows (converted to digits by the CTA), B 64 matrix rows (TMA):
//   column pass  A[n2][n1] = src[n1][n2], B = matrix [u][n1],
//                D[n2][u] -> out[u][n2];
//   row pass     A[r][n2] = src[r][n2],   B = matrix [v][n2],
//                D[r][v]  -> out[r][v].
// Each pass reads src and writes dst (out of place: a tile's output rows are
// other tiles' input rows).
//
// Roles in a CTA (one per SM: 224 KiB of stage buffers, 448 of the 512
// tensor-memory columns): warp 16 lane 0 issues the TMA copies of the data
// words (four 16 KiB stages), warp 18 lane 0 those of the matrix digit
// planes (four 16 KiB stages), each as far ahead as its stages allow;
// warps 0-7 turn the staged data words into digit planes (three 32 KiB
// stages); warp 17 lane 0 issues the MMAs; warps 8-15, and warps 0-7 in
// the gap between their conversions, run the epilogue (warp w reads
// tensor-memory lanes 32 (w % 4) .. and 16 of the 64 columns of each
// diagonal).  The accumulators are one set: the next tile's MMAs start
// when the epilogue has read them (and zeroed 4-6) (two sets of half-width tiles
// were measured slower: each 32-column tile converts the whole data block
// again, and the extra digit traffic through shared memory costs more
// than the overlap gains).
// mbarriers between the roles, every wait bounded (about a second of SM
// clock) -- on expiry the call records
// NTT_ERR_TIMEOUT, all roles leave their loops, and the CTA waits (bounded)
// for its copies and products in flight before it frees its tensor memory.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "fused.cuh"
#include "plan.hpp"

namespace nttgb {

constexpr uint32_t kT5M = 128, kT5N = 64, kT5KC = 32;   // K chunks of 32: 64-byte operand rows
constexpr uint32_t kT5Dig = 4, kT5Diag = 7;
constexpr uint32_t kT5Row = kT5KC * 2;                 // bytes of one operand row (fp16)
constexpr uint32_t kT5StageA = kT5Dig * kT5M * kT5Row;   // 32 KiB
constexpr uint32_t kT5StageB = kT5Dig * kT5N * kT5Row;   // 16 KiB
constexpr uint32_t kT5StageR = kT5M * kT5KC * 4;          // 16 KiB of data words
constexpr uint32_t kT5NA = 3, kT5NB = 4, kT5NR = 4;       // digit / matrix / data-word stage buffers
constexpr uint32_t kT5Chunks = 256 / kT5KC;               // K chunks per tile
constexpr uint32_t kT5ConvWarps = 8;                 // warps 0-7: data digits
constexpr uint32_t kT5EpiWarps = 8;                  // warps 8-15: epilogue
// warp 16: TMA of the data words; warp 17: MMAs; warp 18: TMA of the
// matrix digit planes
constexpr uint32_t kT5TmaWarp = kT5ConvWarps + kT5EpiWarps, kT5MmaWarp = kT5TmaWarp + 1,
                   kT5TmaBWarp = kT5MmaWarp + 1;
constexpr uint32_t kT5Threads = (kT5TmaBWarp + 1) * 32;
constexpr uint32_t kT5TmemCols = 512;
constexpr size_t kT5SmemData =
    (size_t)kT5NA * kT5StageA + (size_t)kT5NB * kT5StageB + (size_t)kT5NR * kT5StageR;   // 224 KiB
constexpr size_t kT5Smem = kT5SmemData + 1024 + 256;

struct Tc5Args {
    const uint32_t *src;
    uint32_t *dst;
    CUtensorMap cmap;               // matrix digit planes, fp16 (k: 256, rows), box 32 x 64, 64-byte swizzle
    CUtensorMap dmap;               // src words (256 a row), box 128 x 32 (column pass) or 32 x 128 (row pass)
    uint32_t mat_row0;              // cmap row of (this pass's matrix, limb 0, digit 0, row 0)
    const Tw<uint32_t> *tw;         // [L][256][256] epilogue twiddles, or null
    const LimbConst *lc;
    const uint32_t *wdiag;          // [L][8]: 2^(8 s) mod q for s < 7
    uint32_t *status;
    uint32_t L;
    uint32_t ntiles;                // 8 per transform (2 row blocks x 4 column tiles)
    uint32_t stall_tx;              // test hook: extra bytes CTA 0's first matrix copy waits for
};

namespace {

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ void t5_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void t5_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (tmem) (+)= A (smem) * B (smem)^T, kind::f16, cta_group::1
__device__ __forceinline__ void t5_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on `bar` once every MMA this thread issued before has completed
__device__ __forceinline__ void t5_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void t5_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 64-byte swizzle (rows of 32
// fp16), 8-row atoms of 512 bytes one after another (stride 512 bytes),
// start at `saddr`.
__device__ __forceinline__ uint64_t t5_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);          // start address
    d |= (uint64_t)1u << 16;                          // leading byte offset (unused when swizzled)
    d |= (uint64_t)(512u >> 4) << 32;                 // stride byte offset
    d |= (uint64_t)1u << 46;                          // descriptor version
    d |= (uint64_t)4u << 61;                          // 64-byte swizzle
    return d;
}
// Instruction descriptor, kind::f16: fp16 A and B, fp32 D, both K-major,
// M = 128.
// The four matrix digit planes of a stage lie one after another, so they
// form one 256-row B operand: a single M = 128, N = 256 product of data
// digit plane i with all of them adds A_i B_j to the accumulator of
// diagonal i + j for j = 0..3 at once (columns 64 (i + j), contiguous).
constexpr uint32_t kT5IdescAll = (1u << 4) | (0u << 7) | (0u << 10) | (((kT5Dig * kT5N) >> 3) << 17) |
                                 ((kT5M >> 4) << 24);

__device__ __forceinline__ void t5_st_zero4(uint32_t taddr) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %1, %1, %1};" ::"r"(taddr), "r"(0u) : "memory");
}
__device__ __forceinline__ void t5_st_zero8(uint32_t taddr) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
                 "r"(0u)
                 : "memory");
}
__device__ __forceinline__ void t5_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// byte offset of 16-byte unit `unit` (0..3) of row `row` in a K-major
// 64-byte-swizzled operand (unit index XOR bits 1-2 of the row)
__device__ __forceinline__ uint32_t t5_swz(uint32_t row, uint32_t unit) {
    return (row >> 3) * 512u + (row & 7u) * 64u + ((unit ^ ((row >> 1) & 3u)) << 4);
}

// Balanced digits of eight words as fp16, packed for one 16-byte unit per
// digit plane: out[d] holds digit d of words 0..7.
__device__ __forceinline__ void t5_digits(const uint32_t (&x)[8], uint4 (&out)[4]) {
    uint32_t y[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) y[i] = x[i] + 0x80808080u;
    const __half2 bias = __halves2half2(__ushort_as_half((unsigned short)0x6480u),
                                        __ushort_as_half((unsigned short)0x6480u));   // 1152
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const uint32_t sel = (uint32_t)d | ((uint32_t)d << 4) | ((uint32_t)(4 + d) << 8) | ((uint32_t)(4 + d) << 12);
        uint32_t w[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            uint32_t t = __byte_perm(y[2 * p], y[2 * p + 1], sel);
            t = (t & 0x00FF00FFu) | 0x64006400u;           // fp16 1024 + byte, twice
            __half2 h = __hsub2(*reinterpret_cast<__half2 *>(&t), bias);
            w[p] = *reinterpret_cast<uint32_t *>(&h);
        }
        out[d] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Wait for phase `parity` of `bar`, bounded; false on expiry or abort.
__device__ __forceinline__ bool t5_wait(uint64_t *bar, uint32_t parity, volatile uint32_t *abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > (1ll << 31)) return false;
    }
    return true;
}

__device__ __forceinline__ void t5_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

struct T5Tile {
    uint32_t t, mb, nb, l;
};
__device__ __forceinline__ T5Tile t5_tile(uint32_t tile, uint32_t L) {
    T5Tile r;
    r.t = tile >> 3;
    r.mb = (tile >> 2) & 1u;
    r.nb = tile & 3u;
    r.l = r.t % L;
    return r;
}

}  // namespace

template <bool ROWP>
__global__ void __launch_bounds__(kT5Threads, 1) k_tc5(const __grid_constant__ Tc5Args a) {
    extern __shared__ __align__(1024) unsigned char t5_smem_raw[];
    unsigned char *base = t5_smem_raw + ((1024u - (smem_addr(t5_smem_raw) & 1023u)) & 1023u);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + kT5SmemData);
    // b_full / b_empty: matrix stages (TMA in, products done); r_full /
    // r_empty: data-word stages (TMA in, converted); a_full / a_empty:
    // digit stages (digits written, products done)
    uint64_t *b_full = bars, *b_empty = bars + kT5NB, *r_full = bars + 2 * kT5NB,
             *r_empty = bars + 2 * kT5NB + kT5NR, *a_full = bars + 2 * kT5NB + 2 * kT5NR,
             *a_empty = bars + 2 * kT5NB + 2 * kT5NR + kT5NA, *acc_full = bars + 2 * kT5NB + 2 * kT5NR + 2 * kT5NA,
             *acc_empty = acc_full + 1, *drain = acc_full + 2;
    __shared__ uint32_t s_tmem;
    __shared__ uint32_t s_abort;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr uint32_t NCONV = kT5ConvWarps * 32, NEPI = kT5EpiWarps * 32;

    if (tid == 0) {
        for (int s = 0; s < (int)kT5NB; ++s) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
        }
        for (int s = 0; s < (int)kT5NR; ++s) {
            mbar_init(&r_full[s], 1);
            mbar_init(&r_empty[s], NCONV);
        }
        for (int s = 0; s < (int)kT5NA; ++s) {
            mbar_init(&a_full[s], NCONV);
            mbar_init(&a_empty[s], 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, NCONV + NEPI);
        mbar_init(drain, 1);
        fence_mbar_init();
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(kT5TmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    t5_fence_before();
    __syncthreads();
    t5_fence_after();
    const uint32_t tmem = s_tmem;
    volatile uint32_t *abort_flag = &s_abort;
    const uint32_t ntiles = a.ntiles;
    // stages: A = data digit planes (converted here), B = matrix digit
    // planes (TMA), R = data words of a chunk (TMA, read by the converters)
    auto stage_a = [&](uint32_t s) { return base + (size_t)s * kT5StageA; };
    auto stage_b = [&](uint32_t s) { return base + (size_t)kT5NA * kT5StageA + (size_t)s * kT5StageB; };
    auto stage_r = [&](uint32_t s) {
        return base + (size_t)kT5NA * kT5StageA + (size_t)kT5NB * kT5StageB + (size_t)s * kT5StageR;
    };
    const uint32_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint32_t nchunks = kT5Chunks * my_tiles;
    auto tile_of = [&](uint32_t g) { return blockIdx.x + (g / kT5Chunks) * gridDim.x; };
    bool ok = true;

    if (warp == kT5TmaWarp || warp == kT5TmaBWarp) {
        // ------------------------------------------------ TMA producers
        // chunk g: its data words into R stage g % NR (warp 16) and its
        // matrix digit planes into B stage g % NB (warp 18), each as soon
        // as that stage is free; two threads, so that neither kind of copy
        // waits behind the other's free stage
        if (lane == 0) {
            const bool rw = warp == kT5TmaWarp;
            const uint32_t NS = rw ? kT5NR : kT5NB;
            uint64_t *full = rw ? r_full : b_full, *empty = rw ? r_empty : b_empty;
            uint32_t n = 0;               // copies issued
            for (uint32_t g = 0; g < nchunks && ok; ++g) {
                const T5Tile T = t5_tile(tile_of(g), a.L);
                const uint32_t c = g % kT5Chunks;
                const uint32_t st = g % NS;
                if (g >= NS && !t5_wait(&empty[st], ((g - NS) / NS) & 1u, abort_flag)) { ok = false; break; }
                if (rw) {
                    mbar_expect_tx(&full[st], kT5StageR);
                    // column pass: words src[32 c + k][128 mb + m]; row pass:
                    // src[128 mb + m][32 c + k]
                    if (ROWP)
                        tma_2d_g2s(stage_r(st), &a.dmap, (int)(c * kT5KC), (int)(T.t * 256 + T.mb * kT5M), &full[st]);
                    else
                        tma_2d_g2s(stage_r(st), &a.dmap, (int)(T.mb * kT5M), (int)(T.t * 256 + c * kT5KC), &full[st]);
                } else {
                    const uint32_t mrow0 = a.mat_row0 + T.l * kT5Dig * 256 + T.nb * kT5N;
                    mbar_expect_tx(&full[st], kT5StageB);
                    // (test hook: this copy's barrier waits for bytes that never come)
                    if (a.stall_tx && g == 0 && blockIdx.x == 0) mbar_add_tx(&full[st], a.stall_tx);
                    for (uint32_t d = 0; d < kT5Dig; ++d)
                        tma_2d_g2s(stage_b(st) + d * kT5N * kT5Row, &a.cmap, (int)(c * kT5KC), (int)(mrow0 + d * 256),
                                   &full[st]);
                }
                ++n;
            }
            if (!ok) {
                atomicExch(const_cast<uint32_t *>(abort_flag), 1u);
                // copies still in flight land before the CTA leaves (bounded):
                // chunk h used stage h % NS for its (h / NS + 1)-th phase
                for (uint32_t h = n >= NS ? n - NS : 0; h < n; ++h) {
                    const long long t0 = clock64();
                    while (!mbar_try_wait(&full[h % NS], (h / NS) & 1u) && clock64() - t0 < (1ll << 30)) {
                    }
                }
            }
        }
    } else if (warp == kT5MmaWarp) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t g = 0;
            for (uint32_t ti = 0; ti < my_tiles && ok; ++ti) {
                // accumulators zeroed (at the start, then by each epilogue)
                if (!t5_wait(acc_empty, ti & 1u, abort_flag)) { ok = false; break; }
                t5_fence_after();
                for (uint32_t c = 0; c < kT5Chunks && ok; ++c, ++g) {
                    const uint32_t s = g % kT5NA, sb = g % kT5NB;
                    if (!t5_wait(&b_full[sb], (g / kT5NB) & 1u, abort_flag) ||
                        !t5_wait(&a_full[s], (g / kT5NA) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    t5_fence_after();
                    // descriptors of the stages' digit planes; a digit plane or
                    // a K step of 16 (32 bytes) moves the start address field
                    const uint64_t da = t5_desc(smem_addr(stage_a(s))), db = t5_desc(smem_addr(stage_b(sb)));
#pragma unroll
                    for (uint32_t ks = 0; ks < kT5KC / 16; ++ks) {
#pragma unroll
                        for (uint32_t i = 0; i < kT5Dig; ++i)
                            t5_mma(tmem + i * kT5N, da + ((i * (kT5M * kT5Row) + ks * 32) >> 4),
                                   db + ((ks * 32) >> 4), kT5IdescAll, (c | ks | i) != 0 ? 1u : 0u);
                    }
                    t5_commit(&a_empty[s]);
                    t5_commit(&b_empty[sb]);
                }
                if (ok) t5_commit(acc_full);
            }
            if (!ok) atomicExch(const_cast<uint32_t *>(abort_flag), 1u);
            // every product issued has completed before the CTA frees the
            // tensor memory
            t5_commit(drain);
            const long long t0 = clock64();
            while (!mbar_try_wait(drain, 0) && clock64() - t0 < (1ll << 31)) {
            }
        }
    } else {
        // ------------------------------------- converters (warps 0-7) and
        // epilogue (warps 8-15, and the converters between conversions): the
        // next tile's first digit stages are made while the epilogue drains
        // the accumulators of the last one
        const bool conv = warp < kT5ConvWarps;
        const uint32_t ew = warp - kT5ConvWarps;        // epilogue warp 0..7
        // Data operand A[m][k] of a tile, m < 128, for chunk c (k in 32 c ..):
        //   column pass  m = n2 - 128 mb, k = n1: word src[k][128 mb + m],
        //                staged as R[k][m];
        //   row pass     m = r - 128 mb,  k = n2: word src[128 mb + m][k],
        //                staged as R[m][k].
        // 16-byte unit u (k = 8u .. 8u + 7) of row m is task (m, u); each
        // thread takes TASKS of them (lanes along m for the column pass,
        // along u for the row pass: conflict-free shared-memory reads).
        constexpr uint32_t UNITS = kT5KC / 8;
        constexpr uint32_t TASKS = kT5M * UNITS / NCONV;
        auto task_mu = [&](uint32_t q, uint32_t &m, uint32_t &u) {
            const uint32_t task = tid + q * NCONV;
            if (ROWP) { m = task / UNITS; u = task % UNITS; }
            else { m = task % kT5M; u = task / kT5M; }
        };
        // one chunk: words from R stage sr to digit planes in A stage s
        auto convert_chunk = [&](uint32_t sr, uint32_t s) {
            const uint32_t *R = reinterpret_cast<const uint32_t *>(stage_r(sr));
            uint32_t xw[TASKS][8];
#pragma unroll
            for (uint32_t q = 0; q < TASKS; ++q) {
                uint32_t m, u;
                task_mu(q, m, u);
                if (ROWP) {
                    const uint4 *p = reinterpret_cast<const uint4 *>(R + m * kT5KC + 8 * u);
                    const uint4 v0 = p[0], v1 = p[1];
                    xw[q][0] = v0.x; xw[q][1] = v0.y; xw[q][2] = v0.z; xw[q][3] = v0.w;
                    xw[q][4] = v1.x; xw[q][5] = v1.y; xw[q][6] = v1.z; xw[q][7] = v1.w;
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) xw[q][e] = R[(8 * u + e) * kT5M + m];
                }
            }
            unsigned char *dst = stage_a(s);
#pragma unroll
            for (uint32_t q = 0; q < TASKS; ++q) {
                uint32_t m, u;
                task_mu(q, m, u);
                uint4 dg[4];
                t5_digits(xw[q], dg);
                const uint32_t off = t5_swz(m, u);
#pragma unroll
                for (uint32_t d = 0; d < kT5Dig; ++d) *reinterpret_cast<uint4 *>(dst + d * (kT5M * kT5Row) + off) = dg[d];
            }
            // the words have been used (not only requested), so the stage
            // may take the chunk NR ahead: the TMA copy into it is an
            // async-proxy write, which the barrier does not order after
            // loads still in flight
            t5_arrive(&r_empty[sr]);
            // generic-proxy stores, read next by the tensor cores
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            t5_arrive(&a_full[s]);
        };
        // The epilogue is shared by all 16 warps: warp w reads tensor-memory
        // lanes 32 (w % 4) .. (its rows m) and columns 16 slice .. of each
        // diagonal, slice = w / 4 for the converter warps, 2 + (w - 8) / 4
        // for the epilogue warps.
        const uint32_t quad = warp & 3u;
        const uint32_t slice = conv ? (warp >> 2) : 2 + (ew >> 2);
        constexpr uint32_t kSliceCols = kT5N / 4;
        auto epilogue = [&](uint32_t tile, uint32_t ti) -> bool {
            constexpr uint32_t GW = 4;      // columns a group (tcgen05.ld .x4)
            const T5Tile T = t5_tile(tile, a.L);
            const uint32_t m = 32 * quad + lane;
            const uint32_t n0 = slice * kSliceCols;
            Lc<uint32_t> kk;
            kk.load(a.lc + T.l);
            uint32_t w7[kT5Diag];
#pragma unroll
            for (uint32_t d = 0; d < kT5Diag; ++d) w7[d] = __ldg(a.wdiag + 8 * T.l + d);
            // each diagonal D (|D| <= 2^24) times its weight (< 2^30) is one
            // signed 32 x 32 -> 64-bit multiply-add; |sum| < 7 2^24 q, so
            // adding 7 2^24 q (a multiple of q) makes it positive
            const int64_t off = (int64_t)kk.q * (7ll << 24);
            // output word (row, column) of the transform: column pass
            // out[u][n2] = out[64 nb + n][128 mb + m]; row pass
            // out[r][v] = out[128 mb + m][64 nb + n]
            uint32_t *outt = a.dst + (size_t)T.t * 65536;
            const Tw<uint32_t> *twt = a.tw ? a.tw + (size_t)T.l * 65536 : nullptr;
            auto tw_at = [&](uint32_t n) -> const Tw<uint32_t> * {
                return twt + (ROWP ? (size_t)(T.mb * kT5M + m) * 256 + T.nb * kT5N + n
                                   : (size_t)(T.nb * kT5N + n) * 256 + T.mb * kT5M + m);
            };
            // the inter-step twiddles of the slice, loaded before the wait
            // for the products (their latency overlaps it)
            Tw<uint32_t> tws16[kSliceCols];
            if (twt) {
#pragma unroll
                for (uint32_t cc = 0; cc < kSliceCols; ++cc) tws16[cc] = ldtw(tw_at(n0 + cc));
            }
            if (!t5_wait(acc_full, ti & 1u, abort_flag)) return false;
            t5_fence_after();
#pragma unroll
            for (uint32_t grp = 0; grp < kSliceCols / GW; ++grp) {
                uint32_t f[kT5Diag][GW];
#pragma unroll
                for (uint32_t d = 0; d < kT5Diag; ++d) {
                    const uint32_t taddr = tmem + ((32u * quad) << 16) + d * kT5N + n0 + GW * grp;
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                                 : "=r"(f[d][0]), "=r"(f[d][1]), "=r"(f[d][2]), "=r"(f[d][3])
                                 : "r"(taddr));
                }
                t5_wait_ld();
                // the next tile's first product (digit 0, which does not
                // accumulate) writes diagonals 0-3; 4-6 accumulate onto zeros
#pragma unroll
                for (uint32_t d = kT5Dig; d < kT5Diag; ++d)
                    t5_st_zero4(tmem + ((32u * quad) << 16) + d * kT5N + n0 + GW * grp);
                uint32_t v[GW];
#pragma unroll
                for (uint32_t cc = 0; cc < GW; ++cc) {
                    int64_t comb = off;
#pragma unroll
                    for (uint32_t d = 0; d < kT5Diag; ++d)
                        comb += (int64_t)__float2int_rn(__uint_as_float(f[d][cc])) * (int64_t)(int32_t)w7[d];
                    // in [0, 2q); the Shoup twiddle product takes any word,
                    // so only a pass without twiddles reduces it further
                    const uint32_t r = barrett_lazy((uint64_t)comb, kk);
                    v[cc] = twt ? mul_full<RED_SHOUP>(r, tws16[GW * grp + cc], kk) : csub<uint32_t>(r, kk.q);
                }
                if (ROWP) {
                    *reinterpret_cast<uint4 *>(outt + (size_t)(T.mb * kT5M + m) * 256 + T.nb * kT5N + n0 + GW * grp) =
                        make_uint4(v[0], v[1], v[2], v[3]);
                } else {
#pragma unroll
                    for (uint32_t cc = 0; cc < GW; ++cc)
                        outt[(size_t)(T.nb * kT5N + n0 + GW * grp + cc) * 256 + T.mb * kT5M + m] = v[cc];
                }
            }
            t5_wait_st();
            t5_fence_before();
            t5_arrive(acc_empty);
            return true;
        };

        // diagonals 4-6 start at zero (the first product of a tile, data
        // digit 0 against the four matrix digits, writes 0-3 without
        // accumulating; the rest accumulate): this thread's row, its slice
        for (uint32_t d = kT5Dig; d < kT5Diag; ++d)
            for (uint32_t c8 = 0; c8 < kSliceCols / 8; ++c8)
                t5_st_zero8(tmem + ((32u * quad) << 16) + d * kT5N + slice * kSliceCols + 8 * c8);
        t5_wait_st();
        t5_fence_before();
        t5_arrive(acc_empty);
        if (conv) {
            // chunk g: wait for its data words (TMA) and for its digit stage
            // (the products of chunk g - NA done), then convert.  The
            // converters are idle while a tile's accumulators drain (the
            // next tile's products wait for the drain), so they take half of
            // each epilogue: that of tile i just before chunk NA - 1 of tile
            // i + 1.  Its chunks 0 .. NA - 2 are converted while tile i's
            // last products run; chunk NA - 1's stage frees only when they
            // end, and its digits are needed only NA - 1 chunks of products
            // after the drain
            for (uint32_t g = 0; g < nchunks && ok; ++g) {
                if (g >= kT5Chunks && g % kT5Chunks == kT5NA - 1) {
                    const uint32_t ti = g / kT5Chunks - 1;
                    ok = epilogue(tile_of(kT5Chunks * ti), ti);
                    if (!ok) break;
                }
                const uint32_t sr = g % kT5NR, s = g % kT5NA;
                if (!t5_wait(&r_full[sr], (g / kT5NR) & 1u, abort_flag)) { ok = false; break; }
                if (g >= kT5NA && !t5_wait(&a_empty[s], ((g - kT5NA) / kT5NA) & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                convert_chunk(sr, s);
            }
            // the last tile's accumulators
            if (ok && my_tiles > 0) ok = epilogue(tile_of(kT5Chunks * (my_tiles - 1)), my_tiles - 1);
        } else {
            for (uint32_t ti = 0; ti < my_tiles && ok; ++ti) ok = epilogue(tile_of(kT5Chunks * ti), ti);
        }
        if (!ok) atomicExch(const_cast<uint32_t *>(abort_flag), 1u);
    }
    // ---------------------------------------------------------- teardown
    t5_fence_before();
    __syncthreads();
    if (tid == 0 && *abort_flag) atomicOr(a.status, 2u);
    if (warp == 0) {
        t5_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kT5TmemCols)
                     : "memory");
    }
}

}  // namespace nttgb

namespace nttgb {

namespace {
using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn t5_encoder() {
    static EncodeFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess && fn)
            encode = reinterpret_cast<EncodeFn>(fn);
    }
    return encode;
}
// matrix digit planes: fp16 rows of 256, box of 32 (K) x 64 rows, 64-byte swizzle
cudaError_t make_t5_cmap(CUtensorMap *m, const void *tab, uint64_t rows) {
    EncodeFn encode = t5_encoder();
    if (!encode) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {256, rows};
    cuuint64_t strides[1] = {256 * 2};
    cuuint32_t box[2] = {kT5KC, kT5N};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(tab), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
// data words of a pass: rows of 256 words; box 128 x 32 (column pass:
// 32 rows k of 128 columns m) or 32 x 128 (row pass: 128 rows m of 32 k)
cudaError_t make_t5_dmap(CUtensorMap *m, const void *src, uint64_t ntrans, bool rowp) {
    EncodeFn encode = t5_encoder();
    if (!encode) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {256, ntrans * 256};
    cuuint64_t strides[1] = {256 * 4};
    cuuint32_t box[2] = {rowp ? kT5KC : kT5M, rowp ? kT5M : kT5KC};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void *>(src), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <bool ROWP> cudaError_t t5_launch(const Tc5Args &a, cudaStream_t st) {
    static int sms = 0;
    if (!sms) {
        cudaError_t e = cudaFuncSetAttribute(k_tc5<ROWP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kT5Smem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const unsigned grid = a.ntiles < (uint32_t)sms ? a.ntiles : (unsigned)sms;
    k_tc5<ROWP><<<grid, kT5Threads, kT5Smem, st>>>(a);
    return cudaGetLastError();
}
}  // namespace

// Tables (plan->d_tc5): matrix digit planes [4][L][4 digits][256][256] fp16
// (balanced digits; matrices as in tc.cu: 0 forward column, 1 forward row,
// 2 inverse row, 3 inverse column; row = output index, column = sum index).
// Twiddles and the powers 2^(8 s) mod q come from plan->d_tc (tc.cu layout).
cudaError_t launch_tc5(ntt_plan_s &p, void *data, uint32_t batch, bool inverse, cudaStream_t st) {
    const uint64_t ntrans = (uint64_t)batch * p.L;
    if (ntrans * 8 >= (1ull << 32)) return cudaErrorInvalidValue;
    const uint8_t *mats = reinterpret_cast<const uint8_t *>(p.d_tc);
    const Tw<uint32_t> *tws = reinterpret_cast<const Tw<uint32_t> *>(mats + (size_t)p.L * 16 * 65536);
    const uint32_t *pow8 = reinterpret_cast<const uint32_t *>(tws + (size_t)p.L * 2 * 65536);
    Tc5Args a;
    std::memset(&a, 0, sizeof(a));
    cudaError_t e = make_t5_cmap(&a.cmap, p.d_tc5, (uint64_t)4 * p.L * 1024);
    if (e != cudaSuccess) return e;
    a.lc = p.d_limb;
    a.wdiag = pow8;
    a.status = p.d_status;
    a.L = p.L;
    a.ntiles = (uint32_t)(ntrans * 8);
    a.stall_tx = (p.flags & NTT_TEST_STALL) && !inverse ? 16u : 0u;
    uint32_t *d = reinterpret_cast<uint32_t *>(data), *s = reinterpret_cast<uint32_t *>(p.d_scratch);
    auto row0 = [&](int m) { return (uint32_t)m * p.L * 1024; };
    auto pass = [&](bool rowp, const uint32_t *src, uint32_t *dst) -> cudaError_t {
        a.src = src;
        a.dst = dst;
        cudaError_t pe = make_t5_dmap(&a.dmap, src, ntrans, rowp);
        if (pe != cudaSuccess) return pe;
        return rowp ? t5_launch<true>(a, st) : t5_launch<false>(a, st);
    };
    if (!inverse) {
        a.mat_row0 = row0(0); a.tw = tws;
        if ((e = pass(false, d, s)) != cudaSuccess) return e;
        a.mat_row0 = row0(1); a.tw = nullptr; a.stall_tx = 0;
        e = pass(true, s, d);
    } else {
        a.mat_row0 = row0(2); a.tw = tws + (size_t)p.L * 65536;
        if ((e = pass(true, d, s)) != cudaSuccess) return e;
        a.mat_row0 = row0(3); a.tw = nullptr;
        e = pass(false, s, d);
    }
    p.last_launches += 2;
    return e;
}

}  // namespace nttgb
