// ragged.hpp -- device-side description of a ragged batch.
//
// A ragged batch is a set of jobs (polynomials of any N in 2^12 .. 2^17, any
// limb count, 4- or 8-byte words, forward or inverse).  Its work is a list of
// items -- a range of tiles of one pass of one job -- split into four
// phases that respect the pass order of every transform:
//   0: forward single-pass tiles and forward column passes
//   1: forward chunk passes
//   2: inverse single-pass tiles and inverse chunk passes
//   3: inverse column passes
// The items of each word size run in a persistent cooperative kernel of
// their own (two launches in a row: the 4-byte kernel is not held to the
// 8-byte one's registers); in each, CTAs take items from an atomic counter
// per phase and meet at a grid barrier between phases.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "modarith.cuh"

namespace nttgb {

struct RJob {
    void *data;
    const void *tw[4];          // main forward, main inverse, chunk forward, chunk inverse
    const LimbConst *lc;
    uint64_t ntrans;            // batch * L
    uint32_t logN, L;
};

struct RItem {
    uint32_t job, code, t0, t1; // code: see ragged_code()
};

struct RaggedArgs {
    const RJob *jobs;
    const CUtensorMap *tmaps;   // per job: [0] column strips, [1] 128-byte rows (swizzled)
    const RItem *items;
    uint32_t phase_begin[5];    // items of phase p: [phase_begin[p], phase_begin[p+1])
    uint32_t *counters;         // 4 item counters, zeroed before each launch
    uint32_t *bar_count;        // grid barrier arrivals
    uint32_t *bar_gen;          // grid barrier generation
    uint32_t *status;           // bit 1: a wait ran out of time
    uint32_t *abort_flag;
    uint32_t stall;             // test hook (NTT_TEST_STALL): CTA 0 leaves
                                // before the first grid barrier
};

// Kinds of work items: single-pass 4096-word transforms, column passes with
// 2^5 .. 2^9 rows, 256-word chunk passes; x direction x word size.
enum : uint32_t { RK_SINGLE12 = 0, RK_COLS5 = 1, RK_CHUNKS = 6, RK_KINDS = 7 };
__host__ __device__ constexpr uint32_t ragged_code(bool w64, bool inv, uint32_t kind) {
    return (w64 ? 2 * RK_KINDS : 0) + (inv ? RK_KINDS : 0) + kind;
}

// One persistent kernel per word size (W = uint32_t, uint64_t).
template <int RED, class W> cudaError_t ragged_kernel_launch(const RaggedArgs &a, unsigned grid, cudaStream_t st);
template <int RED, class W> cudaError_t ragged_kernel_config(size_t *smem, int *blocks_per_sm);

}  // namespace nttgb
