// plan.hpp -- internal plan object shared by the API and the launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/ntt.h"
#include "modarith.cuh"

namespace nttgb {

enum FusedMode : int { FUSED_STAGES = 0, FUSED_SINGLE = 1, FUSED_TWO_PASS = 2, FUSED_CLUSTER = 3 };
// Forms of a two-pass direction: chunk pass on one-warp CTAs (2-chunk
// tiles), on 256-thread CTAs (16-chunk tiles), or both passes in one
// streamed launch; the first two again with the chunk pass's exchanges
// between rounds by warp shuffles (4-byte words, table twiddles).
enum TwoPassForm : int { FORM_SMALL = 0, FORM_WIDE = 1, FORM_STREAMED = 2, FORM_SMALL_SHFL = 3, FORM_WIDE_SHFL = 4 };
constexpr int kForms = 5;
inline bool form_is_shfl(int f) { return f == FORM_SMALL_SHFL || f == FORM_WIDE_SHFL; }

// Largest transform done in one pass of the fused kernel (one CTA holds the
// whole transform in shared memory): 2^14 words of 4 bytes, 2^13 of 8.
constexpr int kSingleMaxLog32 = 14;
constexpr int kSingleMaxLog64 = 13;
constexpr int kLogR = 4;          // 16 words per thread in the fused kernel
constexpr int kChunkLog = 8;      // default pass-B sub-transform size 256
// Two-pass splits N = 2^s1 x 2^s2 the per-plan kernels take (the autotuner
// picks one per shape): chunks of 2^7 .. 2^9 words, column passes of
// 2^5 .. 2^9 points.  NTT_STREAMED and NTT_TW_OTF plans and the ragged
// kernel's plans keep s2 = kChunkLog.
constexpr int kChunkLogMin = 7, kChunkLogMax = 9;
constexpr int kColsLogMin = 5, kColsLogMax = 9;
// One pass on a cluster of eight CTAs (cluster.cuh, flag NTT_CLUSTER):
// N = 2^16, 4-byte words.
constexpr int kClusterLogN = 16;
// One-launch two-pass form (stream.cuh): a plan keeps kStreamRing counter
// sets of stream_set_words(L) words (L limb counts, queue head, exit count,
// abort flag), used by its calls in turn.
constexpr uint32_t kStreamRing = 16;
inline constexpr uint32_t stream_set_words(uint32_t L) { return ((L + 3) + 31) & ~31u; }
// ntt_polymul_host pipelines its work in at most kHostChunks chunks of
// whole pairs; fused plans with fewer than kHostMinChunks pairs split each
// pair into limb windows instead, so that there are about kHostMinChunks
// chunks (measured on GB300 at N = 2^16, 32 limbs: 1 pair 0.180 -> 0.157 ms
// with four windows; more or smaller chunks were slower).
constexpr uint32_t kHostChunks = 8;
constexpr uint32_t kHostMinChunks = 4;

}  // namespace nttgb

struct ntt_plan_s {
    uint32_t N = 0, logN = 0, L = 0, flags = 0;
    ntt_variant variant = NTT_FUSED;
    int red = 0;
    bool word64 = false, bitrev_order = false, check = false;
    std::vector<uint64_t> q, psi;
    int device = 0;

    // device memory (all owned)
    nttgb::LimbConst *d_limb = nullptr;
    // variant (per-stage) tables, [L][N] twiddle pairs each
    void *d_w_fwd = nullptr;     // omega^e
    void *d_w_inv = nullptr;     // omega^-e
    void *d_twist = nullptr;     // psi^n
    void *d_untwist = nullptr;   // N^-1 psi^-n
    // fused tables: [L][N] twiddle pairs each for single-pass plans, [L][N1]
    // (the column pass's entries) for two-pass plans
    void *d_main_fwd = nullptr;  // psi^bitrev(i)
    void *d_main_inv = nullptr;  // psi^-bitrev(i)
    void *d_chunk_fwd = nullptr; // pass-B per-chunk layout of psi^bitrev
    void *d_chunk_inv = nullptr;
    // NTT_TW_OTF two-pass plans instead of the chunk tables: [L][N1][8]
    // stage seeds (words) and [L][256] root pairs per direction
    bool tw_otf = false;
    void *d_seed_fwd = nullptr, *d_seed_inv = nullptr;
    void *d_root_fwd = nullptr, *d_root_inv = nullptr;
    void *d_tc = nullptr;        // tensor-core four-step tables (see tc.cu)
    void *d_tc5 = nullptr;       // their matrices as fp16 balanced digits (tc5.cu)
    bool tc_imma = false;        // NTT_TC_IMMA: warp-level mma.sync form
    // cluster form (cluster.cuh): [L][8][8192 + 16] twiddle pairs each
    void *d_clu_fwd = nullptr;
    void *d_clu_inv = nullptr;
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    // two-pass plans: progress counters of the one-launch form (stream.cuh),
    // a ring of sets, one per call
    uint32_t *d_stream_ctr = nullptr;
    uint32_t stream_seq = 0;
    bool streamed = false;       // NTT_STREAMED: both passes in one streamed launch
    uint32_t stream_tiles = 0;   // tiles per streamed work item (0: default)
    // Two-pass form per direction and batch bucket (floor(log2 batch)),
    // from the tuning table at plan creation; -1: the default (FORM_SMALL
    // forward, FORM_WIDE inverse; FORM_STREAMED under NTT_STREAMED).
    int8_t tuned_form[2][32];
    int form_for(uint32_t batch, bool inverse) const {
        uint32_t b = 0;
        while (b < 31 && (2u << b) <= batch) ++b;
        const int t = tuned_form[inverse ? 1 : 0][b];
        // (the streamed form exists for 256-word chunks in rounds of four
        // stages, not with NTT_TW_OTF)
        const bool stream_ok = !tw_otf && s2 == (uint32_t)nttgb::kChunkLog && lr == 4;
        // (the shuffle forms: 4-byte words and twiddle tables)
        const bool shfl_ok = !tw_otf && !word64;
        if (t >= 0 && (t != nttgb::FORM_STREAMED || stream_ok) && (!nttgb::form_is_shfl(t) || shfl_ok)) return t;
        if (streamed && stream_ok) return nttgb::FORM_STREAMED;
        return inverse ? nttgb::FORM_WIDE : nttgb::FORM_SMALL;
    }
    uint32_t *d_status = nullptr;
    uint32_t last_launches = 0;
    uint64_t table_bytes = 0;    // device bytes of the tables above

    // ntt_polymul_host pipeline: copy streams and events, made on first use
    bool aux_ready = false;
    cudaStream_t aux_h2d = nullptr, aux_d2h = nullptr;
    cudaEvent_t aux_ev[2 + 2 * nttgb::kHostChunks] = {};

    int fused_mode = nttgb::FUSED_STAGES;
    uint32_t s1 = 0, s2 = 0;     // two-pass split: N = 2^s1 * 2^s2
    bool split_fixed = false;    // the split and radix were given (autotuner
                                 // candidates, the ragged kernel's plans,
                                 // streamed and on-the-fly-twiddle plans)
    uint32_t lr = 4;             // two-pass passes: rounds of lr stages on
                                 // 2^lr words a thread (4 or 3; tables laid
                                 // out for it)

    size_t word_bytes() const { return word64 ? 8 : 4; }
    size_t limb_words() const { return (size_t)N; }
};

namespace nttgb {

// Launchers (return the CUDA error of the last launch; count launches).
cudaError_t launch_variant(ntt_plan_s &p, ntt_variant v, void *data, uint32_t batch, bool inverse, cudaStream_t st);
cudaError_t launch_fused(ntt_plan_s &p, void *data, uint32_t batch, bool inverse, cudaStream_t st);
cudaError_t launch_pointwise(ntt_plan_s &p, void *c, const void *a, const void *b, uint32_t batch, cudaStream_t st);
cudaError_t launch_bitrev_permute(ntt_plan_s &p, void *data, uint32_t batch, cudaStream_t st);
cudaError_t launch_check_range(ntt_plan_s &p, const void *data, uint32_t batch, cudaStream_t st);
cudaError_t launch_tc(ntt_plan_s &p, void *data, uint32_t batch, bool inverse, cudaStream_t st);
cudaError_t launch_tc5(ntt_plan_s &p, void *data, uint32_t batch, bool inverse, cudaStream_t st);

ntt_status ensure_scratch(ntt_plan_s &p, uint32_t batch, cudaStream_t st);
// The autotuner's choices for the plan's shape (tune.cu): its two-pass
// split (unless fixed), then the forms per direction and batch bucket.
void apply_tuning(ntt_plan_s &p);
// Whether a two-pass split s2 (chunks of 2^s2 words) serves a plan of
// 2^logN words: column passes of 2^5 .. 2^9 points, chunks of 2^7 .. 2^9.
inline bool split_valid(uint32_t logN, uint32_t s2) {
    return s2 >= (uint32_t)kChunkLogMin && s2 <= (uint32_t)kChunkLogMax && logN > s2 &&
           logN - s2 >= (uint32_t)kColsLogMin && logN - s2 <= (uint32_t)kColsLogMax;
}

// Plan builder (ntt_plan_create_ex with a cap on the single-pass size, and
// a given two-pass split and radix: split_log < 0 takes the tuned or
// default ones, radix_log is then ignored).
ntt_status create_plan(ntt_plan_t *plan, uint32_t N, const uint64_t *q, uint32_t L, ntt_variant variant,
                       uint32_t flags, const uint64_t *psi, int single_max_log, int split_log = -1,
                       int radix_log = 4);
ntt_status validate_plan_args(uint32_t N, const uint64_t *q, uint32_t L, uint32_t flags);

// fused path, instantiated in fused_<word>_<reduction>.cu
template <class W, int RED>
cudaError_t run_fused_t(ntt_plan_s &p, void *data, uint32_t batch, bool inverse, cudaStream_t st);
template <class W, int RED>
cudaError_t run_fused_pwinv_t(ntt_plan_s &p, void *c, const void *a, const void *b, uint32_t batch,
                              cudaStream_t st);
cudaError_t launch_fused_pwinv(ntt_plan_s &p, void *c, const void *a, const void *b, uint32_t batch,
                               cudaStream_t st);
// cluster form, instantiated in cluster_<reduction>.cu
template <int RED>
cudaError_t run_cluster(ntt_plan_s &p, void *data, uint32_t batch, bool inverse, cudaStream_t st);

}  // namespace nttgb
