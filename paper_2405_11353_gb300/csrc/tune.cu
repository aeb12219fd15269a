// tune.cu -- autotuner of the two-pass fused path and its table.
//
// A two-pass direction (forward, or inverse with or without the fused
// product) runs in one of three forms: the chunk pass on one-warp CTAs
// (2-chunk tiles), on 256-thread CTAs (16-chunk tiles), or both passes in
// one streamed launch (stream.cuh).  Which is fastest depends on N, the word
// size, the limb count and the batch, so ntt_autotune times all three on
// the current device for one shape and records the fastest per direction
// in a process-wide table keyed by (N, word size, L, reduction, order,
// twiddles made on the fly or read, floor(log2 batch)).  Plans whose chunk
// twiddles are made on the fly (NTT_TW_OTF) have no streamed form: its time
// is reported as -1 and it is never chosen.  ntt_plan_create copies the table's entries for its
// shape into the plan; each call then looks up its batch bucket.  The
// table is also kept in the JSON-lines file named by NTT_TUNE_DB, read at
// first use and rewritten after every tuning, so tuning survives the
// process.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "../../include/ntt.h"
#include "plan.hpp"

namespace nttgb {
namespace {

struct TuneKey {
    uint32_t N, word, L, red, bitrev, bucket, otf;
    bool operator<(const TuneKey &o) const {
        return std::tie(N, word, L, red, bitrev, bucket, otf) <
               std::tie(o.N, o.word, o.L, o.red, o.bitrev, o.bucket, o.otf);
    }
};
struct TuneVal {
    int form[2];
    float ms[2][3];
};

std::mutex g_mu;
std::map<TuneKey, TuneVal> g_table;
bool g_loaded = false;

uint32_t bucket_of(uint32_t batch) {
    uint32_t b = 0;
    while (b < 31 && (2u << b) <= batch) ++b;
    return b;
}

void load_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = std::getenv("NTT_TUNE_DB");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[1024];
    while (std::fgets(line, sizeof(line), f)) {
        TuneKey k;
        TuneVal v;
        int n = std::sscanf(line,
                            "{\"N\": %u, \"word_bytes\": %u, \"L\": %u, \"reduction\": %u, \"bitrev\": %u, "
                            "\"tw_otf\": %u, \"batch_log2\": %u, \"forward_form\": %d, \"inverse_form\": %d, "
                            "\"forward_ms\": [%f, %f, %f], \"inverse_ms\": [%f, %f, %f]}",
                            &k.N, &k.word, &k.L, &k.red, &k.bitrev, &k.otf, &k.bucket, &v.form[0], &v.form[1],
                            &v.ms[0][0], &v.ms[0][1], &v.ms[0][2], &v.ms[1][0], &v.ms[1][1], &v.ms[1][2]);
        if (n != 15) {
            // lines written before the twiddle-mode field existed
            k.otf = 0;
            n = 1 + std::sscanf(line,
                                "{\"N\": %u, \"word_bytes\": %u, \"L\": %u, \"reduction\": %u, \"bitrev\": %u, "
                                "\"batch_log2\": %u, \"forward_form\": %d, \"inverse_form\": %d, "
                                "\"forward_ms\": [%f, %f, %f], \"inverse_ms\": [%f, %f, %f]}",
                                &k.N, &k.word, &k.L, &k.red, &k.bitrev, &k.bucket, &v.form[0], &v.form[1],
                                &v.ms[0][0], &v.ms[0][1], &v.ms[0][2], &v.ms[1][0], &v.ms[1][1], &v.ms[1][2]);
        }
        if (n != 15 || k.bucket > 31 || k.otf > 1 || v.form[0] < 0 || v.form[0] > 2 || v.form[1] < 0 ||
            v.form[1] > 2)
            continue;
        g_table[k] = v;
    }
    std::fclose(f);
}

void save_locked() {
    const char *path = std::getenv("NTT_TUNE_DB");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "w");
    if (!f) return;
    for (const auto &e : g_table) {
        const TuneKey &k = e.first;
        const TuneVal &v = e.second;
        std::fprintf(f,
                     "{\"N\": %u, \"word_bytes\": %u, \"L\": %u, \"reduction\": %u, \"bitrev\": %u, "
                     "\"tw_otf\": %u, \"batch_log2\": %u, \"forward_form\": %d, \"inverse_form\": %d, "
                     "\"forward_ms\": [%.6f, %.6f, %.6f], \"inverse_ms\": [%.6f, %.6f, %.6f]}\n",
                     k.N, k.word, k.L, k.red, k.bitrev, k.otf, k.bucket, v.form[0], v.form[1], v.ms[0][0], v.ms[0][1],
                     v.ms[0][2], v.ms[1][0], v.ms[1][1], v.ms[1][2]);
    }
    std::fclose(f);
}

TuneKey key_of(const ntt_plan_s &p, uint32_t bucket) {
    return TuneKey{p.N, (uint32_t)p.word_bytes(), p.L, (uint32_t)p.red, p.bitrev_order ? 1u : 0u, bucket,
                   p.tw_otf ? 1u : 0u};
}

}  // namespace

// Copy the table's entries for the plan's shape into the plan.
void apply_tuning(ntt_plan_s &p) {
    std::memset(p.tuned_form, -1, sizeof(p.tuned_form));
    if (p.variant != NTT_FUSED || p.fused_mode != FUSED_TWO_PASS || p.streamed) return;
    std::lock_guard<std::mutex> g(g_mu);
    load_locked();
    for (uint32_t b = 0; b < 32; ++b) {
        auto it = g_table.find(key_of(p, b));
        if (it == g_table.end()) continue;
        p.tuned_form[0][b] = (int8_t)it->second.form[0];
        p.tuned_form[1][b] = (int8_t)it->second.form[1];
    }
}

}  // namespace nttgb

extern "C" {

ntt_status ntt_autotune(uint32_t N, const uint64_t *q, uint32_t L, uint32_t flags, uint32_t batch,
                        ntt_stream_t stream, ntt_tune_result *result) {
    if (!q || batch == 0 || (flags & (NTT_STREAMED | NTT_CHECK | NTT_TEST_STALL))) return NTT_ERR_INVALID_ARG;
    ntt_plan_t p = nullptr;
    ntt_status s = ntt_plan_create(&p, N, q, L, NTT_FUSED, flags);
    if (s != NTT_OK) return s;
    if (p->fused_mode != nttgb::FUSED_TWO_PASS) {
        ntt_plan_destroy(p);
        return NTT_ERR_UNSUPPORTED;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)batch * L * N * p->word_bytes();
    void *d = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
        cudaGetLastError();
        ntt_plan_destroy(p);
        return NTT_ERR_OOM;
    }
    nttgb::TuneVal v;
    bool ok = cudaMemsetAsync(d, 0, bytes, st) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
              cudaEventCreate(&e1) == cudaSuccess;
    const uint32_t bucket = nttgb::bucket_of(batch);
    // time every form of each direction on zero words (valid residues)
    for (int dir = 0; dir < 2 && ok; ++dir) {
        for (int form = 0; form < 3 && ok; ++form) {
            if (form == nttgb::FORM_STREAMED && p->tw_otf) {
                v.ms[dir][form] = -1.f;
                continue;
            }
            p->tuned_form[dir][bucket] = (int8_t)form;
            auto call = [&]() {
                return dir == 0 ? ntt_forward(p, d, batch, stream) : ntt_inverse(p, d, batch, stream);
            };
            for (int w = 0; w < 2 && ok; ++w) ok = call() == NTT_OK;
            // about 20 ms of calls, at least 3
            float ms = 0.f;
            ok = ok && cudaEventRecord(e0, st) == cudaSuccess && call() == NTT_OK &&
                 cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            int reps = ms > 0.f ? (int)(20.f / ms) : 3;
            reps = reps < 3 ? 3 : (reps > 200 ? 200 : reps);
            ok = ok && cudaEventRecord(e0, st) == cudaSuccess;
            for (int r = 0; r < reps && ok; ++r) ok = call() == NTT_OK;
            ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            v.ms[dir][form] = ms / (float)reps;
        }
        int best = 0;
        for (int form = 1; form < 3; ++form)
            if (v.ms[dir][form] >= 0.f && v.ms[dir][form] < v.ms[dir][best]) best = form;
        v.form[dir] = best;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const ntt_status dev = ntt_get_device_status(p, stream);
    cudaFree(d);
    if (ok && dev == NTT_OK) {
        std::lock_guard<std::mutex> g(nttgb::g_mu);
        nttgb::load_locked();
        nttgb::g_table[nttgb::key_of(*p, bucket)] = v;
        nttgb::save_locked();
    }
    ntt_plan_destroy(p);
    if (!ok) {
        cudaGetLastError();
        return NTT_ERR_CUDA;
    }
    if (dev != NTT_OK) return dev;
    if (result) {
        for (int f = 0; f < 3; ++f) {
            result->forward_ms[f] = v.ms[0][f];
            result->inverse_ms[f] = v.ms[1][f];
        }
        result->forward_form = v.form[0];
        result->inverse_form = v.form[1];
    }
    return NTT_OK;
}

namespace {
nttgb::TuneKey key_from_flags(uint32_t N, uint32_t L, uint32_t flags, uint32_t batch) {
    const uint32_t red = (flags & NTT_RED_MASK) == NTT_RED_MONTGOMERY ? nttgb::RED_MONTGOMERY
                         : (flags & NTT_RED_MASK) == NTT_RED_BARRETT   ? nttgb::RED_BARRETT
                                                                       : nttgb::RED_SHOUP;
    return nttgb::TuneKey{N, (flags & NTT_WORD64) ? 8u : 4u, L, red, (flags & NTT_ORDER_BITREV) ? 1u : 0u,
                          nttgb::bucket_of(batch), (flags & NTT_TW_OTF) ? 1u : 0u};
}
}  // namespace

ntt_status ntt_tune_set(uint32_t N, uint32_t L, uint32_t flags, uint32_t batch, int32_t forward_form,
                        int32_t inverse_form) {
    if (batch == 0 || L == 0 || forward_form < 0 || forward_form > 2 || inverse_form < 0 || inverse_form > 2)
        return NTT_ERR_INVALID_ARG;
    nttgb::TuneVal v;
    v.form[0] = forward_form;
    v.form[1] = inverse_form;
    for (int d = 0; d < 2; ++d)
        for (int f = 0; f < 3; ++f) v.ms[d][f] = -1.f;      // set by hand, not timed
    std::lock_guard<std::mutex> g(nttgb::g_mu);
    nttgb::load_locked();
    nttgb::g_table[key_from_flags(N, L, flags, batch)] = v;
    nttgb::save_locked();
    return NTT_OK;
}

int32_t ntt_tune_get(uint32_t N, uint32_t L, uint32_t flags, uint32_t batch, int inverse) {
    if (batch == 0) return -1;
    std::lock_guard<std::mutex> g(nttgb::g_mu);
    nttgb::load_locked();
    auto it = nttgb::g_table.find(key_from_flags(N, L, flags, batch));
    return it == nttgb::g_table.end() ? -1 : it->second.form[inverse ? 1 : 0];
}

void ntt_tune_clear(void) {
    std::lock_guard<std::mutex> g(nttgb::g_mu);
    nttgb::g_table.clear();
    nttgb::g_loaded = true;      // do not read the file again
}

int32_t ntt_plan_form(ntt_plan_t plan, uint32_t batch, int inverse) {
    if (!plan || plan->variant != NTT_FUSED || plan->fused_mode != nttgb::FUSED_TWO_PASS) return -1;
    return plan->form_for(batch == 0 ? 1 : batch, inverse != 0);
}

}  // extern "C"
