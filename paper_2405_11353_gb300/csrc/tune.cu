// tune.cu -- autotuner of the two-pass fused path and its tables.
//
// What the two-pass fused path leaves open at run time, per shape (N, word
// size, L, reduction, order, twiddles made on the fly or read):
//   * the split N = 2^s1 x 2^s2: how many stages each pass does (column
//     passes of 2^s1 points, chunks of 2^s2 = 128, 256 or 512 words), and
//     the radix of the register rounds (four stages on 16 words a thread,
//     or three on 8); the plan's twiddle tables are laid out for both, so
//     they are fixed when a plan is made;
//   * per direction (forward, or inverse with or without the fused
//     product) and batch bucket floor(log2 batch), the form: the chunk pass
//     on one-warp CTAs, on 256-thread CTAs, or both passes in one streamed
//     launch (stream.cuh; 256-word chunks only, not with NTT_TW_OTF), and
//     the first two again with the chunk pass's exchanges between rounds by
//     warp shuffles (4-byte words, twiddle tables).
// ntt_autotune times every valid (radix, split) with every form of both
// directions on the current device and records, per (radix, split), the
// fastest form of each direction for the batch's bucket, and for the shape
// the (radix, split) whose two directions together are fastest.
// ntt_plan_create takes the shape's radix and split (before it builds its
// tables) and copies the form entries of that pair;
// each call then looks up its batch bucket.  Both tables are kept in the
// JSON-lines file named by NTT_TUNE_DB, read at first use and rewritten
// after every tuning, so tuning survives the process.
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
    uint32_t N, word, L, red, bitrev, bucket, otf, split, lr;
    bool operator<(const TuneKey &o) const {
        return std::tie(N, word, L, red, bitrev, bucket, otf, split, lr) <
               std::tie(o.N, o.word, o.L, o.red, o.bitrev, o.bucket, o.otf, o.split, o.lr);
    }
};
struct TuneVal {
    int form[2];
    float ms[2][kForms];
};
// shape (a TuneKey without bucket, split and radix) -> chosen split, radix
struct ShapeVal {
    uint32_t split, lr;
};
struct ShapeKey {
    uint32_t N, word, L, red, bitrev, otf;
    bool operator<(const ShapeKey &o) const {
        return std::tie(N, word, L, red, bitrev, otf) < std::tie(o.N, o.word, o.L, o.red, o.bitrev, o.otf);
    }
};

std::mutex g_mu;
std::map<TuneKey, TuneVal> g_table;
std::map<ShapeKey, ShapeVal> g_split;
bool g_loaded = false;

uint32_t bucket_of(uint32_t batch) {
    uint32_t b = 0;
    while (b < 31 && (2u << b) <= batch) ++b;
    return b;
}

// The numbers of the JSON array after `key` (at most kForms; the rest -1).
int read_ms(const char *line, const char *key, float *ms) {
    for (int f = 0; f < kForms; ++f) ms[f] = -1.f;
    const char *s = std::strstr(line, key);
    if (!s || !(s = std::strchr(s, '['))) return 0;
    ++s;
    int n = 0;
    while (n < kForms) {
        char *end = nullptr;
        const float v = std::strtof(s, &end);
        if (end == s) break;
        ms[n++] = v;
        s = end;
        while (*s == ' ' || *s == ',') ++s;
        if (*s == ']') break;
    }
    return n;
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
        ShapeKey sk;
        uint32_t split = 0, lr = 0;
        if (std::sscanf(line,
                        "{\"N\": %u, \"word_bytes\": %u, \"L\": %u, \"reduction\": %u, \"bitrev\": %u, "
                        "\"tw_otf\": %u, \"split_log2\": %u, \"radix_log2\": %u}",
                        &sk.N, &sk.word, &sk.L, &sk.red, &sk.bitrev, &sk.otf, &split, &lr) == 8) {
            if (sk.otf <= 1 && split >= (uint32_t)kChunkLogMin && split <= (uint32_t)kChunkLogMax &&
                (lr == 3 || lr == 4))
                g_split[sk] = ShapeVal{split, lr};
            continue;
        }
        // the fixed fields, in the newest layout first, then in those of
        // older tables: before the radix field (rounds of four), before the
        // split field (256-word chunks), before the twiddle-mode field
        // (table twiddles)
        k.lr = 4;
        int n = std::sscanf(line,
                            "{\"N\": %u, \"word_bytes\": %u, \"L\": %u, \"reduction\": %u, \"bitrev\": %u, "
                            "\"tw_otf\": %u, \"chunk_log2\": %u, \"radix_log2\": %u, \"batch_log2\": %u, "
                            "\"forward_form\": %d, \"inverse_form\": %d,",
                            &k.N, &k.word, &k.L, &k.red, &k.bitrev, &k.otf, &k.split, &k.lr, &k.bucket, &v.form[0],
                            &v.form[1]);
        if (n != 11) {
            k.lr = 4;
            n = 1 + std::sscanf(line,
                                "{\"N\": %u, \"word_bytes\": %u, \"L\": %u, \"reduction\": %u, \"bitrev\": %u, "
                                "\"tw_otf\": %u, \"chunk_log2\": %u, \"batch_log2\": %u, \"forward_form\": %d, "
                                "\"inverse_form\": %d,",
                                &k.N, &k.word, &k.L, &k.red, &k.bitrev, &k.otf, &k.split, &k.bucket, &v.form[0],
                                &v.form[1]);
        }
        if (n != 11) {
            k.split = (uint32_t)kChunkLog;
            n = 2 + std::sscanf(line,
                                "{\"N\": %u, \"word_bytes\": %u, \"L\": %u, \"reduction\": %u, \"bitrev\": %u, "
                                "\"tw_otf\": %u, \"batch_log2\": %u, \"forward_form\": %d, \"inverse_form\": %d,",
                                &k.N, &k.word, &k.L, &k.red, &k.bitrev, &k.otf, &k.bucket, &v.form[0], &v.form[1]);
        }
        if (n != 11) {
            k.otf = 0;
            n = 3 + std::sscanf(line,
                                "{\"N\": %u, \"word_bytes\": %u, \"L\": %u, \"reduction\": %u, \"bitrev\": %u, "
                                "\"batch_log2\": %u, \"forward_form\": %d, \"inverse_form\": %d,",
                                &k.N, &k.word, &k.L, &k.red, &k.bitrev, &k.bucket, &v.form[0], &v.form[1]);
        }
        // the per-form times: five forms, or the first three in older tables
        if (n != 11 || read_ms(line, "\"forward_ms\"", v.ms[0]) < 3 || read_ms(line, "\"inverse_ms\"", v.ms[1]) < 3 ||
            k.bucket > 31 || k.otf > 1 || v.form[0] < 0 || v.form[0] >= kForms || v.form[1] < 0 ||
            v.form[1] >= kForms || k.split < (uint32_t)kChunkLogMin || k.split > (uint32_t)kChunkLogMax ||
            (k.lr != 3 && k.lr != 4))
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
    for (const auto &e : g_split) {
        const ShapeKey &k = e.first;
        std::fprintf(f,
                     "{\"N\": %u, \"word_bytes\": %u, \"L\": %u, \"reduction\": %u, \"bitrev\": %u, "
                     "\"tw_otf\": %u, \"split_log2\": %u, \"radix_log2\": %u}\n",
                     k.N, k.word, k.L, k.red, k.bitrev, k.otf, e.second.split, e.second.lr);
    }
    for (const auto &e : g_table) {
        const TuneKey &k = e.first;
        const TuneVal &v = e.second;
        std::fprintf(f,
                     "{\"N\": %u, \"word_bytes\": %u, \"L\": %u, \"reduction\": %u, \"bitrev\": %u, "
                     "\"tw_otf\": %u, \"chunk_log2\": %u, \"radix_log2\": %u, \"batch_log2\": %u, "
                     "\"forward_form\": %d, \"inverse_form\": %d, \"forward_ms\": [%.6f, %.6f, %.6f, %.6f, %.6f], "
                     "\"inverse_ms\": [%.6f, %.6f, %.6f, %.6f, %.6f]}\n",
                     k.N, k.word, k.L, k.red, k.bitrev, k.otf, k.split, k.lr, k.bucket, v.form[0], v.form[1],
                     v.ms[0][0], v.ms[0][1], v.ms[0][2], v.ms[0][3], v.ms[0][4], v.ms[1][0], v.ms[1][1], v.ms[1][2],
                     v.ms[1][3], v.ms[1][4]);
    }
    std::fclose(f);
}

ShapeKey shape_of(const ntt_plan_s &p) {
    return ShapeKey{p.N, (uint32_t)p.word_bytes(), p.L, (uint32_t)p.red, p.bitrev_order ? 1u : 0u,
                    p.tw_otf ? 1u : 0u};
}
TuneKey key_of(const ntt_plan_s &p, uint32_t bucket) {
    return TuneKey{p.N, (uint32_t)p.word_bytes(), p.L, (uint32_t)p.red, p.bitrev_order ? 1u : 0u, bucket,
                   p.tw_otf ? 1u : 0u, p.s2, p.lr};
}

}  // namespace

// The shape's tuned split (plans whose split is not fixed), then the form
// entries of the plan's split.
void apply_tuning(ntt_plan_s &p) {
    std::memset(p.tuned_form, -1, sizeof(p.tuned_form));
    if (p.variant != NTT_FUSED || p.fused_mode != FUSED_TWO_PASS) return;
    std::lock_guard<std::mutex> g(g_mu);
    load_locked();
    if (!p.split_fixed) {
        auto it = g_split.find(shape_of(p));
        if (it != g_split.end() && split_valid(p.logN, it->second.split)) {
            p.s2 = it->second.split;
            p.s1 = p.logN - p.s2;
            p.lr = it->second.lr;
        }
    }
    if (p.streamed) return;
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
    // the shape's plan with its default split, to validate and size
    ntt_plan_t p0 = nullptr;
    ntt_status s = nttgb::create_plan(&p0, N, q, L, NTT_FUSED, flags, nullptr, -1, nttgb::kChunkLog);
    if (s != NTT_OK) return s;
    if (p0->fused_mode != nttgb::FUSED_TWO_PASS) {
        ntt_plan_destroy(p0);
        return NTT_ERR_UNSUPPORTED;
    }
    const bool otf = p0->tw_otf;
    const uint32_t logN = p0->logN;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)batch * L * N * p0->word_bytes();
    ntt_plan_destroy(p0);
    void *d = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
        cudaGetLastError();
        return NTT_ERR_OOM;
    }
    bool ok = cudaMemsetAsync(d, 0, bytes, st) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
              cudaEventCreate(&e1) == cudaSuccess;
    const uint32_t bucket = nttgb::bucket_of(batch);
    // per candidate (radix, split): rounds of 3 or 4 stages, chunks of 2^7,
    // 2^8, 2^9 words; every form of each direction, timed on zero words
    // (valid residues)
    constexpr int NSPLIT = nttgb::kChunkLogMax - nttgb::kChunkLogMin + 1;
    constexpr int NCFG = 2 * NSPLIT;             // index (lr - 3) * NSPLIT + (s2 - 7)
    nttgb::TuneVal vals[NCFG];
    float total[NCFG];
    nttgb::TuneKey keys[NCFG];
    nttgb::ShapeKey shape{};
    int best = -1;
    ntt_status dev = NTT_OK;
    for (int ci = 0; ci < NCFG && ok; ++ci) {
        const uint32_t lr = 3 + (uint32_t)(ci / NSPLIT);
        const uint32_t s2 = (uint32_t)(nttgb::kChunkLogMin + ci % NSPLIT);
        total[ci] = -1.f;
        if (!nttgb::split_valid(logN, s2) || (otf && (s2 != (uint32_t)nttgb::kChunkLog || lr != 4))) continue;
        ntt_plan_t p = nullptr;
        if (nttgb::create_plan(&p, N, q, L, NTT_FUSED, flags, nullptr, -1, (int)s2, (int)lr) != NTT_OK) continue;
        nttgb::TuneVal &v = vals[ci];
        for (int dir = 0; dir < 2 && ok; ++dir) {
            for (int form = 0; form < nttgb::kForms && ok; ++form) {
                if ((form == nttgb::FORM_STREAMED && (p->tw_otf || s2 != (uint32_t)nttgb::kChunkLog || lr != 4)) ||
                    (nttgb::form_is_shfl(form) && (p->tw_otf || p->word64))) {
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
            int bf = 0;
            for (int form = 1; form < nttgb::kForms; ++form)
                if (v.ms[dir][form] >= 0.f && v.ms[dir][form] < v.ms[dir][bf]) bf = form;
            v.form[dir] = bf;
        }
        if (ok) {
            const ntt_status ds = ntt_get_device_status(p, stream);
            if (ds != NTT_OK) { dev = ds; ok = false; }
        }
        if (ok) {
            total[ci] = v.ms[0][v.form[0]] + v.ms[1][v.form[1]];
            keys[ci] = nttgb::key_of(*p, bucket);
            shape = nttgb::shape_of(*p);
            if (best < 0 || total[ci] < total[best]) best = ci;
        }
        ntt_plan_destroy(p);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    if (!ok) {
        cudaGetLastError();
        return dev != NTT_OK ? dev : NTT_ERR_CUDA;
    }
    if (best < 0) return NTT_ERR_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> g(nttgb::g_mu);
        nttgb::load_locked();
        for (int ci = 0; ci < NCFG; ++ci)
            if (total[ci] >= 0.f) nttgb::g_table[keys[ci]] = vals[ci];
        nttgb::g_split[shape] = nttgb::ShapeVal{(uint32_t)(nttgb::kChunkLogMin + best % NSPLIT),
                                                3u + (uint32_t)(best / NSPLIT)};
        nttgb::save_locked();
    }
    if (result) {
        const nttgb::TuneVal &v = vals[best];
        for (int f = 0; f < nttgb::kForms; ++f) {
            result->forward_ms[f] = v.ms[0][f];
            result->inverse_ms[f] = v.ms[1][f];
        }
        result->forward_form = v.form[0];
        result->inverse_form = v.form[1];
        result->chunk_log2 = nttgb::kChunkLogMin + best % NSPLIT;
        result->radix_log2 = 3 + best / NSPLIT;
        for (int ci = 0; ci < NCFG; ++ci) result->config_ms[ci / NSPLIT][ci % NSPLIT] = total[ci];
    }
    return NTT_OK;
}

namespace {
nttgb::ShapeKey shape_from_flags(uint32_t N, uint32_t L, uint32_t flags) {
    const uint32_t red = (flags & NTT_RED_MASK) == NTT_RED_MONTGOMERY ? nttgb::RED_MONTGOMERY
                         : (flags & NTT_RED_MASK) == NTT_RED_BARRETT   ? nttgb::RED_BARRETT
                                                                       : nttgb::RED_SHOUP;
    return nttgb::ShapeKey{N, (flags & NTT_WORD64) ? 8u : 4u, L, red, (flags & NTT_ORDER_BITREV) ? 1u : 0u,
                           (flags & NTT_TW_OTF) ? 1u : 0u};
}
// (the caller holds g_mu) the split and radix plans of this shape take
nttgb::ShapeVal config_of_locked(const nttgb::ShapeKey &sk) {
    const nttgb::ShapeVal def{(uint32_t)nttgb::kChunkLog, 4u};
    if (sk.otf) return def;
    auto it = nttgb::g_split.find(sk);
    return it == nttgb::g_split.end() ? def : it->second;
}
nttgb::TuneKey key_from_shape(const nttgb::ShapeKey &sk, uint32_t batch, nttgb::ShapeVal c) {
    return nttgb::TuneKey{sk.N, sk.word, sk.L, sk.red, sk.bitrev, nttgb::bucket_of(batch), sk.otf, c.split, c.lr};
}
}  // namespace

ntt_status ntt_tune_set(uint32_t N, uint32_t L, uint32_t flags, uint32_t batch, int32_t forward_form,
                        int32_t inverse_form) {
    if (batch == 0 || L == 0 || forward_form < 0 || forward_form >= nttgb::kForms || inverse_form < 0 ||
        inverse_form >= nttgb::kForms)
        return NTT_ERR_INVALID_ARG;
    nttgb::TuneVal v;
    v.form[0] = forward_form;
    v.form[1] = inverse_form;
    for (int d = 0; d < 2; ++d)
        for (int f = 0; f < nttgb::kForms; ++f) v.ms[d][f] = -1.f;      // set by hand, not timed
    std::lock_guard<std::mutex> g(nttgb::g_mu);
    nttgb::load_locked();
    const nttgb::ShapeKey sk = shape_from_flags(N, L, flags);
    nttgb::g_table[key_from_shape(sk, batch, config_of_locked(sk))] = v;
    nttgb::save_locked();
    return NTT_OK;
}

int32_t ntt_tune_get(uint32_t N, uint32_t L, uint32_t flags, uint32_t batch, int inverse) {
    if (batch == 0) return -1;
    std::lock_guard<std::mutex> g(nttgb::g_mu);
    nttgb::load_locked();
    const nttgb::ShapeKey sk = shape_from_flags(N, L, flags);
    auto it = nttgb::g_table.find(key_from_shape(sk, batch, config_of_locked(sk)));
    return it == nttgb::g_table.end() ? -1 : it->second.form[inverse ? 1 : 0];
}

ntt_status ntt_tune_set_split(uint32_t N, uint32_t L, uint32_t flags, uint32_t chunk_log2, uint32_t radix_log2) {
    uint32_t n = 0;
    while (n < 31 && (1u << n) < N) ++n;
    if (L == 0 || (1u << n) != N || !nttgb::split_valid(n, chunk_log2) || (radix_log2 != 3 && radix_log2 != 4) ||
        ((flags & NTT_TW_OTF) && (chunk_log2 != (uint32_t)nttgb::kChunkLog || radix_log2 != 4)))
        return NTT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(nttgb::g_mu);
    nttgb::load_locked();
    nttgb::g_split[shape_from_flags(N, L, flags)] = nttgb::ShapeVal{chunk_log2, radix_log2};
    nttgb::save_locked();
    return NTT_OK;
}

int32_t ntt_tune_get_split(uint32_t N, uint32_t L, uint32_t flags, int32_t *radix_log2) {
    std::lock_guard<std::mutex> g(nttgb::g_mu);
    nttgb::load_locked();
    auto it = nttgb::g_split.find(shape_from_flags(N, L, flags));
    if (it == nttgb::g_split.end()) {
        if (radix_log2) *radix_log2 = -1;
        return -1;
    }
    if (radix_log2) *radix_log2 = (int32_t)it->second.lr;
    return (int32_t)it->second.split;
}

void ntt_tune_clear(void) {
    std::lock_guard<std::mutex> g(nttgb::g_mu);
    nttgb::g_table.clear();
    nttgb::g_split.clear();
    nttgb::g_loaded = true;      // do not read the file again
}

int32_t ntt_plan_chunk_log2(ntt_plan_t plan) {
    if (!plan || plan->variant != NTT_FUSED || plan->fused_mode != nttgb::FUSED_TWO_PASS) return -1;
    return (int32_t)plan->s2;
}

int32_t ntt_plan_radix_log2(ntt_plan_t plan) {
    if (!plan || plan->variant != NTT_FUSED || plan->fused_mode != nttgb::FUSED_TWO_PASS) return -1;
    return (int32_t)plan->lr;
}

int32_t ntt_plan_form(ntt_plan_t plan, uint32_t batch, int inverse) {
    if (!plan || plan->variant != NTT_FUSED || plan->fused_mode != nttgb::FUSED_TWO_PASS) return -1;
    return plan->form_for(batch == 0 ? 1 : batch, inverse != 0);
}

}  // extern "C"
