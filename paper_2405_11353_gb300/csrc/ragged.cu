// ragged.cu -- heterogeneous batches in one graph-captured persistent launch.
//
// ntt_ragged_create groups the jobs by (N, word size) and builds one fused
// plan per group with the longest prime list of the group (every job's
// primes must be a prefix of it, else the job gets a group of its own), so
// all jobs of a group share twiddle tables.  Transforms of 2^12 words run in
// one pass, larger ones in two (column strips of N/256 rows, then 256-word
// chunks).  The work is cut into items of a few tiles each, ordered by phase
// (see ragged.hpp), and one cooperative launch of the persistent kernel --
// preceded by zeroing the item counters -- is captured into a CUDA graph
// that ntt_ragged_launch replays.  Like the fused plans it works in the
// bit-reversed evaluation order (NTT_ORDER_BITREV is required).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "fused_launch.cuh"
#include "plan.hpp"
#include "ragged.hpp"

using namespace nttgb;

struct ntt_ragged_s {
    std::vector<ntt_plan_t> plans;
    RaggedArgs args{};
    void *d_jobs = nullptr, *d_tmaps = nullptr, *d_items = nullptr, *d_words = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t n_items = 0, n_jobs = 0;
    uint32_t item_tiles = 0;     // tiles per work item (tuned with NTT_RAGGED_TUNE)
    int red = 0;
    unsigned grid = 0;
};

namespace {

constexpr uint32_t kItemTiles = 8;   // default tiles per work item
constexpr uint32_t kTuneItemTiles[4] = {2, 4, 8, 16};

void ragged_free(ntt_ragged_s *r) {
    if (!r) return;
    if (r->exec) cudaGraphExecDestroy(r->exec);
    if (r->graph) cudaGraphDestroy(r->graph);
    void *ptrs[] = {r->d_jobs, r->d_tmaps, r->d_items, r->d_words};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (ntt_plan_t p : r->plans) ntt_plan_destroy(p);
    delete r;
}

cudaError_t kernel_config(int red, size_t *smem, int *bps) {
    switch (red) {
    case RED_SHOUP: return ragged_kernel_config<RED_SHOUP>(smem, bps);
    case RED_BARRETT: return ragged_kernel_config<RED_BARRETT>(smem, bps);
    default: return ragged_kernel_config<RED_MONTGOMERY>(smem, bps);
    }
}

cudaError_t kernel_launch(int red, const RaggedArgs &a, unsigned grid, cudaStream_t st) {
    switch (red) {
    case RED_SHOUP: return ragged_kernel_launch<RED_SHOUP>(a, grid, st);
    case RED_BARRETT: return ragged_kernel_launch<RED_BARRETT>(a, grid, st);
    default: return ragged_kernel_launch<RED_MONTGOMERY>(a, grid, st);
    }
}

}  // namespace

// Job records, tensor maps and work items of item_tiles tiles for the jobs
// with their data at data_of(j), uploaded into r (replacing earlier ones).
template <class DataOf, class PlanOf>
ntt_status build_items(ntt_ragged_s *r, const ntt_job *jobs, uint32_t n_jobs, DataOf data_of, PlanOf plan_of,
                       uint32_t item_tiles) {
    // ---- device job records, tensor maps, work items
    std::vector<RJob> rj(n_jobs);
    std::vector<CUtensorMap> maps(2 * (size_t)n_jobs);
    std::memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
    std::vector<RItem> items[4];
    for (uint32_t j = 0; j < n_jobs; ++j) {
        const ntt_job &J = jobs[j];
        ntt_plan_s &p = *plan_of(j);
        RJob &R = rj[j];
        R.data = data_of(j);
        R.tw[0] = p.d_main_fwd; R.tw[1] = p.d_main_inv; R.tw[2] = p.d_chunk_fwd; R.tw[3] = p.d_chunk_inv;
        R.lc = p.d_limb;
        R.ntrans = (uint64_t)J.batch * J.L;
        R.logN = p.logN;
        R.L = J.L;
        const bool w64 = J.word64 != 0, inv = J.inverse != 0;
        auto add = [&](int phase, uint32_t kind, uint64_t ntiles) {
            for (uint64_t t0 = 0; t0 < ntiles; t0 += item_tiles) {
                uint64_t t1 = std::min<uint64_t>(ntiles, t0 + item_tiles);
                items[phase].push_back({j, ragged_code(w64, inv, kind), (uint32_t)t0, (uint32_t)t1});
            }
        };
        if (p.fused_mode == FUSED_SINGLE) {
            // 4096-word transforms, one per tile
            add(inv ? 2 : 0, RK_SINGLE12, R.ntrans);
        } else {
            const uint32_t s1 = p.s1, N1 = 1u << s1;
            const uint32_t Kc = 4096u >> s1;                    // column-strip width (256 threads)
            cudaError_t e = make_cols_tmap(&maps[2 * j], data_of(j), w64, R.ntrans * N1, 256, Kc, N1 < 256 ? N1 : 256);
            if (e == cudaSuccess && inv) {
                const uint32_t RW = w64 ? 16 : 32;
                e = make_rows_tmap(&maps[2 * j + 1], data_of(j), w64, R.ntrans * p.N / RW, RW, 16 * 256 / RW);
            }
            if (e != cudaSuccess) return NTT_ERR_CUDA;
            const uint64_t cols_tiles = R.ntrans * (256 / Kc), chunk_tiles = R.ntrans * (N1 / 16);
            const uint32_t cols_kind = RK_COLS5 + (s1 - 5);
            if (!inv) { add(0, cols_kind, cols_tiles); add(1, RK_CHUNKS, chunk_tiles); }
            else { add(2, RK_CHUNKS, chunk_tiles); add(3, cols_kind, cols_tiles); }
        }
    }
    std::vector<RItem> all;
    uint32_t begin[5];
    for (int ph = 0; ph < 4; ++ph) {
        begin[ph] = (uint32_t)all.size();
        // larger transforms first: items of 8-byte words and more rows cost more
        std::stable_sort(items[ph].begin(), items[ph].end(),
                         [&](const RItem &a, const RItem &b) { return rj[a.job].logN > rj[b.job].logN; });
        all.insert(all.end(), items[ph].begin(), items[ph].end());
    }
    begin[4] = (uint32_t)all.size();
    r->n_items = begin[4];

    auto up = [&](void **d, const void *h, size_t bytes) -> bool {
        if (cudaMalloc(d, bytes ? bytes : 16) != cudaSuccess) { *d = nullptr; cudaGetLastError(); return false; }
        return bytes == 0 || cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    for (void **d : {&r->d_jobs, &r->d_tmaps, &r->d_items})
        if (*d) { cudaFree(*d); *d = nullptr; }
    if (!up(&r->d_jobs, rj.data(), rj.size() * sizeof(RJob)) ||
        !up(&r->d_tmaps, maps.data(), maps.size() * sizeof(CUtensorMap)) ||
        !up(&r->d_items, all.data(), all.size() * sizeof(RItem)))
        return NTT_ERR_OOM;
    uint32_t *w = reinterpret_cast<uint32_t *>(r->d_words);
    RaggedArgs &a = r->args;
    a.jobs = reinterpret_cast<const RJob *>(r->d_jobs);
    a.tmaps = reinterpret_cast<const CUtensorMap *>(r->d_tmaps);
    a.items = reinterpret_cast<const RItem *>(r->d_items);
    for (int i = 0; i < 5; ++i) a.phase_begin[i] = begin[i];
    a.counters = w;
    a.bar_count = w + 4;
    a.bar_gen = w + 5;
    a.status = w + 6;
    a.abort_flag = w + 7;
    r->item_tiles = item_tiles;
    return NTT_OK;

}

extern "C" {

ntt_status ntt_ragged_create(ntt_ragged_t *out, const ntt_job *jobs, uint32_t n_jobs, uint32_t flags) {
    if (!out) return NTT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!jobs || n_jobs == 0) return NTT_ERR_INVALID_ARG;
    if (flags & ~(NTT_ORDER_BITREV | NTT_RED_MASK | NTT_RAGGED_TUNE | NTT_TEST_STALL)) return NTT_ERR_INVALID_ARG;
    if ((flags & NTT_TEST_STALL) && (flags & NTT_RAGGED_TUNE)) return NTT_ERR_INVALID_ARG;
    if ((flags & NTT_RED_MASK) == NTT_RED_MASK) return NTT_ERR_INVALID_ARG;
    if (!(flags & NTT_ORDER_BITREV)) return NTT_ERR_UNSUPPORTED;
    for (uint32_t j = 0; j < n_jobs; ++j) {
        const ntt_job &J = jobs[j];
        if (!J.d_data || !J.q || J.L == 0 || J.batch == 0 || J.word64 > 1) return NTT_ERR_INVALID_ARG;
        if ((reinterpret_cast<uintptr_t>(J.d_data) & 15u) != 0) return NTT_ERR_ALIGNMENT;
        ntt_status s = validate_plan_args(J.N, J.q, J.L, J.word64 ? NTT_WORD64 : 0u);
        if (s != NTT_OK) return s;
        if (J.N < (1u << 12)) return NTT_ERR_N_RANGE;
        if ((uint64_t)J.batch * J.L >= (1ull << 26)) return NTT_ERR_INVALID_ARG;
    }
    ntt_ragged_s *r = new (std::nothrow) ntt_ragged_s();
    if (!r) return NTT_ERR_OOM;
    r->red = (flags & NTT_RED_MASK) == NTT_RED_BARRETT ? RED_BARRETT
           : (flags & NTT_RED_MASK) == NTT_RED_MONTGOMERY ? RED_MONTGOMERY : RED_SHOUP;
    r->n_jobs = n_jobs;

    // ---- groups: (N, word size) -> longest prime list; jobs use prefixes
    std::vector<uint32_t> order(n_jobs);
    for (uint32_t j = 0; j < n_jobs; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return jobs[a].L > jobs[b].L; });
    struct Group { uint32_t N, w64, leader; ntt_plan_t plan; };
    std::vector<Group> groups;
    std::vector<uint32_t> group_of(n_jobs);
    for (uint32_t j : order) {
        const ntt_job &J = jobs[j];
        int found = -1;
        for (size_t g = 0; g < groups.size(); ++g) {
            const ntt_job &Ld = jobs[groups[g].leader];
            if (groups[g].N == J.N && groups[g].w64 == J.word64 && Ld.L >= J.L &&
                std::equal(J.q, J.q + J.L, Ld.q)) { found = (int)g; break; }
        }
        if (found < 0) {
            groups.push_back({J.N, J.word64, j, nullptr});
            found = (int)groups.size() - 1;
        }
        group_of[j] = (uint32_t)found;
    }
    for (Group &g : groups) {
        const ntt_job &Ld = jobs[g.leader];
        uint32_t pflags = (flags & (NTT_ORDER_BITREV | NTT_RED_MASK)) | (g.w64 ? NTT_WORD64 : 0u);
        ntt_status s = create_plan(&g.plan, g.N, Ld.q, Ld.L, NTT_FUSED, pflags, nullptr, 12);
        if (s != NTT_OK) { ragged_free(r); return s; }
        r->plans.push_back(g.plan);
    }

    // words: 4 item counters, barrier count, barrier generation, status, abort
    if (cudaMalloc(&r->d_words, 16 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(r->d_words, 0, 16 * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        ragged_free(r);
        return NTT_ERR_OOM;
    }
    uint32_t *w = reinterpret_cast<uint32_t *>(r->d_words);
    auto plan_of = [&](uint32_t j) { return groups[group_of[j]].plan; };

    // ---- persistent grid
    size_t smem = 0;
    int bps = 0, dev = 0, sms = 0;
    if (kernel_config(r->red, &smem, &bps) != cudaSuccess || bps < 1) { cudaGetLastError(); ragged_free(r); return NTT_ERR_CUDA; }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(sms * bps);
    r->grid = grid;

    // ---- autotuning of the work-item size: each candidate runs on zeroed
    // scratch copies of the jobs' buffers (same sizes; jobs that share a
    // buffer share its copy), timed over three launches
    uint32_t best_tiles = kItemTiles;
    if (flags & NTT_RAGGED_TUNE) {
        std::map<void *, size_t> need;            // user buffer -> bytes
        for (uint32_t j = 0; j < n_jobs; ++j) {
            const size_t b = (size_t)jobs[j].batch * jobs[j].L * jobs[j].N * (jobs[j].word64 ? 8 : 4);
            size_t &v = need[jobs[j].d_data];
            v = std::max(v, b);
        }
        size_t total = 0;
        std::map<void *, size_t> off;
        for (auto &e : need) { off[e.first] = total; total += (e.second + 255) & ~size_t(255); }
        void *scratch = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaStream_t ts = nullptr;
        bool ok = cudaMalloc(&scratch, total) == cudaSuccess && cudaMemset(scratch, 0, total) == cudaSuccess &&
                  cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) == cudaSuccess;
        float best_ms = 0.f;
        for (uint32_t c = 0; c < 4 && ok; ++c) {
            auto scratch_of = [&](uint32_t j) {
                return (void *)((char *)scratch + off[jobs[j].d_data]);
            };
            if (build_items(r, jobs, n_jobs, scratch_of, plan_of, kTuneItemTiles[c]) != NTT_OK) { ok = false; break; }
            auto launch = [&]() {
                return cudaMemsetAsync(w, 0, 5 * sizeof(uint32_t), ts) == cudaSuccess &&
                       cudaMemsetAsync(w + 7, 0, sizeof(uint32_t), ts) == cudaSuccess &&
                       kernel_launch(r->red, r->args, grid, ts) == cudaSuccess;
            };
            float ms = 0.f;
            ok = launch() && cudaEventRecord(e0, ts) == cudaSuccess;
            for (int k = 0; k < 3 && ok; ++k) ok = launch();
            ok = ok && cudaEventRecord(e1, ts) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            uint32_t status = 0;
            ok = ok && cudaMemcpy(&status, w + 6, sizeof(status), cudaMemcpyDeviceToHost) == cudaSuccess &&
                 status == 0;
            if (ok && (c == 0 || ms < best_ms)) { best_ms = ms; best_tiles = kTuneItemTiles[c]; }
        }
        if (ts) cudaStreamDestroy(ts);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (scratch) cudaFree(scratch);
        if (!ok) { cudaGetLastError(); ragged_free(r); return NTT_ERR_CUDA; }
    }
    ntt_status bs = build_items(r, jobs, n_jobs, [&](uint32_t j) { return jobs[j].d_data; }, plan_of, best_tiles);
    if (bs != NTT_OK) { cudaGetLastError(); ragged_free(r); return bs; }
    r->args.stall = (flags & NTT_TEST_STALL) ? 1u : 0u;
    const RaggedArgs &a = r->args;

    // ---- graph capture
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); ragged_free(r); return NTT_ERR_CUDA; }
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // item counters and the barrier count (a launch whose barrier wait
        // ran out leaves arrivals behind), and the abort flag
        cudaMemsetAsync(w, 0, 5 * sizeof(uint32_t), st);
        cudaMemsetAsync(w + 7, 0, sizeof(uint32_t), st);
        cudaError_t le = kernel_launch(r->red, a, grid, st);
        e = cudaStreamEndCapture(st, &r->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&r->exec, r->graph, 0);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) { cudaGetLastError(); ragged_free(r); return NTT_ERR_CUDA; }
    *out = r;
    return NTT_OK;
}

ntt_status ntt_ragged_launch(ntt_ragged_t r, ntt_stream_t stream) {
    if (!r) return NTT_ERR_INVALID_ARG;
    if (cudaGraphLaunch(r->exec, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return NTT_ERR_CUDA;
    }
    return NTT_OK;
}

ntt_status ntt_ragged_status(ntt_ragged_t r, ntt_stream_t stream) {
    if (!r) return NTT_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) { cudaGetLastError(); return NTT_ERR_CUDA; }
    uint32_t v = 0;
    if (cudaMemcpy(&v, r->args.status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return NTT_ERR_CUDA;
    if (v) cudaMemset(r->args.status, 0, sizeof(uint32_t));
    return (v & 2u) ? NTT_ERR_TIMEOUT : NTT_OK;
}

uint32_t ntt_ragged_item_tiles(ntt_ragged_t r) { return r ? r->item_tiles : 0u; }

void ntt_ragged_destroy(ntt_ragged_t r) {
    if (!r) return;
    cudaDeviceSynchronize();
    ragged_free(r);
}

}  // extern "C"
