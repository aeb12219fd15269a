// ragged.cu -- heterogeneous batches in one graph-captured persistent launch.
//
// ntt_ragged_create groups the jobs by (N, word size) and builds one fused
// plan per group with the longest prime list of the group (every job's
// primes must be a prefix of it, else the job gets a group of its own), so
// all jobs of a group share twiddle tables.  Transforms of 2^12 words run in
// one pass, larger ones in two (column strips of N/256 rows, then 256-word
// chunks).  The work is cut into items of a few tiles each, ordered by phase
// (see ragged.hpp), and the cooperative launches of the persistent kernels
// -- one per word size present, preceded by zeroing the item counters --
// are captured into a CUDA graph that ntt_ragged_launch replays.  Like the fused plans it works in the
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
    RaggedArgs args[2]{};        // per word size (4-byte, 8-byte items)
    uint32_t n_word_items[2] = {0, 0};
    void *d_jobs = nullptr, *d_tmaps = nullptr, *d_items = nullptr, *d_words = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t n_items = 0, n_jobs = 0;
    uint32_t item_tiles = 0;     // tiles per work item (tuned with NTT_RAGGED_TUNE)
    int red = 0;
    unsigned grid[2] = {0, 0};
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

template <class W> cudaError_t kernel_config_w(int red, size_t *smem, int *bps) {
    switch (red) {
    case RED_SHOUP: return ragged_kernel_config<RED_SHOUP, W>(smem, bps);
    case RED_BARRETT: return ragged_kernel_config<RED_BARRETT, W>(smem, bps);
    default: return ragged_kernel_config<RED_MONTGOMERY, W>(smem, bps);
    }
}
cudaError_t kernel_config(int red, bool w64, size_t *smem, int *bps) {
    return w64 ? kernel_config_w<uint64_t>(red, smem, bps) : kernel_config_w<uint32_t>(red, smem, bps);
}

template <class W> cudaError_t kernel_launch_w(int red, const RaggedArgs &a, unsigned grid, cudaStream_t st) {
    switch (red) {
    case RED_SHOUP: return ragged_kernel_launch<RED_SHOUP, W>(a, grid, st);
    case RED_BARRETT: return ragged_kernel_launch<RED_BARRETT, W>(a, grid, st);
    default: return ragged_kernel_launch<RED_MONTGOMERY, W>(a, grid, st);
    }
}

// Device words of a ragged batch: per word-size kernel w its 4 item counters
// (words 5 w .. 5 w + 3) and grid-barrier arrival count (5 w + 4), then the
// shared abort flag -- the 11 words zeroed before every launch -- then the
// barrier generations (11, 12) and the status word (13).
constexpr uint32_t kRwZeroed = 11, kRwAbort = 10, kRwGen = 11, kRwStatus = 13, kRwWords = 16;

// One replay's work on stream st: zero the counters, then the kernel of
// each word size that has items.
cudaError_t launch_all(const ntt_ragged_s *r, cudaStream_t st) {
    uint32_t *w = reinterpret_cast<uint32_t *>(r->d_words);
    cudaError_t e = cudaMemsetAsync(w, 0, kRwZeroed * sizeof(uint32_t), st);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        if (r->n_word_items[k] == 0) continue;
        e = k == 0 ? kernel_launch_w<uint32_t>(r->red, r->args[0], r->grid[0], st)
                   : kernel_launch_w<uint64_t>(r->red, r->args[1], r->grid[1], st);
    }
    return e;
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
    std::vector<RItem> items[2][4];   // [word size][phase]
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
                items[w64 ? 1 : 0][phase].push_back({j, ragged_code(w64, inv, kind), (uint32_t)t0, (uint32_t)t1});
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
    // both kernels' items in one device array: the 4-byte kernel's, then
    // the 8-byte kernel's, each in phase order
    std::vector<RItem> all;
    uint32_t begin[2][5];
    for (int k = 0; k < 2; ++k) {
        for (int ph = 0; ph < 4; ++ph) {
            begin[k][ph] = (uint32_t)all.size();
            // larger transforms first: items of more rows cost more
            std::stable_sort(items[k][ph].begin(), items[k][ph].end(),
                             [&](const RItem &a, const RItem &b) { return rj[a.job].logN > rj[b.job].logN; });
            all.insert(all.end(), items[k][ph].begin(), items[k][ph].end());
        }
        begin[k][4] = (uint32_t)all.size();
    }
    r->n_items = (uint32_t)all.size();

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
    for (int k = 0; k < 2; ++k) {
        RaggedArgs &a = r->args[k];
        a.jobs = reinterpret_cast<const RJob *>(r->d_jobs);
        a.tmaps = reinterpret_cast<const CUtensorMap *>(r->d_tmaps);
        a.items = reinterpret_cast<const RItem *>(r->d_items);
        for (int i = 0; i < 5; ++i) a.phase_begin[i] = begin[k][i];
        a.counters = w + 5 * k;
        a.bar_count = w + 5 * k + 4;
        a.bar_gen = w + kRwGen + k;
        a.status = w + kRwStatus;
        a.abort_flag = w + kRwAbort;
        r->n_word_items[k] = begin[k][4] - begin[k][0];
    }
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

    // counters, barrier words, status, abort flag (kRw*)
    if (cudaMalloc(&r->d_words, kRwWords * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(r->d_words, 0, kRwWords * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        ragged_free(r);
        return NTT_ERR_OOM;
    }
    uint32_t *w = reinterpret_cast<uint32_t *>(r->d_words);
    auto plan_of = [&](uint32_t j) { return groups[group_of[j]].plan; };

    // ---- persistent grids: every CTA of a cooperative launch resident
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int k = 0; k < 2; ++k) {
        size_t smem = 0;
        int bps = 0;
        if (kernel_config(r->red, k == 1, &smem, &bps) != cudaSuccess || bps < 1) {
            cudaGetLastError();
            ragged_free(r);
            return NTT_ERR_CUDA;
        }
        r->grid[k] = (unsigned)(sms * bps);
    }

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
            auto launch = [&]() { return launch_all(r, ts) == cudaSuccess; };
            float ms = 0.f;
            ok = launch() && cudaEventRecord(e0, ts) == cudaSuccess;
            for (int k = 0; k < 3 && ok; ++k) ok = launch();
            ok = ok && cudaEventRecord(e1, ts) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            uint32_t status = 0;
            ok = ok && cudaMemcpy(&status, w + kRwStatus, sizeof(status), cudaMemcpyDeviceToHost) == cudaSuccess &&
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
    // test hook: CTA 0 of the first kernel leaves before its first barrier
    if (flags & NTT_TEST_STALL) r->args[r->n_word_items[0] ? 0 : 1].stall = 1u;

    // ---- graph capture
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); ragged_free(r); return NTT_ERR_CUDA; }
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // item counters and barrier counts (a launch whose barrier wait ran
        // out leaves arrivals behind), the abort flag, then the kernels
        cudaError_t le = launch_all(r, st);
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
    if (cudaMemcpy(&v, r->args[0].status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return NTT_ERR_CUDA;
    if (v) cudaMemset(r->args[0].status, 0, sizeof(uint32_t));
    return (v & 2u) ? NTT_ERR_TIMEOUT : NTT_OK;
}

uint32_t ntt_ragged_item_tiles(ntt_ragged_t r) { return r ? r->item_tiles : 0u; }

void ntt_ragged_destroy(ntt_ragged_t r) {
    if (!r) return;
    cudaDeviceSynchronize();
    ragged_free(r);
}

}  // extern "C"
