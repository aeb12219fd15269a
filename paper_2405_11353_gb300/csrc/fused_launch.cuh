// fused_launch.cuh -- host launcher of the fused path for one (word,
// reduction) pair; each fused_<w>_<red>.cu instantiates it once so the
// kernels compile in parallel.
#pragma once
#include <cstring>

#include <cstdlib>

#include "fused.cuh"
#include "plan.hpp"
#include "stream.cuh"

namespace nttgb {

static_assert(kN2Log == (uint32_t)kChunkLog, "two-pass split must match the plan's chunk size");

template <class W, int RED, bool INV, int LOGS, int KIND, int PP, bool OTF_K = false>
cudaError_t launch_pass(const FArgs<W> &a, uint32_t threads, size_t smem, cudaStream_t st) {
    auto kern = k_fused<W, RED, INV, LOGS, KIND, PP, OTF_K>;
    // persistent grid: as many CTAs as fit on the GPU at once
    static int resident = 0;
    if (!resident) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        // all of the unified L1/shared storage as shared memory: the tiles,
        // not the L1 cache, hold the working set
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)threads, smem);
        if (e != cudaSuccess) return e;
        resident = sms * (per_sm > 0 ? per_sm : 1);
    }
    unsigned grid = a.ntiles < (uint64_t)resident ? (unsigned)a.ntiles : (unsigned)resident;
    if (grid == 0) grid = 1;
    // programmatic dependent launch: the kernel may be scheduled while the
    // previous launch on the stream drains; it waits for that launch's
    // results before touching data (griddep_wait in k_fused)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

// Tensor map of the data viewed as (ntrans * N1) rows of N2 words, with a
// box of K columns by min(N1, 256) rows: one column strip of one transform.
inline cudaError_t make_cols_tmap(CUtensorMap *m, void *data, bool w64, uint64_t rows, uint32_t N2, uint32_t K,
                                  uint32_t box_rows) {
    using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return cudaErrorNotSupported;
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    const size_t wb = w64 ? 8 : 4;
    cuuint64_t dims[2] = {N2, rows};
    cuuint64_t strides[1] = {(cuuint64_t)N2 * wb};
    cuuint32_t box[2] = {K, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(m, w64 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, data, dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor map of the data viewed as rows of 128 bytes (RW words), box of
// box_rows rows, with the 128-byte swizzle.
inline cudaError_t make_rows_tmap(CUtensorMap *m, void *data, bool w64, uint64_t rows, uint32_t RW,
                                  uint32_t box_rows) {
    using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return cudaErrorNotSupported;
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    cuuint64_t dims[2] = {RW, rows};
    cuuint64_t strides[1] = {128};
    cuuint32_t box[2] = {RW, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(m, w64 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, data, dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <class W, int RED, bool INV, int KIND, int PP, bool OTF_K = false, int LOGS = 4>
cudaError_t pass_dispatch(int logS, const FArgs<W> &a, uint32_t threads, size_t smem, cudaStream_t st) {
    constexpr int MAXS = KIND == TK_SINGLE ? (sizeof(W) == 4 ? kSingleMaxLog32 : kSingleMaxLog64)
                                           : (KIND == TK_COLS ? 9 : kChunkLogMax);
    constexpr int MINS = KIND == TK_SINGLE ? 4 : (KIND == TK_COLS ? 5 : kChunkLogMin);
    if constexpr (LOGS > MAXS) {
        return cudaErrorInvalidValue;
    } else {
        // (chunk twiddles made on the fly: 256-word chunks only)
        if constexpr (LOGS >= MINS && !(OTF_K && LOGS != (int)kN2Log)) {
            if (logS == LOGS) return launch_pass<W, RED, INV, LOGS, KIND, PP, OTF_K>(a, threads, smem, st);
        }
        return pass_dispatch<W, RED, INV, KIND, PP, OTF_K, LOGS + 1>(logS, a, threads, smem, st);
    }
}

template <class W, int KIND, int PP> uint32_t tile_k_for(int logS) {
    switch (logS) {
#define NTTGB_CASE(s) case s: return tile_k<W, s, KIND, PP>();
        NTTGB_CASE(4) NTTGB_CASE(5) NTTGB_CASE(6) NTTGB_CASE(7) NTTGB_CASE(8) NTTGB_CASE(9)
        NTTGB_CASE(10) NTTGB_CASE(11) NTTGB_CASE(12) NTTGB_CASE(13) NTTGB_CASE(14)
#undef NTTGB_CASE
    }
    return 1;
}

template <class W, int KIND, bool INV, int PP> size_t smem_for(int logS) {
    switch (logS) {
#define NTTGB_CASE(s) case s: return fused_smem_bytes<W, s, KIND, INV, PP>();
        NTTGB_CASE(4) NTTGB_CASE(5) NTTGB_CASE(6) NTTGB_CASE(7) NTTGB_CASE(8) NTTGB_CASE(9)
        NTTGB_CASE(10) NTTGB_CASE(11) NTTGB_CASE(12) NTTGB_CASE(13) NTTGB_CASE(14)
#undef NTTGB_CASE
    }
    return 0;
}

// Tile geometry: K sub-transforms of 2^logS words per CTA, 2^logS / 16
// threads each.
inline uint32_t ilog2(uint32_t x) { uint32_t r = 0; while ((1u << r) < x) ++r; return r; }

template <class W, int KIND, int P> uint32_t tile_k_p(int logS) {
    switch (logS) {
#define NTTGB_CASE(s) case s: return tile_k<W, s, KIND, P>();
        NTTGB_CASE(4) NTTGB_CASE(5) NTTGB_CASE(6) NTTGB_CASE(7) NTTGB_CASE(8) NTTGB_CASE(9)
        NTTGB_CASE(10) NTTGB_CASE(11) NTTGB_CASE(12) NTTGB_CASE(13) NTTGB_CASE(14)
#undef NTTGB_CASE
    }
    return 1;
}

// Arguments of one pass over `data` (tiles of K sub-transforms of 2^logS
// words), in place, or (out, pw_b set: the inverse chunk pass of the fused
// pointwise + inverse) from `data` times pw_b into `out`.
template <class W, bool INV, int KIND>
cudaError_t fill_pass(FArgs<W> &a, ntt_plan_s &p, W *data, const void *tw, uint64_t ntrans, int logS,
                      bool final_pass, uint32_t K, W *out, const W *pw_b, uint32_t pair_kg = 0) {
    std::memset(&a, 0, sizeof(a));
    a.data = data;
    a.out = out ? out : data;
    a.pw_b = pw_b;
    a.status = p.d_status;
    a.tw = reinterpret_cast<const Tw<W> *>(tw);
    if (KIND == TK_CHUNKS && p.tw_otf && sizeof(W) == 4) {
        // chunk twiddles made on the fly from seeds (NTT_TW_OTF)
        a.tw_seed = reinterpret_cast<const W *>(INV ? p.d_seed_inv : p.d_seed_fwd);
        a.tw_root = reinterpret_cast<const Tw<W> *>(INV ? p.d_root_inv : p.d_root_fwd);
    }
    // every pass reads a table or, for chunk passes, makes one from seeds
    if (!a.tw && !(KIND == TK_CHUNKS && a.tw_seed && a.tw_root)) return cudaErrorInvalidValue;
    a.lc = p.d_limb;
    a.ntrans = ntrans;
    a.logN = p.logN;
    a.L = p.L;
    a.s2 = p.s2;
    a.final_pass = final_pass ? 1u : 0u;
    a.stall_tx = (p.flags & NTT_TEST_STALL) && !INV && KIND != TK_CHUNKS ? 16u : 0u;
    if (KIND == TK_SINGLE) a.ntiles = (ntrans + K - 1) / K;
    else if (KIND == TK_COLS) a.ntiles = ntrans * ((1u << p.s2) / K);
    else a.ntiles = ntrans * ((1u << (p.logN - p.s2)) / K);
    a.logK = ilog2(K);
    if (a.ntiles >= (1ull << 32) || ntrans >= (1ull << 32)) return cudaErrorInvalidValue;   // 32-bit tile cursor
    if (KIND == TK_COLS) {
        const uint32_t N1 = 1u << logS;
        cudaError_t e = make_cols_tmap(&a.tmap, data, sizeof(W) == 8, ntrans * N1, 1u << p.s2, K,
                                       N1 < 256 ? N1 : 256u);
        if (e != cudaSuccess) return e;
    }
    if (KIND == TK_CHUNKS && INV) {
        // inverse chunk tiles: 128-byte rows, swizzled (see fused.cuh); a
        // box holds the tile's K chunks, or one chunk when the tile pairs
        // polynomials (one copy per polynomial)
        const uint32_t RW = 128 / sizeof(W);
        cudaError_t e = make_rows_tmap(&a.tmap, data, sizeof(W) == 8, ntrans * p.N / RW, RW,
                                       (pair_kg ? pair_kg : K) * (1u << logS) / RW);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One pass as its own launch; PP: tile configuration (0, or 3 for
// 16-chunk tiles in a chunk pass).
template <class W, int RED, bool INV, int KIND, int PP = 0, bool OTF_K = false>
cudaError_t run_pass(ntt_plan_s &p, W *data, const void *tw, uint64_t ntrans, int logS, bool final_pass,
                     cudaStream_t st, W *out = nullptr, const W *pw_b = nullptr) {
    FArgs<W> a;
    const uint32_t T = (1u << logS) >> radix_log<PP>();
    const uint32_t K = tile_k_for<W, KIND, PP>(logS);
    constexpr bool paired = paired_chunks<KIND, PP>();
    constexpr uint32_t KG = paired ? pair_positions<KIND, PP>() : 0u;
    // whole polynomial groups of K / KG polynomials
    if (paired && (K % KG != 0 || (ntrans / p.L) % (K / KG) != 0)) return cudaErrorInvalidValue;
    cudaError_t e = fill_pass<W, INV, KIND>(a, p, data, tw, ntrans, logS, final_pass, K, out, pw_b, KG);
    if (e != cudaSuccess) return e;
    size_t smem = smem_for<W, KIND, INV, PP>(logS);
    ++p.last_launches;
    if (OTF_K != (a.tw_seed != nullptr)) return cudaErrorInvalidValue;   // kernel and plan must agree
    return pass_dispatch<W, RED, INV, KIND, PP, OTF_K>(logS, a, K * T, smem, st);
}

// The chunk pass in the plan's form for this direction.  Tiles pair
// polynomials (the same chunk of K polynomials: one twiddle table per tile,
// so a CTA needs less shared memory and more of them fit on an SM) when K
// divides the batch, else they hold K consecutive chunks of one polynomial.
//
// The shuffle forms' chunk passes (bit 6 of P) for 4-byte words: compiled
// in units of their own (fused_u32_<reduction>_shfl.cu), declared here.
template <class W, int RED, bool INV, int LRB>
cudaError_t run_chunk_pass_shfl(ntt_plan_s &p, int form, W *data, const void *tw, uint64_t ntrans, bool final_pass,
                                cudaStream_t st, W *out, const W *pw_b);

template <class W, int RED, bool INV, int LRB = 0>
cudaError_t run_chunk_pass(ntt_plan_s &p, int form, W *data, const void *tw, uint64_t ntrans, bool final_pass,
                           cudaStream_t st, W *out = nullptr, const W *pw_b = nullptr) {
    // (LRB = 16: the plan's rounds are of three stages on 8 words a thread;
    // + 64: exchanges by warp shuffles)
    if constexpr ((LRB & 16) == 0) {
        if (p.lr == 3)
            return run_chunk_pass<W, RED, INV, LRB | 16>(p, form, data, tw, ntrans, final_pass, st, out, pw_b);
    }
    if constexpr ((LRB & 64) == 0 && sizeof(W) == 4) {
        if (form_is_shfl(form) && !p.tw_otf)
            return run_chunk_pass_shfl<W, RED, INV, LRB | 64>(p, form == FORM_SMALL_SHFL ? FORM_SMALL : FORM_WIDE,
                                                              data, tw, ntrans, final_pass, st, out, pw_b);
    }
    if (form_is_shfl(form)) form = form == FORM_SMALL_SHFL ? FORM_SMALL : FORM_WIDE;
    const int logS = (int)p.s2;
    // pairing needs K | batch, and chunks of at least 256 words (each
    // polynomial's box of swizzled rows then starts on a 1 KiB boundary)
    const uint64_t B = logS >= 8 ? ntrans / p.L : 1;
    if constexpr (sizeof(W) == 4 && RED == RED_SHOUP && LRB == 0) {
        // NTT_TW_OTF plans: kernels that make the chunk tables from seeds
        if (p.tw_otf) {
            if (form == FORM_SMALL)
                return B % 2 == 0
                           ? run_pass<W, RED, INV, TK_CHUNKS, 8, true>(p, data, tw, ntrans, logS, final_pass, st, out, pw_b)
                           : run_pass<W, RED, INV, TK_CHUNKS, 0, true>(p, data, tw, ntrans, logS, final_pass, st, out, pw_b);
            return B % 16 == 0
                       ? run_pass<W, RED, INV, TK_CHUNKS, 11, true>(p, data, tw, ntrans, logS, final_pass, st, out, pw_b)
                       : run_pass<W, RED, INV, TK_CHUNKS, 3, true>(p, data, tw, ntrans, logS, final_pass, st, out, pw_b);
        }
    }
    const uint64_t ks = tile_k_for<W, TK_CHUNKS, LRB>(logS), kw = tile_k_for<W, TK_CHUNKS, LRB | 3>(logS);
    if (form == FORM_SMALL)
        return B % ks == 0 && B > 1
                   ? run_pass<W, RED, INV, TK_CHUNKS, LRB | 8>(p, data, tw, ntrans, logS, final_pass, st, out, pw_b)
                   : run_pass<W, RED, INV, TK_CHUNKS, LRB>(p, data, tw, ntrans, logS, final_pass, st, out, pw_b);
    if (B % kw == 0 && B > 1)
        return run_pass<W, RED, INV, TK_CHUNKS, LRB | 11>(p, data, tw, ntrans, logS, final_pass, st, out, pw_b);
    if constexpr (sizeof(W) == 4) {
        // K / 2 polynomials x 2 chunks a tile: two twiddle tables instead of
        // K, so more CTAs fit an SM (a batch of 8 at K = 16: 4 instead of 3)
        if (B % (kw / 2) == 0 && B > 1)
            return run_pass<W, RED, INV, TK_CHUNKS, LRB | 139>(p, data, tw, ntrans, logS, final_pass, st, out, pw_b);
    }
    return run_pass<W, RED, INV, TK_CHUNKS, LRB | 3>(p, data, tw, ntrans, logS, final_pass, st, out, pw_b);
}

#ifdef NTTGB_SHFL_UNIT
template <class W, int RED, bool INV, int LRB>
cudaError_t run_chunk_pass_shfl(ntt_plan_s &p, int form, W *data, const void *tw, uint64_t ntrans, bool final_pass,
                                cudaStream_t st, W *out, const W *pw_b) {
    return run_chunk_pass<W, RED, INV, LRB>(p, form, data, tw, ntrans, final_pass, st, out, pw_b);
}
#endif

// Tuning of the one-launch two-pass form: tiles per work item and the lag
// (in rounds of one limb) between a limb's first and second pass; unset or
// 0 = the defaults below.  Read at each call from NTT_STREAM_TILES /
// NTT_STREAM_LAG (any value gives the same result; only the speed changes).
inline uint32_t stream_env(const char *name) {
    const char *v = std::getenv(name);
    return v ? (uint32_t)std::strtoul(v, nullptr, 10) : 0u;
}

// Both passes of a two-pass transform in one launch (stream.cuh).
template <class W, int RED, bool INV>
cudaError_t run_stream(ntt_plan_s &p, W *data, uint64_t ntrans, cudaStream_t st, W *out, const W *pw_b) {
    const uint32_t env_tiles = p.stream_tiles ? p.stream_tiles : stream_env("NTT_STREAM_TILES");
    const uint32_t env_lag = stream_env("NTT_STREAM_LAG");
    StreamArgs<W> sa;
    std::memset(&sa, 0, sizeof(sa));
    const uint32_t Kc = tile_k_p<W, TK_COLS, stream_p<W>()>((int)p.s1);
    const uint32_t Kh = tile_k<W, kN2Log, TK_CHUNKS, stream_p<W>()>();
    const uint64_t B = ntrans / p.L;
    const uint64_t tpl_cols = B * ((1u << p.s2) / Kc), tpl_chunks = B * ((1u << p.s1) / Kh);
    if (tpl_cols * p.L >= (1ull << 32) || tpl_chunks * p.L >= (1ull << 32)) return cudaErrorInvalidValue;
    W *o = out ? out : data;
    cudaError_t e;
    if (!INV) {
        e = fill_pass<W, false, TK_COLS>(sa.pass[0], p, data, p.d_main_fwd, ntrans, (int)p.s1, false, Kc, nullptr,
                                         nullptr);
        if (e == cudaSuccess)
            e = fill_pass<W, false, TK_CHUNKS>(sa.pass[1], p, data, p.d_chunk_fwd, ntrans, (int)p.s2, true, Kh,
                                               nullptr, nullptr);
        sa.tiles_per_limb[0] = (uint32_t)tpl_cols;
        sa.tiles_per_limb[1] = (uint32_t)tpl_chunks;
    } else {
        e = fill_pass<W, true, TK_CHUNKS>(sa.pass[0], p, data, p.d_chunk_inv, ntrans, (int)p.s2, false, Kh, o, pw_b);
        if (e == cudaSuccess)
            e = fill_pass<W, true, TK_COLS>(sa.pass[1], p, o, p.d_main_inv, ntrans, (int)p.s1, true, Kc, nullptr,
                                            nullptr);
        sa.tiles_per_limb[0] = (uint32_t)tpl_chunks;
        sa.tiles_per_limb[1] = (uint32_t)tpl_cols;
    }
    if (e != cudaSuccess) return e;
    int resident = 0;
    e = stream_resident<W, RED, INV>((int)p.s1, &resident);
    if (e != cudaSuccess) return e;
    // work items of up to 4 tiles (4 KiB ... 32 KiB each), fewer when the
    // first pass would otherwise have less than two items per CTA
    uint32_t g = env_tiles;
    if (!g) {
        const uint64_t first_tiles = (uint64_t)sa.tiles_per_limb[0] * p.L;
        const uint64_t per = first_tiles / (2ull * (uint64_t)resident);
        g = per >= 4 ? 4u : (per >= 2 ? 2u : 1u);
    }
    uint32_t slots = 0;
    for (int i = 0; i < 2; ++i) {
        sa.tiles_per_item[i] = g < sa.tiles_per_limb[i] ? g : sa.tiles_per_limb[i];
        sa.items_per_limb[i] = (sa.tiles_per_limb[i] + sa.tiles_per_item[i] - 1) / sa.tiles_per_item[i];
        slots += sa.items_per_limb[i];
    }
    sa.L = p.L;
    // the second pass of a limb starts about two grids of items after its
    // first pass (so its first-pass tiles are done), plus one round; the
    // intermediate then held in L2 is about lag rounds of one limb
    sa.lag = env_lag ? env_lag : (2u * (uint32_t)resident + slots - 1) / slots + 1;
    sa.ctr = p.d_stream_ctr + (size_t)(p.stream_seq++ % kStreamRing) * stream_set_words(p.L);
    ++p.last_launches;
    switch (p.s1) {
    case 6: return stream_launch<W, RED, INV, 6>(sa, st);
    case 7: return stream_launch<W, RED, INV, 7>(sa, st);
    case 8: return stream_launch<W, RED, INV, 8>(sa, st);
    case 9: return stream_launch<W, RED, INV, 9>(sa, st);
    }
    return cudaErrorInvalidValue;
}

// The column pass of a two-pass plan, in the plan's radix.
template <class W, int RED, bool INV>
cudaError_t run_cols_pass(ntt_plan_s &p, W *data, const void *tw, uint64_t ntrans, bool final_pass,
                          cudaStream_t st) {
    // (bit 5: rows of 2^s2 words other than 256, read from the arguments)
    if (p.s2 != kN2Log) {
        if (p.lr == 3) return run_pass<W, RED, INV, TK_COLS, 48>(p, data, tw, ntrans, (int)p.s1, final_pass, st);
        return run_pass<W, RED, INV, TK_COLS, 32>(p, data, tw, ntrans, (int)p.s1, final_pass, st);
    }
    if (p.lr == 3) return run_pass<W, RED, INV, TK_COLS, 16>(p, data, tw, ntrans, (int)p.s1, final_pass, st);
    return run_pass<W, RED, INV, TK_COLS>(p, data, tw, ntrans, (int)p.s1, final_pass, st);
}

template <class W, int RED>
cudaError_t run_fused_t(ntt_plan_s &p, void *data_v, uint32_t batch, bool inverse, cudaStream_t st) {
    W *data = reinterpret_cast<W *>(data_v);
    const uint64_t ntrans = (uint64_t)batch * p.L;
    cudaError_t e;
    if (p.fused_mode == FUSED_SINGLE) {
        if (!inverse) return run_pass<W, RED, false, TK_SINGLE>(p, data, p.d_main_fwd, ntrans, p.logN, true, st);
        return run_pass<W, RED, true, TK_SINGLE>(p, data, p.d_main_inv, ntrans, p.logN, true, st);
    }
    const int form = p.form_for(batch, inverse);
    if (form == FORM_STREAMED) {
        if (!inverse) return run_stream<W, RED, false>(p, data, ntrans, st, nullptr, nullptr);
        return run_stream<W, RED, true>(p, data, ntrans, st, nullptr, nullptr);
    }
    if (!inverse) {
        e = run_cols_pass<W, RED, false>(p, data, p.d_main_fwd, ntrans, false, st);
        if (e != cudaSuccess) return e;
        return run_chunk_pass<W, RED, false>(p, form, data, p.d_chunk_fwd, ntrans, true, st);
    }
    e = run_chunk_pass<W, RED, true>(p, form, data, p.d_chunk_inv, ntrans, false, st);
    if (e != cudaSuccess) return e;
    return run_cols_pass<W, RED, true>(p, data, p.d_main_inv, ntrans, true, st);
}

// c = inverse(a (.) b) for two-pass plans: the product is taken in the
// first inverse pass (its first round reads b beside a), which writes c;
// the second pass runs on c in place.
template <class W, int RED>
cudaError_t run_fused_pwinv_t(ntt_plan_s &p, void *c, const void *a, const void *b, uint32_t batch,
                              cudaStream_t st) {
    const uint64_t ntrans = (uint64_t)batch * p.L;
    W *cw = reinterpret_cast<W *>(c);
    const int form = p.form_for(batch, true);
    if (form == FORM_STREAMED)
        return run_stream<W, RED, true>(p, const_cast<W *>(reinterpret_cast<const W *>(a)), ntrans, st, cw,
                                        reinterpret_cast<const W *>(b));
    cudaError_t e = run_chunk_pass<W, RED, true>(p, form, const_cast<W *>(reinterpret_cast<const W *>(a)),
                                                 p.d_chunk_inv, ntrans, false, st, cw,
                                                 reinterpret_cast<const W *>(b));
    if (e != cudaSuccess) return e;
    return run_cols_pass<W, RED, true>(p, cw, p.d_main_inv, ntrans, true, st);
}

}  // namespace nttgb
