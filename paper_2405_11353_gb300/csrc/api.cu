// api.cu -- the C ABI of libnttgb: validation, plan building, dispatch.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "host_nt.hpp"
#include "plan.hpp"

using nttgb::LimbConst;
namespace H = nttgb::host;
using u128 = unsigned __int128;

namespace {

constexpr uint32_t kKnownFlags =
    NTT_WORD64 | NTT_ORDER_BITREV | NTT_RED_MASK | NTT_CHECK | NTT_CLUSTER | NTT_STREAMED |
    NTT_TC_IMMA | NTT_TW_OTF | NTT_TEST_STALL;
constexpr uint32_t kMaxLimbs = 4096;

int red_of(uint32_t flags) {
    switch (flags & NTT_RED_MASK) {
    case NTT_RED_BARRETT: return nttgb::RED_BARRETT;
    case NTT_RED_MONTGOMERY: return nttgb::RED_MONTGOMERY;
    default: return nttgb::RED_SHOUP;
    }
}

bool is_pow2(uint32_t x) { return x && !(x & (x - 1)); }

// Twiddle pair (value, companion) for the plan's reduction.
struct Enc {
    uint64_t q;
    int W;          // 32 or 64
    int red;
    uint64_t qinv;  // q^-1 mod 2^W
    void operator()(uint64_t w, uint64_t &v, uint64_t &c) const {
        const u128 R = (u128)1 << W;
        if (red == nttgb::RED_SHOUP) {
            v = w;
            c = (uint64_t)(((u128)w << W) / q);
        } else if (red == nttgb::RED_MONTGOMERY) {
            uint64_t wm = (uint64_t)(((u128)w % q) * (R % q) % q);
            v = wm;
            c = W == 32 ? (uint64_t)((uint32_t)wm * (uint32_t)qinv) : wm * qinv;
        } else {
            v = w;
            c = 0;
        }
    }
};

// Writes a [L][N] table of pairs in the word type into `out` (bytes).
void put_pair(std::vector<uint8_t> &out, size_t idx, uint64_t v, uint64_t c, bool w64) {
    if (w64) {
        uint64_t *p = reinterpret_cast<uint64_t *>(out.data()) + 2 * idx;
        p[0] = v; p[1] = c;
    } else {
        uint32_t *p = reinterpret_cast<uint32_t *>(out.data()) + 2 * idx;
        p[0] = (uint32_t)v; p[1] = (uint32_t)c;
    }
}

// Device copy of a host table; its size is added to *total.
ntt_status upload(void **dptr, const std::vector<uint8_t> &h, uint64_t *total) {
    *total += h.size();
    if (cudaMalloc(dptr, h.size()) != cudaSuccess) { *dptr = nullptr; cudaGetLastError(); return NTT_ERR_OOM; }
    if (cudaMemcpy(*dptr, h.data(), h.size(), cudaMemcpyHostToDevice) != cudaSuccess) return NTT_ERR_CUDA;
    return NTT_OK;
}

void free_plan_memory(ntt_plan_s *p) {
    void *ptrs[] = {p->d_limb,      p->d_w_fwd,     p->d_w_inv,   p->d_twist,    p->d_untwist,
                    p->d_main_fwd,  p->d_main_inv,  p->d_chunk_fwd, p->d_chunk_inv, p->d_tc,
                    p->d_clu_fwd,   p->d_clu_inv,   p->d_scratch,  p->d_status,
                    p->d_stream_ctr, p->d_tc5, p->d_seed_fwd, p->d_seed_inv,
                    p->d_root_fwd,  p->d_root_inv};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (p->aux_ready) {
        cudaStreamDestroy(p->aux_h2d);
        cudaStreamDestroy(p->aux_d2h);
        for (cudaEvent_t e : p->aux_ev) cudaEventDestroy(e);
    }
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

namespace nttgb {
ntt_status validate_plan_args(uint32_t N, const uint64_t *q, uint32_t L, uint32_t flags);
}

namespace {

ntt_status validate(uint32_t N, const uint64_t *q, uint32_t L, uint32_t flags) {
    if (!q || L == 0 || L > kMaxLimbs) return NTT_ERR_INVALID_ARG;
    if (flags & ~kKnownFlags) return NTT_ERR_INVALID_ARG;
    if ((flags & NTT_RED_MASK) == NTT_RED_MASK) return NTT_ERR_INVALID_ARG;
    if (!is_pow2(N)) return NTT_ERR_N_NOT_POW2;
    if (N < 2 || N > (1u << 17)) return NTT_ERR_N_RANGE;
    const uint64_t limit = (flags & NTT_WORD64) ? (1ull << 60) : (1ull << 30);
    for (uint32_t l = 0; l < L; ++l) {
        if (q[l] >= limit || q[l] < 3) return NTT_ERR_Q_WIDTH;
        if (!H::is_prime(q[l])) return NTT_ERR_Q_NOT_PRIME;
        if ((q[l] - 1) % (2ull * N) != 0) return NTT_ERR_Q_NOT_NTT_FRIENDLY;
    }
    return NTT_OK;
}

// Tensor-core four-step tables for N = 2^16 (layout described in tc.cu).
// With k1 = bitrev8(u), k2 = bitrev8(v):
//   forward column matrix  [u][n1] = psi^(256 (2 k1 + 1) n1)
//   forward row matrix     [v][n2] = psi^(512 k2 n2)
//   inverse row matrix     [n2][v] = psi^(-512 k2 n2) / 256
//   inverse column matrix  [n1][u] = psi^(-256 (2 k1 + 1) n1) / 256
//   forward twiddle        [u][n2] = psi^(n2 (2 k1 + 1))
//   inverse twiddle        [u][n2] = psi^(-n2 (2 k1 + 1))
// each matrix as four 8-bit digit planes; twiddles as Shoup pairs.
// IEEE half-precision bits of a small integer (|d| <= 2048: exact).
uint16_t half_bits(int d) {
    if (d == 0) return 0;
    const uint16_t sign = d < 0 ? 0x8000u : 0u;
    uint32_t a = (uint32_t)(d < 0 ? -d : d), e = 0;
    while ((a >> (e + 1)) != 0) ++e;
    const uint32_t mant = (a << (10 - e)) & 0x3FFu;
    return (uint16_t)(sign | ((e + 15) << 10) | mant);
}

// Matrices of the tensor-core form as balanced 8-bit digits in fp16
// (tc5.cu): v = sum_d c_d 256^d, c_d = byte d of (v + 0x80808080) - 128.
void build_tc5_digits(const std::vector<uint8_t> &tc, uint32_t L, std::vector<uint8_t> &out) {
    out.assign((size_t)4 * L * 4 * 65536 * 2, 0);
    uint16_t *h = reinterpret_cast<uint16_t *>(out.data());
    for (size_t ml = 0; ml < (size_t)4 * L; ++ml)
        for (size_t e = 0; e < 65536; ++e) {
            uint32_t v = 0;
            for (int d = 0; d < 4; ++d) v |= (uint32_t)tc[(ml * 4 + d) * 65536 + e] << (8 * d);
            const uint32_t y = v + 0x80808080u;
            for (int d = 0; d < 4; ++d) h[(ml * 4 + d) * 65536 + e] = half_bits((int)((y >> (8 * d)) & 255u) - 128);
        }
}

void build_tc_tables(ntt_plan_s *p, std::vector<uint8_t> &out) {
    const uint32_t L = p->L, N = p->N;
    const size_t mat_bytes = (size_t)4 * L * 4 * 65536, tw_bytes = (size_t)2 * L * 65536 * 8;
    out.assign(mat_bytes + tw_bytes + (size_t)L * 8 * 4, 0);
    uint8_t *mats = out.data();
    uint32_t *tws = reinterpret_cast<uint32_t *>(out.data() + mat_bytes);
    uint32_t *pow8 = reinterpret_cast<uint32_t *>(out.data() + mat_bytes + tw_bytes);
    std::vector<uint64_t> pw(N), pwi(N);
    for (uint32_t l = 0; l < L; ++l) {
        const uint64_t q = p->q[l], psi = p->psi[l], psi_inv = H::invm(psi, q);
        const uint64_t inv256 = H::invm(256, q);
        pw[0] = pwi[0] = 1;
        for (uint32_t i = 1; i < N; ++i) { pw[i] = H::mulm(pw[i - 1], psi, q); pwi[i] = H::mulm(pwi[i - 1], psi_inv, q); }
        // psi^e and psi^-e for any e >= 0 (psi^N = -1)
        auto P = [&](uint64_t e, bool inv) -> uint64_t {
            e %= 2ull * N;
            const std::vector<uint64_t> &t = inv ? pwi : pw;
            return e < N ? t[e] : (q - t[e - N]) % q;
        };
        auto put_mat = [&](int m, uint32_t row, uint32_t col, uint64_t v) {
            uint8_t *base = mats + ((size_t)m * L + l) * 4 * 65536 + (size_t)row * 256 + col;
            for (int d = 0; d < 4; ++d) base[(size_t)d * 65536] = (uint8_t)((v >> (8 * d)) & 255u);
        };
        for (uint32_t u = 0; u < 256; ++u) {
            const uint64_t k1 = H::bitrev(u, 8);
            for (uint32_t n = 0; n < 256; ++n) {
                put_mat(0, u, n, P(256ull * (2 * k1 + 1) * n, false));
                put_mat(1, u, n, P(512ull * k1 * n, false));                       // u plays v, k1 plays k2
                put_mat(2, n, u, H::mulm(P(512ull * k1 * n, true), inv256, q));     // [n2][v]
                put_mat(3, n, u, H::mulm(P(256ull * (2 * k1 + 1) * n, true), inv256, q));  // [n1][u]
                const uint64_t wf = P((uint64_t)n * (2 * k1 + 1), false), wi = P((uint64_t)n * (2 * k1 + 1), true);
                const size_t at = ((size_t)0 * L + l) * 65536 + (size_t)u * 256 + n;
                const size_t ai = ((size_t)1 * L + l) * 65536 + (size_t)u * 256 + n;
                tws[2 * at] = (uint32_t)wf;
                tws[2 * at + 1] = (uint32_t)(((u128)wf << 32) / q);
                tws[2 * ai] = (uint32_t)wi;
                tws[2 * ai + 1] = (uint32_t)(((u128)wi << 32) / q);
            }
        }
        for (int s = 0; s < 8; ++s) pow8[l * 8 + s] = (uint32_t)H::powm(2, 8ull * s, q);
    }
}

ntt_status build_tables(ntt_plan_s *p) {
    const uint32_t N = p->N, L = p->L, n = p->logN;
    const bool w64 = p->word64;
    const int W = w64 ? 64 : 32;
    const size_t pair_bytes = w64 ? 16 : 8;
    const bool variant_tabs = (p->variant != NTT_FUSED && p->variant != NTT_TC_FOURSTEP) ||
                              p->fused_mode == nttgb::FUSED_STAGES;
    const bool clu_tabs = p->variant == NTT_FUSED && p->fused_mode == nttgb::FUSED_CLUSTER;
    const bool fused_tabs = p->variant == NTT_FUSED && p->fused_mode != nttgb::FUSED_STAGES && !clu_tabs;
    const bool two_pass = fused_tabs && p->fused_mode == nttgb::FUSED_TWO_PASS;
    const bool chunk_tabs = two_pass && !p->tw_otf;
    const bool otf_tabs = two_pass && p->tw_otf;

    std::vector<LimbConst> lc(L);
    std::vector<uint8_t> wf, wi, tw, ut, mf, mi, cf, ci;
    const size_t tab_bytes = (size_t)L * N * pair_bytes;
    if (variant_tabs) { wf.resize(tab_bytes); wi.resize(tab_bytes); tw.resize(tab_bytes); ut.resize(tab_bytes); }
    const uint32_t N1 = 1u << p->s1, N2 = 1u << p->s2;
    // fused main tables: [L][N] (single pass), or [L][N1] for the column
    // pass of two-pass plans (the chunk pass has its own tables or seeds)
    const uint32_t NM = two_pass ? N1 : N;
    if (fused_tabs) { mf.resize((size_t)L * NM * pair_bytes); mi.resize(mf.size()); }
    const uint32_t CP = nttgb::chunk_tab_pitch_rt(w64, p->s2);
    const size_t chunk_limb = (size_t)N1 * CP;       // pairs per limb, chunk tables
    if (chunk_tabs) { cf.resize(L * chunk_limb * pair_bytes); ci.resize(L * chunk_limb * pair_bytes); }
    // NTT_TW_OTF (4-byte words): per limb, 8 stage seeds per chunk and the
    // 256-entry root table of the chunk stages (see the kernels' staging)
    std::vector<uint8_t> sf, si, rf, ri;
    if (otf_tabs) {
        sf.resize((size_t)L * N1 * 8 * 4); si.resize(sf.size());
        rf.resize((size_t)L * N2 * 8); ri.resize(rf.size());
    }
    std::vector<uint8_t> kf, ki;   // cluster form tables (below)
    if (clu_tabs) { kf.resize((size_t)L * 8 * (8192 + 16) * pair_bytes); ki.resize(kf.size()); }
    // main-table position of entry i (see level_pos in modarith.cuh)
    auto main_pos = [&](uint32_t i) -> uint32_t {
        return p->fused_mode == nttgb::FUSED_SINGLE ? nttgb::level_pos(i, n) : nttgb::level_pos(i, p->s1, p->lr);
    };

    std::vector<uint64_t> pw(N), pwi(N);
    for (uint32_t l = 0; l < L; ++l) {
        const uint64_t q = p->q[l], psi = p->psi[l];
        const uint64_t psi_inv = H::invm(psi, q);
        const uint64_t ninv = H::invm(N % q, q);
        const uint64_t qinv64 = H::inv_pow2_64(q);
        Enc enc{q, W, p->red, w64 ? qinv64 : (uint64_t)(uint32_t)qinv64};

        LimbConst &c = lc[l];
        std::memset(&c, 0, sizeof(c));
        c.q = q;
        c.two_q = 2 * q;
        c.qinv = enc.qinv;
        const u128 R = (u128)1 << W;
        uint64_t rmod = (uint64_t)(R % q);
        c.r2 = H::mulm(rmod, rmod, q);
        c.r2c = w64 ? c.r2 * qinv64 : (uint64_t)((uint32_t)c.r2 * (uint32_t)qinv64);
        c.bits = (uint32_t)H::bit_length(q);
        if (w64) c.mu = (uint64_t)(((u128)1 << (2 * c.bits + 3)) / q);
        else c.mu = (uint64_t)((((u128)1) << 64) / q);
        enc(ninv, c.ninv_w, c.ninv_c);
        // N^-1 * psi^-bitrev(1) = N^-1 psi^-(N/2)
        enc(H::mulm(ninv, H::powm(psi_inv, N / 2, q), q), c.ninv_w1_w, c.ninv_w1_c);

        pw[0] = 1; pwi[0] = 1;
        for (uint32_t i = 1; i < N; ++i) { pw[i] = H::mulm(pw[i - 1], psi, q); pwi[i] = H::mulm(pwi[i - 1], psi_inv, q); }
        const size_t base = (size_t)l * N;
        uint64_t v, cc;
        if (variant_tabs) {
            // omega^e = psi^(2e): e < N/2 from the psi powers, the rest by omega^(N/2) = -1
            for (uint32_t e = 0; e < N; ++e) {
                uint64_t ex = 2ull * e % (2ull * N);
                uint64_t om = ex < N ? pw[ex] : (q - pw[ex - N]) % q;
                uint64_t omi = ex < N ? pwi[ex] : (q - pwi[ex - N]) % q;
                enc(om, v, cc); put_pair(wf, base + e, v, cc, w64);
                enc(omi, v, cc); put_pair(wi, base + e, v, cc, w64);
                enc(pw[e], v, cc); put_pair(tw, base + e, v, cc, w64);
                enc(H::mulm(ninv, pwi[e], q), v, cc); put_pair(ut, base + e, v, cc, w64);
            }
        }
        if (fused_tabs) {
            // entry i < NM: psi^bitrev_n(i) (for two-pass plans i < N1, the
            // column pass's stages)
            for (uint32_t i = 0; i < NM; ++i) {
                uint32_t r = H::bitrev(i, (int)n);
                enc(pw[r], v, cc); put_pair(mf, (size_t)l * NM + main_pos(i), v, cc, w64);
                enc(pwi[r], v, cc); put_pair(mi, (size_t)l * NM + main_pos(i), v, cc, w64);
            }
        }
        if (chunk_tabs) {
            // chunk r of the second pass: local entry 2^s + i' is global
            // entry 2^s (N1 + r) + i' of the bit-reversed psi table
            const size_t cbase = (size_t)l * chunk_limb;
            for (uint32_t r = 0; r < N1; ++r) {
                for (uint32_t j = CP - 1; j >= 1 && j >= N2; --j) {
                    put_pair(cf, cbase + (size_t)r * CP + j, 0, 0, w64);
                    put_pair(ci, cbase + (size_t)r * CP + j, 0, 0, w64);
                }
                put_pair(cf, cbase + (size_t)r * CP, 0, 0, w64);
                put_pair(ci, cbase + (size_t)r * CP, 0, 0, w64);
                for (uint32_t s = 0; s < p->s2; ++s)
                    for (uint32_t ip = 0; ip < (1u << s); ++ip) {
                        uint32_t gi = (1u << s) * (N1 + r) + ip;
                        uint32_t e = H::bitrev(gi, (int)n);
                        size_t at = cbase + (size_t)r * CP + nttgb::level_pos((1u << s) + ip, p->s2, p->lr);
                        enc(pw[e], v, cc); put_pair(cf, at, v, cc, w64);
                        enc(pwi[e], v, cc); put_pair(ci, at, v, cc, w64);
                    }
            }
        }
    }
    if (otf_tabs) {
        // chunk r, stage s (0 = first of the pass), entry i < 2^s: with
        // m = 2^s (N1 + r) + i, bitrev_n(m) = 2^(7-s) (1 + 2 bitrev_s1(r)) +
        // 2^(n-s) bitrev_s(i) (the bit fields of m are disjoint), so
        // psi^bitrev(m) = A_s(r) * B_s(i):
        //   seeds [l][r][s]        A_s(r), plain words
        //   roots [l][level_pos]   B_s(i) as Shoup pairs, entry 2^s + i in
        //                          the chunk tables' level-transposed order
        std::vector<uint64_t> pw2(N), pwi2(N);
        for (uint32_t l = 0; l < L; ++l) {
            const uint64_t q = p->q[l], psi = p->psi[l], psi_inv = H::invm(psi, q);
            Enc enc{q, W, p->red, (uint64_t)(uint32_t)H::inv_pow2_64(q)};
            pw2[0] = 1; pwi2[0] = 1;
            for (uint32_t i = 1; i < N; ++i) { pw2[i] = H::mulm(pw2[i - 1], psi, q); pwi2[i] = H::mulm(pwi2[i - 1], psi_inv, q); }
            uint32_t *sfw = reinterpret_cast<uint32_t *>(sf.data()) + (size_t)l * N1 * 8;
            uint32_t *siw = reinterpret_cast<uint32_t *>(si.data()) + (size_t)l * N1 * 8;
            for (uint32_t r = 0; r < N1; ++r)
                for (uint32_t s = 0; s < p->s2; ++s) {
                    const uint64_t e = (1ull << (p->s2 - 1 - s)) * (1 + 2 * (uint64_t)H::bitrev(r, (int)p->s1));
                    sfw[r * 8 + s] = (uint32_t)pw2[e];
                    siw[r * 8 + s] = (uint32_t)pwi2[e];
                }
            const size_t rb = (size_t)l * N2;
            uint64_t v, cc;
            put_pair(rf, rb, 0, 0, w64);
            put_pair(ri, rb, 0, 0, w64);
            for (uint32_t s = 0; s < p->s2; ++s)
                for (uint32_t ip = 0; ip < (1u << s); ++ip) {
                    const uint64_t e = (1ull << (n - s)) * (uint64_t)H::bitrev(ip, (int)s);
                    const size_t at = rb + nttgb::level_pos((1u << s) + ip, p->s2, p->lr);
                    enc(pw2[e], v, cc); put_pair(rf, at, v, cc, w64);
                    enc(pwi2[e], v, cc); put_pair(ri, at, v, cc, w64);
                }
        }
    }
    std::vector<uint8_t> tcb;
    std::vector<uint8_t> tc5b;
    if (p->variant == NTT_TC_FOURSTEP) {
        build_tc_tables(p, tcb);
        if (!p->tc_imma) build_tc5_digits(tcb, L, tc5b);
    }
    if (clu_tabs) {
        // cluster form (cluster.cuh), word index g = 8192 k + 1024 r + j; per
        // (limb, CTA c) a slice of 8192 + 16 pairs: block (c, r) of 1024
        // points after six stages at 1024 r (local entry 2^s + i' = global
        // entry 2^(s+6) + (8c + r) 2^s + i', level_pos layout); then round A
        // (stages 1, 2, 4 across k: entries 1..7) at 8192 + e; then round X
        // (stages 8, 16, 32 across r in block c: local entry 2^a + b =
        // global entry 2^(a+3) + c 2^a + b) at 8200 + e.
        const size_t SL = 8192 + 16;
        for (uint32_t l = 0; l < L; ++l) {
            const uint64_t q = p->q[l], psi = p->psi[l], psi_inv = H::invm(psi, q);
            Enc enc{q, W, p->red, (uint64_t)(uint32_t)H::inv_pow2_64(q)};
            uint64_t v, cc;
            std::vector<uint64_t> pw(N), pwi(N);
            pw[0] = 1; pwi[0] = 1;
            for (uint32_t i = 1; i < N; ++i) { pw[i] = H::mulm(pw[i - 1], psi, q); pwi[i] = H::mulm(pwi[i - 1], psi_inv, q); }
            auto put_both = [&](size_t at, uint32_t gidx) {
                const uint32_t e = H::bitrev(gidx, (int)n);
                enc(pw[e], v, cc); put_pair(kf, at, v, cc, w64);
                enc(pwi[e], v, cc); put_pair(ki, at, v, cc, w64);
            };
            for (uint32_t c = 0; c < 8; ++c) {
                const size_t sb = ((size_t)l * 8 + c) * SL;
                for (uint32_t r = 0; r < 8; ++r) {
                    const size_t kb = sb + (size_t)r * 1024;
                    put_pair(kf, kb, 0, 0, w64);
                    put_pair(ki, kb, 0, 0, w64);
                    for (uint32_t s = 0; s < 10; ++s)
                        for (uint32_t ip = 0; ip < (1u << s); ++ip)
                            put_both(kb + nttgb::level_pos((1u << s) + ip, 10),
                                     (1u << (s + 6)) + (8 * c + r) * (1u << s) + ip);
                }
                for (uint32_t e = 0; e < 16; ++e) { put_pair(kf, sb + 8192 + e, 0, 0, w64); put_pair(ki, sb + 8192 + e, 0, 0, w64); }
                for (uint32_t a = 0; a < 3; ++a)
                    for (uint32_t b = 0; b < (1u << a); ++b) {
                        const uint32_t e = (1u << a) + b;
                        put_both(sb + 8192 + e, e);
                        put_both(sb + 8200 + e, (1u << (a + 3)) + c * (1u << a) + b);
                    }
            }
        }
    }
    std::vector<uint8_t> lcb(sizeof(LimbConst) * L);
    std::memcpy(lcb.data(), lc.data(), lcb.size());
    ntt_status s;
    if (!tcb.empty() && (s = upload(&p->d_tc, tcb, &p->table_bytes)) != NTT_OK) return s;
    if (!tc5b.empty() && (s = upload(&p->d_tc5, tc5b, &p->table_bytes)) != NTT_OK) return s;
    if ((s = upload((void **)&p->d_limb, lcb, &p->table_bytes)) != NTT_OK) return s;
    if (variant_tabs) {
        if ((s = upload(&p->d_w_fwd, wf, &p->table_bytes)) != NTT_OK) return s;
        if ((s = upload(&p->d_w_inv, wi, &p->table_bytes)) != NTT_OK) return s;
        if ((s = upload(&p->d_twist, tw, &p->table_bytes)) != NTT_OK) return s;
        if ((s = upload(&p->d_untwist, ut, &p->table_bytes)) != NTT_OK) return s;
    }
    if (fused_tabs) {
        if ((s = upload(&p->d_main_fwd, mf, &p->table_bytes)) != NTT_OK) return s;
        if ((s = upload(&p->d_main_inv, mi, &p->table_bytes)) != NTT_OK) return s;
    }
    if (clu_tabs) {
        if ((s = upload(&p->d_clu_fwd, kf, &p->table_bytes)) != NTT_OK) return s;
        if ((s = upload(&p->d_clu_inv, ki, &p->table_bytes)) != NTT_OK) return s;
    }
    if (chunk_tabs) {
        if ((s = upload(&p->d_chunk_fwd, cf, &p->table_bytes)) != NTT_OK) return s;
        if ((s = upload(&p->d_chunk_inv, ci, &p->table_bytes)) != NTT_OK) return s;
    }
    if (otf_tabs) {
        if ((s = upload(&p->d_seed_fwd, sf, &p->table_bytes)) != NTT_OK) return s;
        if ((s = upload(&p->d_seed_inv, si, &p->table_bytes)) != NTT_OK) return s;
        if ((s = upload(&p->d_root_fwd, rf, &p->table_bytes)) != NTT_OK) return s;
        if ((s = upload(&p->d_root_inv, ri, &p->table_bytes)) != NTT_OK) return s;
    }
    if (cudaMalloc((void **)&p->d_status, sizeof(uint32_t)) != cudaSuccess) { cudaGetLastError(); return NTT_ERR_OOM; }
    if (cudaMemset(p->d_status, 0, sizeof(uint32_t)) != cudaSuccess) return NTT_ERR_CUDA;
    if (two_pass) {
        const size_t bytes = (size_t)nttgb::kStreamRing * nttgb::stream_set_words(L) * sizeof(uint32_t);
        if (cudaMalloc((void **)&p->d_stream_ctr, bytes) != cudaSuccess) { cudaGetLastError(); return NTT_ERR_OOM; }
        if (cudaMemset(p->d_stream_ctr, 0, bytes) != cudaSuccess) return NTT_ERR_CUDA;
    }
    return NTT_OK;
}

bool needs_scratch(const ntt_plan_s &p) {
    switch (p.variant) {
    case NTT_PEASE: case NTT_PEASE_NC: case NTT_STOCKHAM: case NTT_SIXSTEP: return true;
    case NTT_TC_FOURSTEP: return !p.tc_imma;     // tcgen05 passes run out of place
    default: return false;
    }
}

// A view of a fused plan (single-pass or two-pass) restricted to its limbs
// l0 .. l0 + lw - 1: every device table is per limb, so the view is the
// plan with its limb count cut and its table pointers advanced by l0 limbs.
// It shares the plan's status word and counter sets.
ntt_plan_s limb_window(const ntt_plan_s &p, uint32_t l0, uint32_t lw) {
    ntt_plan_s v = p;
    v.q.clear();
    v.psi.clear();
    v.L = lw;
    const size_t pair = p.word64 ? 16 : 8;
    const size_t main_limb = p.fused_mode == nttgb::FUSED_TWO_PASS ? ((size_t)1 << p.s1) : (size_t)p.N;
    auto adv = [&](void *ptr, size_t bytes_per_limb) -> void * {
        return ptr ? reinterpret_cast<uint8_t *>(ptr) + (size_t)l0 * bytes_per_limb : nullptr;
    };
    v.d_limb = p.d_limb + l0;
    v.d_main_fwd = adv(p.d_main_fwd, main_limb * pair);
    v.d_main_inv = adv(p.d_main_inv, main_limb * pair);
    if (p.fused_mode == nttgb::FUSED_TWO_PASS) {
        const size_t N1 = (size_t)1 << p.s1;
        const size_t CP = nttgb::chunk_tab_pitch_rt(p.word64, p.s2);
        v.d_chunk_fwd = adv(p.d_chunk_fwd, N1 * CP * pair);
        v.d_chunk_inv = adv(p.d_chunk_inv, N1 * CP * pair);
        v.d_seed_fwd = adv(p.d_seed_fwd, N1 * 8 * 4);
        v.d_seed_inv = adv(p.d_seed_inv, N1 * 8 * 4);
        v.d_root_fwd = adv(p.d_root_fwd, ((size_t)1 << p.s2) * 8);
        v.d_root_inv = adv(p.d_root_inv, ((size_t)1 << p.s2) * 8);
    }
    return v;
}

ntt_status run_transform(ntt_plan_t plan, void *d_data, uint32_t batch, ntt_stream_t stream, bool inverse,
                         uint32_t limbs = 0) {
    if (!plan || !d_data || batch == 0) return NTT_ERR_INVALID_ARG;
    if (!aligned16(d_data)) return NTT_ERR_ALIGNMENT;
    if (limbs > plan->L) return NTT_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (limbs && limbs != plan->L) {
        // polynomials of the plan's first `limbs` primes: every table is per
        // limb, so a view of the plan with a smaller L serves them
        ntt_plan_s view = *plan;
        view.L = limbs;
        view.q.clear();
        view.psi.clear();
        ntt_status s = run_transform(&view, d_data, batch, stream, inverse, 0);
        plan->last_launches = view.last_launches;
        plan->stream_seq = view.stream_seq;
        // the view may have grown (freed and replaced) the scratch buffer
        plan->d_scratch = view.d_scratch;
        plan->scratch_bytes = view.scratch_bytes;
        return s;
    }
    ntt_plan_s &p = *plan;
    p.last_launches = 0;
    if (needs_scratch(p)) {
        ntt_status s = nttgb::ensure_scratch(p, batch, st);
        if (s != NTT_OK) return s;
    }
    cudaError_t e = cudaSuccess;
    if (p.check) e = nttgb::launch_check_range(p, d_data, batch, st);
    if (e == cudaSuccess) {
        if (p.variant == NTT_TC_FOURSTEP) {
            // works in bit-reversed order, like the fused kernels
            if (inverse && !p.bitrev_order) e = nttgb::launch_bitrev_permute(p, d_data, batch, st);
            if (e == cudaSuccess)
                e = p.tc_imma ? nttgb::launch_tc(p, d_data, batch, inverse, st)
                              : nttgb::launch_tc5(p, d_data, batch, inverse, st);
            if (e == cudaSuccess && !inverse && !p.bitrev_order) e = nttgb::launch_bitrev_permute(p, d_data, batch, st);
        } else if (p.variant != NTT_FUSED || p.fused_mode == nttgb::FUSED_STAGES) {
            ntt_variant v = p.variant == NTT_FUSED ? NTT_FLAT : p.variant;
            e = nttgb::launch_variant(p, v, d_data, batch, inverse, st);
        } else {
            // the fused kernels work in bit-reversed order
            if (inverse && !p.bitrev_order) e = nttgb::launch_bitrev_permute(p, d_data, batch, st);
            if (e == cudaSuccess) e = nttgb::launch_fused(p, d_data, batch, inverse, st);
            if (e == cudaSuccess && !inverse && !p.bitrev_order) e = nttgb::launch_bitrev_permute(p, d_data, batch, st);
        }
    }
    if (e != cudaSuccess) { cudaGetLastError(); return NTT_ERR_CUDA; }
    return NTT_OK;
}

}  // namespace

namespace nttgb {

ntt_status validate_plan_args(uint32_t N, const uint64_t *q, uint32_t L, uint32_t flags) {
    return validate(N, q, L, flags);
}

ntt_status ensure_scratch(ntt_plan_s &p, uint32_t batch, cudaStream_t st) {
    size_t need = (size_t)batch * p.L * p.N * p.word_bytes();
    if (need <= p.scratch_bytes) return NTT_OK;
    if (cudaStreamSynchronize(st) != cudaSuccess) { cudaGetLastError(); return NTT_ERR_CUDA; }
    if (p.d_scratch) cudaFree(p.d_scratch);
    p.d_scratch = nullptr;
    p.scratch_bytes = 0;
    if (cudaMalloc(&p.d_scratch, need) != cudaSuccess) { cudaGetLastError(); p.d_scratch = nullptr; return NTT_ERR_OOM; }
    p.scratch_bytes = need;
    return NTT_OK;
}

}  // namespace nttgb

extern "C" {

const char *ntt_status_string(ntt_status s) {
    switch (s) {
    case NTT_OK: return "NTT_OK";
    case NTT_ERR_INVALID_ARG: return "NTT_ERR_INVALID_ARG: invalid argument";
    case NTT_ERR_N_NOT_POW2: return "NTT_ERR_N_NOT_POW2: N is not a power of two";
    case NTT_ERR_N_RANGE: return "NTT_ERR_N_RANGE: N outside 2^1..2^17";
    case NTT_ERR_Q_NOT_PRIME: return "NTT_ERR_Q_NOT_PRIME: modulus is not prime";
    case NTT_ERR_Q_NOT_NTT_FRIENDLY: return "NTT_ERR_Q_NOT_NTT_FRIENDLY: q != 1 mod 2N";
    case NTT_ERR_Q_WIDTH: return "NTT_ERR_Q_WIDTH: modulus too wide for the word size";
    case NTT_ERR_ALIGNMENT: return "NTT_ERR_ALIGNMENT: device pointer not 16-byte aligned";
    case NTT_ERR_CUDA: return "NTT_ERR_CUDA: CUDA runtime error";
    case NTT_ERR_OOM: return "NTT_ERR_OOM: device allocation failed";
    case NTT_ERR_INPUT_RANGE: return "NTT_ERR_INPUT_RANGE: input word >= q";
    case NTT_ERR_TIMEOUT: return "NTT_ERR_TIMEOUT: bounded device wait expired";
    case NTT_ERR_UNSUPPORTED: return "NTT_ERR_UNSUPPORTED: not supported by this build";
    case NTT_ERR_PSI: return "NTT_ERR_PSI: psi is not a primitive 2N-th root of unity";
    case NTT_ERR_SCRATCH_LIMIT: return "NTT_ERR_SCRATCH_LIMIT: batch exceeds the fixed 8 MiB scratch array";
    }
    return "NTT_ERR_UNKNOWN";
}

ntt_status ntt_validate(uint32_t N, const uint64_t *q, uint32_t L, uint32_t flags) {
    return validate(N, q, L, flags);
}

ntt_status ntt_default_psi(uint64_t q, uint32_t N, uint64_t *psi_out) {
    if (!psi_out || !is_pow2(N) || q < 3 || q >= (1ull << 62)) return NTT_ERR_INVALID_ARG;
    if (!H::is_prime(q)) return NTT_ERR_Q_NOT_PRIME;
    if ((q - 1) % (2ull * N) != 0) return NTT_ERR_Q_NOT_NTT_FRIENDLY;
    uint64_t g = H::smallest_generator(q);
    *psi_out = H::powm(g, (q - 1) / (2ull * N), q);
    return NTT_OK;
}

ntt_status ntt_find_primes(uint32_t bits, uint32_t m, uint32_t count, uint64_t *out) {
    if (!out || bits < 3 || bits > 62 || m >= bits || count == 0) return NTT_ERR_INVALID_ARG;
    const uint64_t top = 1ull << bits, low = 1ull << (bits - 1), step = 1ull << m;
    uint32_t found = 0;
    for (uint64_t k = 1; found < count; ++k) {
        if (k * step >= top) break;
        uint64_t q = top - k * step + 1;
        if (q <= low) break;
        if (H::is_prime(q)) out[found++] = q;
    }
    return found == count ? NTT_OK : NTT_ERR_INVALID_ARG;
}

ntt_status ntt_limb_shard(uint32_t L, uint32_t world, uint32_t rank, uint32_t *first, uint32_t *count) {
    if (!first || !count || world == 0 || rank >= world || L < world) return NTT_ERR_INVALID_ARG;
    const uint32_t base = L / world, extra = L % world;
    *count = base + (rank < extra ? 1u : 0u);
    *first = rank * base + (rank < extra ? rank : extra);
    return NTT_OK;
}

}  // extern "C"

namespace nttgb {

// Plan builder behind ntt_plan_create_ex.  single_max_log >= 0 caps the
// size done in one fused pass (the ragged kernel uses 12).
ntt_status create_plan(ntt_plan_t *plan, uint32_t N, const uint64_t *q, uint32_t L, ntt_variant variant,
                       uint32_t flags, const uint64_t *psi, int single_max_log, int split_log, int radix_log) {
    if (!plan) return NTT_ERR_INVALID_ARG;
    *plan = nullptr;
    if ((int)variant < NTT_DIT || (int)variant > NTT_TC_FOURSTEP) return NTT_ERR_INVALID_ARG;
    ntt_status s = validate(N, q, L, flags);
    if (s != NTT_OK) return s;
    // the tensor-core four-step form: N = 2^16, 4-byte words, Shoup twiddles
    if (variant == NTT_TC_FOURSTEP &&
        (N != (1u << 16) || (flags & NTT_WORD64) || (flags & NTT_RED_MASK) != NTT_RED_SHOUP))
        return NTT_ERR_UNSUPPORTED;
    // twiddles made on the fly: the fused path's chunk pass, 4-byte words,
    // Shoup pairs; not with the streamed one-launch form
    if ((flags & NTT_TW_OTF) && (variant != NTT_FUSED || (flags & NTT_WORD64) ||
                                 (flags & NTT_RED_MASK) != NTT_RED_SHOUP || (flags & NTT_STREAMED)))
        return NTT_ERR_UNSUPPORTED;
    ntt_plan_s *p = new (std::nothrow) ntt_plan_s();
    if (!p) return NTT_ERR_OOM;
    p->N = N;
    while ((1u << p->logN) < N) ++p->logN;
    p->L = L;
    p->flags = flags;
    p->variant = variant;
    p->red = red_of(flags);
    p->word64 = (flags & NTT_WORD64) != 0;
    p->bitrev_order = (flags & NTT_ORDER_BITREV) != 0;
    p->check = (flags & NTT_CHECK) != 0;
    p->tc_imma = (flags & NTT_TC_IMMA) != 0;
    p->q.assign(q, q + L);
    p->psi.resize(L);
    for (uint32_t l = 0; l < L; ++l) {
        if (psi) {
            if (psi[l] == 0 || psi[l] >= q[l] || H::powm(psi[l], N, q[l]) != q[l] - 1) { delete p; return NTT_ERR_PSI; }
            p->psi[l] = psi[l];
        } else {
            ntt_default_psi(q[l], N, &p->psi[l]);
        }
    }
    if (variant == NTT_FUSED) {
        int single_max = p->word64 ? nttgb::kSingleMaxLog64 : nttgb::kSingleMaxLog32;
        if (single_max_log >= 0 && single_max_log < single_max) single_max = single_max_log;
        if (p->logN < 4) p->fused_mode = nttgb::FUSED_STAGES;
        else if ((int)p->logN <= single_max) p->fused_mode = nttgb::FUSED_SINGLE;
        else if ((int)p->logN == nttgb::kClusterLogN && !p->word64 && single_max_log < 0 &&
                 (flags & NTT_CLUSTER))
            p->fused_mode = nttgb::FUSED_CLUSTER;
        else {
            p->fused_mode = nttgb::FUSED_TWO_PASS;
            p->streamed = (flags & NTT_STREAMED) != 0;
            p->tw_otf = (flags & NTT_TW_OTF) != 0;
            p->s2 = nttgb::kChunkLog;
            // streamed, on-the-fly-twiddle and ragged-kernel plans keep the
            // 256-word chunks; others may take a given or tuned split
            p->split_fixed = p->streamed || p->tw_otf || single_max_log >= 0;
            if (split_log >= 0) {
                if (p->split_fixed && (split_log != nttgb::kChunkLog || radix_log != 4)) {
                    delete p;
                    return NTT_ERR_UNSUPPORTED;
                }
                if (!nttgb::split_valid(p->logN, (uint32_t)split_log) || (radix_log != 3 && radix_log != 4)) {
                    delete p;
                    return NTT_ERR_UNSUPPORTED;
                }
                p->s2 = (uint32_t)split_log;
                p->lr = (uint32_t)radix_log;
                p->split_fixed = true;
            }
            p->s1 = p->logN - p->s2;
        }
    }
    nttgb::apply_tuning(*p);
    cudaGetDevice(&p->device);
    s = build_tables(p);
    if (s != NTT_OK) { free_plan_memory(p); delete p; cudaGetLastError(); return s; }
    *plan = p;
    return NTT_OK;
}

}  // namespace nttgb

extern "C" {

ntt_status ntt_plan_create_ex(ntt_plan_t *plan, uint32_t N, const uint64_t *q, uint32_t L, ntt_variant variant,
                              uint32_t flags, const uint64_t *psi) {
    return nttgb::create_plan(plan, N, q, L, variant, flags, psi, -1);
}

ntt_status ntt_plan_create(ntt_plan_t *plan, uint32_t N, const uint64_t *q, uint32_t L, ntt_variant variant,
                           uint32_t flags) {
    return ntt_plan_create_ex(plan, N, q, L, variant, flags, nullptr);
}

void ntt_plan_destroy(ntt_plan_t plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    free_plan_memory(plan);
    delete plan;
}

ntt_status ntt_plan_reserve(ntt_plan_t plan, uint32_t max_batch, ntt_stream_t stream) {
    if (!plan || max_batch == 0) return NTT_ERR_INVALID_ARG;
    if (!needs_scratch(*plan)) return NTT_OK;
    return nttgb::ensure_scratch(*plan, max_batch, reinterpret_cast<cudaStream_t>(stream));
}

ntt_status ntt_forward(ntt_plan_t plan, void *d_data, uint32_t batch, ntt_stream_t stream) {
    return run_transform(plan, d_data, batch, stream, false);
}

ntt_status ntt_inverse(ntt_plan_t plan, void *d_data, uint32_t batch, ntt_stream_t stream) {
    return run_transform(plan, d_data, batch, stream, true);
}

ntt_status ntt_forward_prefix(ntt_plan_t plan, void *d_data, uint32_t batch, uint32_t limbs, ntt_stream_t stream) {
    if (limbs == 0) return NTT_ERR_INVALID_ARG;
    return run_transform(plan, d_data, batch, stream, false, limbs);
}

ntt_status ntt_inverse_prefix(ntt_plan_t plan, void *d_data, uint32_t batch, uint32_t limbs, ntt_stream_t stream) {
    if (limbs == 0) return NTT_ERR_INVALID_ARG;
    return run_transform(plan, d_data, batch, stream, true, limbs);
}

ntt_status ntt_pointwise_mul(ntt_plan_t plan, void *d_c, const void *d_a, const void *d_b, uint32_t batch,
                             ntt_stream_t stream) {
    if (!plan || !d_c || !d_a || !d_b || batch == 0) return NTT_ERR_INVALID_ARG;
    if (!aligned16(d_c) || !aligned16(d_a) || !aligned16(d_b)) return NTT_ERR_ALIGNMENT;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    plan->last_launches = 0;
    cudaError_t e = cudaSuccess;
    if (plan->check) {
        e = nttgb::launch_check_range(*plan, d_a, batch, st);
        if (e == cudaSuccess) e = nttgb::launch_check_range(*plan, d_b, batch, st);
    }
    if (e == cudaSuccess) e = nttgb::launch_pointwise(*plan, d_c, d_a, d_b, batch, st);
    if (e != cudaSuccess) { cudaGetLastError(); return NTT_ERR_CUDA; }
    return NTT_OK;
}

ntt_status ntt_pointwise_inverse(ntt_plan_t plan, void *d_c, const void *d_a, const void *d_b, uint32_t batch,
                                 ntt_stream_t stream) {
    if (!plan || !d_c || !d_a || !d_b || batch == 0) return NTT_ERR_INVALID_ARG;
    if (!aligned16(d_c) || !aligned16(d_a) || !aligned16(d_b)) return NTT_ERR_ALIGNMENT;
    ntt_plan_s &p = *plan;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // one fused launch pair where the inverse starts with the chunk pass on
    // bit-reversed input; otherwise the product, then the inverse
    if (p.variant == NTT_FUSED && p.fused_mode == nttgb::FUSED_TWO_PASS && p.bitrev_order && !p.check) {
        p.last_launches = 0;   // (each pass counts itself)
        if (nttgb::launch_fused_pwinv(p, d_c, d_a, d_b, batch, st) != cudaSuccess) {
            cudaGetLastError();
            return NTT_ERR_CUDA;
        }
        return NTT_OK;
    }
    ntt_status s = ntt_pointwise_mul(plan, d_c, d_a, d_b, batch, stream);
    if (s != NTT_OK) return s;
    const uint32_t pw = p.last_launches;
    s = ntt_inverse(plan, d_c, batch, stream);
    p.last_launches += pw;
    return s;
}

ntt_status ntt_polymul_host(ntt_plan_t plan, void *h_out, const void *h_in, void *d_work, uint32_t pairs,
                            ntt_stream_t stream) {
    if (!plan || !h_out || !h_in || !d_work || pairs == 0) return NTT_ERR_INVALID_ARG;
    if (!aligned16(d_work)) return NTT_ERR_ALIGNMENT;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ntt_plan_s &p = *plan;
    // Chunks run as a three-stage pipeline: host-to-device copies on one
    // stream, the transforms on the caller's stream, device-to-host copies
    // on a third, chained by events, so the copies of one chunk overlap the
    // arithmetic of the others and each other.  A chunk is g whole pairs, or
    // -- fused plans with one or two pairs -- a window of lw limbs of one
    // pair (the limbs are independent), so that even one pair is pipelined.
    // Chunk (pair p0, limbs l0..) keeps its inputs at d_work + 2 (p0 L + l0) N
    // words as [a | b].
    if (!p.aux_ready) {
        if (cudaStreamCreateWithFlags(&p.aux_h2d, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&p.aux_d2h, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return NTT_ERR_CUDA;
        }
        for (cudaEvent_t &e : p.aux_ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); return NTT_ERR_CUDA; }
        p.aux_ready = true;
    }
    const uint32_t K = nttgb::kHostChunks, KMIN = nttgb::kHostMinChunks;
    const size_t limb = (size_t)p.N * p.word_bytes(), poly = (size_t)p.L * limb;
    const bool windows = pairs * 2 <= KMIN && p.L > 1 && p.variant == NTT_FUSED &&
                         (p.fused_mode == nttgb::FUSED_SINGLE || p.fused_mode == nttgb::FUSED_TWO_PASS);
    uint32_t g = 1, lw = p.L;
    if (windows) {
        const uint32_t per_pair = (KMIN / pairs < p.L) ? KMIN / pairs : p.L;   // windows per pair
        lw = (p.L + per_pair - 1) / per_pair;
    } else {
        g = (pairs + K - 1) / K;
    }
    const uint32_t wpp = (p.L + lw - 1) / lw;                 // windows per pair
    const uint32_t chunks = windows ? pairs * wpp : (pairs + g - 1) / g;
    const uint8_t *hi = reinterpret_cast<const uint8_t *>(h_in);
    uint8_t *ho = reinterpret_cast<uint8_t *>(h_out);
    uint8_t *d = reinterpret_cast<uint8_t *>(d_work);
    cudaEvent_t *ev = p.aux_ev;   // [0]: start, [1]: end, then per chunk (copied in, computed)
    bool ok = cudaEventRecord(ev[0], st) == cudaSuccess && cudaStreamWaitEvent(p.aux_h2d, ev[0], 0) == cudaSuccess &&
              cudaStreamWaitEvent(p.aux_d2h, ev[0], 0) == cudaSuccess;
    uint32_t launches = 0;
    ntt_status s = NTT_OK;
    for (uint32_t c = 0; c < chunks && ok && s == NTT_OK; ++c) {
        // pairs p0 .. p0 + gc - 1, limbs l0 .. l0 + lc - 1
        const uint32_t p0 = windows ? c / wpp : c * g;
        const uint32_t gc = windows ? 1 : (pairs - p0 < g ? pairs - p0 : g);
        const uint32_t l0 = windows ? (c % wpp) * lw : 0;
        const uint32_t lc = windows ? (p.L - l0 < lw ? p.L - l0 : lw) : p.L;
        const size_t part = (size_t)gc * lc * limb;           // one operand of the chunk
        uint8_t *dc = d + 2 * ((size_t)p0 * poly + (size_t)l0 * limb);
        cudaEvent_t e_in = ev[2 + 2 * c], e_done = ev[3 + 2 * c];
        ok = cudaMemcpyAsync(dc, hi + (size_t)p0 * poly + l0 * limb, part, cudaMemcpyHostToDevice, p.aux_h2d) ==
                 cudaSuccess &&
             cudaMemcpyAsync(dc + part, hi + ((size_t)pairs + p0) * poly + l0 * limb, part, cudaMemcpyHostToDevice,
                             p.aux_h2d) == cudaSuccess &&
             cudaEventRecord(e_in, p.aux_h2d) == cudaSuccess && cudaStreamWaitEvent(st, e_in, 0) == cudaSuccess;
        if (!ok) break;
        if (windows && lc != p.L) {
            // the limb window as a plan of its own: every table is per limb
            ntt_plan_s view = limb_window(p, l0, lc);
            s = ntt_forward(&view, dc, 2, stream);
            launches += view.last_launches;
            if (s == NTT_OK) { s = ntt_pointwise_inverse(&view, dc, dc, dc + part, 1, stream); launches += view.last_launches; }
            p.stream_seq = view.stream_seq;
        } else {
            s = ntt_forward(plan, dc, 2 * gc, stream);
            launches += p.last_launches;
            if (s == NTT_OK) { s = ntt_pointwise_inverse(plan, dc, dc, dc + part, gc, stream); launches += p.last_launches; }
        }
        if (s != NTT_OK) break;
        ok = cudaEventRecord(e_done, st) == cudaSuccess && cudaStreamWaitEvent(p.aux_d2h, e_done, 0) == cudaSuccess &&
             cudaMemcpyAsync(ho + (size_t)p0 * poly + l0 * limb, dc, part, cudaMemcpyDeviceToHost, p.aux_d2h) ==
                 cudaSuccess;
    }
    // the caller's stream resumes after the last copy out (also on an error,
    // so no work of this call outlives what the caller waits for)
    const bool joined = cudaEventRecord(ev[1], p.aux_d2h) == cudaSuccess && cudaStreamWaitEvent(st, ev[1], 0) == cudaSuccess;
    p.last_launches = launches;
    if (s != NTT_OK) return s;
    if (!ok || !joined) { cudaGetLastError(); return NTT_ERR_CUDA; }
    return NTT_OK;
}

ntt_status ntt_get_device_status(ntt_plan_t plan, ntt_stream_t stream) {
    if (!plan) return NTT_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) { cudaGetLastError(); return NTT_ERR_CUDA; }
    uint32_t v = 0;
    if (cudaMemcpy(&v, plan->d_status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return NTT_ERR_CUDA;
    if (v) cudaMemset(plan->d_status, 0, sizeof(uint32_t));
    if (v & 2u) return NTT_ERR_TIMEOUT;
    if (v & 1u) return NTT_ERR_INPUT_RANGE;
    return NTT_OK;
}

ntt_status ntt_plan_get_psi(ntt_plan_t plan, uint64_t *psi_out) {
    if (!plan || !psi_out) return NTT_ERR_INVALID_ARG;
    for (uint32_t l = 0; l < plan->L; ++l) psi_out[l] = plan->psi[l];
    return NTT_OK;
}

uint32_t ntt_plan_last_launches(ntt_plan_t plan) { return plan ? plan->last_launches : 0; }

uint64_t ntt_plan_table_bytes(ntt_plan_t plan) { return plan ? plan->table_bytes : 0; }

}  // extern "C"
