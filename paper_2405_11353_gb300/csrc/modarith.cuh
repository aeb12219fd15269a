// modarith.cuh -- modular arithmetic over Z_q on the integer pipes.
//
// Words are uint32_t (q < 2^30) or uint64_t (q < 2^60).  Three reductions for
// the twiddle product x * w mod q, selected per plan (Sec. III-C: modular
// reduction dominates the butterfly; Algorithm 4 is the one-compare add,
// Algorithm 5 the precomputed-quotient product after HEAX):
//
//   Shoup      w' = floor(w 2^W / q);  qh = hi(x w');  r = lo(x w) - lo(qh q)
//              (written lo(x w) + lo(qh (-q)): one multiply-add)
//              r in [0, 2q) for every x < 2^W (Algorithm 5 without its final
//              correction -- the lazy form).
//   Montgomery w_m = w R mod q, c = w_m q^-1 mod R (R = 2^W);  m = lo(x c);
//              t = hi(x w_m) - hi(m q) in (-q, q);  t + q in (0, 2q) and
//              t = x w (mod q) because lo(x w_m) = lo(m q) exactly.
//   Barrett    u32: z = x w (64 bits), qh = hi64(z mu), mu = floor(2^64 / q).
//              u64: z = x w (128 bits), qh = ((z >> (b-2)) mu) >> (b+5),
//              mu = floor(2^(2b+3) / q), b = bit length of q, x < 4q.
//              Both give qh in {floor(z/q) - 1, floor(z/q)}: r in [0, 2q).
//
// Butterflies keep values lazily reduced (Harvey): the forward (Cooley-Tukey,
// Eq. 4-5) one maps [0,4q)^2 -> [0,4q)^2, the inverse (Gentleman-Sande, Eq. 6)
// one maps [0,2q)^2 -> [0,2q)^2.  Outputs are brought to [0,q) once, at the
// end of a transform.  The one-compare corrections of Algorithm 4 are written
// branch-free as an unsigned minimum: min(x, x - c) is x - c when x >= c and
// x otherwise (the subtraction wraps to a large value).
#pragma once
#include <cstdint>

namespace nttgb {

enum Red : int { RED_SHOUP = 0, RED_BARRETT = 1, RED_MONTGOMERY = 2 };

// Per-limb constants, one record per RNS limb, in device memory.
struct LimbConst {
    uint64_t q;
    uint64_t two_q;
    uint64_t qinv;      // q^-1 mod 2^W (Montgomery)
    uint64_t r2;        // R^2 mod q, Montgomery form of R (to leave the domain)
    uint64_t r2c;       // r2 * qinv mod 2^W
    uint64_t mu;        // Barrett constant (see above)
    uint32_t bits;      // bit length of q
    uint32_t pad0;
    // N^-1 folded into the last inverse stage: twiddle pairs (value, companion)
    uint64_t ninv_w, ninv_c;          // N^-1
    uint64_t ninv_w1_w, ninv_w1_c;    // N^-1 * psi^-bitrev(1) (fused path)
};

// A twiddle and its companion (Shoup quotient or Montgomery q^-1 product).
template <class W> struct Tw { W w; W c; };

__device__ __forceinline__ uint32_t mulhi(uint32_t a, uint32_t b) { return __umulhi(a, b); }
__device__ __forceinline__ uint64_t mulhi(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

template <class W> __device__ __forceinline__ W umin(W a, W b) { return a < b ? a : b; }

// x - c if x >= c else x  (c <= 2^(W-1), x < 2c + c)
template <class W> __device__ __forceinline__ W csub(W x, W c) { return umin<W>(x, x - c); }

template <class W> struct Lc {
    W q, two_q, qinv, r2, r2c;
    W nq;               // -q mod 2^W: lo(x w) - lo(qh q) as one multiply-add
    uint64_t mu;
    uint32_t bits;
    __device__ __forceinline__ void load(const LimbConst *p) {
        q = (W)p->q; two_q = (W)p->two_q; qinv = (W)p->qinv;
        r2 = (W)p->r2; r2c = (W)p->r2c; mu = p->mu; bits = p->bits;
        nq = (W)0 - q;
    }
};

// ---------------------------------------------------------------- Barrett
__device__ __forceinline__ uint32_t barrett_lazy(uint64_t z, const Lc<uint32_t> &k) {
    // z < 2^64; qh in {floor(z/q)-1, floor(z/q)}
    uint64_t qh = __umul64hi(z, k.mu);
    return (uint32_t)z - (uint32_t)qh * k.q;
}

__device__ __forceinline__ uint64_t shr128(uint64_t lo, uint64_t hi, uint32_t s) {
    // (hi:lo) >> s for 0 < s < 128
    if (s >= 64) return hi >> (s - 64);
    return (lo >> s) | (hi << (64 - s));
}

__device__ __forceinline__ uint64_t barrett_lazy64(uint64_t zlo, uint64_t zhi, const Lc<uint64_t> &k) {
    // z < 4 q^2 < 2^(2b+2)
    uint64_t z1 = shr128(zlo, zhi, k.bits - 2);
    uint64_t plo = z1 * k.mu;
    uint64_t phi = __umul64hi(z1, k.mu);
    uint64_t qh = shr128(plo, phi, k.bits + 5);
    return zlo - qh * k.q;
}

// -------------------------------------------------- lazy twiddle product
// x * w mod q in [0, 2q).  Preconditions: x < 4q (Barrett); any x (others).
template <int RED> __device__ __forceinline__ uint32_t mul_lazy(uint32_t x, Tw<uint32_t> t, const Lc<uint32_t> &k) {
    if (RED == RED_SHOUP) {
        uint32_t qh = __umulhi(x, t.c);
        return x * t.w + qh * k.nq;
    } else if (RED == RED_MONTGOMERY) {
        uint32_t m = x * t.c;
        uint32_t t1 = __umulhi(x, t.w);
        uint32_t t2 = __umulhi(m, k.q);
        return t1 - t2 + k.q;
    } else {
        return barrett_lazy((uint64_t)x * t.w, k);
    }
}

template <int RED> __device__ __forceinline__ uint64_t mul_lazy(uint64_t x, Tw<uint64_t> t, const Lc<uint64_t> &k) {
    if (RED == RED_SHOUP) {
        uint64_t qh = __umul64hi(x, t.c);
        return x * t.w + qh * k.nq;
    } else if (RED == RED_MONTGOMERY) {
        uint64_t m = x * t.c;
        uint64_t t1 = __umul64hi(x, t.w);
        uint64_t t2 = __umul64hi(m, k.q);
        return t1 - t2 + k.q;
    } else {
        return barrett_lazy64(x * t.w, __umul64hi(x, t.w), k);
    }
}

// Fully reduced twiddle product, x < 4q.
template <int RED, class W> __device__ __forceinline__ W mul_full(W x, Tw<W> t, const Lc<W> &k) {
    return csub<W>(mul_lazy<RED>(x, t, k), k.q);
}

// a * b mod q for two variable operands in [0, q); result in [0, q).
// Barrett for Shoup/Barrett plans; Montgomery: REDC(a b) = a b R^-1, then a
// product with the constant R^2 (Montgomery form of R) restores a b.
template <int RED> __device__ __forceinline__ uint32_t mul_var(uint32_t a, uint32_t b, const Lc<uint32_t> &k) {
    if (RED == RED_MONTGOMERY) {
        uint32_t lo = a * b;
        uint32_t hi = __umulhi(a, b);
        uint32_t m = lo * k.qinv;
        uint32_t t = hi - __umulhi(m, k.q) + k.q;           // (0, 2q)
        Tw<uint32_t> r2{k.r2, k.r2c};
        return csub<uint32_t>(mul_lazy<RED_MONTGOMERY>(t, r2, k), k.q);
    } else {
        return csub<uint32_t>(barrett_lazy((uint64_t)a * b, k), k.q);
    }
}

template <int RED> __device__ __forceinline__ uint64_t mul_var(uint64_t a, uint64_t b, const Lc<uint64_t> &k) {
    if (RED == RED_MONTGOMERY) {
        uint64_t lo = a * b;
        uint64_t hi = __umul64hi(a, b);
        uint64_t m = lo * k.qinv;
        uint64_t t = hi - __umul64hi(m, k.q) + k.q;
        Tw<uint64_t> r2{k.r2, k.r2c};
        return csub<uint64_t>(mul_lazy<RED_MONTGOMERY>(t, r2, k), k.q);
    } else {
        return csub<uint64_t>(barrett_lazy64(a * b, __umul64hi(a, b), k), k.q);
    }
}

// ------------------------------------------------------------ butterflies
// Forward Cooley-Tukey (Eq. 4-5): (U, V) -> (U + wV, U - wV), [0,4q) lazy.
template <int RED, class W> __device__ __forceinline__ void ct_bfly(W &u, W &v, Tw<W> t, const Lc<W> &k) {
    W a = csub<W>(u, k.two_q);
    W b = mul_lazy<RED>(v, t, k);
    u = a + b;
    v = a - b + k.two_q;
}

// Inverse Gentleman-Sande (Eq. 6): (U, V) -> (U + V, (U - V) w), [0,2q) lazy.
template <int RED, class W> __device__ __forceinline__ void gs_bfly(W &u, W &v, Tw<W> t, const Lc<W> &k) {
    W s = u + v;
    W d = u - v + k.two_q;
    u = csub<W>(s, k.two_q);
    v = mul_lazy<RED>(d, t, k);
}

// Last inverse stage with N^-1 folded in: (U, V) -> ((U+V) N^-1, (U-V) w N^-1).
template <int RED, class W> __device__ __forceinline__ void gs_bfly_last(W &u, W &v, Tw<W> tn, Tw<W> twn, const Lc<W> &k) {
    W s = u + v;
    W d = u - v + k.two_q;
    u = mul_lazy<RED>(s, tn, k);
    v = mul_lazy<RED>(d, twn, k);
}

// Shoup quotient of a twiddle made on the device: floor(w 2^32 / q) for
// w < q < 2^30, from mu = floor(2^64 / q) = vh 2^32 + vl.  The Barrett
// estimate floor(w 2^32 mu / 2^64) = w vh + hi(w vl) is floor(w 2^32 / q)
// or one less (w 2^32 / 2^64 < 1/4); it is below 2^32, so it may be formed
// modulo 2^32, and so may the remainder w 2^32 - e q, which lies in
// [0, 2q): one comparison settles it.
__device__ __forceinline__ uint32_t shoup_quotient(uint32_t w, const Lc<uint32_t> &k) {
    const uint32_t vh = (uint32_t)(k.mu >> 32), vl = (uint32_t)k.mu;
    uint32_t e = w * vh + __umulhi(w, vl);
    const uint32_t r = 0u - e * k.q;
    return r >= k.q ? e + 1 : e;
}

// Fully reduced add / sub (Algorithm 4 with the >= reading), a, b in [0, q).
template <class W> __device__ __forceinline__ W add_mod(W a, W b, W q) { return csub<W>(a + b, q); }
template <class W> __device__ __forceinline__ W sub_mod(W a, W b, W q) { return csub<W>(a - b + q, q); }

template <class W> __device__ __forceinline__ Tw<W> ldtw(const Tw<W> *p) {
    Tw<W> t;
    if (sizeof(W) == 4) {
        uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        t.w = (W)v.x; t.c = (W)v.y;
    } else {
        ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
        t.w = (W)v.x; t.c = (W)v.y;
    }
    return t;
}

// ------------------------------------------------ fused-path table layout
// A sub-transform of 2^LOGS points uses the table entries 1 .. 2^LOGS - 1,
// entry 2^l + i for its stage l (l = 0 first in the forward order).  The
// fused kernels process the stages in rounds of LR (4, or 3) with a thread
// holding 2^LR words; in a full round starting at bit LO the thread tau
// needs, for stage l, 2^(l+LO+LR-LOGS) consecutive entries starting at
// 2^l + (tau >> LO) * count.  The table is stored "level-transposed" so
// that entry j of every thread of one stage are adjacent:
//   position(2^l + hi * count + j) = 2^l + j * (2^l / count) + hi.
// Stages of the short round (the top LOGS mod LR bits) keep their order.
inline uint32_t level_pos(uint32_t idx, uint32_t LOGS, uint32_t LR = 4) {
    if (idx == 0) return 0;
    uint32_t l = 0;
    while ((idx >> (l + 1)) != 0) ++l;
    const uint32_t b = LOGS - 1 - l;                 // the index bit this stage pairs
    const uint32_t full_top = (LOGS / LR) * LR;      // bits >= full_top: short round
    if (b >= full_top) return idx;
    const uint32_t LO = (b / LR) * LR, d = b - LO;
    const uint32_t cnt = 1u << (LR - 1 - d);
    const uint32_t ntau = (1u << l) / cnt;
    const uint32_t off = idx - (1u << l);
    return (1u << l) + (off % cnt) * ntau + off / cnt;
}

// Pairs per chunk table of a 2^LOGS-word chunk (2^LOGS entries + 64
// bytes, so the tables of neighbouring chunks of a tile fall on different
// bank halves in shared memory).
template <class W, int LOGS = 8> __host__ __device__ constexpr uint32_t chunk_tab_pitch() {
    return (1u << LOGS) + 64u / (2u * (uint32_t)sizeof(W));
}
inline uint32_t chunk_tab_pitch_rt(bool w64, uint32_t logs) { return (1u << logs) + (w64 ? 4u : 8u); }

}  // namespace nttgb
