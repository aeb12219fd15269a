// host_nt.hpp -- host-side number theory for plan building.
//
// Primality: Miller-Rabin with the seven bases {2, 325, 9375, 28178, 450775,
// 9780504, 1795265022} (J. Sinclair's set), which decides every 64-bit n.
// Factoring q-1 (for the generator search): Pollard-Brent rho with the same
// primality test at the leaves.  A generator g has order q-1 iff
// g^((q-1)/p) != 1 for each prime p | q-1; psi = g^((q-1)/(2N)) with g the
// smallest generator (the root convention of the C ABI).
#pragma once
#include <algorithm>
#include <cstdint>
#include <vector>

namespace nttgb {
namespace host {

using u128 = unsigned __int128;

inline uint64_t mulm(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }

inline uint64_t powm(uint64_t b, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    b %= m;
    for (; e; e >>= 1) {
        if (e & 1) r = mulm(r, b, m);
        b = mulm(b, b, m);
    }
    return r;
}

inline uint64_t invm(uint64_t a, uint64_t p) { return powm(a, p - 2, p); }

inline bool is_prime(uint64_t n) {
    if (n < 2) return false;
    static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t p : small) {
        if (n == p) return true;
        if (n % p == 0) return false;
    }
    uint64_t d = n - 1;
    int s = __builtin_ctzll(d);
    d >>= s;
    static const uint64_t bases[] = {2, 325, 9375, 28178, 450775, 9780504, 1795265022};
    for (uint64_t a : bases) {
        uint64_t x = a % n;
        if (x == 0) continue;
        x = powm(x, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int r = 1; r < s && witness; ++r) {
            x = mulm(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

inline uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) { uint64_t t = a % b; a = b; b = t; }
    return a;
}

// One non-trivial factor of composite odd n (Pollard-Brent).
inline uint64_t rho(uint64_t n) {
    if (n % 2 == 0) return 2;
    for (uint64_t c = 1;; ++c) {
        uint64_t y = 2, x = 2, g = 1, q = 1, ys = 2;
        const uint64_t m = 64;
        uint64_t r = 1;
        auto f = [&](uint64_t v) { return (uint64_t)(((u128)v * v + c) % n); };
        do {
            x = y;
            for (uint64_t i = 0; i < r; ++i) y = f(y);
            uint64_t k = 0;
            do {
                ys = y;
                for (uint64_t i = 0; i < std::min(m, r - k); ++i) {
                    y = f(y);
                    q = mulm(q, x > y ? x - y : y - x, n);
                }
                g = gcd64(q, n);
                k += m;
            } while (k < r && g == 1);
            r <<= 1;
        } while (g == 1);
        if (g == n) {
            do {
                ys = f(ys);
                g = gcd64(x > ys ? x - ys : ys - x, n);
            } while (g == 1);
        }
        if (g != n) return g;
    }
}

inline void factor_into(uint64_t n, std::vector<uint64_t> &out) {
    if (n == 1) return;
    for (uint64_t p : {2ull, 3ull, 5ull, 7ull}) {
        if (n % p == 0) {
            out.push_back(p);
            while (n % p == 0) n /= p;
        }
    }
    if (n == 1) return;
    if (is_prime(n)) { out.push_back(n); return; }
    uint64_t d = rho(n);
    factor_into(d, out);
    factor_into(n / d, out);
}

inline std::vector<uint64_t> distinct_prime_factors(uint64_t n) {
    std::vector<uint64_t> f;
    factor_into(n, f);
    std::sort(f.begin(), f.end());
    f.erase(std::unique(f.begin(), f.end()), f.end());
    return f;
}

inline uint64_t smallest_generator(uint64_t q) {
    std::vector<uint64_t> f = distinct_prime_factors(q - 1);
    for (uint64_t g = 2; g < q; ++g) {
        bool ok = true;
        for (uint64_t p : f)
            if (powm(g, (q - 1) / p, q) == 1) { ok = false; break; }
        if (ok) return g;
    }
    return 0;
}

inline uint32_t bitrev(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i, x >>= 1) r = (r << 1) | (x & 1u);
    return r;
}

inline int bit_length(uint64_t x) { return x ? 64 - __builtin_clzll(x) : 0; }

// q^-1 mod 2^64 by Newton iteration (q odd): x <- x (2 - q x) doubles the
// number of correct low bits; x = q is correct to 3 bits.
inline uint64_t inv_pow2_64(uint64_t q) {
    uint64_t x = q;
    for (int i = 0; i < 6; ++i) x *= 2 - q * x;
    return x;
}

}  // namespace host
}  // namespace nttgb
