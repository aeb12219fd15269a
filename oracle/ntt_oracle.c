/*
 * ntt_oracle.c -- CPU oracle for the batched negacyclic NTT.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  The CUDA
 * product path never includes, links or calls anything in this directory, and
 * this file includes nothing from the product.
 *
 * Everything here is written for clarity, not speed: every modular product is
 * a 128-bit multiply followed by the C `%` operator, every sum is reduced with
 * `%`, and no lazy reduction, Shoup/Barrett/Montgomery trick, tiling or
 * reordering is used.
 *
 * Paper: "NTTSuite: Number Theoretic Transform Benchmarks for Accelerating
 * Encrypted Computation" (arXiv 2405.11353).
 *   - Eq. 1-3 (Sec. II, "Twiddle Factors"): X[k] = sum_{n<N} x[n] W_N^{kn},
 *     W_N = g^{(P-1)/N}.  The paper states the cyclic transform only; the
 *     negacyclic (x^N + 1) form used here twists by psi, a primitive 2N-th
 *     root with psi^2 = W_N:  X[k] = sum_n a[n] psi^{(2k+1) n}.
 *   - Eq. 4 and Algorithm 1 (Sec. II, "Decimation in Time"): the iterative
 *     radix-2 DIT that the O(N log N) path below follows, with the index
 *     typos read as stated in the comments of orc_ntt_fwd_fast.
 *   - Sec. I: the NTT reduces a polynomial product to a pointwise product.
 *   - orc_base_conv: the fast RNS base conversion that follows the inverse
 *     transform in the homomorphic schemes Sec. I motivates; the paper does
 *     not define it, the definition is stated above the function.
 *
 * Conventions (readings of points the paper leaves open):
 *   - generator g of Z_q^* = the smallest integer >= 2 of multiplicative
 *     order q-1; psi = g^{(q-1)/(2N)} mod q.
 *   - forward output in natural order k = 0..N-1; the inverse maps it back.
 *   - primes of a given width: q = 2^b - k 2^m + 1 for k = 1, 2, ... keeping
 *     the primes with 2^(b-1) < q < 2^b, in that (descending) order.
 *
 * Parity status: every function below is pinned by the "not gpu" tests in
 * tests/test_oracle_pins.py (closed forms, invariants, brute force on tiny
 * inputs, library primality / primitive-root routines, hand-derived values).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- Z_q ops */

uint64_t orc_mulmod(uint64_t a, uint64_t b, uint64_t q)
{
    return (uint64_t)(((u128)a * (u128)b) % (u128)q);
}

uint64_t orc_addmod(uint64_t a, uint64_t b, uint64_t q)
{
    return (uint64_t)(((u128)a + (u128)b) % (u128)q);
}

uint64_t orc_submod(uint64_t a, uint64_t b, uint64_t q)
{
    /* a, b < q: a + (q - b) < 2q, computed in 128 bits to stay exact. */
    return (uint64_t)(((u128)a + (u128)(q - (b % q))) % (u128)q);
}

uint64_t orc_powmod(uint64_t base, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    uint64_t b = base % q;
    while (e) {
        if (e & 1u) r = orc_mulmod(r, b, q);
        b = orc_mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}

/* Inverse by Fermat's little theorem (q prime). */
uint64_t orc_invmod(uint64_t a, uint64_t q)
{
    return orc_powmod(a, q - 2, q);
}

/* ------------------------------------------------------- number theory */

/* Deterministic Miller-Rabin: the first twelve primes as bases decide
 * primality exactly for every n < 3.3e24, hence for all 64-bit n. */
int orc_is_prime(uint64_t n)
{
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; ++i) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1u) == 0) { d >>= 1; ++s; }
    for (int i = 0; i < 12; ++i) {
        uint64_t x = orc_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; ++r) {
            x = orc_mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* Distinct prime factors of n by trial division; returns their count. */
int orc_prime_factors(uint64_t n, uint64_t *out, int cap)
{
    int cnt = 0;
    if (n % 2 == 0) {
        if (cnt < cap) out[cnt] = 2;
        ++cnt;
        while (n % 2 == 0) n /= 2;
    }
    for (uint64_t d = 3; d <= n / d; d += 2) {
        if (n % d == 0) {
            if (cnt < cap) out[cnt] = d;
            ++cnt;
            while (n % d == 0) n /= d;
        }
    }
    if (n > 1) {
        if (cnt < cap) out[cnt] = n;
        ++cnt;
    }
    return cnt;
}

/* Smallest generator of Z_q^* (q prime): g has order q-1 iff
 * g^((q-1)/p) != 1 for every prime p dividing q-1. */
uint64_t orc_generator(uint64_t q)
{
    uint64_t f[64];
    int nf = orc_prime_factors(q - 1, f, 64);
    for (uint64_t g = 2; g < q; ++g) {
        int ok = 1;
        for (int i = 0; i < nf; ++i) {
            if (orc_powmod(g, (q - 1) / f[i], q) == 1) { ok = 0; break; }
        }
        if (ok) return g;
    }
    return 0;
}

/* psi = g^((q-1)/(2N)); 0 if 2N does not divide q-1. */
uint64_t orc_psi(uint64_t q, uint64_t N)
{
    if (N == 0 || (q - 1) % (2 * N) != 0) return 0;
    return orc_powmod(orc_generator(q), (q - 1) / (2 * N), q);
}

/* The first `count` primes q = 2^bits - k 2^m + 1 (k = 1, 2, ...) with
 * 2^(bits-1) < q < 2^bits.  Returns how many were found. */
int orc_find_primes(int bits, int m, int count, uint64_t *out)
{
    int found = 0;
    uint64_t top = (uint64_t)1 << bits;
    uint64_t low = (uint64_t)1 << (bits - 1);
    uint64_t step = (uint64_t)1 << m;
    for (uint64_t k = 1; found < count; ++k) {
        if (k * step >= top) break;
        uint64_t q = top - k * step + 1;
        if (q <= low) break;
        if (orc_is_prime(q)) out[found++] = q;
    }
    return found;
}

/* ------------------------------------------------- definitional O(N^2) */

/* One Horner step acc * x + c, reduced once: acc, x < q < 2^62 and
 * c < 2^64, so the 128-bit sum is exact before the `%`. */
static uint64_t horner_step(uint64_t acc, uint64_t x, uint64_t c, uint64_t q)
{
    return (uint64_t)(((u128)acc * (u128)x + (u128)c) % (u128)q);
}

/* X[k] = sum_{n<N} a[n] psi^{(2k+1) n}: the polynomial a evaluated at the
 * root psi^(2k+1) of x^N + 1, by Horner's rule. */
uint64_t orc_ntt_fwd_at(uint64_t q, uint64_t psi, uint64_t N,
                        const uint64_t *a, uint64_t k)
{
    uint64_t x = orc_powmod(psi, 2 * k + 1, q);
    uint64_t acc = 0;
    for (uint64_t n = N; n-- > 0;)
        acc = horner_step(acc, x, a[n], q);
    return acc;
}

/* a[n] = N^-1 psi^-n sum_{k<N} X[k] psi^{-2nk}. */
uint64_t orc_ntt_inv_at(uint64_t q, uint64_t psi, uint64_t N,
                        const uint64_t *X, uint64_t n)
{
    uint64_t psi_inv = orc_invmod(psi, q);
    uint64_t y = orc_powmod(psi_inv, 2 * n, q);
    uint64_t acc = 0;
    for (uint64_t k = N; k-- > 0;)
        acc = horner_step(acc, y, X[k], q);
    acc = orc_mulmod(acc, orc_powmod(psi_inv, n, q), q);
    return orc_mulmod(acc, orc_invmod(N % q, q), q);
}

void orc_ntt_fwd_naive(uint64_t q, uint64_t psi, uint64_t N,
                       const uint64_t *a, uint64_t *X)
{
    for (uint64_t k = 0; k < N; ++k) X[k] = orc_ntt_fwd_at(q, psi, N, a, k);
}

void orc_ntt_inv_naive(uint64_t q, uint64_t psi, uint64_t N,
                       const uint64_t *X, uint64_t *a)
{
    for (uint64_t n = 0; n < N; ++n) a[n] = orc_ntt_inv_at(q, psi, N, X, n);
}

/* c = a * b mod (x^N + 1, q): schoolbook, with x^N = -1. */
void orc_negacyclic_mul(uint64_t q, uint64_t N, const uint64_t *a,
                        const uint64_t *b, uint64_t *c)
{
    for (uint64_t i = 0; i < N; ++i) c[i] = 0;
    for (uint64_t i = 0; i < N; ++i) {
        for (uint64_t j = 0; j < N; ++j) {
            uint64_t p = orc_mulmod(a[i], b[j], q);
            if (i + j < N)
                c[i + j] = orc_addmod(c[i + j], p, q);
            else
                c[i + j - N] = orc_submod(c[i + j - N], p, q);
        }
    }
}

/* Coefficient j of a * b mod (x^N + 1, q):
 * sum_{i<=j} a[i] b[j-i] - sum_{i>j} a[i] b[N+j-i]. */
uint64_t orc_negacyclic_mul_at(uint64_t q, uint64_t N, const uint64_t *a,
                               const uint64_t *b, uint64_t j)
{
    uint64_t acc = 0;
    for (uint64_t i = 0; i < N; ++i) {
        if (i <= j)
            acc = orc_addmod(acc, orc_mulmod(a[i], b[j - i], q), q);
        else
            acc = orc_submod(acc, orc_mulmod(a[i], b[N + j - i], q), q);
    }
    return acc;
}

/* c[k] = a[k] b[k] mod q. */
void orc_pointwise(uint64_t q, uint64_t n, const uint64_t *a,
                   const uint64_t *b, uint64_t *c)
{
    for (uint64_t k = 0; k < n; ++k) c[k] = orc_mulmod(a[k], b[k], q);
}

/* ------------------------------------------------ textbook O(N log N) */

static uint64_t bitrev(uint64_t x, int bits)
{
    uint64_t r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

static int log2u(uint64_t N)
{
    int L = 0;
    while (((uint64_t)1 << L) < N) ++L;
    return L;
}

/* Out-of-place reorder: out[i] = in[brv(i)] (an involution). */
void orc_bitrev_permute(uint64_t N, const uint64_t *in, uint64_t *out)
{
    int L = log2u(N);
    for (uint64_t i = 0; i < N; ++i) out[i] = in[bitrev(i, L)];
}

/* Cyclic N-point transform with root w, following Algorithm 1: reorder
 * the input by bit reversal, then for stages s = 1..L with m = 2^s, for each
 * k < m/2 take tw = W[(N/m) k] = w^{k N/m} and for j = 0, m, 2m, ... apply
 * the butterfly f1 = x[j+k], f2 = tw x[j+k+m/2], x[j+k] = f1 + f2,
 * x[j+k+m/2] = f1 - f2.  (The printed listing writes the stage size as
 * 1 << i and runs k to n-1; the butterfly recurrence of Eq. 4 needs
 * m = 2^s and k < m/2, which is what is used.) */
static void cyclic_dit(uint64_t q, uint64_t w, uint64_t N, uint64_t *x)
{
    int L = log2u(N);
    uint64_t *W = (uint64_t *)malloc(sizeof(uint64_t) * (N / 2 + 1));
    uint64_t *t = (uint64_t *)malloc(sizeof(uint64_t) * N);
    W[0] = 1;
    for (uint64_t i = 1; i <= N / 2; ++i) W[i] = orc_mulmod(W[i - 1], w, q);
    orc_bitrev_permute(N, x, t);
    memcpy(x, t, sizeof(uint64_t) * N);
    for (int s = 1; s <= L; ++s) {
        uint64_t m = (uint64_t)1 << s;
        for (uint64_t k = 0; k < m / 2; ++k) {
            uint64_t tw = W[(N / m) * k];
            for (uint64_t j = 0; j < N; j += m) {
                uint64_t f1 = x[j + k];
                uint64_t f2 = orc_mulmod(tw, x[j + k + m / 2], q);
                x[j + k] = orc_addmod(f1, f2, q);
                x[j + k + m / 2] = orc_submod(f1, f2, q);
            }
        }
    }
    free(W);
    free(t);
}

/* Negacyclic forward: twist a[n] psi^n, then the cyclic DIT with w = psi^2. */
void orc_ntt_fwd_fast(uint64_t q, uint64_t psi, uint64_t N,
                      const uint64_t *a, uint64_t *X)
{
    uint64_t p = 1;
    for (uint64_t n = 0; n < N; ++n) {
        X[n] = orc_mulmod(a[n] % q, p, q);
        p = orc_mulmod(p, psi, q);
    }
    cyclic_dit(q, orc_mulmod(psi, psi, q), N, X);
}

/* Negacyclic inverse: cyclic DIT with w = psi^-2, then scale by
 * N^-1 psi^-n. */
void orc_ntt_inv_fast(uint64_t q, uint64_t psi, uint64_t N,
                      const uint64_t *X, uint64_t *a)
{
    uint64_t psi_inv = orc_invmod(psi, q);
    uint64_t n_inv = orc_invmod(N % q, q);
    for (uint64_t k = 0; k < N; ++k) a[k] = X[k] % q;
    cyclic_dit(q, orc_mulmod(psi_inv, psi_inv, q), N, a);
    uint64_t p = n_inv;
    for (uint64_t n = 0; n < N; ++n) {
        a[n] = orc_mulmod(a[n], p, q);
        p = orc_mulmod(p, psi_inv, q);
    }
}

/* ----------------------------------------------------- batched wrappers */

/* data layout [batch][L][N]; limb l uses q[l], psi[l].  dir 0 = forward,
 * 1 = inverse.  fast != 0 selects the O(N log N) path, else O(N^2).
 * Independent transforms run in parallel (OpenMP) when compiled with it. */
void orc_ntt_batch(int dir, int fast, uint64_t N, uint32_t L, uint32_t batch,
                   const uint64_t *q, const uint64_t *psi,
                   const uint64_t *in, uint64_t *out)
{
    long total = (long)batch * (long)L;
#pragma omp parallel for schedule(dynamic, 1)
    for (long t = 0; t < total; ++t) {
        uint32_t l = (uint32_t)(t % L);
        const uint64_t *src = in + (size_t)t * N;
        uint64_t *dst = out + (size_t)t * N;
        if (dir == 0) {
            if (fast) orc_ntt_fwd_fast(q[l], psi[l], N, src, dst);
            else orc_ntt_fwd_naive(q[l], psi[l], N, src, dst);
        } else {
            if (fast) orc_ntt_inv_fast(q[l], psi[l], N, src, dst);
            else orc_ntt_inv_naive(q[l], psi[l], N, src, dst);
        }
    }
}

/* Sampled check support: out[i] = X[k_i] (dir 0) or a[n_i] (dir 1) of
 * transform t_i of a [batch][L][N] array. */
void orc_ntt_batch_at(int dir, uint64_t N, uint32_t L, const uint64_t *q,
                      const uint64_t *psi, const uint64_t *in, uint64_t count,
                      const uint64_t *t_idx, const uint64_t *k_idx,
                      uint64_t *out)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)count; ++i) {
        uint64_t t = t_idx[i];
        uint32_t l = (uint32_t)(t % L);
        const uint64_t *src = in + (size_t)t * N;
        out[i] = dir == 0 ? orc_ntt_fwd_at(q[l], psi[l], N, src, k_idx[i])
                          : orc_ntt_inv_at(q[l], psi[l], N, src, k_idx[i]);
    }
}

/* Pointwise product of [batch][L][N] arrays, limb l modulo q[l]. */
void orc_pointwise_batch(uint64_t N, uint32_t L, uint32_t batch,
                         const uint64_t *q, const uint64_t *a,
                         const uint64_t *b, uint64_t *c)
{
    long total = (long)batch * (long)L;
#pragma omp parallel for schedule(static)
    for (long t = 0; t < total; ++t) {
        uint32_t l = (uint32_t)(t % L);
        orc_pointwise(q[l], N, a + (size_t)t * N, b + (size_t)t * N,
                      c + (size_t)t * N);
    }
}

/* ------------------------------------------------- RNS base conversion */
/*
 * Fast base conversion of RNS residues (the basis-extension step that
 * follows the inverse transform in RNS homomorphic schemes, the setting
 * Sec. I motivates the NTT with; the paper itself defines no conversion).
 * For a coefficient with residues x_i = x mod q_i (i < L), Q = prod_i q_i
 * and qhat_i = Q / q_i:
 *     y_i = x_i * qhat_i^{-1} mod q_i
 *     z_j = ( sum_i y_i * qhat_i ) mod p_j            (j < K)
 * with the sum taken exactly; written out here as
 *     z_j = sum_i y_i * (qhat_i mod p_j)   mod p_j.
 * The exact sum v = sum_i y_i qhat_i satisfies v = x (mod Q) and
 * 0 <= v < L Q, so z_j = (x + alpha Q) mod p_j for one integer
 * 0 <= alpha < L (the conversion is approximate by that multiple of Q).
 * x: [batch][L][N], z: [batch][K][N]; the q_i pairwise coprime.
 */

/* qhat_i mod m = prod_{k != i} q_k mod m */
static uint64_t qhat_mod(uint32_t L, const uint64_t *q, uint32_t i, uint64_t m)
{
    uint64_t r = 1 % m;
    for (uint32_t k = 0; k < L; ++k)
        if (k != i) r = orc_mulmod(r, q[k] % m, m);
    return r;
}

void orc_base_conv(uint32_t L, const uint64_t *q, uint32_t K, const uint64_t *p,
                   uint64_t N, uint32_t batch, const uint64_t *x, uint64_t *z)
{
    uint64_t *qinv = (uint64_t *)malloc(sizeof(uint64_t) * L);
    uint64_t *qm = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)L * K);
    for (uint32_t i = 0; i < L; ++i) {
        qinv[i] = orc_invmod(qhat_mod(L, q, i, q[i]), q[i]);
        for (uint32_t j = 0; j < K; ++j) qm[(size_t)i * K + j] = qhat_mod(L, q, i, p[j]);
    }
    long total = (long)batch * (long)N;
#pragma omp parallel for schedule(static)
    for (long t = 0; t < total; ++t) {
        const uint64_t b = (uint64_t)t / N, n = (uint64_t)t % N;
        for (uint32_t j = 0; j < K; ++j) {
            uint64_t acc = 0;
            for (uint32_t i = 0; i < L; ++i) {
                const uint64_t xi = x[(b * L + i) * N + n];
                const uint64_t yi = orc_mulmod(xi, qinv[i], q[i]);
                acc = orc_addmod(acc, orc_mulmod(yi % p[j], qm[(size_t)i * K + j], p[j]), p[j]);
            }
            z[(b * K + j) * N + n] = acc;
        }
    }
    free(qinv);
    free(qm);
}

/* Threads an OpenMP region would use (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
