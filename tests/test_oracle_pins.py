"""Pins for the CPU oracle: checks against facts fixed outside the oracle.

Nothing here compares the oracle with a retyped copy of itself.  The pins are
hand-worked examples (tests/golden), closed forms, algebraic invariants of
the negacyclic transform (convolution theorem against the schoolbook
product in Z_q[x]/(x^N+1), roundtrip, linearity, evaluation at the roots of
x^N+1), library routines (sympy primality, primitive roots, polynomial
evaluation) and brute force on tiny inputs.
"""
import os
import random

import numpy as np
import pytest

sympy = pytest.importorskip("sympy")

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows[key] = [int(v) for v in vals]
    return rows


# ------------------------------------------------------------ hand examples
def test_worked_example_q5_n2_all_inputs(orc):
    g = _read_golden("q5_n2.txt")
    q, N = g["q"][0], g["N"][0]
    assert orc.generator(q) == g["g"][0]
    psi = orc.psi(q, N)
    assert psi == g["psi"][0]
    for a0 in range(q):
        for a1 in range(q):
            X = orc.ntt_fwd([a0, a1], q, psi)
            for k in range(N):
                c0, c1 = g["X%d" % k]
                assert int(X[k]) == (c0 * a0 + c1 * a1) % q
            back = orc.ntt_inv(X, q, psi)
            assert list(back) == [a0, a1]


def test_worked_example_q17_n4(orc):
    g = _read_golden("q17_n4.txt")
    q, N = g["q"][0], g["N"][0]
    assert orc.generator(q) == g["g"][0]
    psi = orc.psi(q, N)
    assert psi == g["psi"][0]
    for k, r in enumerate(g["points"]):
        assert pow(psi, 2 * k + 1, q) == r
    for fast in (False, True):
        assert list(orc.ntt_fwd(g["a"], q, psi, fast)) == g["A"]
        assert list(orc.ntt_fwd(g["b"], q, psi, fast)) == g["B"]
        assert list(orc.ntt_fwd(g["c"], q, psi, fast)) == g["C"]
        assert list(orc.ntt_inv(g["A"], q, psi, fast)) == g["a"]
        assert list(orc.ntt_inv(g["C"], q, psi, fast)) == g["c"]
    assert list(orc.negacyclic_mul(g["a"], g["b"], q)) == g["c"]
    assert list(orc.pointwise(g["A"], g["B"], q)) == g["C"]


# ------------------------------------------------------------- number theory
STRONG_PSEUDOPRIMES = [
    2047, 1373653, 25326001, 3215031751, 2152302898747, 3474749660383,
    341550071728321, 3825123056546413051,
]
CARMICHAEL = [561, 1105, 1729, 2465, 2821, 6601, 8911, 41041, 825265]


def test_is_prime_against_sympy(orc):
    rng = random.Random(7)
    for n in list(range(0, 2000)) + STRONG_PSEUDOPRIMES + CARMICHAEL:
        assert orc.is_prime(n) == sympy.isprime(n), n
    for bits in (30, 31, 60, 62, 63, 64):
        for _ in range(300):
            n = rng.getrandbits(bits) | 1
            assert orc.is_prime(n) == sympy.isprime(n), n
    # Mersenne prime 2^61 - 1 and the largest 64-bit prime
    assert orc.is_prime((1 << 61) - 1)
    assert orc.is_prime(18446744073709551557)
    assert not orc.is_prime(18446744073709551615)


def test_generator_is_smallest_primitive_root(orc):
    for q in [5, 17, 97, 257, 7681, 12289, 65537, 786433]:
        assert orc.generator(q) == sympy.primitive_root(q), q
    for q in orc.find_primes(30, 17, 6) + orc.find_primes(60, 17, 4):
        assert orc.generator(q) == sympy.primitive_root(q), q


def test_prime_factors(orc):
    for n in [2, 12, 12288, 2 ** 17 * 3 * 7, 1 << 40, 999983 * 1000003]:
        assert sorted(orc.prime_factors(n)) == sorted(sympy.primefactors(n))


@pytest.mark.parametrize("bits,m,count", [(30, 15, 8), (30, 17, 32), (60, 17, 24),
                                          (30, 18, 32), (60, 18, 32)])
def test_find_primes_is_descending_list(orc, bits, m, count):
    got = orc.find_primes(bits, m, count)
    want = []
    k = 1
    while len(want) < count:
        q = (1 << bits) - k * (1 << m) + 1
        assert q > (1 << (bits - 1))
        if sympy.isprime(q):
            want.append(q)
        k += 1
    assert got == want
    for q in got:
        assert (q - 1) % (1 << m) == 0
        assert (1 << (bits - 1)) < q < (1 << bits)


@pytest.mark.parametrize("q,N", [(12289, 1024), (12289, 2048), (17, 8), (7681, 256)])
def test_psi_primitive_2n_root(orc, q, N):
    psi = orc.psi(q, N)
    assert pow(psi, 2 * N, q) == 1
    assert pow(psi, N, q) == q - 1
    # order exactly 2N: psi^(2N/p) != 1 for p = 2 (the only prime factor)
    assert pow(psi, N, q) != 1


def test_psi_config_primes(orc):
    for bits, m, cnt, N in [(30, 15, 8, 1 << 14), (60, 17, 24, 1 << 16),
                            (30, 17, 32, 1 << 16), (30, 18, 8, 1 << 17),
                            (60, 18, 8, 1 << 17)]:
        for q in orc.find_primes(bits, m, cnt):
            psi = orc.psi(q, N)
            assert pow(psi, 2 * N, q) == 1 and pow(psi, N, q) == q - 1
            # psi for a smaller N is the matching power of the larger one
            assert orc.psi(q, N // 2) == pow(psi, 2, q)


def test_psi_rejects_non_friendly(orc):
    assert orc.psi(12289, 1 << 13) == 0      # 2^14 does not divide 12288
    assert orc.psi(17, 16) == 0


# --------------------------------------------------------------- closed forms
@pytest.mark.parametrize("q,N", [(12289, 1024), (17, 4), (7681, 64)])
def test_delta_closed_forms(orc, q, N):
    psi = orc.psi(q, N)
    d0 = np.zeros(N, np.uint64)
    d0[0] = 1
    assert np.all(orc.ntt_fwd(d0, q, psi, fast=True) == 1)
    for j in (1, 2, N - 1):
        dj = np.zeros(N, np.uint64)
        dj[j] = 1
        X = orc.ntt_fwd(dj, q, psi, fast=True)
        assert [int(v) for v in X] == [pow(psi, (2 * k + 1) * j, q) for k in range(N)]
        # the inverse of those values is the delta again
        assert np.array_equal(orc.ntt_inv(X, q, psi), dj)
    c = np.zeros(N, np.uint64)
    c[0] = 1234 % q
    assert np.all(orc.ntt_fwd(c, q, psi) == 1234 % q)


def test_negacyclic_coefficient_matches_full_product(orc):
    rng = random.Random(4)
    for q, N in [(17, 4), (12289, 64), (1152921504606830593, 32)]:
        a, b = _rand(rng, q, N), _rand(rng, q, N)
        c = orc.negacyclic_mul(a, b, q)
        for j in range(N):
            assert orc.negacyclic_mul_at(a, b, q, j) == int(c[j])
    g = _read_golden("q17_n4.txt")
    assert [orc.negacyclic_mul_at(g["a"], g["b"], 17, j) for j in range(4)] == g["c"]


def test_negacyclic_wrap(orc):
    q, N = 12289, 16
    a = np.zeros(N, np.uint64)
    b = np.zeros(N, np.uint64)
    a[N - 1] = 1
    b[1] = 1
    c = orc.negacyclic_mul(a, b, q)
    assert int(c[0]) == q - 1 and np.all(c[1:] == 0)
    # x^i * x^j lands on x^(i+j) with sign (-1)^floor((i+j)/N)
    for i, j in [(3, 5), (10, 9), (15, 15)]:
        a = np.zeros(N, np.uint64)
        b = np.zeros(N, np.uint64)
        a[i] = 2
        b[j] = 3
        c = orc.negacyclic_mul(a, b, q)
        s = i + j
        want = np.zeros(N, np.uint64)
        want[s % N] = 6 if s < N else q - 6
        assert np.array_equal(c, want)


# ------------------------------------------------------------------ invariants
def _rand(rng, q, N):
    return np.array([rng.randrange(q) for _ in range(N)], dtype=np.uint64)


@pytest.mark.parametrize("q,N", [(12289, 64), (7681, 128), (17, 8),
                                 (1152921504606830593, 32), (1073479681, 256)])
def test_convolution_theorem(orc, q, N):
    if orc.psi(q, N) == 0:
        pytest.skip("q not NTT-friendly for N")
    psi = orc.psi(q, N)
    rng = random.Random(q ^ N)
    for _ in range(3):
        a, b = _rand(rng, q, N), _rand(rng, q, N)
        c = orc.negacyclic_mul(a, b, q)
        for fast in (False, True):
            A = orc.ntt_fwd(a, q, psi, fast)
            B = orc.ntt_fwd(b, q, psi, fast)
            assert np.array_equal(orc.ntt_inv(orc.pointwise(A, B, q), q, psi, fast), c)


@pytest.mark.parametrize("fast", [False, True])
def test_roundtrip_and_linearity(orc, fast):
    rng = random.Random(3)
    for q, N in [(12289, 1024), (1073479681, 512), (1152921504606830593, 256)]:
        psi = orc.psi(q, N)
        assert psi
        a, b = _rand(rng, q, N), _rand(rng, q, N)
        s = rng.randrange(q)
        A = orc.ntt_fwd(a, q, psi, fast)
        B = orc.ntt_fwd(b, q, psi, fast)
        assert np.array_equal(orc.ntt_inv(A, q, psi, fast), a)
        lin = np.array([(s * int(x) + int(y)) % q for x, y in zip(a, b)], np.uint64)
        want = np.array([(s * int(x) + int(y)) % q for x, y in zip(A, B)], np.uint64)
        assert np.array_equal(orc.ntt_fwd(lin, q, psi, fast), want)


def test_evaluation_at_roots_with_sympy(orc):
    """X[k] is a(x) evaluated at psi^(2k+1), the N distinct roots of x^N+1."""
    x = sympy.symbols("x")
    rng = random.Random(11)
    for q, N in [(12289, 32), (1073479681, 16), (1152921504606830593, 8)]:
        psi = orc.psi(q, N)
        a = _rand(rng, q, N)
        X = orc.ntt_fwd(a, q, psi)
        poly = sympy.Poly([int(v) for v in a[::-1]], x)
        pts = [pow(psi, 2 * k + 1, q) for k in range(N)]
        assert len(set(pts)) == N
        for k, r in enumerate(pts):
            assert pow(r, N, q) == q - 1
            assert int(X[k]) == int(poly.eval(r)) % q


def test_fast_equals_naive(orc):
    rng = random.Random(5)
    cases = [(12289, 1 << n) for n in range(1, 12)]
    cases += [(q, 1 << n) for q in orc.find_primes(30, 15, 2) for n in (5, 9, 12)]
    cases += [(q, 1 << n) for q in orc.find_primes(60, 17, 2) for n in (4, 10, 12)]
    for q, N in cases:
        psi = orc.psi(q, N)
        a = _rand(rng, q, N)
        A = orc.ntt_fwd(a, q, psi, fast=False)
        assert np.array_equal(orc.ntt_fwd(a, q, psi, fast=True), A), (q, N)
        assert np.array_equal(orc.ntt_inv(A, q, psi, fast=True), a), (q, N)


def test_point_evaluation_matches_full(orc):
    rng = random.Random(9)
    q, N = 1073479681, 128
    psi = orc.psi(q, N)
    a = _rand(rng, q, N)
    A = orc.ntt_fwd(a, q, psi)
    for k in (0, 1, 77, N - 1):
        assert orc.ntt_fwd_at(a, q, psi, k) == int(A[k])
        assert orc.ntt_inv_at(A, q, psi, k) == int(a[k])


def test_bitrev_permutation(orc):
    assert list(orc.bitrev_permute(np.arange(8, dtype=np.uint64))) == [0, 4, 2, 6, 1, 5, 3, 7]
    x = np.arange(1024, dtype=np.uint64)
    assert np.array_equal(orc.bitrev_permute(orc.bitrev_permute(x)), x)


def test_modular_ops_brute_force(orc):
    q = 12289
    rng = random.Random(1)
    for _ in range(2000):
        a, b = rng.randrange(q), rng.randrange(q)
        assert orc.mulmod(a, b, q) == a * b % q
    Q = 1152921504606830593
    for _ in range(2000):
        a, b = rng.randrange(Q), rng.randrange(Q)
        assert orc.mulmod(a, b, Q) == a * b % Q
        assert orc.lib().orc_submod(a, b, Q) == (a - b) % Q
        assert orc.lib().orc_addmod(a, b, Q) == (a + b) % Q


def test_batch_wrappers(orc):
    import ntt_synth
    qs = orc.find_primes(30, 15, 3)
    N = 256
    psis = [orc.psi(q, N) for q in qs]
    data = ntt_synth.rns_batch(42, qs, N, 4)
    out = orc.ntt_batch(data, qs, psis)
    naive = orc.ntt_batch(data, qs, psis, fast=False)
    assert np.array_equal(out, naive)
    for p in range(4):
        for l in range(3):
            assert np.array_equal(out[p, l], orc.ntt_fwd(data[p, l], qs[l], psis[l]))
    back = orc.ntt_batch(out, qs, psis, inverse=True)
    assert np.array_equal(back, data)
    t, k = ntt_synth.sample_indices(1, 12, N, 50)
    got = orc.ntt_batch_at(data, qs, psis, t, k)
    assert np.array_equal(got, out.reshape(12, N)[t.astype(int), k.astype(int)])


def test_pointwise_batch_limb_by_limb(orc):
    """orc_pointwise_batch on [batch][L][N] arrays at odd L and batch: every
    (polynomial, limb) block equals orc_pointwise with that limb's prime
    (itself pinned by the q = 17 worked example below), so a wrong limb
    index (t % L) or a wrong block stride fails.  The primes differ in
    every limb, and one block is also checked against Python integers."""
    import ntt_synth
    g = _read_golden("q17_n4.txt")
    assert orc.pointwise(g["A"], g["B"], 17).tolist() == g["C"]
    for B, L, N, bits in ((3, 5, 16, 30), (5, 3, 64, 60), (1, 7, 8, 30), (7, 1, 32, 60)):
        qs = orc.find_primes(bits, 8, L)
        assert len(set(qs)) == L
        a = ntt_synth.rns_batch(71 + B, qs, N, B)
        b = ntt_synth.rns_batch(97 + B, qs, N, B)
        c = orc.pointwise_batch(a, b, qs)
        assert c.shape == (B, L, N)
        for p in range(B):
            for l in range(L):
                assert np.array_equal(c[p, l], orc.pointwise(a[p, l], b[p, l], qs[l])), (B, L, p, l)
        p, l = B - 1, L - 1
        assert [int(v) for v in c[p, l]] == [int(x) * int(y) % qs[l] for x, y in zip(a[p, l], b[p, l])]
    # a limb index taken from the wrong prime would change these: the same
    # residues multiplied under two different primes give different products
    qs = orc.find_primes(30, 8, 2)
    a = np.full((1, 2, 4), (1 << 29) + 12345, dtype=np.uint64)
    c = orc.pointwise_batch(a, a, qs)
    assert [int(c[0, l, 0]) for l in range(2)] == [((1 << 29) + 12345) ** 2 % q for q in qs]
    assert int(c[0, 0, 0]) != int(c[0, 1, 0])


def test_synth_residues_in_range():
    import ntt_synth
    for q in (12289, (1 << 30) - 35, 1152921504606830593):
        v = ntt_synth.uniform_residues(123, q, 10000)
        assert v.size == 10000 and int(v.max()) < q
        # the stream is deterministic
        assert np.array_equal(v, ntt_synth.uniform_residues(123, q, 10000))
    # SplitMix64 reference outputs for seed 0 (first three values of the
    # published generator seeded with 0)
    first = [int(v) for v in ntt_synth.splitmix64(0, 3)]
    assert first == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


# ------------------------------------------------------ RNS base conversion
def test_base_conv_worked_example(orc):
    g = _read_golden("bconv_q5_7_p11_13.txt")
    qs, ps = g.pop("q"), g.pop("p")
    for key, (x0, x1, y0, y1, v, z0, z1) in g.items():
        x = np.array([[[x0], [x1]]], dtype=np.uint64)
        assert orc.base_conv(x, qs, ps)[0, :, 0].tolist() == [z0, z1], key


def _crt_check(orc, qs, ps, X):
    """z_j = (X + alpha Q) mod p_j for one alpha in [0, L) (the approximate
    fast conversion), X given by its residues."""
    Q = 1
    for q in qs:
        Q *= q
    x = np.array([[[X % q] for q in qs]], dtype=np.uint64)
    z = [int(v) for v in orc.base_conv(x, qs, ps)[0, :, 0]]
    # residues reassembled by the library CRT give X back
    assert int(sympy.ntheory.modular.crt(qs, [int(v) for v in x[0, :, 0]])[0]) == X
    # alpha from the first target prime, then checked on every one
    alpha = (z[0] - X) * pow(Q, -1, ps[0]) % ps[0]
    assert 0 <= alpha < len(qs)
    assert z == [(X + alpha * Q) % p for p in ps]
    return alpha


def test_base_conv_is_x_plus_small_multiple_of_Q(orc):
    rng = random.Random(11)
    qs = orc.find_primes(30, 17, 6)
    ps = orc.find_primes(31, 17, 5)
    Q = 1
    for q in qs:
        Q *= q
    alphas = set()
    for X in [0, 1, 2, Q - 1, Q // 2] + [rng.randrange(Q) for _ in range(200)]:
        alphas.add(_crt_check(orc, qs, ps, X))
    assert len(alphas) > 1          # the multiple of Q really varies


def test_base_conv_special_cases(orc):
    rng = random.Random(12)
    qs = orc.find_primes(30, 17, 4)
    ps = orc.find_primes(31, 17, 3)
    x = np.array([[[rng.randrange(q) for _ in range(64)] for q in qs]], dtype=np.uint64)
    # one source prime: qhat = 1, the conversion is plain reduction
    z1 = orc.base_conv(x[:, :1], qs[:1], ps)
    assert np.array_equal(z1[0], np.stack([x[0, 0] % p for p in ps]))
    # a target prime of the source basis returns that limb (Q = 0 mod q_i)
    z = orc.base_conv(x, qs, [qs[2], ps[0], qs[0]])
    assert np.array_equal(z[0, 0], x[0, 2]) and np.array_equal(z[0, 2], x[0, 0])
    # zero maps to zero; batches convert independently
    assert not orc.base_conv(np.zeros((2, 4, 8), np.uint64), qs, ps).any()
    xb = np.concatenate([x, x[:, :, ::-1].copy()])
    zb = orc.base_conv(xb, qs, ps)
    assert np.array_equal(zb[1], orc.base_conv(x[:, :, ::-1].copy(), qs, ps)[0])


def test_chunk_twiddle_factorization(orc):
    """The identity the on-the-fly chunk twiddles rest on: for the two-pass
    split N = N1 x 256, entry 2^s + i of chunk r, psi^bitrev_n(2^s (N1 + r) + i),
    equals A_s(r) B_s(i) with A_s(r) = psi^(2^(7-s) (1 + 2 bitrev(r))) and
    B_s(i) = psi^(2^(n-s) bitrev_s(i)).  Checked over every (r, s, i) for
    N = 2^13 and, for a sample of chunks, N = 2^17."""
    def brv(x, b):
        return int(format(x, "0%db" % b)[::-1], 2) if b else 0

    for n, chunks in ((13, range(32)), (17, (0, 1, 77, 300, 511))):
        N, s1 = 1 << n, n - 8
        q = orc.find_primes(30, 18, 1)[0]
        psi = orc.psi(q, N)
        for r in chunks:
            for s in range(8):
                a = orc.powmod(psi, (1 << (7 - s)) * (1 + 2 * brv(r, s1)), q)
                for i in range(1 << s):
                    b = orc.powmod(psi, (1 << (n - s)) * brv(i, s), q)
                    want = orc.powmod(psi, brv((1 << s) * ((1 << s1) + r) + i, n), q)
                    assert orc.mulmod(a, b, q) == want, (n, r, s, i)
