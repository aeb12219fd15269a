"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Every comparison is exact: the transform over Z_q has a unique result for a
given (q, psi, order), so every variant and reduction must reproduce the
oracle word for word.  Inputs come from the seeded generators in ntt_synth;
expected values only from oracle/.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import ntt_synth  # noqa: E402
from parity_helpers import check_definition_samples  # noqa: E402


@pytest.fixture(scope="module")
def nt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2405_11353_gb300 as nt
    torch.cuda.init()
    return nt


ALL_VARIANTS = ["dit", "dif", "flat", "pease", "pease_nc", "stockham", "sixstep", "fused"]


def to_dev(host, w64):
    a = np.ascontiguousarray(host.astype(np.uint64 if w64 else np.uint32))
    return torch.from_numpy(a.view(np.int64 if w64 else np.int32).reshape(-1).copy()).cuda()


def to_host(t, w64, shape):
    a = t.cpu().numpy().view(np.uint64 if w64 else np.uint32)
    return a.reshape(shape).astype(np.uint64)


class Plan:
    def __init__(self, nt, N, qs, variant="fused", red="shoup", w64=False, bitrev=False, check=False,
                 extra_flags=0):
        self.nt = nt
        flags = nt.REDUCTIONS[red] | extra_flags
        if w64:
            flags |= nt.NTT_WORD64
        if bitrev:
            flags |= nt.NTT_ORDER_BITREV
        if check:
            flags |= nt.NTT_CHECK
        self.h = nt.ntt_plan_create(N, qs, nt.VARIANTS[variant], flags)
        self.N, self.L, self.w64, self.bitrev = N, len(qs), w64, bitrev

    def fwd(self, t, batch):
        self.nt.ntt_forward(self.h, t, batch)

    def inv(self, t, batch):
        self.nt.ntt_inverse(self.h, t, batch)

    def close(self):
        self.nt.ntt_plan_destroy(self.h)


def reorder(X, bitrev, orc):
    """Oracle output (natural order) in the plan's output order."""
    if not bitrev:
        return X
    B, L, N = X.shape
    return np.stack([np.stack([orc.bitrev_permute(X[b, l]) for l in range(L)]) for b in range(B)])


def primes_for(orc, N, w64, L):
    bits = 60 if w64 else 30
    m = max(18, N.bit_length())
    return orc.find_primes(bits, m, L)


def roundtrip_check(nt, orc, N, qs, batch, variant, red="shoup", w64=False, bitrev=False, seed=1,
                    naive=False, extra_flags=0):
    psis = [orc.psi(q, N) for q in qs]
    host = ntt_synth.rns_batch(seed, qs, N, batch)
    want = orc.ntt_batch(host, qs, psis, fast=not naive)
    p = Plan(nt, N, qs, variant, red, w64, bitrev, extra_flags=extra_flags)
    try:
        assert nt.ntt_plan_get_psi(p.h, len(qs)) == psis
        d = to_dev(host, w64)
        p.fwd(d, batch)
        got = to_host(d, w64, host.shape)
        assert np.array_equal(got, reorder(want, bitrev, orc)), (variant, red, N, w64, bitrev)
        p.inv(d, batch)
        back = to_host(d, w64, host.shape)
        assert np.array_equal(back, host), ("inverse", variant, red, N, w64, bitrev)
        assert nt.ntt_get_device_status(p.h) == nt.NTT_OK
    finally:
        p.close()


# ------------------------------------------------------------------ variants
@pytest.mark.parametrize("variant", ALL_VARIANTS)
@pytest.mark.parametrize("bitrev", [False, True])
def test_variants_all_sizes_u32(nt, orc, variant, bitrev):
    for n in range(1, 13):
        N = 1 << n
        qs = [12289] if N <= 2048 else []
        qs += primes_for(orc, N, False, 2)
        roundtrip_check(nt, orc, N, qs, 3, variant, bitrev=bitrev, seed=n, naive=N <= 256)


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_variants_large_u32(nt, orc, variant):
    for n in (13, 14, 15, 16, 17):
        N = 1 << n
        qs = primes_for(orc, N, False, 2)
        roundtrip_check(nt, orc, N, qs, 2, variant, seed=100 + n)


@pytest.mark.parametrize("variant", ["dit", "dif", "flat", "pease", "pease_nc", "stockham", "sixstep", "fused"])
def test_variants_u64(nt, orc, variant):
    for n in (1, 2, 5, 10, 12, 13, 14, 15, 16, 17):
        N = 1 << n
        qs = primes_for(orc, N, True, 2)
        roundtrip_check(nt, orc, N, qs, 2, variant, w64=True, seed=200 + n)


@pytest.mark.parametrize("red", ["shoup", "barrett", "montgomery"])
@pytest.mark.parametrize("w64", [False, True])
@pytest.mark.parametrize("variant", ["fused", "flat"])
def test_reductions(nt, orc, red, w64, variant):
    for n in (4, 10, 13, 14, 16, 17):
        N = 1 << n
        qs = primes_for(orc, N, w64, 3)
        roundtrip_check(nt, orc, N, qs, 2, variant, red=red, w64=w64, seed=300 + n,
                        bitrev=(n % 2 == 0))


# ------------------------------------------------------------ workloads
def polymul_pipeline(nt, orc, N, qs, pairs, variant, red="shoup", w64=False, bitrev=False, seed=1, samples=0):
    """forward (2*pairs polys) -> pointwise -> inverse; returns GPU and oracle.
    Every stage is compared in full with the O(N log N) oracle; with
    samples > 0, that many coefficients of every forward transform and of
    every inverse transform are also checked against the O(N^2) definition."""
    psis = [orc.psi(q, N) for q in qs]
    host = ntt_synth.rns_batch(seed, qs, N, 2 * pairs)
    p = Plan(nt, N, qs, variant, red, w64, bitrev)
    try:
        d = to_dev(host, w64)
        p.fwd(d, 2 * pairs)
        fwd = to_host(d, w64, host.shape)
        half = pairs * len(qs) * N
        nt.ntt_pointwise_mul(p.h, d, d, d[half:], pairs)
        prod = to_host(d[:half], w64, (pairs, len(qs), N))
        p.inv(d, pairs)
        out = to_host(d[:half], w64, (pairs, len(qs), N))
        assert nt.ntt_get_device_status(p.h) == nt.NTT_OK
    finally:
        p.close()
    A = orc.ntt_batch(host, qs, psis)
    assert np.array_equal(fwd, reorder(A, bitrev, orc))
    P = orc.pointwise_batch(A[:pairs], A[pairs:], qs)
    assert np.array_equal(prod, reorder(P, bitrev, orc))
    want = orc.ntt_batch(P, qs, psis, inverse=True)
    assert np.array_equal(out, want)
    if samples:
        check_definition_samples(orc, host, qs, psis, fwd, seed, samples, bitrev=bitrev)
        check_definition_samples(orc, P, qs, psis, out, seed + 1, samples, inverse=True)
    return host, out


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_workload_n1024_q12289_64polys(nt, orc, variant):
    """N = 1024, q = 12289, 64 polys: forward, 32 pointwise products,
    inverse; every output against the O(N^2) oracle and a few products
    against the schoolbook negacyclic product."""
    N, qs = 1024, [12289]
    psis = [orc.psi(12289, N)]
    host = ntt_synth.rns_batch(1001, qs, N, 64)
    want = orc.ntt_batch(host, qs, psis, fast=False)
    p = Plan(nt, N, qs, variant)
    try:
        d = to_dev(host, False)
        p.fwd(d, 64)
        assert np.array_equal(to_host(d, False, host.shape), want)
        half = 32 * N
        nt.ntt_pointwise_mul(p.h, d, d, d[half:], 32)
        p.inv(d, 32)
        out = to_host(d[:half], False, (32, 1, N))
    finally:
        p.close()
    P = orc.pointwise_batch(want[:32], want[32:], qs)
    assert np.array_equal(out, orc.ntt_batch(P, qs, psis, inverse=True, fast=False))
    for i in (0, 17, 31):
        assert np.array_equal(out[i, 0], orc.negacyclic_mul(host[i, 0], host[32 + i, 0], 12289))


@pytest.mark.parametrize("bitrev", [True, False])
def test_workload_n2p14_L8_128polys(nt, orc, bitrev):
    """N = 2^14, 8 30-bit primes, 128 polys: forward, 64 x 8 pointwise
    products, inverse; all in full against the O(N log N) oracle and 256
    coefficients of each of the 1024 forward and 512 inverse transforms
    against the O(N^2) definition."""
    qs = orc.find_primes(30, 15, 8)
    polymul_pipeline(nt, orc, 1 << 14, qs, 64, "fused", bitrev=bitrev, seed=1002, samples=256)


@pytest.mark.parametrize("red", ["montgomery", "shoup"])
def test_workload_n2p16_L24_u64(nt, orc, red):
    """N = 2^16, 24 60-bit primes, 8 polys: forward + inverse, full
    comparison with the O(N log N) oracle and 256 coefficients of each of
    the 192 forward transforms against the O(N^2) definition."""
    N = 1 << 16
    qs = orc.find_primes(60, 17, 24)
    psis = [orc.psi(q, N) for q in qs]
    host = ntt_synth.rns_batch(1003, qs, N, 8)
    p = Plan(nt, N, qs, "fused", red, w64=True, bitrev=True)
    try:
        d = to_dev(host, True)
        p.fwd(d, 8)
        got = to_host(d, True, host.shape)
        p.inv(d, 8)
        back = to_host(d, True, host.shape)
    finally:
        p.close()
    want = orc.ntt_batch(host, qs, psis)
    assert np.array_equal(got, reorder(want, True, orc))
    assert np.array_equal(back, host)
    assert check_definition_samples(orc, host, qs, psis, got, 1003, 256, bitrev=True) == 192 * 256


def test_workload_n2p16_L32_u32(nt, orc):
    """N = 2^16, 32 30-bit primes, 16 polys, butterfly form, as bench.py
    runs it: forward, 8 x 32 pointwise products, inverse; in full against
    the O(N log N) oracle and 256 coefficients of each of the 512 forward
    and 256 inverse transforms against the O(N^2) definition."""
    qs = orc.find_primes(30, 17, 32)
    host, out = polymul_pipeline(nt, orc, 1 << 16, qs, 8, "fused", bitrev=True, seed=1005, samples=256)
    # sampled coefficients of products against the schoolbook definition
    for i, l, j in [(0, 0, 0), (3, 5, 12345), (7, 31, (1 << 16) - 1), (5, 17, 40000)]:
        assert int(out[i, l, j]) == orc.negacyclic_mul_at(host[i, l], host[8 + i, l], qs[l], j)


# ----------------------------------------- N = 2^16: two-pass and cluster
@pytest.mark.parametrize("red", ["shoup", "barrett", "montgomery"])
@pytest.mark.parametrize("form", ["two_launch", "streamed", "cluster"])
def test_n2p16_u32_two_pass_and_cluster(nt, orc, red, form):
    """The fused forms of N = 2^16 with 4-byte words (the two-pass split as
    two launches or in one streamed launch; one pass on clusters of eight
    CTAs), both orders, batch sizes that give clusters one transform, none,
    or uneven ranges, and limb changes inside a cluster's range."""
    N = 1 << 16
    extra = {"two_launch": 0, "streamed": nt.NTT_STREAMED, "cluster": nt.NTT_CLUSTER}[form]
    qs = primes_for(orc, N, False, 10)
    for i, (batch, L, bitrev) in enumerate([(1, 1, True), (3, 5, False), (10, 10, True), (1, 7, True)]):
        roundtrip_check(nt, orc, N, qs[:L], batch, "fused", red=red, bitrev=bitrev, seed=1600 + i,
                        extra_flags=extra)


@pytest.mark.parametrize("tiles,lag", [("1", "1"), ("3", "1"), ("8", "2"), ("64", "1"), ("5", "40")])
def test_stream_form_item_sizes_and_lags(nt, orc, monkeypatch, tiles, lag):
    """The one-launch two-pass form under other work-item sizes and lags
    (the smallest lag makes second-pass items wait on first-pass items still
    in flight): forward, pointwise-fused inverse and their launch counts, for
    4- and 8-byte words and every column-pass size (N = 2^14 .. 2^17)."""
    monkeypatch.setenv("NTT_STREAM_TILES", tiles)
    monkeypatch.setenv("NTT_STREAM_LAG", lag)
    for n, w64, L, pairs in [(16, False, 6, 2), (15, False, 3, 1), (17, False, 2, 1), (14, True, 5, 2),
                             (16, True, 3, 1)]:
        N = 1 << n
        qs = primes_for(orc, N, w64, L)
        psis = [orc.psi(q, N) for q in qs]
        host = ntt_synth.rns_batch(1700 + n, qs, N, 2 * pairs)
        p = Plan(nt, N, qs, "fused", w64=w64, bitrev=True, extra_flags=nt.NTT_STREAMED)
        try:
            d = to_dev(host, w64)
            p.fwd(d, 2 * pairs)
            assert nt.ntt_plan_last_launches(p.h) == 1
            fwd = to_host(d, w64, host.shape)
            half = pairs * L * N
            c = torch.empty_like(d[:half])
            nt.ntt_pointwise_inverse(p.h, c, d[:half], d[half:], pairs)
            assert nt.ntt_plan_last_launches(p.h) == 1
            out = to_host(c, w64, (pairs, L, N))
            assert nt.ntt_get_device_status(p.h) == nt.NTT_OK
        finally:
            p.close()
        A = orc.ntt_batch(host, qs, psis)
        assert np.array_equal(fwd, reorder(A, True, orc)), (n, w64)
        P = orc.pointwise_batch(A[:pairs], A[pairs:], qs)
        assert np.array_equal(out, orc.ntt_batch(P, qs, psis, inverse=True)), (n, w64)


def test_stream_and_two_launch_forms_agree_on_the_workload_shape(nt, orc):
    """N = 2^16, 32 limbs, 16 polynomials: the streamed form (NTT_STREAMED)
    and the two launches give the same words, forward and inverse, over
    five calls in a row (the plan's counter sets are reused and reset by
    every call)."""
    N = 1 << 16
    qs = orc.find_primes(30, 17, 32)
    host = ntt_synth.rns_batch(1705, qs, N, 16)
    ps = Plan(nt, N, qs, "fused", bitrev=True, extra_flags=nt.NTT_STREAMED)
    p2 = Plan(nt, N, qs, "fused", bitrev=True)
    try:
        a, b = to_dev(host, False), to_dev(host, False)
        for _ in range(5):
            ps.fwd(a, 16)
            p2.fwd(b, 16)
            assert torch.equal(a, b)
            ps.inv(a, 16)
            p2.inv(b, 16)
            assert torch.equal(a, b)
        assert nt.ntt_plan_last_launches(p2.h) == 2
        assert np.array_equal(to_host(a, False, host.shape), host)
        assert nt.ntt_get_device_status(ps.h) == nt.NTT_OK
    finally:
        ps.close()
        p2.close()


def test_n2p16_u32_cluster_polymul_and_launches(nt, orc):
    """The cluster form through a forward / pointwise / inverse pipeline of
    the 32-limb workload shape (fewer polynomials), one launch per call."""
    N = 1 << 16
    qs = orc.find_primes(30, 17, 32)
    pairs = 2
    psis = [orc.psi(q, N) for q in qs]
    host = ntt_synth.rns_batch(1606, qs, N, 2 * pairs)
    p = Plan(nt, N, qs, "fused", bitrev=True, extra_flags=nt.NTT_CLUSTER)
    try:
        d = to_dev(host, False)
        p.fwd(d, 2 * pairs)
        assert nt.ntt_plan_last_launches(p.h) == 1
        fwd = to_host(d, False, host.shape)
        half = pairs * len(qs) * N
        nt.ntt_pointwise_mul(p.h, d, d, d[half:], pairs)
        p.inv(d, pairs)
        assert nt.ntt_plan_last_launches(p.h) == 1
        out = to_host(d[:half], False, (pairs, len(qs), N))
        assert nt.ntt_get_device_status(p.h) == nt.NTT_OK
    finally:
        p.close()
    A = orc.ntt_batch(host, qs, psis)
    assert np.array_equal(fwd, reorder(A, True, orc))
    P = orc.pointwise_batch(A[:pairs], A[pairs:], qs)
    assert np.array_equal(out, orc.ntt_batch(P, qs, psis, inverse=True))


# ------------------------------------------------------------- edge cases
def test_ragged_tail_tiles(nt, orc):
    # single-pass tiles hold 4 transforms at N = 1024: 5 limbs x 1 poly
    qs = primes_for(orc, 1024, False, 5)
    roundtrip_check(nt, orc, 1024, qs, 1, "fused", seed=7)
    roundtrip_check(nt, orc, 256, qs[:3], 1, "fused", seed=8)


def test_batch_one_and_max_size(nt, orc):
    for w64 in (False, True):
        qs = primes_for(orc, 1 << 17, w64, 1)
        roundtrip_check(nt, orc, 1 << 17, qs, 1, "fused", w64=w64, seed=9)


def test_check_flag_reports_out_of_range(nt, orc):
    N, qs = 1024, [12289]
    host = ntt_synth.rns_batch(5, qs, N, 2)
    p = Plan(nt, N, qs, "fused", check=True)
    try:
        d = to_dev(host, False)
        p.fwd(d, 2)
        assert nt.ntt_get_device_status(p.h) == nt.NTT_OK
        bad = host.copy()
        bad[1, 0, 77] = 12289
        d = to_dev(bad, False)
        p.fwd(d, 2)
        assert nt.ntt_get_device_status(p.h) == nt.NTT_ERR_INPUT_RANGE
        # the status is sticky until read, then cleared
        assert nt.ntt_get_device_status(p.h) == nt.NTT_OK
    finally:
        p.close()


def test_argument_errors(nt, orc):
    p = Plan(nt, 1024, [12289], "fused")
    try:
        d = torch.zeros(4 * 1024 + 4, dtype=torch.int32, device="cuda")
        with pytest.raises(nt.NttError) as e:
            nt.ntt_forward(p.h, d.data_ptr() + 4, 1)
        assert e.value.status == nt.NTT_ERR_ALIGNMENT
        with pytest.raises(nt.NttError) as e:
            nt.ntt_forward(p.h, d, 0)
        assert e.value.status == nt.NTT_ERR_INVALID_ARG
        with pytest.raises(nt.NttError) as e:
            nt.ntt_pointwise_mul(p.h, d, d.data_ptr() + 8, d, 1)
        assert e.value.status == nt.NTT_ERR_ALIGNMENT
    finally:
        p.close()


def test_pointwise_aliasing_and_reductions(nt, orc):
    N = 1 << 12
    for w64 in (False, True):
        qs = primes_for(orc, N, w64, 3)
        a = ntt_synth.rns_batch(11, qs, N, 2)
        b = ntt_synth.rns_batch(12, qs, N, 2)
        want = orc.pointwise_batch(a, b, qs)
        for red in ("shoup", "barrett", "montgomery"):
            p = Plan(nt, N, qs, "fused", red, w64)
            try:
                da, db = to_dev(a, w64), to_dev(b, w64)
                nt.ntt_pointwise_mul(p.h, db, da, db, 2)     # c aliases b
                assert np.array_equal(to_host(db, w64, a.shape), want), (red, w64)
            finally:
                p.close()


def test_pointwise_edge_values(nt, orc):
    """Products of q-1, q-2, 1, 0 and (q-1)/2 with each other, every reduction."""
    N = 1024
    for w64 in (False, True):
        qs = primes_for(orc, N, w64, 2)
        edge = lambda q: [0, 1, 2, q - 1, q - 2, (q - 1) // 2, (q + 1) // 2, q // 3]
        a = np.zeros((1, 2, N), np.uint64)
        b = np.zeros((1, 2, N), np.uint64)
        for l, q in enumerate(qs):
            e = edge(q)
            pairs = [(x, y) for x in e for y in e]
            for i, (x, y) in enumerate(pairs):
                a[0, l, i], b[0, l, i] = x, y
        want = orc.pointwise_batch(a, b, qs)
        for red in ("shoup", "barrett", "montgomery"):
            p = Plan(nt, N, qs, "fused", red, w64)
            try:
                da, db = to_dev(a, w64), to_dev(b, w64)
                nt.ntt_pointwise_mul(p.h, da, da, db, 1)
                assert np.array_equal(to_host(da, w64, a.shape), want), (red, w64)
            finally:
                p.close()


def test_extreme_inputs_all_q_minus_1(nt, orc):
    """Inputs at q-1 everywhere drive the lazy butterflies to their bounds."""
    for w64 in (False, True):
        N = 1 << 16
        qs = primes_for(orc, N, w64, 2)
        host = np.zeros((2, 2, N), np.uint64)
        for l, q in enumerate(qs):
            host[:, l, :] = q - 1
        psis = [orc.psi(q, N) for q in qs]
        want = orc.ntt_batch(host, qs, psis)
        for red in ("shoup", "barrett", "montgomery"):
            p = Plan(nt, N, qs, "fused", red, w64)
            try:
                d = to_dev(host, w64)
                p.fwd(d, 2)
                assert np.array_equal(to_host(d, w64, host.shape), want), (red, w64)
                p.inv(d, 2)
                assert np.array_equal(to_host(d, w64, host.shape), host), (red, w64)
            finally:
                p.close()


@pytest.mark.parametrize("red", ["shoup", "barrett", "montgomery"])
def test_pointwise_inverse_fused_and_fallback(nt, orc, red):
    """c = INTT(a (.) b) through the fused entry point: the two-pass sizes
    in bit-reversed order take the product inside the first inverse pass
    (u32 N = 2^15, 2^16, 2^17; u64 N = 2^16); N = 2^12, natural order and
    NTT_CHECK plans run the two steps.  c aliasing a, aliasing b, or apart."""
    # (log N, u64, bit-reversed, flags, launches: 2 fused (the two passes),
    # 1 with NTT_STREAMED; else the product (with NTT_CHECK: + a range check
    # of each operand), then the inverse (+ its range check, + the order
    # permutation, + its two launches))
    cases = [(15, False, True, 0, 2), (16, False, True, 0, 2), (17, False, True, 0, 2), (16, True, True, 0, 2),
             (16, False, True, nt.NTT_STREAMED, 1), (16, True, True, nt.NTT_STREAMED, 1),
             (12, False, True, 0, 2), (16, False, False, 0, 4), (16, False, True, nt.NTT_CHECK, 6)]
    for i, (n, w64, bitrev, extra, launches) in enumerate(cases):
        N, batch = 1 << n, 3
        qs = primes_for(orc, N, w64, 2)
        psis = [orc.psi(q, N) for q in qs]
        A = ntt_synth.rns_batch(1700 + i, qs, N, batch)
        Bm = ntt_synth.rns_batch(1750 + i, qs, N, batch)
        fa, fb = orc.ntt_batch(A, qs, psis), orc.ntt_batch(Bm, qs, psis)
        want = orc.ntt_batch(orc.pointwise_batch(fa, fb, qs), qs, psis, inverse=True)
        p = Plan(nt, N, qs, "fused", red=red, w64=w64, bitrev=bitrev, extra_flags=extra)
        try:
            for mode in ("c=a", "c=b", "apart"):
                da, db = to_dev(reorder(fa, bitrev, orc), w64), to_dev(reorder(fb, bitrev, orc), w64)
                dc = da if mode == "c=a" else db if mode == "c=b" else torch.zeros_like(da)
                nt.ntt_pointwise_inverse(p.h, dc, da, db, batch)
                assert np.array_equal(to_host(dc, w64, A.shape), want), (n, w64, bitrev, extra, mode)
                if mode == "apart":
                    assert np.array_equal(to_host(db, w64, A.shape), reorder(fb, bitrev, orc))
            assert nt.ntt_plan_last_launches(p.h) == launches
            assert nt.ntt_get_device_status(p.h) == nt.NTT_OK
        finally:
            p.close()


@pytest.mark.parametrize("red", ["shoup", "barrett", "montgomery"])
@pytest.mark.parametrize("w64", [False, True])
def test_paired_chunk_tiles(nt, orc, red, w64):
    """Chunk-pass tiles that pair polynomials (the same chunk of K
    polynomials, one twiddle table per tile) run when K divides the batch:
    K = 2 in the one-warp form, K = 16 in the 16-chunk form.  Batches 2, 16
    and 32 take them, 17 and 1 the unpaired tiles; every form of both
    directions, and the pointwise product fused into the paired inverse."""
    N = 1 << (15 if w64 else 16)
    qs = primes_for(orc, N, w64, 3)
    psis = [orc.psi(q, N) for q in qs]
    flags = nt.REDUCTIONS[red] | nt.NTT_ORDER_BITREV | (nt.NTT_WORD64 if w64 else 0)
    for i, batch in enumerate((2, 16, 17, 1, 32)):
        for form in ("small", "wide"):
            nt.ntt_tune_clear()
            nt.ntt_tune_set(N, len(qs), flags, batch, nt.FORMS[form], nt.FORMS[form])
            try:
                roundtrip_check(nt, orc, N, qs, batch, "fused", red=red, w64=w64, bitrev=True, seed=1900 + i)
            finally:
                nt.ntt_tune_clear()
    batch = 16
    A = ntt_synth.rns_batch(1950, qs, N, batch)
    Bm = ntt_synth.rns_batch(1951, qs, N, batch)
    fa, fb = orc.ntt_batch(A, qs, psis), orc.ntt_batch(Bm, qs, psis)
    want = orc.ntt_batch(orc.pointwise_batch(fa, fb, qs), qs, psis, inverse=True)
    p = Plan(nt, N, qs, "fused", red=red, w64=w64, bitrev=True)
    try:
        assert nt.ntt_plan_form(p.h, batch, True) == nt.NTT_FORM_WIDE
        da, db = to_dev(reorder(fa, True, orc), w64), to_dev(reorder(fb, True, orc), w64)
        dc = torch.zeros_like(da)
        nt.ntt_pointwise_inverse(p.h, dc, da, db, batch)
        assert np.array_equal(to_host(dc, w64, A.shape), want)
        assert nt.ntt_get_device_status(p.h) == nt.NTT_OK
    finally:
        p.close()


def test_paired_chunk_tiles_twiddles_on_the_fly(nt, orc):
    """The same pairing in the kernels that make the chunk twiddles from
    seeds (NTT_TW_OTF), both forms, batches that pair and that do not."""
    N = 1 << 16
    qs = primes_for(orc, N, False, 3)
    flags = nt.NTT_ORDER_BITREV | nt.NTT_TW_OTF
    for i, batch in enumerate((2, 16, 3)):
        for form in ("small", "wide"):
            nt.ntt_tune_clear()
            nt.ntt_tune_set(N, len(qs), flags, batch, nt.FORMS[form], nt.FORMS[form])
            try:
                roundtrip_check(nt, orc, N, qs, batch, "fused", bitrev=True, seed=1960 + i,
                                extra_flags=nt.NTT_TW_OTF)
            finally:
                nt.ntt_tune_clear()


def test_polymul_host_entry(nt, orc):
    """The host-buffer entry point: copies, transforms and products in one
    call, pipelined in chunks of pairs (1, 3 and 13 pairs: one chunk, chunks
    of one pair, chunks of two with a short last one); two calls back to back
    on one non-default stream, read after synchronising only that stream."""
    N = 2048
    qs = primes_for(orc, N, False, 2)
    p = Plan(nt, N, qs, "fused", bitrev=True)
    stream = torch.cuda.Stream()
    try:
        for pairs in (1, 3, 13):
            work = torch.empty(2 * pairs * 2 * N, dtype=torch.int32, device="cuda")
            runs = []
            for seed in (21, 22):
                host = ntt_synth.rns_batch(seed + 100 * pairs, qs, N, 2 * pairs).astype(np.uint32)
                h_in = torch.from_numpy(host.view(np.int32).copy()).pin_memory()
                h_out = torch.zeros(pairs * 2 * N, dtype=torch.int32).pin_memory()
                nt.ntt_polymul_host(p.h, h_out, h_in, work, pairs, stream.cuda_stream)
                runs.append((host, h_out))
            stream.synchronize()
            for host, h_out in runs:
                got = h_out.numpy().view(np.uint32).reshape(pairs, 2, N)
                for i in range(pairs):
                    for l in range(2):
                        assert np.array_equal(got[i, l].astype(np.uint64),
                                              orc.negacyclic_mul(host[i, l], host[pairs + i, l], qs[l]))
    finally:
        p.close()


def test_polymul_host_limb_windows(nt, orc):
    """One or two pairs are pipelined as windows of limbs (an uneven last
    window with 5 limbs), 3 or 9 pairs as chunks of whole pairs.  On a
    two-pass size in both orders and on a single-pass size; every product
    coefficient against the oracle's transform pipeline, a sample against
    the schoolbook product."""
    for n, L, bitrev in ((16, 5, True), (15, 5, False), (12, 3, True)):
        N = 1 << n
        qs = primes_for(orc, N, False, L)
        psis = [orc.psi(q, N) for q in qs]
        p = Plan(nt, N, qs, "fused", bitrev=bitrev)
        try:
            for pairs in (1, 2, 3, 9):
                host = ntt_synth.rns_batch(3000 + n + pairs, qs, N, 2 * pairs).astype(np.uint32)
                h_in = torch.from_numpy(host.view(np.int32).copy()).pin_memory()
                h_out = torch.zeros(pairs * L * N, dtype=torch.int32).pin_memory()
                work = torch.empty(2 * pairs * L * N, dtype=torch.int32, device="cuda")
                nt.ntt_polymul_host(p.h, h_out, h_in, work, pairs)
                torch.cuda.synchronize()
                got = h_out.numpy().view(np.uint32).reshape(pairs, L, N).astype(np.uint64)
                A = orc.ntt_batch(host, qs, psis)
                want = orc.ntt_batch(orc.pointwise_batch(A[:pairs], A[pairs:], qs), qs, psis, inverse=True)
                assert np.array_equal(got, want), (n, L, pairs)
                assert int(got[0, L - 1, N - 1]) == orc.negacyclic_mul_at(host[0, L - 1], host[pairs, L - 1],
                                                                        qs[L - 1], N - 1)
            assert nt.ntt_get_device_status(p.h) == nt.NTT_OK
        finally:
            p.close()


def test_dependent_launches_around_other_kernels(nt, orc):
    """The library's passes are dependent launches: each waits for the
    previous launch on the stream before it touches data.  Interleave them
    with PyTorch kernels on the same stream (which read their output and
    write their input) and with back-to-back calls on one buffer, for the
    two-pass, single-pass and per-stage (variant) paths."""
    for N, variant, L, batch in ((1 << 16, "fused", 3, 2), (1 << 12, "fused", 2, 3), (1 << 10, "stockham", 2, 2)):
        qs = primes_for(orc, N, False, L)
        psis = [orc.psi(q, N) for q in qs]
        host = ntt_synth.rns_batch(3100 + N.bit_length(), qs, N, batch)
        want = reorder(orc.ntt_batch(host, qs, psis), True, orc) if variant == "fused" else \
            orc.ntt_batch(host, qs, psis)
        p = Plan(nt, N, qs, variant, bitrev=(variant == "fused"))
        try:
            d = to_dev(host, False)
            for _ in range(3):
                p.fwd(d, batch)
                e = d.clone()                     # a PyTorch kernel reads the transform
                assert np.array_equal(to_host(e, False, host.shape), want)
                p.inv(e, batch)
                d.copy_(e)                        # ... and writes the next input
                p.fwd(d, batch)
                p.inv(d, batch)                   # back to back on one buffer
            assert np.array_equal(to_host(d, False, host.shape), host)
            assert nt.ntt_get_device_status(p.h) == nt.NTT_OK
        finally:
            p.close()


def test_two_streams(nt, orc):
    N = 1 << 14
    qs = primes_for(orc, N, False, 2)
    psis = [orc.psi(q, N) for q in qs]
    h1 = ntt_synth.rns_batch(31, qs, N, 4)
    h2 = ntt_synth.rns_batch(32, qs, N, 4)
    p1 = Plan(nt, N, qs, "fused")
    p2 = Plan(nt, N, qs, "stockham")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    try:
        d1, d2 = to_dev(h1, False), to_dev(h2, False)
        torch.cuda.synchronize()
        for _ in range(3):
            nt.ntt_forward(p1.h, d1, 4, s1)
            nt.ntt_forward(p2.h, d2, 4, s2)
            nt.ntt_inverse(p1.h, d1, 4, s1)
            nt.ntt_inverse(p2.h, d2, 4, s2)
        nt.ntt_forward(p1.h, d1, 4, s1)
        nt.ntt_forward(p2.h, d2, 4, s2)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(d1, False, h1.shape), orc.ntt_batch(h1, qs, psis))
        assert np.array_equal(to_host(d2, False, h2.shape), orc.ntt_batch(h2, qs, psis))
    finally:
        p1.close()
        p2.close()


@pytest.mark.parametrize("variant", ["fused", "stockham"])
def test_limb_prefix_entry_points(nt, orc, variant):
    """Polynomials of the plan's first 3 of 5 primes (an RNS level below the top)."""
    cases = [(12, False, 0), (16, False, 0), (14, True, 0)]
    if variant == "fused":
        cases.append((16, False, nt.NTT_CLUSTER))
    for n, w64, extra in cases:
        N = 1 << n
        qs = primes_for(orc, N, w64, 5)
        psis = [orc.psi(q, N) for q in qs[:3]]
        host = ntt_synth.rns_batch(41 + n, qs[:3], N, 2)
        p = Plan(nt, N, qs, variant, w64=w64, bitrev=True, extra_flags=extra)
        try:
            d = to_dev(host, w64)
            nt.ntt_forward_prefix(p.h, d, 2, 3)
            got = to_host(d, w64, host.shape)
            assert np.array_equal(got, reorder(orc.ntt_batch(host, qs[:3], psis), True, orc))
            nt.ntt_inverse_prefix(p.h, d, 2, 3)
            assert np.array_equal(to_host(d, w64, host.shape), host)
            with pytest.raises(nt.NttError):
                nt.ntt_forward_prefix(p.h, d, 2, 6)
        finally:
            p.close()


@pytest.mark.parametrize("form", ["two_launch", "streamed", "cluster"])
def test_bounded_wait_reports_timeout_and_context_survives(nt, orc, form):
    """Failure path on the GPU without a fault: with the test hook, one CTA's
    first tile waits for bytes that never arrive; its wait gives up after
    about a second, the call reports NTT_ERR_TIMEOUT, and the next plan on
    the same context works."""
    N = 1 << 16
    qs = primes_for(orc, N, False, 2)
    host = ntt_synth.rns_batch(61, qs, N, 2)
    extra = {"two_launch": 0, "streamed": nt.NTT_STREAMED, "cluster": nt.NTT_CLUSTER}[form]
    p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, nt.NTT_ORDER_BITREV | nt.NTT_TEST_STALL | extra)
    try:
        d = to_dev(host, False)
        nt.ntt_forward(p, d, 2)
        assert nt.ntt_get_device_status(p) == nt.NTT_ERR_TIMEOUT
    finally:
        nt.ntt_plan_destroy(p)
    roundtrip_check(nt, orc, N, qs, 2, "fused", bitrev=True, seed=62)
