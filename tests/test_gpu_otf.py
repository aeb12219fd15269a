"""Chunk-pass twiddles made on the fly (NTT_TW_OTF) against the CPU oracle.

The second pass of a two-pass plan stages each chunk's table as
A_s(r) * B_s(i) (eight seeds per chunk, one 255-entry root table per limb)
with a Shoup quotient computed on the device, instead of reading the
per-chunk tables.  The transform does not change, so every output must equal
the oracle's word for word, in both chunk-pass forms and both directions.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import ntt_synth  # noqa: E402


@pytest.fixture(scope="module")
def nt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2405_11353_gb300 as nt
    torch.cuda.init()
    return nt


def to_dev(host):
    return torch.from_numpy(np.ascontiguousarray(host.astype(np.uint32)).view(np.int32).reshape(-1).copy()).cuda()


def to_host(t, shape):
    return t.cpu().numpy().view(np.uint32).reshape(shape).astype(np.uint64)


def reorder(X, bitrev, orc):
    if not bitrev:
        return X
    return np.stack([np.stack([orc.bitrev_permute(x) for x in row]) for row in X])


@pytest.mark.parametrize("fwd_form,inv_form", [(0, 1), (1, 0)])
def test_otf_matches_oracle_every_two_pass_size(nt, orc, fwd_form, inv_form):
    """N = 2^15, 2^16, 2^17 (column passes of 128, 256, 512 points), odd
    limb counts and batches, both orders, both chunk-pass forms per
    direction (set through the tuning table): forward against the oracle,
    inverse back to the input, and the product fused into the inverse."""
    try:
        for i, (n, L, pairs, bitrev) in enumerate([(15, 3, 1, True), (16, 5, 2, False), (17, 2, 1, True),
                                                    (16, 1, 3, True)]):
            N = 1 << n
            qs = orc.find_primes(30, 18, L)
            psis = [orc.psi(q, N) for q in qs]
            flags = nt.NTT_TW_OTF | (nt.NTT_ORDER_BITREV if bitrev else 0)
            for b in (pairs, 2 * pairs):
                nt.ntt_tune_set(N, L, flags, b, fwd_form, inv_form)
            host = ntt_synth.rns_batch(2100 + i, qs, N, 2 * pairs)
            p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, flags)
            try:
                assert nt.ntt_plan_form(p, 2 * pairs) == fwd_form
                assert nt.ntt_plan_form(p, pairs, True) == inv_form
                d = to_dev(host)
                nt.ntt_forward(p, d, 2 * pairs)
                fwd = to_host(d, host.shape)
                half = pairs * L * N
                c = torch.empty_like(d[:half])
                nt.ntt_pointwise_inverse(p, c, d[:half], d[half:], pairs)
                prod_inv = to_host(c, (pairs, L, N))
                nt.ntt_inverse(p, d, 2 * pairs)
                back = to_host(d, host.shape)
                assert nt.ntt_get_device_status(p) == nt.NTT_OK
            finally:
                nt.ntt_plan_destroy(p)
            A = orc.ntt_batch(host, qs, psis)
            assert np.array_equal(fwd, reorder(A, bitrev, orc)), (n, L)
            assert np.array_equal(back, host), (n, L)
            if bitrev:
                P = orc.pointwise_batch(A[:pairs], A[pairs:], qs)
                assert np.array_equal(prod_inv, orc.ntt_batch(P, qs, psis, inverse=True)), (n, L)
    finally:
        nt.ntt_tune_clear()


def test_otf_and_table_plans_agree_on_the_workload_shape(nt, orc):
    """N = 2^16, 32 limbs, 16 polynomials (the benchmark's shape): the plan
    that makes its chunk twiddles and the one that reads them give the same
    words forward, for the fused product + inverse, and back; a sample of
    outputs against the oracle's O(N) evaluation."""
    N = 1 << 16
    qs = orc.find_primes(30, 17, 32)
    host = ntt_synth.rns_batch(2110, qs, N, 16)
    pa = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, nt.NTT_ORDER_BITREV | nt.NTT_TW_OTF)
    pb = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, nt.NTT_ORDER_BITREV)
    try:
        a, b = to_dev(host), to_dev(host)
        nt.ntt_forward(pa, a, 16)
        nt.ntt_forward(pb, b, 16)
        assert torch.equal(a, b)
        half = 8 * 32 * N
        ca, cb = torch.empty_like(a[:half]), torch.empty_like(b[:half])
        nt.ntt_pointwise_inverse(pa, ca, a[:half], a[half:], 8)
        nt.ntt_pointwise_inverse(pb, cb, b[:half], b[half:], 8)
        assert torch.equal(ca, cb)
        fwd = to_host(a, host.shape)
        nt.ntt_inverse(pa, a, 16)
        assert np.array_equal(to_host(a, host.shape), host)
        assert nt.ntt_get_device_status(pa) == nt.NTT_OK
    finally:
        nt.ntt_plan_destroy(pa)
        nt.ntt_plan_destroy(pb)
    for poly, l, pos in [(0, 0, 0), (3, 31, 1), (15, 17, 65535), (9, 4, 40001)]:
        k = int(format(pos, "016b")[::-1], 2)     # bit-reversed output order
        assert int(fwd[poly, l, pos]) == orc.ntt_fwd_at(host[poly, l], qs[l], orc.psi(qs[l], N), k)


def test_otf_extreme_inputs_and_prefix(nt, orc):
    """All words q - 1 (the largest lazy intermediates) and the limb-prefix
    entry points on an OTF plan."""
    N, L = 1 << 16, 4
    qs = orc.find_primes(30, 17, L)
    psis = [orc.psi(q, N) for q in qs]
    host = np.stack([np.stack([np.full(N, q - 1, dtype=np.uint64) for q in qs])] * 2)
    p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, nt.NTT_TW_OTF)
    try:
        d = to_dev(host)
        nt.ntt_forward(p, d, 2)
        assert np.array_equal(to_host(d, host.shape), orc.ntt_batch(host, qs, psis))
        nt.ntt_inverse(p, d, 2)
        assert np.array_equal(to_host(d, host.shape), host)
        # the first two limbs only, as a batch of two-limb polynomials
        h2 = ntt_synth.rns_batch(2120, qs[:2], N, 3)
        d2 = to_dev(h2)
        nt.ntt_forward_prefix(p, d2, 3, 2)
        assert np.array_equal(to_host(d2, h2.shape), orc.ntt_batch(h2, qs[:2], psis[:2]))
        assert nt.ntt_get_device_status(p) == nt.NTT_OK
    finally:
        nt.ntt_plan_destroy(p)


def test_otf_single_pass_sizes_unchanged_and_autotune(nt, orc):
    """Below the two-pass range the flag changes nothing; the autotuner
    times no streamed form for OTF plans (-1) and never picks it."""
    N = 1 << 12
    qs = orc.find_primes(30, 17, 3)
    psis = [orc.psi(q, N) for q in qs]
    host = ntt_synth.rns_batch(2130, qs, N, 2)
    p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, nt.NTT_TW_OTF)
    try:
        d = to_dev(host)
        nt.ntt_forward(p, d, 2)
        assert np.array_equal(to_host(d, host.shape), orc.ntt_batch(host, qs, psis))
        assert nt.ntt_plan_form(p, 2) == -1
    finally:
        nt.ntt_plan_destroy(p)
    try:
        r = nt.ntt_autotune(1 << 15, orc.find_primes(30, 17, 4), nt.NTT_TW_OTF, 4)
        assert r["forward_ms"][2] == -1 and r["inverse_ms"][2] == -1
        assert r["forward_ms"][0] > 0 and r["forward_ms"][1] > 0
        assert r["forward_form"] in (0, 1) and r["inverse_form"] in (0, 1)
        assert nt.ntt_tune_get(1 << 15, 4, nt.NTT_TW_OTF, 4) == r["forward_form"]
    finally:
        nt.ntt_tune_clear()


def test_otf_table_bytes(nt, orc):
    """The chunk tables (N1 chunks x 264 pairs of 4-byte words per limb and
    direction) give way to 8 seeds per chunk and 256 root pairs per limb."""
    N, L = 1 << 16, 32
    qs = orc.find_primes(30, 17, L)
    pa = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, nt.NTT_TW_OTF)
    pb = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, 0)
    try:
        N1 = N >> 8
        chunk = 2 * L * N1 * 264 * 8
        seeds = 2 * L * (N1 * 8 * 4 + 256 * 8)
        assert nt.ntt_plan_table_bytes(pb) - nt.ntt_plan_table_bytes(pa) == chunk - seeds
        assert nt.ntt_plan_table_bytes(pb) > chunk
    finally:
        nt.ntt_plan_destroy(pa)
        nt.ntt_plan_destroy(pb)


def test_otf_with_range_check_and_natural_order(nt, orc):
    """NTT_TW_OTF with NTT_CHECK (the product then runs apart from the
    inverse) and in natural order (a permutation around the passes): the
    product of two polynomials against the oracle's pipeline, and a word
    >= q reported."""
    N, L = 1 << 15, 2
    qs = orc.find_primes(30, 17, L)
    psis = [orc.psi(q, N) for q in qs]
    host = ntt_synth.rns_batch(2140, qs, N, 2)
    for flags in (nt.NTT_TW_OTF | nt.NTT_CHECK | nt.NTT_ORDER_BITREV, nt.NTT_TW_OTF):
        p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, flags)
        try:
            d = to_dev(host)
            nt.ntt_forward(p, d, 2)
            c = torch.empty_like(d[:L * N])
            nt.ntt_pointwise_inverse(p, c, d[:L * N], d[L * N:], 1)
            got = to_host(c, (1, L, N))
            assert nt.ntt_get_device_status(p) == nt.NTT_OK
            if flags & nt.NTT_CHECK:
                bad = to_dev(host)
                bad[5] = qs[0]                     # one word equal to q
                nt.ntt_forward(p, bad, 2)
                assert nt.ntt_get_device_status(p) == nt.NTT_ERR_INPUT_RANGE
        finally:
            nt.ntt_plan_destroy(p)
        A = orc.ntt_batch(host, qs, psis)
        want = orc.ntt_batch(orc.pointwise_batch(A[:1], A[1:], qs), qs, psis, inverse=True)
        assert np.array_equal(got, want), flags
