"""Two-pass forms chosen by the tuning table, and the autotuner itself:
every combination of forward and inverse form is bit-exact against the
oracle, and a tuning run records forms that the next plan uses."""
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
    yield nt
    nt.ntt_tune_clear()


def to_dev(h, w64):
    a = np.ascontiguousarray(h.astype(np.uint64 if w64 else np.uint32))
    return torch.from_numpy(a.view(np.int64 if w64 else np.int32).reshape(-1).copy()).cuda()


def to_host(t, w64, shape):
    return t.cpu().numpy().view(np.uint64 if w64 else np.uint32).reshape(shape).astype(np.uint64)


def bitrev_rows(X, orc):
    B, L, N = X.shape
    return np.stack([np.stack([orc.bitrev_permute(X[b, l]) for l in range(L)]) for b in range(B)])


@pytest.mark.parametrize("n,w64", [(16, False), (15, True)])
def test_every_form_pair_bit_exact(nt, orc, n, w64):
    """Every (forward, inverse) pair of the five forms; 8-byte plans take
    the shuffle forms as their shared-memory defaults."""
    N, L, pairs = 1 << n, 3, 2
    qs = orc.find_primes(60 if w64 else 30, 18, L)
    psis = [orc.psi(q, N) for q in qs]
    host = ntt_synth.rns_batch(2300 + n, qs, N, 2 * pairs)
    A = orc.ntt_batch(host, qs, psis)
    want_prod = orc.ntt_batch(orc.pointwise_batch(A[:pairs], A[pairs:], qs), qs, psis, inverse=True)
    flags = nt.NTT_ORDER_BITREV | (nt.NTT_WORD64 if w64 else 0)
    try:
        shfl = (nt.NTT_FORM_SMALL_SHFL, nt.NTT_FORM_WIDE_SHFL)
        for fwd in range(5):
            for inv in range(5):
                nt.ntt_tune_set(N, L, flags, 2 * pairs, fwd, inv)     # forward batch
                nt.ntt_tune_set(N, L, flags, pairs, fwd, inv)         # product batch
                p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, flags)
                try:
                    assert nt.ntt_plan_form(p, 2 * pairs) == (nt.NTT_FORM_SMALL if w64 and fwd in shfl else fwd)
                    assert nt.ntt_plan_form(p, pairs, True) == (nt.NTT_FORM_WIDE if w64 and inv in shfl else inv)
                    d = to_dev(host, w64)
                    nt.ntt_forward(p, d, 2 * pairs)
                    assert nt.ntt_plan_last_launches(p) == (1 if fwd == 2 else 2)
                    assert np.array_equal(to_host(d, w64, host.shape), bitrev_rows(A, orc)), (fwd, inv)
                    half = pairs * L * N
                    c = torch.empty_like(d[:half])
                    nt.ntt_pointwise_inverse(p, c, d[:half], d[half:], pairs)
                    assert np.array_equal(to_host(c, w64, (pairs, L, N)), want_prod), (fwd, inv)
                    nt.ntt_inverse(p, d, 2 * pairs)
                    assert np.array_equal(to_host(d, w64, host.shape), host), (fwd, inv)
                    assert nt.ntt_get_device_status(p) == nt.NTT_OK
                finally:
                    nt.ntt_plan_destroy(p)
    finally:
        nt.ntt_tune_clear()


def test_autotune_records_forms_the_next_plan_uses(nt, orc):
    N, L, batch = 1 << 16, 5, 4
    qs = orc.find_primes(30, 17, L)
    flags = nt.NTT_ORDER_BITREV
    try:
        r = nt.ntt_autotune(N, qs, flags, batch)
        assert r["forward_form"] in range(5) and r["inverse_form"] in range(5)
        # splits 2^7 x 2^9, 2^8 x 2^8, 2^9 x 2^7 and both radices are all
        # valid at N = 2^16; the chosen pair has the smallest forward +
        # inverse time
        assert r["chunk_log2"] in (7, 8, 9) and r["radix_log2"] in (3, 4)
        assert sorted(r["config_ms"]) == ["%d,%d" % (lr, s2) for lr in (3, 4) for s2 in (7, 8, 9)]
        assert all(ms > 0 for ms in r["config_ms"].values())
        assert r["config_ms"]["%d,%d" % (r["radix_log2"], r["chunk_log2"])] == min(r["config_ms"].values())
        # (the streamed form exists only with 256-word chunks and radix 16)
        streamed_ok = r["chunk_log2"] == 8 and r["radix_log2"] == 4
        for ms in (r["forward_ms"], r["inverse_ms"]):
            assert len(ms) == 5 and all(v > 0 for v in ms[:2] + ms[3:]) and (ms[2] > 0) == streamed_ok
        assert r["forward_ms"][r["forward_form"]] == min(v for v in r["forward_ms"] if v > 0)
        assert nt.ntt_tune_get_split(N, L, flags) == (r["chunk_log2"], r["radix_log2"])
        assert nt.ntt_tune_get(N, L, flags, batch) == r["forward_form"]
        p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, flags)
        try:
            assert nt.ntt_plan_chunk_log2(p) == r["chunk_log2"]
            assert nt.ntt_plan_radix_log2(p) == r["radix_log2"]
            assert nt.ntt_plan_form(p, batch) == r["forward_form"]
            assert nt.ntt_plan_form(p, batch, True) == r["inverse_form"]
            assert nt.ntt_plan_form(p, 4 * batch) == nt.NTT_FORM_SMALL        # untuned bucket: default
            psis = [orc.psi(q, N) for q in qs]
            host = ntt_synth.rns_batch(2310, qs, N, batch)
            d = to_dev(host, False)
            nt.ntt_forward(p, d, batch)
            assert np.array_equal(to_host(d, False, host.shape), bitrev_rows(orc.ntt_batch(host, qs, psis), orc))
            nt.ntt_inverse(p, d, batch)
            assert np.array_equal(to_host(d, False, host.shape), host)
        finally:
            nt.ntt_plan_destroy(p)
        with pytest.raises(nt.NttError) as e:
            nt.ntt_autotune(1 << 12, qs, flags, 2)                           # single-pass size
        assert e.value.status == nt.NTT_ERR_UNSUPPORTED
    finally:
        nt.ntt_tune_clear()


# (log N, 8-byte words): the splits each size takes, chunks of 2^s2 words
SPLITS = [(15, False, (7, 8, 9)), (16, False, (7, 8, 9)), (17, False, (8, 9)), (14, True, (7, 8, 9)),
          (16, True, (7, 8, 9))]


@pytest.mark.parametrize("shfl", [False, True])
@pytest.mark.parametrize("radix", [4, 3])
@pytest.mark.parametrize("n,w64,splits", SPLITS)
def test_every_split_bit_exact(nt, orc, n, w64, splits, radix, shfl):
    """Every split N = 2^s1 x 2^s2 a size takes, in both radices (rounds of
    four stages on 16 words a thread, or three on 8), with both chunk-pass
    forms -- with shared-memory exchanges, and (4-byte words) with warp
    shuffles --, batches whose tiles pair polynomials (one chunk of K
    polynomials, or two chunks of K / 2) and batches that do not: forward,
    the product fused into the inverse, and the inverse, bit-exact."""
    if shfl and w64:
        pytest.skip("the shuffle forms are for 4-byte words")
    N, L = 1 << n, 3
    qs = orc.find_primes(60 if w64 else 30, 18, L)
    psis = [orc.psi(q, N) for q in qs]
    flags = nt.NTT_ORDER_BITREV | (nt.NTT_WORD64 if w64 else 0)
    try:
        for s2 in splits:
            small, wide = ((nt.NTT_FORM_SMALL_SHFL, nt.NTT_FORM_WIDE_SHFL) if shfl
                           else (nt.NTT_FORM_SMALL, nt.NTT_FORM_WIDE))
            # (8 and 12 on 256-thread tiles: K / 2 polynomials x 2 chunks a
            # tile where K / 2 divides the batch and K does not)
            for batch, form in ((4, small), (3, wide), (16, wide), (2, small), (8, wide), (12, wide)):
                nt.ntt_tune_clear()
                nt.ntt_tune_set_split(N, L, flags, s2, radix)
                nt.ntt_tune_set(N, L, flags, batch, form, form)
                pairs = batch // 2
                if pairs:
                    nt.ntt_tune_set(N, L, flags, pairs, form, form)
                host = ntt_synth.rns_batch(2400 + 10 * s2 + batch + 100 * radix, qs, N, batch)
                A = orc.ntt_batch(host, qs, psis)
                p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, flags)
                try:
                    assert (nt.ntt_plan_chunk_log2(p), nt.ntt_plan_radix_log2(p)) == (s2, radix)
                    assert nt.ntt_plan_form(p, batch) == form
                    d = to_dev(host, w64)
                    nt.ntt_forward(p, d, batch)
                    assert np.array_equal(to_host(d, w64, host.shape), bitrev_rows(A, orc)), (s2, batch, form)
                    if pairs:
                        want = orc.ntt_batch(orc.pointwise_batch(A[:pairs], A[pairs:2 * pairs], qs), qs, psis,
                                             inverse=True)
                        half = pairs * L * N
                        c = torch.empty_like(d[:half])
                        nt.ntt_pointwise_inverse(p, c, d[:half], d[half:2 * half], pairs)
                        assert np.array_equal(to_host(c, w64, (pairs, L, N)), want), (s2, batch, form)
                    nt.ntt_inverse(p, d, batch)
                    assert np.array_equal(to_host(d, w64, host.shape), host), (s2, batch, form)
                    assert nt.ntt_get_device_status(p) == nt.NTT_OK
                finally:
                    nt.ntt_plan_destroy(p)
    finally:
        nt.ntt_tune_clear()


@pytest.mark.parametrize("red", ["barrett", "montgomery"])
@pytest.mark.parametrize("radix", [4, 3])
def test_shuffle_forms_other_reductions(nt, orc, red, radix):
    """The shuffle forms with Barrett and Montgomery twiddles (each has its
    own kernels): forward, product + inverse and inverse against the
    oracle, paired and unpaired tiles."""
    N, L = 1 << 16, 3
    qs = orc.find_primes(30, 17, L)
    psis = [orc.psi(q, N) for q in qs]
    flags = nt.NTT_ORDER_BITREV | (nt.NTT_RED_BARRETT if red == "barrett" else nt.NTT_RED_MONTGOMERY)
    try:
        for batch, fwd, inv in ((4, nt.NTT_FORM_SMALL_SHFL, nt.NTT_FORM_WIDE_SHFL),
                                (3, nt.NTT_FORM_WIDE_SHFL, nt.NTT_FORM_SMALL_SHFL)):
            nt.ntt_tune_clear()
            nt.ntt_tune_set_split(N, L, flags, 8, radix)
            nt.ntt_tune_set(N, L, flags, batch, fwd, inv)
            pairs = batch // 2
            nt.ntt_tune_set(N, L, flags, pairs, fwd, inv)
            host = ntt_synth.rns_batch(2500 + batch + 10 * radix, qs, N, batch)
            A = orc.ntt_batch(host, qs, psis)
            p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, flags)
            try:
                assert (nt.ntt_plan_form(p, batch), nt.ntt_plan_form(p, pairs, True)) == (fwd, inv)
                d = to_dev(host, False)
                nt.ntt_forward(p, d, batch)
                assert np.array_equal(to_host(d, False, host.shape), bitrev_rows(A, orc)), batch
                want = orc.ntt_batch(orc.pointwise_batch(A[:pairs], A[pairs:2 * pairs], qs), qs, psis,
                                     inverse=True)
                half = pairs * L * N
                c = torch.empty_like(d[:half])
                nt.ntt_pointwise_inverse(p, c, d[:half], d[half:2 * half], pairs)
                assert np.array_equal(to_host(c, False, (pairs, L, N)), want), batch
                nt.ntt_inverse(p, d, batch)
                assert np.array_equal(to_host(d, False, host.shape), host), batch
                assert nt.ntt_get_device_status(p) == nt.NTT_OK
            finally:
                nt.ntt_plan_destroy(p)
    finally:
        nt.ntt_tune_clear()


def test_split_limits(nt, orc):
    """Splits and radices a size cannot take are refused; streamed and
    on-the-fly twiddle plans keep 256-word chunks and radix 16 whatever the
    table says, and a radix-8 or non-256 split plan has no streamed form."""
    qs = orc.find_primes(30, 18, 2)
    f = nt.NTT_ORDER_BITREV
    with pytest.raises(nt.NttError):
        nt.ntt_tune_set_split(1 << 17, 2, f, 7)                      # 2^10-point columns
    with pytest.raises(nt.NttError):
        nt.ntt_tune_set_split(1 << 15, 2, f | nt.NTT_TW_OTF, 9)
    with pytest.raises(nt.NttError):
        nt.ntt_tune_set_split(1 << 16, 2, f, 8, 5)
    try:
        nt.ntt_tune_set_split(1 << 16, 2, f | nt.NTT_STREAMED, 9, 3)
        p = nt.ntt_plan_create(1 << 16, qs, nt.NTT_FUSED, f | nt.NTT_STREAMED)
        try:
            assert (nt.ntt_plan_chunk_log2(p), nt.ntt_plan_radix_log2(p)) == (8, 4)
            assert nt.ntt_plan_form(p, 4) == nt.NTT_FORM_STREAMED
        finally:
            nt.ntt_plan_destroy(p)
        for s2, radix in ((9, 4), (8, 3)):
            nt.ntt_tune_clear()
            nt.ntt_tune_set_split(1 << 16, 2, f, s2, radix)
            nt.ntt_tune_set(1 << 16, 2, f, 4, nt.NTT_FORM_STREAMED, nt.NTT_FORM_STREAMED)
            p = nt.ntt_plan_create(1 << 16, qs, nt.NTT_FUSED, f)
            try:
                assert (nt.ntt_plan_chunk_log2(p), nt.ntt_plan_radix_log2(p)) == (s2, radix)
                # no streamed form there: the defaults serve
                assert nt.ntt_plan_form(p, 4) == nt.NTT_FORM_SMALL
                assert nt.ntt_plan_form(p, 4, True) == nt.NTT_FORM_WIDE
            finally:
                nt.ntt_plan_destroy(p)
    finally:
        nt.ntt_tune_clear()
