"""The tensor-core four-step form (N = 2^16, 8-bit digit products on the
integer tensor cores) against the oracle and against the butterfly form."""
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


def dev(h):
    return torch.from_numpy(np.ascontiguousarray(h.astype(np.uint32)).view(np.int32).reshape(-1).copy()).cuda()


def host(t, shape):
    return t.cpu().numpy().view(np.uint32).reshape(shape).astype(np.uint64)


def bitrev_rows(X, orc):
    B, L, N = X.shape
    return np.stack([np.stack([orc.bitrev_permute(X[b, l]) for l in range(L)]) for b in range(B)])


@pytest.mark.parametrize("L,batch", [(2, 1), (32, 16)])
def test_tc_forward_inverse_bit_exact(nt, orc, L, batch):
    N = 1 << 16
    qs = orc.find_primes(30, 17, L)
    psis = [orc.psi(q, N) for q in qs]
    h = ntt_synth.rns_batch(1005, qs, N, batch)
    p = nt.ntt_plan_create(N, qs, nt.NTT_TC_FOURSTEP, nt.NTT_ORDER_BITREV)
    try:
        d = dev(h)
        nt.ntt_forward(p, d, batch)
        got = host(d, h.shape)
        want = bitrev_rows(orc.ntt_batch(h, qs, psis), orc)
        assert np.array_equal(got, want)
        nt.ntt_inverse(p, d, batch)
        assert np.array_equal(host(d, h.shape), h)
    finally:
        nt.ntt_plan_destroy(p)


def test_tc_matches_butterfly_form_and_natural_order(nt, orc):
    N, L, batch = 1 << 16, 4, 3
    qs = orc.find_primes(30, 17, L)
    h = ntt_synth.rns_batch(77, qs, N, batch)
    outs = []
    for variant, flags in [(nt.NTT_TC_FOURSTEP, 0), (nt.NTT_FUSED, 0)]:
        p = nt.ntt_plan_create(N, qs, variant, flags)
        try:
            d = dev(h)
            nt.ntt_forward(p, d, batch)
            outs.append(host(d, h.shape))
            nt.ntt_inverse(p, d, batch)
            assert np.array_equal(host(d, h.shape), h)
        finally:
            nt.ntt_plan_destroy(p)
    assert np.array_equal(outs[0], outs[1])
    psis = [orc.psi(q, N) for q in qs]
    assert np.array_equal(outs[0], orc.ntt_batch(h, qs, psis))


def test_tc_extreme_inputs(nt, orc):
    """All words q-1: every digit product and diagonal sum at its maximum."""
    N = 1 << 16
    qs = orc.find_primes(30, 17, 2)
    h = np.zeros((1, 2, N), np.uint64)
    for l, q in enumerate(qs):
        h[0, l] = q - 1
    p = nt.ntt_plan_create(N, qs, nt.NTT_TC_FOURSTEP, nt.NTT_ORDER_BITREV)
    try:
        d = dev(h)
        nt.ntt_forward(p, d, 1)
        psis = [orc.psi(q, N) for q in qs]
        assert np.array_equal(host(d, h.shape), bitrev_rows(orc.ntt_batch(h, qs, psis), orc))
    finally:
        nt.ntt_plan_destroy(p)


def test_tc_rejects_unsupported(nt, orc):
    qs = orc.find_primes(30, 17, 1)
    for N, flags in [(1 << 14, 0), (1 << 16, nt.NTT_RED_MONTGOMERY)]:
        with pytest.raises(nt.NttError) as e:
            nt.ntt_plan_create(N, qs if N == 1 << 16 else orc.find_primes(30, 15, 1),
                               nt.NTT_TC_FOURSTEP, flags)
        assert e.value.status == nt.NTT_ERR_UNSUPPORTED
