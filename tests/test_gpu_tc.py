"""The tensor-core four-step form (N = 2^16, 8-bit digit products) against
the oracle and against the butterfly form, in both of its forms: tcgen05
(balanced digits in fp16, fp32 diagonals in tensor memory; the default) and
the warp-level integer MMA (NTT_TC_IMMA)."""
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


def dev(h):
    return torch.from_numpy(np.ascontiguousarray(h.astype(np.uint32)).view(np.int32).reshape(-1).copy()).cuda()


def host(t, shape):
    return t.cpu().numpy().view(np.uint32).reshape(shape).astype(np.uint64)


def bitrev_rows(X, orc):
    B, L, N = X.shape
    return np.stack([np.stack([orc.bitrev_permute(X[b, l]) for l in range(L)]) for b in range(B)])


FORMS = ["tcgen05", "imma"]


def form_flags(nt, form):
    return nt.NTT_TC_IMMA if form == "imma" else 0


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("L,batch", [(2, 1), (3, 5), (32, 16)])
def test_tc_forward_inverse_bit_exact(nt, orc, form, L, batch):
    N = 1 << 16
    qs = orc.find_primes(30, 17, L)
    psis = [orc.psi(q, N) for q in qs]
    h = ntt_synth.rns_batch(1005, qs, N, batch)
    p = nt.ntt_plan_create(N, qs, nt.NTT_TC_FOURSTEP, nt.NTT_ORDER_BITREV | form_flags(nt, form))
    try:
        d = dev(h)
        nt.ntt_forward(p, d, batch)
        got = host(d, h.shape)
        want = bitrev_rows(orc.ntt_batch(h, qs, psis), orc)
        assert np.array_equal(got, want)
        if L * batch >= 256:
            # the full workload (512 transforms): 256 coefficients of each
            # against the O(N^2) definition as well
            check_definition_samples(orc, h, qs, psis, got, 1005, 256, bitrev=True)
        nt.ntt_inverse(p, d, batch)
        assert np.array_equal(host(d, h.shape), h)
        assert nt.ntt_get_device_status(p) == nt.NTT_OK
    finally:
        nt.ntt_plan_destroy(p)


def test_tc_matches_butterfly_form_and_natural_order(nt, orc):
    N, L, batch = 1 << 16, 4, 3
    qs = orc.find_primes(30, 17, L)
    h = ntt_synth.rns_batch(77, qs, N, batch)
    outs = []
    for variant, flags in [(nt.NTT_TC_FOURSTEP, 0), (nt.NTT_TC_FOURSTEP, nt.NTT_TC_IMMA), (nt.NTT_FUSED, 0)]:
        p = nt.ntt_plan_create(N, qs, variant, flags)
        try:
            d = dev(h)
            nt.ntt_forward(p, d, batch)
            outs.append(host(d, h.shape))
            nt.ntt_inverse(p, d, batch)
            assert np.array_equal(host(d, h.shape), h)
        finally:
            nt.ntt_plan_destroy(p)
    assert np.array_equal(outs[0], outs[2])
    assert np.array_equal(outs[1], outs[2])
    psis = [orc.psi(q, N) for q in qs]
    assert np.array_equal(outs[0], orc.ntt_batch(h, qs, psis))


@pytest.mark.parametrize("form", FORMS)
def test_tc_extreme_inputs(nt, orc, form):
    """Words that put the digits at their extremes, against the matrices of
    12 primes: q - 1 (unsigned digits all large), 0x3F7F7F80 (balanced
    digits -128, -128, -128, 64), 0x3F7F7F7F (127, 127, 127, 63: the
    largest positive digits a word below 2^30 has), 0 and alternating
    patterns, forward and back.  The fp32 accumulation in the tensor core is
    exact only if it keeps 24 significand bits; this is the check."""
    N = 1 << 16
    qs = orc.find_primes(30, 17, 12)
    h = np.zeros((3, 12, N), np.uint64)
    for l, q in enumerate(qs):
        h[0, l] = q - 1
        h[1, l, 0::2] = 0x3F7F7F80 % q
        h[1, l, 1::4] = 0
        h[1, l, 3::4] = 0x00808080
        h[2, l] = 0x3F7F7F7F % q
        h[2, l, 1::3] = 0x3F7F7F80 % q
    p = nt.ntt_plan_create(N, qs, nt.NTT_TC_FOURSTEP, nt.NTT_ORDER_BITREV | form_flags(nt, form))
    try:
        d = dev(h)
        nt.ntt_forward(p, d, 3)
        psis = [orc.psi(q, N) for q in qs]
        assert np.array_equal(host(d, h.shape), bitrev_rows(orc.ntt_batch(h, qs, psis), orc))
        nt.ntt_inverse(p, d, 3)
        assert np.array_equal(host(d, h.shape), h)
    finally:
        nt.ntt_plan_destroy(p)


def test_tc_rejects_unsupported(nt, orc):
    qs = orc.find_primes(30, 17, 1)
    for N, flags in [(1 << 14, 0), (1 << 16, nt.NTT_RED_MONTGOMERY)]:
        with pytest.raises(nt.NttError) as e:
            nt.ntt_plan_create(N, qs if N == 1 << 16 else orc.find_primes(30, 15, 1),
                               nt.NTT_TC_FOURSTEP, flags)
        assert e.value.status == nt.NTT_ERR_UNSUPPORTED


def test_tc_bounded_wait_reports_timeout_and_context_survives(nt, orc):
    """Failure path of the tcgen05 kernel without a fault: with the test
    hook, CTA 0's first matrix copy waits for bytes that never arrive; the
    MMA thread's wait gives up after about a second, every role leaves its
    loop, the CTA frees its tensor memory, the call reports
    NTT_ERR_TIMEOUT, and the next plan on the same context is bit-exact."""
    N = 1 << 16
    qs = orc.find_primes(30, 17, 2)
    h = ntt_synth.rns_batch(63, qs, N, 2)
    p = nt.ntt_plan_create(N, qs, nt.NTT_TC_FOURSTEP, nt.NTT_ORDER_BITREV | nt.NTT_TEST_STALL)
    try:
        d = dev(h)
        nt.ntt_forward(p, d, 2)
        assert nt.ntt_get_device_status(p) == nt.NTT_ERR_TIMEOUT
    finally:
        nt.ntt_plan_destroy(p)
    p = nt.ntt_plan_create(N, qs, nt.NTT_TC_FOURSTEP, nt.NTT_ORDER_BITREV)
    try:
        d = dev(h)
        nt.ntt_forward(p, d, 2)
        psis = [orc.psi(q, N) for q in qs]
        assert np.array_equal(host(d, h.shape), bitrev_rows(orc.ntt_batch(h, qs, psis), orc))
        assert nt.ntt_get_device_status(p) == nt.NTT_OK
    finally:
        nt.ntt_plan_destroy(p)
