"""Fast RNS base conversion on the GPU (ntt_bconv, through the C ABI)
against the CPU oracle: bit-exact, every output word or sampled columns at
the full workload size."""
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


def bases(orc, L, K):
    qs = orc.find_primes(30, 17, L)
    ps = orc.find_primes(29, 17, K)          # a disjoint basis (29-bit primes)
    return qs, ps


def run(nt, x, qs, ps):
    B, L, N = x.shape
    h = nt.ntt_bconv_create(qs, ps, N)
    try:
        d_in = dev(x)
        d_out = torch.zeros(B * len(ps) * N, dtype=torch.int32, device="cuda")
        nt.ntt_bconv(h, d_out, d_in, B)
        torch.cuda.synchronize()
        return host(d_out, (B, len(ps), N))
    finally:
        nt.ntt_bconv_destroy(h)


@pytest.mark.parametrize("L,K,N,B", [(1, 1, 1, 1), (3, 5, 7, 2), (8, 8, 4096, 3), (17, 4, 1000, 1),
                                     (12, 30, 777, 2), (64, 64, 512, 1), (5, 64, 33, 3), (33, 2, 2048, 2)])
def test_bconv_matches_oracle(nt, orc, L, K, N, B):
    qs, ps = bases(orc, L, K)
    x = ntt_synth.rns_batch(2000 + L * 7 + K, qs, N, B)
    assert np.array_equal(run(nt, x, qs, ps), orc.base_conv(x, qs, ps))


def test_bconv_extreme_and_overlapping_bases(nt, orc):
    """Every residue q_i - 1 or 0 (largest and smallest products), and a
    target basis that shares primes with the source (those limbs come back
    unchanged)."""
    qs, ps = bases(orc, 32, 8)
    N = 256
    x = np.zeros((2, 32, N), np.uint64)
    for i, q in enumerate(qs):
        x[0, i] = q - 1
        x[1, i, ::2] = q - 1
    tgt = [qs[3], ps[0], qs[31], ps[1]]
    got = run(nt, x, qs, tgt)
    assert np.array_equal(got, orc.base_conv(x, qs, tgt))
    assert np.array_equal(got[:, 0], x[:, 3]) and np.array_equal(got[:, 2], x[:, 31])


def test_bconv_workload_size_sampled(nt, orc):
    """N = 2^16, 32 limbs -> 32 limbs, 8 polynomials (the bench workload):
    1024 sampled coefficients against the oracle run on those columns."""
    qs, ps = bases(orc, 32, 32)
    N, B = 1 << 16, 8
    x = ntt_synth.rns_batch(2100, qs, N, B)
    got = run(nt, x, qs, ps)
    rng = np.random.default_rng(2101)
    bs = rng.integers(0, B, 1024)
    ns = rng.integers(0, N, 1024)
    cols = np.ascontiguousarray(x[bs, :, ns].T[None])          # [1][L][1024]
    want = orc.base_conv(cols, qs, ps)[0]                     # [K][1024]
    assert np.array_equal(got[bs, :, ns].T, want)


def test_bconv_rejects_bad_arguments(nt, orc):
    qs, ps = bases(orc, 4, 4)
    for args, status in [((qs, [], 16), nt.NTT_ERR_INVALID_ARG), ((qs, ps, 0), nt.NTT_ERR_INVALID_ARG),
                         ((qs + [qs[0]], ps, 16), nt.NTT_ERR_INVALID_ARG),
                         ((qs, ps + [(1 << 30) + 3], 16), nt.NTT_ERR_Q_WIDTH),
                         ((qs[:3] + [qs[3] + 2], ps, 16), nt.NTT_ERR_Q_NOT_PRIME),
                         ((orc.find_primes(30, 17, 65), ps, 16), nt.NTT_ERR_INVALID_ARG)]:
        with pytest.raises(nt.NttError) as e:
            nt.ntt_bconv_create(*args)
        assert e.value.status == status
    h = nt.ntt_bconv_create(qs, ps, 16)
    try:
        x = torch.zeros(4 * 16, dtype=torch.int32, device="cuda")
        with pytest.raises(nt.NttError):
            nt.ntt_bconv(h, x, x, 0)
    finally:
        nt.ntt_bconv_destroy(h)
