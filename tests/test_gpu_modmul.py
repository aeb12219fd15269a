"""Row a2 (modular multiplication) on its own: every pair (a, b) in
[0, 12289)^2 through the product of two variable operands (Barrett for
Shoup/Barrett plans, Montgomery for Montgomery plans), with 4- and 8-byte
words, plus the edge values of 30- and 60-bit primes, against the oracle's
128-bit products.  (The twiddle product, Shoup / Barrett / Montgomery with a
precomputed operand, is exercised by every transform in the parity tests.)"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2405_11353_gb300 as nt
    torch.cuda.init()
    return nt


def to_dev(a, w64):
    a = np.ascontiguousarray(a.astype(np.uint64 if w64 else np.uint32))
    return torch.from_numpy(a.view(np.int64 if w64 else np.int32).reshape(-1).copy()).cuda()


def to_host(t, w64):
    return t.cpu().numpy().view(np.uint64 if w64 else np.uint32).astype(np.uint64)


@pytest.mark.parametrize("w64", [False, True])
@pytest.mark.parametrize("red", ["barrett", "montgomery"])
def test_all_pairs_q12289(nt, orc, w64, red):
    q, N = 12289, 2048
    flags = nt.REDUCTIONS[red] | (nt.NTT_WORD64 if w64 else 0)
    p = nt.ntt_plan_create(N, [q], nt.NTT_FUSED, flags)
    try:
        av = np.arange(q, dtype=np.uint64)
        for b0 in range(0, q, 2048):                     # 2048 values of b at a time
            bv = np.arange(b0, min(q, b0 + 2048), dtype=np.uint64)
            a = np.tile(av, bv.size)
            b = np.repeat(bv, q)
            n = a.size
            pad = (-n) % N
            a = np.concatenate([a, np.zeros(pad, np.uint64)])
            b = np.concatenate([b, np.zeros(pad, np.uint64)])
            batch = a.size // N
            da, db = to_dev(a, w64), to_dev(b, w64)
            dc = torch.empty_like(da)
            nt.ntt_pointwise_mul(p, dc, da, db, batch)
            got = to_host(dc, w64)
            want = orc.pointwise_batch(a.reshape(batch, 1, N), b.reshape(batch, 1, N), [q]).reshape(-1)
            assert np.array_equal(got, want), (red, w64, b0)
    finally:
        nt.ntt_plan_destroy(p)


@pytest.mark.parametrize("w64", [False, True])
@pytest.mark.parametrize("red", ["shoup", "barrett", "montgomery"])
def test_edge_values_wide_primes(nt, orc, w64, red):
    """{0, 1, 2, q/2, q-2, q-1} and random values, all pairs, for the first and
    last primes of the workloads (30-bit: 2^30 - k 2^17 + 1; 60-bit)."""
    bits = 60 if w64 else 30
    qs = orc.find_primes(bits, 17, 24)
    N = 1 << 16
    rng = np.random.default_rng(5 + w64)
    for q in (qs[0], qs[-1]):
        edge = [0, 1, 2, q // 2, q - 2, q - 1] + [int(v) for v in rng.integers(0, q, 10, dtype=np.uint64)]
        a = np.array([x for x in edge for _ in edge], dtype=np.uint64)
        b = np.array([y for _ in edge for y in edge], dtype=np.uint64)
        a = np.resize(a, N)
        b = np.resize(b, N)
        flags = nt.REDUCTIONS[red] | (nt.NTT_WORD64 if w64 else 0)
        p = nt.ntt_plan_create(N, [q], nt.NTT_FUSED, flags)
        try:
            da, db = to_dev(a, w64), to_dev(b, w64)
            dc = torch.empty_like(da)
            nt.ntt_pointwise_mul(p, dc, da, db, 1)
            got = to_host(dc, w64)
        finally:
            nt.ntt_plan_destroy(p)
        want = orc.pointwise_batch(a.reshape(1, 1, N), b.reshape(1, 1, N), [q]).reshape(-1)
        assert np.array_equal(got, want), (red, w64, q)
