"""Ragged batches (one graph-captured persistent launch over heterogeneous
jobs) against the CPU oracle, bit for bit."""
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


def dev(host, w64):
    a = np.ascontiguousarray(host.astype(np.uint64 if w64 else np.uint32))
    return torch.from_numpy(a.view(np.int64 if w64 else np.int32).reshape(-1).copy()).cuda()


def back(t, w64, shape):
    return t.cpu().numpy().view(np.uint64 if w64 else np.uint32).reshape(shape).astype(np.uint64)


def bitrev_rows(X, orc):
    B, L, N = X.shape
    return np.stack([np.stack([orc.bitrev_permute(X[b, l]) for l in range(L)]) for b in range(B)])


PRIMES = {}


def primes(orc, w64, count=32):
    key = (w64, count)
    if key not in PRIMES:
        PRIMES[key] = orc.find_primes(60 if w64 else 30, 18, count)
    return PRIMES[key]


def run(nt, jobs, flags=None):
    flags = nt.NTT_ORDER_BITREV if flags is None else flags
    r = nt.ntt_ragged_create(jobs, flags)
    try:
        nt.ntt_ragged_launch(r)
        assert nt.ntt_ragged_status(r) == nt.NTT_OK
        torch.cuda.synchronize()
    finally:
        nt.ntt_ragged_destroy(r)


def test_ragged_mixed_forward_and_inverse(nt, orc):
    specs = []
    for n in range(12, 18):
        for w64 in (False, True):
            specs.append(dict(N=1 << n, w64=w64, L=1 + (n + w64) % 3, batch=1 + (n % 2)))
    hosts, tens, jobs = [], [], []
    for i, sp in enumerate(specs):
        qs = primes(orc, sp["w64"])[:sp["L"]]
        h = ntt_synth.rns_batch(500 + i, qs, sp["N"], sp["batch"])
        t = dev(h, sp["w64"])
        hosts.append((h, qs))
        tens.append(t)
        jobs.append(dict(data=t, q=qs, N=sp["N"], batch=sp["batch"], word64=sp["w64"], inverse=False))
    run(nt, jobs)
    fwd = []
    for (h, qs), t, sp in zip(hosts, tens, specs):
        psis = [orc.psi(q, sp["N"]) for q in qs]
        want = bitrev_rows(orc.ntt_batch(h, qs, psis), orc)
        got = back(t, sp["w64"], h.shape)
        assert np.array_equal(got, want), sp
        fwd.append(got)
    # inverse jobs on the forward outputs
    for j in jobs:
        j["inverse"] = True
    run(nt, jobs)
    for (h, qs), t, sp in zip(hosts, tens, specs):
        assert np.array_equal(back(t, sp["w64"], h.shape), h), sp


def test_ragged_roundtrip_in_one_launch(nt, orc):
    """A forward and an inverse job on the same buffer: all forward work
    completes before any inverse work, so the set is a round trip."""
    hosts, jobs = [], []
    for i, (n, w64, L) in enumerate([(12, False, 3), (13, True, 2), (16, False, 4), (17, True, 1)]):
        qs = primes(orc, w64)[:L]
        h = ntt_synth.rns_batch(700 + i, qs, 1 << n, 2)
        t = dev(h, w64)
        hosts.append((h, t, w64))
        for inv in (False, True):
            jobs.append(dict(data=t, q=qs, N=1 << n, batch=2, word64=w64, inverse=inv))
    run(nt, jobs)
    for h, t, w64 in hosts:
        assert np.array_equal(back(t, w64, h.shape), h)


def c4_jobs(orc):
    specs = ntt_synth.ragged_jobs(**{"seed": 1004, "jobs": 512})
    for s in specs:
        s["q"] = primes(orc, s["word"] == 64)[:s["L"]]
    return specs


def _brv(k, bits):
    return int(format(int(k), "0%db" % bits)[::-1], 2)


def test_ragged_c4_full_size(nt, orc):
    """The 512-job workload (N = 2^12..2^17, L = 1..32, half 30-bit / half
    60-bit): a forward+inverse round trip in one graph launch returns every
    input; a forward-only launch matches the O(N log N) oracle on every
    coefficient of every job, and, for the transforms with N > 2^14, 256
    coefficients each drawn at random match the O(N^2) definition."""
    specs = c4_jobs(orc)
    hosts, tens, jobs = [], [], []
    for i, s in enumerate(specs):
        w64 = s["word"] == 64
        h = ntt_synth.rns_batch(ntt_synth.stream_seed(1004, i, 99), s["q"], 1 << s["logN"], 1)
        t = dev(h, w64)
        hosts.append(h)
        tens.append(t)
        jobs.append(dict(data=t, q=s["q"], N=1 << s["logN"], batch=1, word64=w64, inverse=False))
    # round trip
    rt = jobs + [dict(j, inverse=True) for j in jobs]
    run(nt, rt)
    for s, h, t in zip(specs, hosts, tens):
        assert np.array_equal(back(t, s["word"] == 64, h.shape), h), s
    # forward only: every job in full, large transforms also by definition
    run(nt, jobs)
    n_sampled = 0
    for i, (s, h) in enumerate(zip(specs, hosts)):
        n, L = s["logN"], s["L"]
        N, w64 = 1 << n, s["word"] == 64
        got = back(tens[i], w64, h.shape)
        psis = [orc.psi(q, N) for q in s["q"]]
        want = orc.ntt_batch(h, s["q"], psis)
        assert np.array_equal(got, bitrev_rows(want, orc)), (i, s)
        if n > 14:
            t_idx = np.repeat(np.arange(L, dtype=np.uint64), 256)
            _, k_idx = ntt_synth.sample_indices(ntt_synth.stream_seed(1004, i, 7), 1, N, 256 * L)
            vals = orc.ntt_batch_at(h, s["q"], psis, t_idx, k_idx)
            pos = [_brv(k, n) for k in k_idx]
            assert np.array_equal(got.reshape(L, N)[t_idx.astype(int), pos], vals), (i, s)
            n_sampled += L
    assert n_sampled > 4000          # about half of the 8536 transforms


def test_ragged_errors(nt, orc):
    qs = primes(orc, False)[:2]
    t = torch.zeros(2 * 4096, dtype=torch.int32, device="cuda")
    ok = dict(data=t, q=qs, N=4096, batch=1, word64=False, inverse=False)
    with pytest.raises(nt.NttError) as e:
        nt.ntt_ragged_create([dict(ok, N=2048)], nt.NTT_ORDER_BITREV)
    assert e.value.status == nt.NTT_ERR_N_RANGE
    with pytest.raises(nt.NttError) as e:
        nt.ntt_ragged_create([ok], 0)
    assert e.value.status == nt.NTT_ERR_UNSUPPORTED
    with pytest.raises(nt.NttError) as e:
        nt.ntt_ragged_create([dict(ok, data=t.data_ptr() + 4)], nt.NTT_ORDER_BITREV)
    assert e.value.status == nt.NTT_ERR_ALIGNMENT
    with pytest.raises(nt.NttError) as e:
        nt.ntt_ragged_create([dict(ok, q=[12289, 7681])], nt.NTT_ORDER_BITREV)
    assert e.value.status == nt.NTT_ERR_Q_NOT_NTT_FRIENDLY
    with pytest.raises(nt.NttError) as e:
        nt.ntt_ragged_create([], nt.NTT_ORDER_BITREV)
    assert e.value.status == nt.NTT_ERR_INVALID_ARG


@pytest.mark.parametrize("red", ["barrett", "montgomery"])
def test_ragged_other_reductions(nt, orc, red):
    hosts, jobs = [], []
    for i, (n, w64) in enumerate([(12, False), (14, True), (16, False)]):
        qs = primes(orc, w64)[:2]
        h = ntt_synth.rns_batch(900 + i, qs, 1 << n, 1)
        t = dev(h, w64)
        hosts.append((h, qs, t, w64, 1 << n))
        jobs.append(dict(data=t, q=qs, N=1 << n, batch=1, word64=w64, inverse=False))
    run(nt, jobs, nt.NTT_ORDER_BITREV | nt.REDUCTIONS[red])
    for h, qs, t, w64, N in hosts:
        want = bitrev_rows(orc.ntt_batch(h, qs, [orc.psi(q, N) for q in qs]), orc)
        assert np.array_equal(back(t, w64, h.shape), want)


def test_ragged_autotuned_item_size(nt, orc):
    """NTT_RAGGED_TUNE: the work-item size is timed on scratch copies (the
    jobs' buffers are untouched by the creation), one of 2/4/8/16 tiles is
    captured, and the launch is bit-exact (forward jobs of every kind)."""
    specs = [(12, False, 3, 2), (13, True, 2, 1), (14, False, 4, 3), (16, False, 5, 2), (16, True, 3, 1),
             (17, False, 2, 1)]
    hosts, tens, jobs = [], [], []
    for i, (n, w64, L, batch) in enumerate(specs):
        qs = primes(orc, w64)[:L]
        h = ntt_synth.rns_batch(900 + i, qs, 1 << n, batch)
        t = dev(h, w64)
        hosts.append((h, qs, n, w64))
        tens.append(t)
        jobs.append(dict(data=t, q=qs, N=1 << n, batch=batch, word64=w64, inverse=False))
    r = nt.ntt_ragged_create(jobs, nt.NTT_ORDER_BITREV | nt.NTT_RAGGED_TUNE)
    try:
        assert nt.ntt_ragged_item_tiles(r) in (2, 4, 8, 16)
        torch.cuda.synchronize()
        for (h, qs, n, w64), t in zip(hosts, tens):
            assert np.array_equal(back(t, w64, h.shape), h)            # creation left the data alone
        nt.ntt_ragged_launch(r)
        assert nt.ntt_ragged_status(r) == nt.NTT_OK
        torch.cuda.synchronize()
    finally:
        nt.ntt_ragged_destroy(r)
    for (h, qs, n, w64), t in zip(hosts, tens):
        psis = [orc.psi(q, 1 << n) for q in qs]
        assert np.array_equal(back(t, w64, h.shape), bitrev_rows(orc.ntt_batch(h, qs, psis), orc)), (n, w64)
    r = nt.ntt_ragged_create(jobs, nt.NTT_ORDER_BITREV)
    try:
        assert nt.ntt_ragged_item_tiles(r) == 8                     # the default without tuning
    finally:
        nt.ntt_ragged_destroy(r)


def test_ragged_barrier_timeout_reported_and_context_survives(nt, orc):
    """Failure path of the grid barrier without a fault: with the test hook,
    CTA 0 leaves before the first barrier, the other CTAs' bounded wait runs
    out (about two seconds), the launch reports NTT_ERR_TIMEOUT, a second
    launch of the same set does the same (the barrier count is reset per
    launch), and a regular set on the same context is then bit-exact."""
    specs = [(12, False, 3), (16, False, 2), (14, True, 2)]
    hosts, jobs = [], []
    for i, (n, w64, L) in enumerate(specs):
        qs = primes(orc, w64)[:L]
        h = ntt_synth.rns_batch(1200 + i, qs, 1 << n, 2)
        t = dev(h, w64)
        hosts.append((h, qs, t, n, w64))
        jobs.append(dict(data=t, q=qs, N=1 << n, batch=2, word64=w64, inverse=False))
    with pytest.raises(nt.NttError) as e:
        nt.ntt_ragged_create(jobs, nt.NTT_ORDER_BITREV | nt.NTT_TEST_STALL | nt.NTT_RAGGED_TUNE)
    assert e.value.status == nt.NTT_ERR_INVALID_ARG
    r = nt.ntt_ragged_create(jobs, nt.NTT_ORDER_BITREV | nt.NTT_TEST_STALL)
    try:
        for _ in range(2):
            nt.ntt_ragged_launch(r)
            assert nt.ntt_ragged_status(r) == nt.NTT_ERR_TIMEOUT
            assert nt.ntt_ragged_status(r) == nt.NTT_OK          # read and cleared
    finally:
        nt.ntt_ragged_destroy(r)
    for h, qs, t, n, w64 in hosts:
        t.copy_(dev(h, w64))
    run(nt, jobs)
    for h, qs, t, n, w64 in hosts:
        psis = [orc.psi(q, 1 << n) for q in qs]
        assert np.array_equal(back(t, w64, h.shape), bitrev_rows(orc.ntt_batch(h, qs, psis), orc)), (n, w64)


@pytest.mark.parametrize("w64", [False, True])
def test_ragged_one_word_size(nt, orc, w64):
    """A set whose jobs all have one word size runs one persistent kernel
    (the other has no items and is not launched): every job's forward output
    bit-exact, and the barrier test hook lands on the kernel that exists
    (NTT_ERR_TIMEOUT, then a regular set is bit-exact again)."""
    specs = [(12, 2), (15, 3), (16, 1)]
    hosts, jobs = [], []
    for i, (n, L) in enumerate(specs):
        qs = primes(orc, w64)[:L]
        h = ntt_synth.rns_batch(1300 + i + 10 * w64, qs, 1 << n, 2)
        t = dev(h, w64)
        hosts.append((h, qs, t, n))
        jobs.append(dict(data=t, q=qs, N=1 << n, batch=2, word64=w64, inverse=False))

    def check():
        for h, qs, t, n in hosts:
            psis = [orc.psi(q, 1 << n) for q in qs]
            assert np.array_equal(back(t, w64, h.shape), bitrev_rows(orc.ntt_batch(h, qs, psis), orc)), (n, w64)

    run(nt, jobs)
    check()
    r = nt.ntt_ragged_create(jobs, nt.NTT_ORDER_BITREV | nt.NTT_TEST_STALL)
    try:
        nt.ntt_ragged_launch(r)
        assert nt.ntt_ragged_status(r) == nt.NTT_ERR_TIMEOUT
    finally:
        nt.ntt_ragged_destroy(r)
    for h, qs, t, n in hosts:
        t.copy_(dev(h, w64))
    run(nt, jobs)
    check()
