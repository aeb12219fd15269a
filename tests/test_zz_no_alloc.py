"""ntt_forward_noalloc: the forward transform for callers that must not
allocate device memory (a framework owning every byte through its own pool,
a loop that cannot take cudaMalloc's implicit synchronisation, a plugin under
a fixed budget).  It must give exactly what ntt_forward gives on the same
plan -- and what the CPU oracle gives -- call after call, while its fixed
scratch array keeps the previous call's contents, and it must not change the
device's free memory.  Collected last (file name) so a failure here never
hides the other tests."""
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


def _dev(host, w64):
    a = np.ascontiguousarray(host.astype(np.uint64 if w64 else np.uint32))
    return torch.from_numpy(a.view(np.int64 if w64 else np.int32).reshape(-1).copy()).cuda()


def _host(t, w64, shape):
    return t.cpu().numpy().view(np.uint64 if w64 else np.uint32).reshape(shape).astype(np.uint64)


def _oracle_forward(orc, host, qs, N, bitrev):
    X = orc.ntt_batch(host, qs, [orc.psi(q, N) for q in qs])
    if bitrev:
        B, L, _ = X.shape
        X = np.stack([np.stack([orc.bitrev_permute(X[b, l]) for l in range(L)]) for b in range(B)])
    return X


@pytest.mark.parametrize("red", ["shoup", "barrett", "montgomery"])
@pytest.mark.parametrize("w64,bitrev,variant", [(False, False, "stockham"), (True, True, "pease"),
                                                (False, True, "dit")])
def test_noalloc_matches_ntt_forward_and_oracle_twice(nt, orc, red, w64, bitrev, variant):
    N, L, batch = 1 << 12, 3, 4
    qs = nt.ntt_find_primes(60 if w64 else 30, 17, L)
    flags = (nt.NTT_WORD64 if w64 else 0) | (nt.NTT_ORDER_BITREV if bitrev else 0) | nt.REDUCTIONS[red]
    plan = nt.ntt_plan_create(N, qs, nt.VARIANTS[variant], flags)
    try:
        for call in range(2):                     # two calls in a row
            host = ntt_synth.rns_batch(77 + call, qs, N, batch)
            ref = _dev(host, w64)
            got = _dev(host, w64)
            nt.ntt_forward(plan, ref, batch)
            nt.ntt_forward_noalloc(plan, got, batch)
            # twist + 12 Stockham stages (an even count: the result is back
            # in the caller's buffer, no copy) (+ the bit-reversal permutation)
            assert nt.ntt_plan_last_launches(plan) == 1 + 12 + (1 if bitrev else 0)
            torch.cuda.synchronize()
            assert torch.equal(ref, got), "call %d differs from ntt_forward" % call
            want = _oracle_forward(orc, host, qs, N, bitrev)
            assert np.array_equal(_host(got, w64, host.shape), want), "call %d differs from the oracle" % call
        assert nt.ntt_get_device_status(plan) == nt.NTT_OK
    finally:
        nt.ntt_plan_destroy(plan)


def test_noalloc_full_array_and_limits(nt, orc):
    """The largest batch the 8 MiB array takes (one 32-limb polynomial of
    2^16 u32 words) bit for bit against ntt_forward and sampled oracle
    values; one more polynomial is rejected."""
    N = 1 << 16
    qs = nt.ntt_find_primes(30, 17, 32)
    plan = nt.ntt_plan_create(N, qs, nt.NTT_STOCKHAM, 0)
    try:
        for call in range(2):
            host = ntt_synth.rns_batch(500 + call, qs, N, 1)
            ref = _dev(host, False)
            got = _dev(host, False)
            nt.ntt_forward(plan, ref, 1)
            nt.ntt_forward_noalloc(plan, got, 1)        # exactly 8 MiB: accepted
            torch.cuda.synchronize()
            assert torch.equal(ref, got), "call %d differs from ntt_forward" % call
            t, k = ntt_synth.sample_indices(500 + call, 32, N, 64)
            psis = [orc.psi(q, N) for q in qs]
            vals = orc.ntt_batch_at(host, qs, psis, t, k)
            gh = _host(got, False, (32, N))
            assert np.array_equal(gh[t.astype(int), k.astype(int)], vals)
        d = torch.zeros(2 * 32 * N, dtype=torch.int32, device="cuda")
        with pytest.raises(nt.NttError) as e:
            nt.ntt_forward_noalloc(plan, d, 2)          # 16 MiB: rejected
        assert e.value.status == nt.NTT_ERR_SCRATCH_LIMIT
        torch.cuda.synchronize()
    finally:
        nt.ntt_plan_destroy(plan)


def test_noalloc_rejects_fused_plans_and_serves_tensor_core_plans(nt):
    """Fused plans with N >= 16 have no per-stage tables and are rejected;
    tensor-core four-step plans carry them and give ntt_forward's result,
    in both output orders."""
    d = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
    fused = nt.ntt_plan_create(1024, [12289], nt.NTT_FUSED, 0)
    try:
        with pytest.raises(nt.NttError) as e:
            nt.ntt_forward_noalloc(fused, d, 1)
        assert e.value.status == nt.NTT_ERR_UNSUPPORTED
    finally:
        nt.ntt_plan_destroy(fused)
    N = 1 << 16
    qs = nt.ntt_find_primes(30, 17, 2)
    host = ntt_synth.rns_batch(41, qs, N, 1)
    for flags in (0, nt.NTT_ORDER_BITREV):
        plan = nt.ntt_plan_create(N, qs, nt.NTT_TC_FOURSTEP, flags)
        try:
            ref = _dev(host, False)
            got = _dev(host, False)
            nt.ntt_forward(plan, ref, 1)
            nt.ntt_forward_noalloc(plan, got, 1)
            torch.cuda.synchronize()
            assert torch.equal(ref, got), "flags %#x" % flags
        finally:
            nt.ntt_plan_destroy(plan)


def test_noalloc_reports_input_range_under_check(nt):
    """NTT_CHECK: an input word >= q is recorded in the plan's status word,
    as ntt_forward records it; in-range input leaves the status clear."""
    N, L = 1 << 10, 2
    qs = nt.ntt_find_primes(30, 17, L)
    plan = nt.ntt_plan_create(N, qs, nt.NTT_STOCKHAM, nt.NTT_CHECK)
    try:
        host = ntt_synth.rns_batch(9, qs, N, 2)
        d = _dev(host, False)
        nt.ntt_forward_noalloc(plan, d, 2)
        assert nt.ntt_plan_last_launches(plan) == 1 + 1 + 10    # range check, twist, 10 stages
        assert nt.ntt_get_device_status(plan) == nt.NTT_OK
        host[1, 1, 123] = qs[1]                  # one word equal to its prime
        d = _dev(host, False)
        nt.ntt_forward_noalloc(plan, d, 2)
        assert nt.ntt_get_device_status(plan) == nt.NTT_ERR_INPUT_RANGE
        assert nt.ntt_get_device_status(plan) == nt.NTT_OK      # read and cleared
    finally:
        nt.ntt_plan_destroy(plan)


def test_noalloc_leaves_free_memory_unchanged(nt):
    """A call does not change the device's free memory, while a regular
    ntt_forward on a fresh plan of the same shape (which grows its scratch
    buffer) visibly does -- so the check can see an allocation."""
    N, L, batch = 1 << 16, 32, 1
    qs = nt.ntt_find_primes(30, 17, L)
    host = ntt_synth.rns_batch(31, qs, N, batch)
    plan = nt.ntt_plan_create(N, qs, nt.NTT_STOCKHAM, 0)
    try:
        d = _dev(host, False)
        nt.ntt_forward_noalloc(plan, d, batch)   # first call on the device: symbol lookup
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(3):
            nt.ntt_forward_noalloc(plan, d, batch)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, "free memory changed by %d bytes" % (free0 - free1)
        big = torch.zeros(4 * L * N, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free2, _ = torch.cuda.mem_get_info()
        nt.ntt_forward(plan, big, 4)             # grows the plan's scratch to 32 MiB
        torch.cuda.synchronize()
        free3, _ = torch.cuda.mem_get_info()
        assert free2 - free3 >= 32 << 20, "a 32 MiB scratch allocation was not visible"
    finally:
        nt.ntt_plan_destroy(plan)
