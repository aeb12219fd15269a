"""ntt_forward_noalloc: the forward transform for callers that must not
allocate device memory (a framework owning every byte through its own pool,
a loop that cannot take cudaMalloc's implicit synchronisation, a plugin under
a fixed budget).  It must give exactly what ntt_forward gives on the same
plan, call after call, while its fixed scratch array keeps the previous
call's contents.  Collected last (file name) so a failure here never hides
the other tests."""
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


@pytest.mark.parametrize("w64,bitrev,variant", [(False, False, "stockham"), (True, True, "pease"),
                                                (False, True, "dit")])
def test_noalloc_matches_ntt_forward_twice(nt, w64, bitrev, variant):
    N, L, batch = 1 << 12, 3, 4
    qs = nt.ntt_find_primes(60 if w64 else 30, 17, L)
    flags = (nt.NTT_WORD64 if w64 else 0) | (nt.NTT_ORDER_BITREV if bitrev else 0)
    plan = nt.ntt_plan_create(N, qs, nt.VARIANTS[variant], flags)
    try:
        for call in range(2):                     # two calls in a row
            host = ntt_synth.rns_batch(77 + call, qs, N, batch)
            ref = _dev(host, w64)
            got = _dev(host, w64)
            nt.ntt_forward(plan, ref, batch)
            nt.ntt_forward_noalloc(plan, got, batch)
            torch.cuda.synchronize()
            assert torch.equal(ref, got), "call %d differs" % call
    finally:
        nt.ntt_plan_destroy(plan)


def test_noalloc_rejects_oversized_batches(nt):
    N = 1 << 16
    qs = nt.ntt_find_primes(30, 17, 32)
    plan = nt.ntt_plan_create(N, qs, nt.NTT_STOCKHAM, 0)
    try:
        d = torch.zeros(2 * 32 * N, dtype=torch.int32, device="cuda")
        nt.ntt_forward_noalloc(plan, d, 1)        # exactly 8 MiB: accepted
        with pytest.raises(nt.NttError) as e:
            nt.ntt_forward_noalloc(plan, d, 2)    # 16 MiB: rejected
        assert e.value.status == nt.NTT_ERR_SCRATCH_LIMIT
        torch.cuda.synchronize()
    finally:
        nt.ntt_plan_destroy(plan)
    fused = nt.ntt_plan_create(1024, [12289], nt.NTT_FUSED, 0)
    try:
        d = torch.zeros(1024, dtype=torch.int32, device="cuda")
        with pytest.raises(nt.NttError) as e:
            nt.ntt_forward_noalloc(fused, d, 1)
        assert e.value.status == nt.NTT_ERR_UNSUPPORTED
    finally:
        nt.ntt_plan_destroy(fused)
