"""The N > 1 path of bench.py, on CPU: one process per rank over gloo.

Every transform is independent, so ranks run replicas with no data-path
collective; the only cross-rank step is the max-over-ranks of the timings
(and, in the reference arm, ranks other than 0 exit without work)."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    slowest = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    rate = bench.job_rate(768, world, 100, slowest)
    q.put((rank, slowest, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in res:
        assert slowest == 20.0
        assert rate == pytest.approx(768 * 2 * 100 / 0.020)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(10, 1, 5, 1000.0) == 50.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


# ------------------------------------------------------------ limb sharding
def _shard_worker(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import ntt_synth
    import oracle
    import paper_2405_11353_gb300 as nt
    from paper_2405_11353_gb300.shard import gather_limbs
    out = []
    for L, N, B in ((7, 64, 3), (2, 16, 1), (9, 32, 2)):
        qs = oracle.find_primes(30, 12, L)
        psis = [oracle.psi(p, N) for p in qs]
        full = ntt_synth.rns_batch(1234 + L, qs, N, B)        # the whole job (same on every rank)
        first, cnt = nt.ntt_limb_shard(L, world, rank)
        local = np.ascontiguousarray(full[:, first:first + cnt])   # this rank's limbs
        # the rank's transforms over its own primes (the oracle stands in
        # for the GPU kernels on this host)
        X = oracle.ntt_batch(local, qs[first:first + cnt], psis[first:first + cnt])
        t = torch.from_numpy(X.view(np.int64).reshape(-1).copy())
        g = gather_limbs(t, B, L, N).numpy().view(np.uint64)
        want = oracle.ntt_batch(full, qs, psis)
        out.append((L, first, cnt, bool(np.array_equal(g, want)), g.shape))
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_limb_sharding_gather_gloo_world2():
    """Two ranks each transform their slice of the limbs (7, 2 and 9 limbs:
    uneven and minimal splits); the all-gather restores [batch][L][N] in
    limb order on both ranks, equal to the transform of the whole job."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for (L, f0, c0, ok0, shape0), (L1, f1, c1, ok1, shape1) in zip(res[0], res[1]):
        assert L == L1 and f0 == 0 and f1 == c0 and c0 + c1 == L and c0 - c1 in (0, 1)
        assert ok0 and ok1 and shape0 == shape1 and shape0[1] == L


def test_limb_shard_partition_host():
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2405_11353_gb300 as nt
    for L in (1, 2, 7, 32, 33, 256):
        for world in range(1, min(L, 9) + 1):
            spans = [nt.ntt_limb_shard(L, world, r) for r in range(world)]
            assert spans[0][0] == 0
            for (f, c), (f2, _) in zip(spans, spans[1:]):
                assert f + c == f2 and c >= 1
            assert sum(c for _, c in spans) == L
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    for bad in ((4, 0, 0), (4, 2, 2), (3, 4, 0)):
        with pytest.raises(nt.NttError) as e:
            nt.ntt_limb_shard(*bad)
        assert e.value.status == 1          # NTT_ERR_INVALID_ARG
