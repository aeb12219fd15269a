"""Limb sharding across processes, one GPU each.

Each rank transforms its contiguous slice of the RNS limbs (ntt_limb_shard)
with a plan over those limbs' primes; nothing is exchanged on the transform
path.  gather_limbs is the one exchange: an all-gather that restores
[batch][L][N] on every rank before a step that reads all limbs of a
coefficient (the RNS base conversion, ntt_bconv).  The collective is
torch.distributed's (NCCL between GPUs, gloo on the host); no library kernel
touches another rank's memory.
"""
from . import ntt_limb_shard


def gather_limbs(local, batch, L, N, group=None):
    """All-gather of limb slices.

    local: this rank's [batch][count][N] words (a torch tensor of any
    integer dtype, flat or shaped), count from ntt_limb_shard(L, world,
    rank).  Returns a [batch][L][N] tensor of the same dtype and device on
    every rank, limbs in rank order.  Slices are padded to the largest count
    so that every rank sends the same number of words."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    shards = [ntt_limb_shard(L, world, r) for r in range(world)]
    first, count = shards[rank]
    cmax = max(c for _, c in shards)
    x = local.reshape(batch, count, N)
    buf = torch.zeros((batch, cmax, N), dtype=x.dtype, device=x.device)
    buf[:, :count] = x
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([parts[r][:, :c] for r, (_, c) in enumerate(shards)], dim=1)
