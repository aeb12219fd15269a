"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This module holds no arithmetic of the transform: it draws random numbers,
describes workload shapes and nothing else.  Both the CUDA path and the CPU
oracle receive the same arrays from here.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): state advances by the odd constant
0x9E3779B97F4A7C15 and each output is the state passed through the
variant-13 finaliser.  The i-th output of a stream seeded with s is therefore
mix(s + (i + 1) * gamma), which numpy evaluates for many i at once.

Residues uniform in [0, q): each draw keeps its top bit_length(q) bits and is
rejected when >= q (acceptance > 1/2); the accepted draws, in stream order,
are the coefficients.

Per-(polynomial, limb) stream seed: seed XOR (poly * 2^20 + limb), with
seed = 1000 + workload index (C1..C5 -> 1001..1005).
"""
import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed, count, start=0):
    """Outputs start .. start+count-1 of the SplitMix64 stream seeded `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GAMMA)


def uniform_residues(seed, q, n):
    """n values uniform in [0, q) drawn from one SplitMix64 stream."""
    bits = int(q).bit_length()
    shift = np.uint64(64 - bits)
    qq = np.uint64(q)
    out = np.empty(0, dtype=np.uint64)
    start = 0
    while out.size < n:
        need = n - out.size
        block = int(need * 2.2) + 64
        cand = splitmix64(seed, block, start) >> shift
        start += block
        out = np.concatenate([out, cand[cand < qq][:need]])
    return out


def stream_seed(seed, poly, limb):
    return (int(seed) ^ (int(poly) * (1 << 20) + int(limb))) & 0xFFFFFFFFFFFFFFFF


def rns_batch(seed, qs, N, batch, dtype=np.uint64):
    """[batch][L][N] residues, limb l uniform in [0, qs[l])."""
    L = len(qs)
    out = np.empty((batch, L, N), dtype=dtype)
    for p in range(batch):
        for l, q in enumerate(qs):
            out[p, l] = uniform_residues(stream_seed(seed, p, l), q, N)
    return out


# ----------------------------------------------------------- workload shapes
# (sizes only; prime lists come from the oracle in tests and from the
# library's own prime search in bench.py, and a test checks they agree)
WORKLOADS = {
    "C1": dict(seed=1001, N=1 << 10, L=1, bits=None, fixed_q=12289, m=None,
               batch=64, word=32,
               desc="plain NTT, 7 variants: N=1024, q=12289, u32, 64 polys"),
    "C2": dict(seed=1002, N=1 << 14, L=8, bits=30, m=15, batch=128, word=32,
               desc="RNS batch: N=2^14, L=8 30-bit primes = 1 mod 2^15, u32, "
                    "128 polys (64 two-poly ciphertexts)"),
    "C3": dict(seed=1003, N=1 << 16, L=24, bits=60, m=17, batch=8, word=64,
               desc="wide-word: N=2^16, L=24 60-bit primes = 1 mod 2^17, u64, "
                    "8 polys"),
    "C4": dict(seed=1004, jobs=512, logN=(12, 17), L=(1, 32), m=18,
               desc="ragged: 512 polys, N log-uniform 2^12..2^17, L uniform "
                    "1..32, half 30-bit / half 60-bit primes = 1 mod 2^18"),
    "C5": dict(seed=1005, N=1 << 16, L=32, bits=30, m=17, batch=16, word=32,
               desc="tensor-core form: N=2^16, L=32 30-bit primes = 1 mod "
                    "2^17, u32, 16 polys"),
}


def ragged_jobs(seed=1004, jobs=512, logN=(12, 17), Lrange=(1, 32)):
    """Descriptors of the ragged workload: list of dicts with logN, L, word.

    Job j draws logN uniform in logN[0]..logN[1] and L uniform in
    Lrange[0]..Lrange[1] from one SplitMix64 stream (two draws per job,
    reduced by rejection like the residues); even jobs use 30-bit primes
    (u32 words), odd jobs 60-bit primes (u64 words)."""
    nN = logN[1] - logN[0] + 1
    nL = Lrange[1] - Lrange[0] + 1
    a = uniform_residues(seed, nN, jobs)
    b = uniform_residues(seed ^ 0x5A5A5A5A, nL, jobs)
    out = []
    for j in range(jobs):
        out.append(dict(logN=logN[0] + int(a[j]), L=Lrange[0] + int(b[j]),
                        word=32 if j % 2 == 0 else 64))
    return out


def sample_indices(seed, total, N, count):
    """`count` (transform, coefficient) index pairs for sampled checks."""
    t = splitmix64(seed ^ 0x77, count) % np.uint64(total)
    k = splitmix64(seed ^ 0x99, count) % np.uint64(N)
    return t.astype(np.uint64), k.astype(np.uint64)


def log2(n):
    v = int(math.log2(n))
    assert (1 << v) == n
    return v
