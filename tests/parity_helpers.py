"""Sampled checks against the O(N^2) definition (Eq. 3 with the negacyclic
twist), shared by the GPU parity tests.  Expected values come only from the
oracle; the sample positions from ntt_synth's seeded generator."""
import numpy as np

import ntt_synth


def bitrev_positions(k, bits):
    """bitrev_bits(k) for an array of indices."""
    k = np.asarray(k, dtype=np.uint64)
    r = np.zeros_like(k)
    for i in range(bits):
        r |= ((k >> np.uint64(i)) & np.uint64(1)) << np.uint64(bits - 1 - i)
    return r


def check_definition_samples(orc, inp, qs, psis, got, seed, per=256, bitrev=False, inverse=False):
    """`per` coefficients of every transform of `got` ([batch][L][N], the
    library's output for input `inp`) against the O(N^2) oracle: forward
    X[k] = sum_n a[n] psi^((2k+1) n), or the inverse a[n]; with bitrev the
    library's position p holds X[bitrev(p)] (forward outputs only).  Returns
    the number of values checked."""
    B, L, N = inp.shape
    T = B * L
    n = ntt_synth.log2(N)
    t_idx = np.repeat(np.arange(T, dtype=np.uint64), per)
    _, k_idx = ntt_synth.sample_indices(seed, 1, N, T * per)
    vals = orc.ntt_batch_at(inp, qs, psis, t_idx, k_idx, inverse=inverse)
    pos = bitrev_positions(k_idx, n) if bitrev else k_idx
    flat = np.asarray(got).reshape(T, N)
    sel = flat[t_idx.astype(np.int64), pos.astype(np.int64)].astype(np.uint64)
    bad = np.nonzero(sel != vals)[0]
    assert bad.size == 0, "definition mismatch at transform %d coefficient %d: %d != %d" % (
        int(t_idx[bad[0]]), int(k_idx[bad[0]]), int(sel[bad[0]]), int(vals[bad[0]]))
    return int(vals.size)
