"""The sampled O(N^2) check used by the GPU parity tests, exercised on the
CPU: it accepts the oracle's own O(N log N) output (natural and bit-reversed
order, forward and inverse) and rejects an output with one wrong value."""
import numpy as np
import pytest

import ntt_synth
from parity_helpers import bitrev_positions, check_definition_samples


def test_bitrev_positions():
    assert bitrev_positions(np.arange(8), 3).tolist() == [0, 4, 2, 6, 1, 5, 3, 7]
    assert bitrev_positions([1, 2 ** 15], 16).tolist() == [2 ** 15, 1]


@pytest.mark.parametrize("bitrev", [False, True])
def test_samples_accept_oracle_and_reject_a_planted_error(orc, bitrev):
    N = 1 << 10
    qs = orc.find_primes(30, 12, 3)
    psis = [orc.psi(q, N) for q in qs]
    a = ntt_synth.rns_batch(5, qs, N, 2)
    X = orc.ntt_batch(a, qs, psis)
    got = X
    if bitrev:
        got = np.stack([np.stack([orc.bitrev_permute(X[b, l]) for l in range(3)]) for b in range(2)])
    assert check_definition_samples(orc, a, qs, psis, got, 9, per=N, bitrev=bitrev) == 6 * N
    assert check_definition_samples(orc, X, qs, psis, a, 10, per=64, inverse=True) == 6 * 64
    # one transform wrong by one in every coefficient (a sampled check
    # cannot miss it: every transform gets `per` samples)
    bad = got.copy()
    bad[1, 2] = (bad[1, 2] + 1) % qs[2]
    with pytest.raises(AssertionError):
        check_definition_samples(orc, a, qs, psis, bad, 9, per=N, bitrev=bitrev)
