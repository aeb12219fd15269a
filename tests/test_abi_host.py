"""C-ABI checks that need no GPU: the library loads, exports every symbol
include/ntt.h declares, and its host-side validation and number theory agree
with the oracle."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nt():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2405_11353_gb300 as nt
    return nt


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ntt_[a-z0-9_]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(nt):
    declared = _declared()
    assert len(declared) >= 15
    lib = nt.lib()
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert declared == set(nt.EXPORTS)


def test_validation_codes(nt):
    v = nt.ntt_validate
    assert v(1024, [12289]) == nt.NTT_OK
    assert v(1000, [12289]) == nt.NTT_ERR_N_NOT_POW2
    assert v(0, [12289]) == nt.NTT_ERR_N_NOT_POW2
    assert v(1, [12289]) == nt.NTT_ERR_N_RANGE
    assert v(1 << 18, [(1 << 30) - 2 ** 19 + 1]) == nt.NTT_ERR_N_RANGE
    assert v(1024, [12287]) == nt.NTT_ERR_Q_NOT_PRIME          # 11 * 1117
    assert v(1024, [12289, 12287]) == nt.NTT_ERR_Q_NOT_PRIME
    assert v(4096, [12289]) == nt.NTT_ERR_Q_NOT_NTT_FRIENDLY   # 8192 does not divide 12288
    assert v(1024, [(1 << 30) + 1]) == nt.NTT_ERR_Q_WIDTH     # above the u32 limit
    q60 = 1152921504606830593
    assert v(1024, [q60]) == nt.NTT_ERR_Q_WIDTH
    assert v(1024, [q60], nt.NTT_WORD64) == nt.NTT_OK
    assert v(1024, [(1 << 61) - 1], nt.NTT_WORD64) == nt.NTT_ERR_Q_WIDTH
    assert v(1024, [12289], 0x40000) == nt.NTT_ERR_INVALID_ARG
    assert v(1024, [12289], nt.NTT_RED_MASK) == nt.NTT_ERR_INVALID_ARG
    assert v(1024, []) == nt.NTT_ERR_INVALID_ARG


def test_plan_create_rejects_before_touching_cuda(nt):
    with pytest.raises(nt.NttError) as e:
        nt.ntt_plan_create(1000, [12289])
    assert e.value.status == nt.NTT_ERR_N_NOT_POW2
    with pytest.raises(nt.NttError) as e:
        nt.ntt_plan_create(1024, [12289], variant=42)
    assert e.value.status == nt.NTT_ERR_INVALID_ARG
    with pytest.raises(nt.NttError) as e:
        nt.ntt_plan_create(1024, [12289], psi=[2])
    assert e.value.status == nt.NTT_ERR_PSI


def test_entry_points_reject_null(nt):
    lib = nt.lib()
    assert lib.ntt_forward(None, None, 1, None) == nt.NTT_ERR_INVALID_ARG
    assert lib.ntt_inverse(None, None, 1, None) == nt.NTT_ERR_INVALID_ARG
    assert lib.ntt_pointwise_mul(None, None, None, None, 1, None) == nt.NTT_ERR_INVALID_ARG
    assert lib.ntt_get_device_status(None, None) == nt.NTT_ERR_INVALID_ARG
    assert lib.ntt_plan_last_launches(None) == 0
    lib.ntt_plan_destroy(None)


def test_status_strings(nt):
    for code, name in nt.STATUS_NAMES.items():
        assert nt.ntt_status_string(code).startswith(name)


@pytest.mark.parametrize("bits,m,count", [(30, 15, 8), (60, 17, 24), (30, 17, 32),
                                          (30, 18, 32), (60, 18, 32)])
def test_primes_match_oracle(nt, orc, bits, m, count):
    assert nt.ntt_find_primes(bits, m, count) == orc.find_primes(bits, m, count)


def test_default_psi_matches_oracle(nt, orc):
    cases = [(12289, 1024), (17, 4), (5, 2), (7681, 256)]
    cases += [(q, 1 << 14) for q in orc.find_primes(30, 15, 8)]
    cases += [(q, 1 << 16) for q in orc.find_primes(60, 17, 6)]
    cases += [(q, 1 << 17) for q in orc.find_primes(60, 18, 4)]
    for q, N in cases:
        assert nt.ntt_default_psi(q, N) == orc.psi(q, N), (q, N)


def test_otf_flag_combinations_rejected_before_touching_cuda(nt):
    """NTT_TW_OTF needs the fused variant, 4-byte words, Shoup twiddles and
    the two-launch forms."""
    q = 1073479681   # 30-bit, 1 mod 2^18
    q60 = 1152921504606830593
    for N, qs, variant, flags in [(1 << 16, [q], nt.NTT_DIT, 0),
                                  (1024, [q60], nt.NTT_FUSED, nt.NTT_WORD64),
                                  (1 << 16, [q], nt.NTT_FUSED, nt.NTT_RED_BARRETT),
                                  (1 << 16, [q], nt.NTT_FUSED, nt.NTT_RED_MONTGOMERY),
                                  (1 << 16, [q], nt.NTT_FUSED, nt.NTT_STREAMED),
                                  (1 << 16, [q], nt.NTT_TC_FOURSTEP, 0)]:
        with pytest.raises(nt.NttError) as e:
            nt.ntt_plan_create(N, qs, variant, flags | nt.NTT_TW_OTF)
        assert e.value.status == nt.NTT_ERR_UNSUPPORTED, (variant, flags)
