"""CPU oracle for the batched negacyclic NTT -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library never imports it, and it imports nothing from the product.

The arithmetic lives in ``ntt_oracle.c`` (plain C, 128-bit ``%`` for every
modular operation).  This module compiles it with gcc on first use and wraps
it with ctypes.  See the header of ``ntt_oracle.c`` for the passages of the
paper each function follows and for the conventions (generator, psi, output
order, prime list).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ntt_oracle.c")
_LIB = os.path.join(_HERE, "libntt_oracle.so")
_lock = threading.Lock()
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force=False):
    """Compile the oracle shared library with gcc (OpenMP over transforms)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            u64 = ctypes.c_uint64
            sig = {
                "orc_mulmod": (u64, [u64, u64, u64]),
                "orc_addmod": (u64, [u64, u64, u64]),
                "orc_submod": (u64, [u64, u64, u64]),
                "orc_powmod": (u64, [u64, u64, u64]),
                "orc_invmod": (u64, [u64, u64]),
                "orc_is_prime": (ctypes.c_int, [u64]),
                "orc_prime_factors": (ctypes.c_int, [u64, _u64p, ctypes.c_int]),
                "orc_generator": (u64, [u64]),
                "orc_psi": (u64, [u64, u64]),
                "orc_find_primes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, _u64p]),
                "orc_ntt_fwd_at": (u64, [u64, u64, u64, _u64p, u64]),
                "orc_ntt_inv_at": (u64, [u64, u64, u64, _u64p, u64]),
                "orc_ntt_fwd_naive": (None, [u64, u64, u64, _u64p, _u64p]),
                "orc_ntt_inv_naive": (None, [u64, u64, u64, _u64p, _u64p]),
                "orc_ntt_fwd_fast": (None, [u64, u64, u64, _u64p, _u64p]),
                "orc_ntt_inv_fast": (None, [u64, u64, u64, _u64p, _u64p]),
                "orc_negacyclic_mul": (None, [u64, u64, _u64p, _u64p, _u64p]),
                "orc_pointwise": (None, [u64, u64, _u64p, _u64p, _u64p]),
                "orc_negacyclic_mul_at": (u64, [u64, u64, _u64p, _u64p, u64]),
                "orc_bitrev_permute": (None, [u64, _u64p, _u64p]),
                "orc_ntt_batch": (None, [ctypes.c_int, ctypes.c_int, u64,
                                         ctypes.c_uint32, ctypes.c_uint32,
                                         _u64p, _u64p, _u64p, _u64p]),
                "orc_ntt_batch_at": (None, [ctypes.c_int, u64, ctypes.c_uint32,
                                            _u64p, _u64p, _u64p, u64, _u64p,
                                            _u64p, _u64p]),
                "orc_pointwise_batch": (None, [u64, ctypes.c_uint32,
                                               ctypes.c_uint32, _u64p, _u64p,
                                               _u64p, _u64p]),
                "orc_base_conv": (None, [ctypes.c_uint32, _u64p, ctypes.c_uint32,
                                         _u64p, u64, ctypes.c_uint32, _u64p, _u64p]),
                "orc_num_threads": (ctypes.c_int, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(arr):
    assert arr.dtype == np.uint64 and arr.flags.c_contiguous
    return arr.ctypes.data_as(_u64p)


def _u64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint64))


# ------------------------------------------------------------ scalar helpers
def mulmod(a, b, q):
    return lib().orc_mulmod(a, b, q)


def powmod(b, e, q):
    return lib().orc_powmod(b, e, q)


def is_prime(n):
    return bool(lib().orc_is_prime(n))


def prime_factors(n):
    buf = np.zeros(64, dtype=np.uint64)
    c = lib().orc_prime_factors(n, _p(buf), 64)
    return [int(v) for v in buf[:c]]


def generator(q):
    return int(lib().orc_generator(q))


def psi(q, N):
    return int(lib().orc_psi(q, N))


def find_primes(bits, m, count):
    buf = np.zeros(count, dtype=np.uint64)
    c = lib().orc_find_primes(bits, m, count, _p(buf))
    if c != count:
        raise ValueError("only %d primes of %d bits = 1 mod 2^%d" % (c, bits, m))
    return [int(v) for v in buf]


def num_threads():
    return int(lib().orc_num_threads())


# ---------------------------------------------------------- single transforms
def ntt_fwd(a, q, psi_, fast=False):
    a = _u64(a)
    out = np.zeros_like(a)
    f = lib().orc_ntt_fwd_fast if fast else lib().orc_ntt_fwd_naive
    f(q, psi_, a.size, _p(a), _p(out))
    return out


def ntt_inv(X, q, psi_, fast=False):
    X = _u64(X)
    out = np.zeros_like(X)
    f = lib().orc_ntt_inv_fast if fast else lib().orc_ntt_inv_naive
    f(q, psi_, X.size, _p(X), _p(out))
    return out


def ntt_fwd_at(a, q, psi_, k):
    a = _u64(a)
    return int(lib().orc_ntt_fwd_at(q, psi_, a.size, _p(a), k))


def ntt_inv_at(X, q, psi_, n):
    X = _u64(X)
    return int(lib().orc_ntt_inv_at(q, psi_, X.size, _p(X), n))


def negacyclic_mul(a, b, q):
    a = _u64(a)
    b = _u64(b)
    c = np.zeros_like(a)
    lib().orc_negacyclic_mul(q, a.size, _p(a), _p(b), _p(c))
    return c


def negacyclic_mul_at(a, b, q, j):
    a = _u64(a)
    b = _u64(b)
    return int(lib().orc_negacyclic_mul_at(q, a.size, _p(a), _p(b), j))


def pointwise(a, b, q):
    a = _u64(a)
    b = _u64(b)
    c = np.zeros_like(a)
    lib().orc_pointwise(q, a.size, _p(a), _p(b), _p(c))
    return c


def bitrev_permute(x):
    x = _u64(x)
    out = np.zeros_like(x)
    lib().orc_bitrev_permute(x.size, _p(x), _p(out))
    return out


# ------------------------------------------------------------------- batches
def ntt_batch(data, qs, psis, inverse=False, fast=True):
    """data: [batch][L][N] (any integer dtype) -> uint64 result, same shape."""
    d = _u64(data)
    B, L, N = d.shape
    q = _u64(qs)
    p = _u64(psis)
    assert q.size == L and p.size == L
    out = np.zeros_like(d)
    lib().orc_ntt_batch(1 if inverse else 0, 1 if fast else 0, N, L, B,
                        _p(q), _p(p), _p(d), _p(out))
    return out


def ntt_batch_at(data, qs, psis, t_idx, k_idx, inverse=False):
    """Sampled outputs: value k_idx[i] of transform t_idx[i] (t = b*L + l)."""
    d = _u64(data)
    B, L, N = d.shape
    q = _u64(qs)
    p = _u64(psis)
    t = _u64(t_idx)
    k = _u64(k_idx)
    out = np.zeros(t.size, dtype=np.uint64)
    lib().orc_ntt_batch_at(1 if inverse else 0, N, L, _p(q), _p(p), _p(d),
                           t.size, _p(t), _p(k), _p(out))
    return out


def pointwise_batch(a, b, qs):
    a = _u64(a)
    b = _u64(b)
    B, L, N = a.shape
    q = _u64(qs)
    c = np.zeros_like(a)
    lib().orc_pointwise_batch(N, L, B, _p(q), _p(a), _p(b), _p(c))
    return c


def base_conv(data, qs, ps):
    """Fast RNS base conversion of [batch][L][N] residues modulo qs to
    [batch][K][N] residues modulo ps (see orc_base_conv)."""
    d = _u64(data)
    B, L, N = d.shape
    q = _u64(qs)
    p = _u64(ps)
    assert q.size == L
    out = np.zeros((B, p.size, N), dtype=np.uint64)
    lib().orc_base_conv(L, _p(q), p.size, _p(p), N, B, _p(d), _p(out))
    return out
