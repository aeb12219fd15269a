"""Python binding of libnttgb (batched negacyclic NTT for GB300, sm_103a).

Argument marshalling only: every function forwards to the C entry point of
the same name in ``libnttgb.so`` (declared in ``include/ntt.h``); all
arithmetic runs in the library's CUDA kernels.  Data arguments may be torch
tensors (their ``data_ptr()`` is passed) or integer addresses; stream
arguments may be a ``torch.cuda.Stream``, an integer handle or ``None``
(the current torch stream when torch is initialised, else the legacy
stream).  A non-OK status raises ``NttError``.

The library must have been built (``python -m paper_2405_11353_gb300.build``
or ``__graft_entry__.build()``); importing this package without it raises.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnttgb.so")

# ------------------------------------------------------------- constants
NTT_OK = 0
STATUS_NAMES = {
    0: "NTT_OK", 1: "NTT_ERR_INVALID_ARG", 2: "NTT_ERR_N_NOT_POW2",
    3: "NTT_ERR_N_RANGE", 4: "NTT_ERR_Q_NOT_PRIME", 5: "NTT_ERR_Q_NOT_NTT_FRIENDLY",
    6: "NTT_ERR_Q_WIDTH", 7: "NTT_ERR_ALIGNMENT", 8: "NTT_ERR_CUDA", 9: "NTT_ERR_OOM",
    10: "NTT_ERR_INPUT_RANGE", 11: "NTT_ERR_TIMEOUT", 12: "NTT_ERR_UNSUPPORTED",
    13: "NTT_ERR_PSI", 14: "NTT_ERR_SCRATCH_LIMIT",
}
for _v, _n in STATUS_NAMES.items():
    globals()[_n] = _v

NTT_DIT, NTT_DIF, NTT_FLAT, NTT_PEASE, NTT_PEASE_NC, NTT_STOCKHAM, NTT_SIXSTEP, \
    NTT_FUSED, NTT_TC_FOURSTEP = range(9)
VARIANTS = {"dit": NTT_DIT, "dif": NTT_DIF, "flat": NTT_FLAT, "pease": NTT_PEASE,
            "pease_nc": NTT_PEASE_NC, "stockham": NTT_STOCKHAM, "sixstep": NTT_SIXSTEP,
            "fused": NTT_FUSED, "tc_fourstep": NTT_TC_FOURSTEP}

NTT_WORD64 = 0x1
NTT_ORDER_BITREV = 0x2
NTT_RED_SHOUP = 0x00
NTT_RED_BARRETT = 0x10
NTT_RED_MONTGOMERY = 0x20
NTT_RED_MASK = 0x30
NTT_CHECK = 0x100
NTT_CLUSTER = 0x200
NTT_STREAMED = 0x400
NTT_TC_IMMA = 0x800
NTT_RAGGED_TUNE = 0x1000
NTT_TW_OTF = 0x2000
NTT_TEST_STALL = 0x8000
REDUCTIONS = {"shoup": NTT_RED_SHOUP, "barrett": NTT_RED_BARRETT,
              "montgomery": NTT_RED_MONTGOMERY}

# every symbol include/ntt.h declares
EXPORTS = [
    "ntt_plan_create", "ntt_plan_create_ex", "ntt_plan_destroy", "ntt_plan_reserve",
    "ntt_forward", "ntt_inverse", "ntt_pointwise_mul", "ntt_polymul_host",
    "ntt_get_device_status", "ntt_plan_get_psi", "ntt_plan_last_launches",
    "ntt_status_string", "ntt_validate", "ntt_default_psi", "ntt_find_primes",
    "ntt_ragged_create", "ntt_ragged_launch", "ntt_ragged_status", "ntt_ragged_destroy",
    "ntt_forward_noalloc", "ntt_forward_prefix", "ntt_inverse_prefix", "ntt_pointwise_inverse",
    "ntt_bconv_create", "ntt_bconv", "ntt_bconv_destroy", "ntt_measure_int_mad_rate",
    "ntt_autotune", "ntt_plan_form", "ntt_tune_set", "ntt_tune_get", "ntt_tune_clear",
    "ntt_ragged_item_tiles", "ntt_plan_table_bytes", "ntt_limb_shard",
    "ntt_tune_set_split", "ntt_tune_get_split", "ntt_plan_chunk_log2", "ntt_plan_radix_log2",
]


class NttError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__("%s: %s" % (where, STATUS_NAMES.get(status, status)))


class NttJob(ctypes.Structure):
    _fields_ = [("d_data", ctypes.c_void_p), ("q", ctypes.POINTER(ctypes.c_uint64)),
                ("N", ctypes.c_uint32), ("L", ctypes.c_uint32), ("batch", ctypes.c_uint32),
                ("word64", ctypes.c_uint32), ("inverse", ctypes.c_int32),
                ("reserved", ctypes.c_uint32)]


class NttTuneResult(ctypes.Structure):
    _fields_ = [("forward_ms", ctypes.c_float * 5), ("inverse_ms", ctypes.c_float * 5),
                ("forward_form", ctypes.c_int32), ("inverse_form", ctypes.c_int32),
                ("chunk_log2", ctypes.c_int32), ("radix_log2", ctypes.c_int32),
                ("config_ms", (ctypes.c_float * 3) * 2)]


NTT_FORM_SMALL, NTT_FORM_WIDE, NTT_FORM_STREAMED, NTT_FORM_SMALL_SHFL, NTT_FORM_WIDE_SHFL = 0, 1, 2, 3, 4
FORMS = {"small": NTT_FORM_SMALL, "wide": NTT_FORM_WIDE, "streamed": NTT_FORM_STREAMED,
         "small_shfl": NTT_FORM_SMALL_SHFL, "wide_shfl": NTT_FORM_WIDE_SHFL}

_lib = None


def lib():
    """The loaded library (ctypes.CDLL); raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libnttgb.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, u32, u64, st = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        u64p = ctypes.POINTER(ctypes.c_uint64)
        sig = {
            "ntt_plan_create": (st, [ctypes.POINTER(vp), u32, u64p, u32, st, u32]),
            "ntt_plan_create_ex": (st, [ctypes.POINTER(vp), u32, u64p, u32, st, u32, u64p]),
            "ntt_plan_destroy": (None, [vp]),
            "ntt_plan_reserve": (st, [vp, u32, vp]),
            "ntt_forward": (st, [vp, vp, u32, vp]),
            "ntt_inverse": (st, [vp, vp, u32, vp]),
            "ntt_pointwise_mul": (st, [vp, vp, vp, vp, u32, vp]),
            "ntt_pointwise_inverse": (st, [vp, vp, vp, vp, u32, vp]),
            "ntt_polymul_host": (st, [vp, vp, vp, vp, u32, vp]),
            "ntt_get_device_status": (st, [vp, vp]),
            "ntt_plan_get_psi": (st, [vp, u64p]),
            "ntt_plan_last_launches": (u32, [vp]),
            "ntt_plan_table_bytes": (u64, [vp]),
            "ntt_status_string": (ctypes.c_char_p, [st]),
            "ntt_validate": (st, [u32, u64p, u32, u32]),
            "ntt_default_psi": (st, [u64, u32, u64p]),
            "ntt_find_primes": (st, [u32, u32, u32, u64p]),
            "ntt_ragged_create": (st, [ctypes.POINTER(vp), ctypes.POINTER(NttJob), u32, u32]),
            "ntt_ragged_launch": (st, [vp, vp]),
            "ntt_ragged_status": (st, [vp, vp]),
            "ntt_ragged_destroy": (None, [vp]),
            "ntt_forward_noalloc": (st, [vp, vp, u32, vp]),
            "ntt_forward_prefix": (st, [vp, vp, u32, u32, vp]),
            "ntt_inverse_prefix": (st, [vp, vp, u32, u32, vp]),
            "ntt_bconv_create": (st, [ctypes.POINTER(vp), u64p, u32, u64p, u32, u32]),
            "ntt_bconv": (st, [vp, vp, vp, u32, vp]),
            "ntt_bconv_destroy": (None, [vp]),
            "ntt_measure_int_mad_rate": (st, [ctypes.c_int, u32, vp, ctypes.c_size_t, ctypes.POINTER(u32), vp]),
            "ntt_autotune": (st, [u32, u64p, u32, u32, u32, vp, ctypes.POINTER(NttTuneResult)]),
            "ntt_plan_form": (ctypes.c_int32, [vp, u32, ctypes.c_int]),
            "ntt_tune_set": (st, [u32, u32, u32, u32, ctypes.c_int32, ctypes.c_int32]),
            "ntt_tune_get": (ctypes.c_int32, [u32, u32, u32, u32, ctypes.c_int]),
            "ntt_tune_clear": (None, []),
            "ntt_ragged_item_tiles": (u32, [vp]),
            "ntt_limb_shard": (st, [u32, u32, u32, ctypes.POINTER(u32), ctypes.POINTER(u32)]),
            "ntt_tune_set_split": (st, [u32, u32, u32, u32, u32]),
            "ntt_tune_get_split": (ctypes.c_int32, [u32, u32, u32, ctypes.POINTER(ctypes.c_int32)]),
            "ntt_plan_chunk_log2": (ctypes.c_int32, [vp]),
            "ntt_plan_radix_log2": (ctypes.c_int32, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):          # numpy array (host buffers)
        return x.ctypes.data
    raise TypeError("expected a tensor, array or integer address, got %r" % type(x))


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status, where):
    if status != NTT_OK:
        raise NttError(status, where)


def _u64arr(vals):
    vals = [int(v) for v in vals]
    return (ctypes.c_uint64 * len(vals))(*vals)


# ------------------------------------------------------------ entry points
def ntt_plan_create(N, q, variant=NTT_FUSED, flags=0, psi=None):
    """Returns a plan handle (int).  q: sequence of L primes."""
    h = ctypes.c_void_p()
    qa = _u64arr(q)
    if psi is None:
        s = lib().ntt_plan_create(ctypes.byref(h), N, qa, len(q), variant, flags)
    else:
        s = lib().ntt_plan_create_ex(ctypes.byref(h), N, qa, len(q), variant, flags, _u64arr(psi))
    _check(s, "ntt_plan_create")
    return h.value


def ntt_plan_destroy(plan):
    lib().ntt_plan_destroy(plan)


def ntt_plan_reserve(plan, max_batch, stream=None):
    _check(lib().ntt_plan_reserve(plan, max_batch, _stream(stream)), "ntt_plan_reserve")


def ntt_forward(plan, data, batch, stream=None):
    _check(lib().ntt_forward(plan, _ptr(data), batch, _stream(stream)), "ntt_forward")


def ntt_inverse(plan, data, batch, stream=None):
    _check(lib().ntt_inverse(plan, _ptr(data), batch, _stream(stream)), "ntt_inverse")


def ntt_forward_prefix(plan, data, batch, limbs, stream=None):
    _check(lib().ntt_forward_prefix(plan, _ptr(data), batch, limbs, _stream(stream)),
           "ntt_forward_prefix")


def ntt_inverse_prefix(plan, data, batch, limbs, stream=None):
    _check(lib().ntt_inverse_prefix(plan, _ptr(data), batch, limbs, _stream(stream)),
           "ntt_inverse_prefix")


def ntt_pointwise_mul(plan, c, a, b, batch, stream=None):
    _check(lib().ntt_pointwise_mul(plan, _ptr(c), _ptr(a), _ptr(b), batch, _stream(stream)),
           "ntt_pointwise_mul")


def ntt_pointwise_inverse(plan, c, a, b, batch, stream=None):
    _check(lib().ntt_pointwise_inverse(plan, _ptr(c), _ptr(a), _ptr(b), batch, _stream(stream)),
           "ntt_pointwise_inverse")


def ntt_polymul_host(plan, h_out, h_in, d_work, pairs, stream=None):
    _check(lib().ntt_polymul_host(plan, _ptr(h_out), _ptr(h_in), _ptr(d_work), pairs,
                                  _stream(stream)), "ntt_polymul_host")


def ntt_get_device_status(plan, stream=None):
    """Returns the raw status code (does not raise)."""
    return lib().ntt_get_device_status(plan, _stream(stream))


def ntt_plan_get_psi(plan, L):
    out = (ctypes.c_uint64 * L)()
    _check(lib().ntt_plan_get_psi(plan, out), "ntt_plan_get_psi")
    return [int(v) for v in out]


def ntt_plan_last_launches(plan):
    return int(lib().ntt_plan_last_launches(plan))


def ntt_plan_table_bytes(plan):
    return int(lib().ntt_plan_table_bytes(plan))


def ntt_status_string(status):
    return lib().ntt_status_string(status).decode()


def ntt_validate(N, q, flags=0):
    """Returns the raw status code of the host-side checks (no GPU used)."""
    return lib().ntt_validate(N, _u64arr(q), len(q), flags)


def ntt_default_psi(q, N):
    out = ctypes.c_uint64()
    _check(lib().ntt_default_psi(q, N, ctypes.byref(out)), "ntt_default_psi")
    return int(out.value)


def ntt_find_primes(bits, m, count):
    out = (ctypes.c_uint64 * count)()
    _check(lib().ntt_find_primes(bits, m, count, out), "ntt_find_primes")
    return [int(v) for v in out]


def ntt_limb_shard(L, world, rank):
    """(first, count): the contiguous slice of the L limbs that `rank` of
    `world` holds (host-only)."""
    f, c = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().ntt_limb_shard(L, world, rank, ctypes.byref(f), ctypes.byref(c)), "ntt_limb_shard")
    return int(f.value), int(c.value)


def ntt_forward_noalloc(plan, data, batch, stream=None):
    """Forward transform that allocates nothing (fixed 8 MiB scratch array in
    the library), for callers that must not allocate device memory."""
    _check(lib().ntt_forward_noalloc(plan, _ptr(data), batch, _stream(stream)),
           "ntt_forward_noalloc")


def ntt_ragged_create(jobs, flags=0):
    """jobs: list of dicts with data, q, N, batch, word64, inverse."""
    arr = (NttJob * len(jobs))()
    keep = []
    for i, j in enumerate(jobs):
        qa = _u64arr(j["q"])
        keep.append(qa)
        arr[i].d_data = _ptr(j["data"])
        arr[i].q = ctypes.cast(qa, ctypes.POINTER(ctypes.c_uint64))
        arr[i].N = j["N"]
        arr[i].L = len(j["q"])
        arr[i].batch = j.get("batch", 1)
        arr[i].word64 = 1 if j.get("word64") else 0
        arr[i].inverse = 1 if j.get("inverse") else 0
    h = ctypes.c_void_p()
    _check(lib().ntt_ragged_create(ctypes.byref(h), arr, len(jobs), flags), "ntt_ragged_create")
    return h.value


def ntt_ragged_launch(r, stream=None):
    _check(lib().ntt_ragged_launch(r, _stream(stream)), "ntt_ragged_launch")


def ntt_ragged_status(r, stream=None):
    return lib().ntt_ragged_status(r, _stream(stream))


def ntt_ragged_destroy(r):
    lib().ntt_ragged_destroy(r)


def ntt_bconv_create(q, p, N):
    """Fast RNS base conversion plan from primes q (L) to primes p (K) for
    polynomials of N coefficients; returns a handle (int)."""
    h = ctypes.c_void_p()
    _check(lib().ntt_bconv_create(ctypes.byref(h), _u64arr(q), len(q), _u64arr(p), len(p), N),
           "ntt_bconv_create")
    return h.value


def ntt_bconv(plan, out, inp, batch, stream=None):
    _check(lib().ntt_bconv(plan, _ptr(out), _ptr(inp), batch, _stream(stream)), "ntt_bconv")


def ntt_bconv_destroy(plan):
    lib().ntt_bconv_destroy(plan)


def ntt_measure_int_mad_rate(high, iters, scratch, stream=None):
    """Launch the integer multiply-add rate kernel; returns the operation
    count of the launch (the caller times it)."""
    blocks = ctypes.c_uint32()
    nbytes = scratch.numel() * scratch.element_size()
    _check(lib().ntt_measure_int_mad_rate(1 if high else 0, iters, _ptr(scratch), nbytes, ctypes.byref(blocks),
                                          _stream(stream)), "ntt_measure_int_mad_rate")
    return blocks.value * 256 * 8 * iters


def ntt_autotune(N, q, flags, batch, stream=None):
    """Time every two-pass radix, split and form for this shape, record
    the fastest; returns {"forward_ms": [...], "inverse_ms": [...] (per form,
    at the chosen radix and split), "forward_form", "inverse_form",
    "chunk_log2", "radix_log2" (the chosen split and radix), "config_ms":
    {"radix_log2,chunk_log2": fastest forward + inverse ms, for the valid
    pairs}}."""
    r = NttTuneResult()
    _check(lib().ntt_autotune(N, _u64arr(q), len(q), flags, batch, _stream(stream), ctypes.byref(r)),
           "ntt_autotune")
    return {"forward_ms": list(r.forward_ms), "inverse_ms": list(r.inverse_ms),
            "forward_form": r.forward_form, "inverse_form": r.inverse_form,
            "chunk_log2": r.chunk_log2, "radix_log2": r.radix_log2,
            "config_ms": {"%d,%d" % (3 + i, 7 + j): r.config_ms[i][j] for i in range(2) for j in range(3)
                          if r.config_ms[i][j] >= 0}}


def ntt_plan_form(plan, batch, inverse=False):
    return lib().ntt_plan_form(plan, batch, 1 if inverse else 0)


def ntt_tune_set(N, L, flags, batch, forward_form, inverse_form):
    _check(lib().ntt_tune_set(N, L, flags, batch, forward_form, inverse_form), "ntt_tune_set")


def ntt_tune_get(N, L, flags, batch, inverse=False):
    return lib().ntt_tune_get(N, L, flags, batch, 1 if inverse else 0)


def ntt_tune_set_split(N, L, flags, chunk_log2, radix_log2=4):
    _check(lib().ntt_tune_set_split(N, L, flags, chunk_log2, radix_log2), "ntt_tune_set_split")


def ntt_tune_get_split(N, L, flags):
    """(chunk_log2, radix_log2) recorded for the shape, or (-1, -1)."""
    r = ctypes.c_int32()
    s = lib().ntt_tune_get_split(N, L, flags, ctypes.byref(r))
    return int(s), int(r.value)


def ntt_plan_chunk_log2(plan):
    return lib().ntt_plan_chunk_log2(plan)


def ntt_plan_radix_log2(plan):
    return lib().ntt_plan_radix_log2(plan)


def ntt_tune_clear():
    lib().ntt_tune_clear()


def ntt_ragged_item_tiles(r):
    return lib().ntt_ragged_item_tiles(r)
