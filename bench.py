"""Batched negacyclic NTT throughput on one GB300 (or N, one process each).

Workload (one step): 16 polynomials of N = 2^16 coefficients, L = 32 RNS
limbs modulo 30-bit primes q = 1 mod 2^17 (u32 words): forward NTT of all 16
(ntt_forward), then pointwise product of the 8 pairs and inverse NTT of the 8
products (ntt_pointwise_inverse: the product is taken inside the first
inverse pass) -- 768 transforms per step.  Fused butterfly path, Shoup
reduction, bit-reversed evaluation order.  Inputs are seeded synthetic residues (no dataset exists
for this method); four copies of the batch rotate so every step reads a
working set (4 x 128 MiB) larger than L2.

Several GPUs (torchrun, one process each): the limbs are sharded -- the job
is 16 polynomials of 32 x world limbs and each rank transforms its own 32
(ntt_limb_shard); no data moves between ranks in the step.

Output: detail lines for the side measurements, then one JSON line (rank
0, printed last).  `value` is NTTs per second for the whole job, from K
steps run back to back; `roofline` describes the forward transform (the
dominant call), timed by events around each call in a second run of the
same K steps; `cpu_baseline` times the CPU oracle on a bounded sample;
`e2e` is the same metric through ntt_polymul_host with pinned host buffers;
`side` closes the line with the side measurements' headline figures.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import itertools
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ntt_synth  # noqa: E402

METRIC = "batched NTT throughput (NTTs/s, GB/s vs HBM peak) at N=2^16; ragged vs plain"
N, L, POLYS, BITS, M = 1 << 16, 32, 16, 30, 17
PAIRS = POLYS // 2
WORD = 4
NTT_PER_STEP = (POLYS + PAIRS) * L
ROTATE = 4
WORKLOAD = ("N=2^16, L=32 primes q<2^30 (q=1 mod 2^17), u32, 16 polys: forward NTT x16, "
            "pointwise x8 fused with inverse NTT x8 per step")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def tensor_peak():
    """Dense bf16 tensor-core peak (burst) in TFLOP/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


# measured 32-bit multiply-add rates (filled by measure_int_mad_rate)
_MAD_RATES = {}


def traffic_from_profiles(digest):
    """Per-launch DRAM bytes of the forward transform from the committed ncu
    figures (profiles/fused_forward_n65536_L32_u32.traffic.txt: `key: value`
    lines), if they were taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "fused_forward_n65536_L32_u32.traffic.txt")
    vals = {}
    try:
        for line in open(p):
            line = line.split("#", 1)[0].strip()
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    except OSError:
        return None
    if vals.get("source_digest") != digest:
        return None
    try:
        return int(vals["forward_dram_bytes_per_call"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, parts in rows:
            for i, n in enumerate(names):
                if parts[5 + i].lower() == "active":
                    reasons.add(n)
        load = [r[0] for r in rows]
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def max_over_ranks(x, dist=None, device=None):
    """The largest of each rank's x (timings are taken as the slowest rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_step_per_rank, world, steps, elapsed_ms):
    """Whole-job throughput: units every rank processed / the slowest time."""
    return units_per_step_per_rank * world * steps / (elapsed_ms / 1000.0)


# ----------------------------------------------------------------- oracle arm
def oracle_sample(qs, seconds=12.0, max_reps=200):
    """The CPU oracle (O(N log N) path, OpenMP over transforms) running the
    step's pipeline on one pair of polynomials x all limbs, repeated for
    about `seconds`.  Returns (NTTs/s, threads, description)."""
    import oracle
    psis = [oracle.psi(q, N) for q in qs]
    host = ntt_synth.rns_batch(1005, qs, N, 2)
    done = 0
    t0 = time.perf_counter()
    reps = 0
    while reps < max_reps:
        A = oracle.ntt_batch(host, qs, psis)
        P = oracle.pointwise_batch(A[:1], A[1:], qs)
        oracle.ntt_batch(P, qs, psis, inverse=True)
        done += 3 * L
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    desc = ("oracle O(N log N) path: forward of 2 polys, pointwise, inverse of 1 product, "
            "x %d limbs, %d repetitions (%d NTTs in %.1f s)" % (L, reps, done, dt))
    return done / dt, oracle.num_threads(), desc


def oracle_naive_n1024(polys=256):
    """For the record: the oracle's O(N^2) definition (Horner at each
    psi^(2k+1)) on `polys` transforms at N = 1024, q = 12289.  (One
    transform at N = 2^16 would be 4.3e9 modular products, minutes of CPU;
    it is not timed.)"""
    import oracle
    q = 12289
    psi = oracle.psi(q, 1024)
    host = ntt_synth.rns_batch(1001, [q], 1024, polys)
    t0 = time.perf_counter()
    oracle.ntt_batch(host, [q], [psi], fast=False)
    dt = time.perf_counter() - t0
    return {"value": polys / dt, "unit": "NTT/s",
            "sample": "oracle O(N^2) forward, N=1024, q=12289, %d transforms in %.2f s" % (polys, dt)}


def oracle_naive_n65536():
    """For the record: the oracle's O(N^2) definition on one transform at
    N = 2^16 (q < 2^30): all 2^16 outputs, each a Horner evaluation at
    psi^(2k+1) (2^32 modular steps), spread over the host cores."""
    import oracle
    q = oracle.find_primes(BITS, M, 1)[0]
    n = 1 << 16
    psi = oracle.psi(q, n)
    host = ntt_synth.rns_batch(1005, [q], n, 1)
    k = np.arange(n, dtype=np.uint64)
    t0 = time.perf_counter()
    oracle.ntt_batch_at(host, [q], [psi], np.zeros(n, dtype=np.uint64), k)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "NTT/s", "seconds_per_transform": dt, "cores": oracle.num_threads(),
            "sample": "oracle O(N^2) forward, N=2^16, one transform (2^32 Horner steps)"}


def _sig(x, n=4):
    """x rounded to n significant digits (compact JSON)."""
    if isinstance(x, float):
        return float("%.*g" % (n, x))
    return x


def _pick(d, *path):
    for k in path:
        if not isinstance(d, dict) or k not in d:
            return None
        d = d[k]
    return _sig(d)


def side_summary(extras):
    """The side measurements' headline figures, compact, for the main line."""
    g = lambda *p: _pick(extras, *p)  # noqa: E731
    out = {}
    if "ragged" in extras:
        out["ragged"] = {"ntt_s": g("ragged", "value"), "ms": g("ragged", "ms_per_step"),
                         "transforms": g("ragged", "transforms_per_step"),
                         "plain_ms": g("ragged", "plain_ms_per_step"),
                         "speedup_vs_plain": g("ragged", "speedup_vs_plain"),
                         "hbm_frac": g("ragged", "roofline", "frac"), "status": g("ragged", "device_status"),
                         "item_tiles": g("ragged", "item_tiles_autotuned")}
    if "tc_fourstep" in extras:
        out["tc_fourstep"] = {"tcgen05_ms": g("tc_fourstep", "tensor_core", "ms_per_call"),
                              "mma_sync_ms": g("tc_fourstep", "tensor_core_mma_sync", "ms_per_call"),
                              "butterfly_ms": g("tc_fourstep", "butterfly", "ms_per_call"),
                              "tcgen05_over_butterfly": g("tc_fourstep", "tensor_core", "ratio_to_butterfly"),
                              "tensor_frac": g("tc_fourstep", "tensor_core", "roofline", "frac")}
    if "wide_word_u64" in extras:
        out["wide_word_u64"] = {"shoup_ms": g("wide_word_u64", "shoup", "ms_per_step"),
                                "montgomery_ms": g("wide_word_u64", "montgomery", "ms_per_step"),
                                "barrett_ms": g("wide_word_u64", "barrett", "ms_per_step"),
                                "shoup_int_frac": g("wide_word_u64", "shoup", "int_roofline", "frac"),
                                "shoup_hbm_frac": g("wide_word_u64", "shoup", "roofline", "frac"),
                                "montgomery_int_frac": g("wide_word_u64", "montgomery", "int_roofline", "frac")}
    if "rns_n2p14" in extras:
        out["rns_n2p14"] = {"ms": g("rns_n2p14", "ms_per_step"), "ntt_s": g("rns_n2p14", "value")}
    if "variants_n1024" in extras:
        ms = [(k, v.get("ms_per_step")) for k, v in extras["variants_n1024"].items() if isinstance(v, dict)]
        ms = [(k, m) for k, m in ms if m]
        if ms:
            out["variants_n1024_ms_min_max"] = [_sig(min(m for _, m in ms)), _sig(max(m for _, m in ms))]
    if "cluster_form" in extras:
        out["forward_ms_by_form"] = {k: _sig(v.get("forward_ms")) for k, v in extras["cluster_form"].items()
                                     if isinstance(v, dict)}
    errors = [k for k, v in extras.items() if isinstance(v, dict) and "error" in v]
    if errors:
        out["errors"] = errors
    return out


def run_reference(args):
    """The oracle as the reference arm: each step is the step's pipeline on
    one pair of polynomials x all 32 limbs (96 NTTs).  When K such steps
    would take more than about a minute, only the first ones that fit are
    timed (reported as timed_steps)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    qs = oracle.find_primes(BITS, M, L)
    t0 = time.perf_counter()
    for _ in range(args.warmup):
        oracle_sample(qs, seconds=0.0, max_reps=1)
    est = (time.perf_counter() - t0) / max(1, args.warmup)
    timed = max(1, min(args.steps, int(60.0 / max(est, 1e-3))))
    t0 = time.perf_counter()
    v, cores, desc = oracle_sample(qs, seconds=1e9, max_reps=timed)
    total = time.perf_counter() - t0
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "NTT/s",
        "n_gpus": args.gpus, "steps": args.steps, "timed_steps": timed, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total / timed, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64 (128-bit % per product)",
        "data": "synthetic (seeded SplitMix64 residues)",
        "config": {"workload": WORKLOAD, "N": N, "L": L, "polys": POLYS, "word": "u32",
                   "sample": "each step: 1 pair x 32 limbs (96 NTTs)"},
        "cpu_baseline": {"value": v, "unit": "NTT/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": v, "unit": "NTT/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ side workloads
def _time_loop(torch, stream, fn, reps, warm=3):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_int_mad_rate(nt, torch, dev, stream, iters=4096, reps=5):
    """32-bit integer multiply-add rates (mad.lo, mad.hi) over all SMs."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    scratch = torch.empty(sms * 8 * 256, dtype=torch.int32, device=dev)
    sh = stream.cuda_stream
    rates = []
    for high in (False, True):
        for _ in range(2):
            nt.ntt_measure_int_mad_rate(high, iters, scratch, sh)
        ms = _time_loop(torch, stream, lambda: nt.ntt_measure_int_mad_rate(high, iters, scratch, sh), reps, warm=0)
        ops = sms * 8 * 256 * 8 * iters
        rates.append(ops / (ms / 1e3))
    _MAD_RATES["lo"], _MAD_RATES["hi"] = rates[0], rates[1]
    return rates[0], rates[1]



def ragged_vs_plain(nt, torch, dev, reps=10):
    """The 512-polynomial ragged workload (N = 2^12..2^17 log-uniform, L =
    1..32, half 30-bit / half 60-bit primes = 1 mod 2^18): forward + inverse
    of every job in one graph launch, against the same jobs through the
    per-plan API (one plan per (N, word size), ntt_*_prefix per job)."""
    specs = ntt_synth.ragged_jobs(seed=1004, jobs=512)
    plist = {32: nt.ntt_find_primes(30, 18, 32), 64: nt.ntt_find_primes(60, 18, 32)}
    bufs, jobs = [], []
    bytes_total, ntt_total = 0, 0
    for i, sp in enumerate(specs):
        qs = plist[sp["word"]][:sp["L"]]
        N = 1 << sp["logN"]
        h = ntt_synth.rns_batch(ntt_synth.stream_seed(1004, i, 99), qs, N, 1,
                                dtype=np.uint32 if sp["word"] == 32 else np.uint64)
        t = torch.from_numpy(h.view(np.int32 if sp["word"] == 32 else np.int64).reshape(-1).copy()).to(dev)
        bufs.append(t)
        jobs.append(dict(data=t, q=qs, N=N, batch=1, word64=sp["word"] == 64, inverse=False))
        bytes_total += N * sp["L"] * sp["word"] // 8
        ntt_total += sp["L"]
    flags = nt.NTT_ORDER_BITREV | nt.NTT_RED_SHOUP
    # the work-item size is autotuned at creation (on scratch copies)
    r = nt.ntt_ragged_create(jobs + [dict(j, inverse=True) for j in jobs], flags | nt.NTT_RAGGED_TUNE)
    item_tiles = nt.ntt_ragged_item_tiles(r)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    try:
        ms_r = _time_loop(torch, stream, lambda: nt.ntt_ragged_launch(r, sh), reps)
        status = nt.ntt_ragged_status(r, sh)
    finally:
        nt.ntt_ragged_destroy(r)
    plans = {}
    for sp in specs:
        key = (sp["logN"], sp["word"])
        if key not in plans:
            plans[key] = nt.ntt_plan_create(1 << sp["logN"], plist[sp["word"]], nt.NTT_FUSED,
                                            flags | (nt.NTT_WORD64 if sp["word"] == 64 else 0))

    def plain():
        for sp, t in zip(specs, bufs):
            p = plans[(sp["logN"], sp["word"])]
            nt.ntt_forward_prefix(p, t, 1, sp["L"], sh)
            nt.ntt_inverse_prefix(p, t, 1, sp["L"], sh)
    try:
        ms_p = _time_loop(torch, stream, plain, max(2, reps // 2))
    finally:
        for p in plans.values():
            nt.ntt_plan_destroy(p)
    n_step = 2 * ntt_total
    # forward + inverse, each reads and writes the data once, plus each
    # (N, word) group's twiddle pairs (its longest prime list) once per direction
    group_l = {}
    for sp in specs:
        key = (sp["logN"], sp["word"])
        group_l[key] = max(group_l.get(key, 0), sp["L"])
    table_bytes = sum((1 << n) * l * 2 * (w // 8) for (n, w), l in group_l.items())
    bytes_step = 2 * (2 * bytes_total + table_bytes)
    peak, peak_kind = peaks()
    gbs = bytes_step / (ms_r / 1e3) / 1e9
    return {"workload": "512 polys, N=2^12..2^17, L=1..32, half u32/half u64; forward+inverse",
            "transforms_per_step": n_step, "value": n_step / (ms_r / 1e3), "unit": "NTT/s",
            "ms_per_step": ms_r, "algorithmic_gbs": gbs,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "algorithmic_bytes_per_launch": bytes_step,
                         "peak_source": "%s hbm_gbs" % peak_kind},
            "plain_value": n_step / (ms_p / 1e3), "plain_ms_per_step": ms_p,
            "speedup_vs_plain": ms_p / ms_r, "device_status": status, "item_tiles_autotuned": item_tiles,
            "note": "ragged = one graph-captured cooperative launch; plain = ntt_forward_prefix/"
                    "ntt_inverse_prefix per job on shared (N, word) plans"}


def wide_word(nt, torch, dev, reps=50):
    """N = 2^16, 24 primes q < 2^60 (= 1 mod 2^17), u64, 8 polys: forward +
    inverse, Montgomery and Shoup."""
    qs = nt.ntt_find_primes(60, 17, 24)
    N, B = 1 << 16, 8
    host = ntt_synth.rns_batch(1003, qs, N, B, dtype=np.uint64)
    d = torch.from_numpy(host.view(np.int64).reshape(-1).copy()).to(dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    out = {"workload": "N=2^16, L=24 primes q<2^60, u64, 8 polys: forward + inverse"}
    for red in ("montgomery", "shoup", "barrett"):
        p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED,
                               nt.NTT_WORD64 | nt.NTT_ORDER_BITREV | nt.REDUCTIONS[red])
        try:
            def step():
                nt.ntt_forward(p, d, B, sh)
                nt.ntt_inverse(p, d, B, sh)
            ms = _time_loop(torch, stream, step, reps)
        finally:
            nt.ntt_plan_destroy(p)
        out[red] = {"value": 2 * B * 24 / (ms / 1e3), "unit": "NTT/s", "ms_per_step": ms}
    # HBM: forward + inverse of 192 transforms (data read + written once per
    # direction) + 24 limbs x N twiddle pairs of 16 bytes per direction
    peak, peak_kind = peaks()
    byts = 2 * (2 * N * 8 * B * 24 + 24 * N * 16)
    # integer multiply pipe: a 64 x 64-bit product from 32-bit multiplies:
    # low half 3 mul.lo + 1 mul.hi, high half 4 mul.lo + 4 mul.hi; per
    # butterfly Shoup takes one high and two low halves (10 lo + 6 hi),
    # Montgomery one low and two high halves (11 lo + 9 hi)
    bfly = 2 * B * 24 * (N // 2) * 16
    lo_rate, hi_rate = _MAD_RATES.get("lo"), _MAD_RATES.get("hi")
    for red, (nlo, nhi) in (("shoup", (10, 6)), ("montgomery", (11, 9))):
        ms = out[red]["ms_per_step"]
        gbs = byts / (ms / 1e3) / 1e9
        out[red]["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                                "peak_source": "%s hbm_gbs" % peak_kind}
        if lo_rate and hi_rate:
            t_min = bfly * (nlo / lo_rate + nhi / hi_rate)
            out[red]["int_roofline"] = {
                "bound": "alu", "frac": t_min / (ms / 1e3), "unit": "32-bit multiplies",
                "multiplies_per_butterfly": {"mad.lo": nlo, "mad.hi": nhi},
                "floor_ms": t_min * 1e3,
                "peak_source": "measured mad.lo %.2f T/s, mad.hi %.2f T/s" % (lo_rate / 1e12, hi_rate / 1e12)}
    return out


def tc_fourstep(nt, torch, dev, reps=20):
    """N = 2^16, 32 primes q < 2^30, u32, 16 polys: the forward transform as
    the tensor-core four-step form (8-bit digit products on tcgen05, and on
    the warp-level mma.sync u8 -> s32) against the butterfly form on the
    same data."""
    qs = nt.ntt_find_primes(30, 17, 32)
    N, B = 1 << 16, 16
    host = ntt_synth.rns_batch(1005, qs, N, B, dtype=np.uint32)
    d = torch.from_numpy(host.view(np.int32).reshape(-1).copy()).to(dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    out = {"workload": "N=2^16, L=32 primes q<2^30, u32, 16 polys: forward transform"}
    macs = 2 * 2 * 256 * 256 * 256 * 16 * B * 32 / 2   # 2 passes x 256^3 per transform x 16 digit pairs
    for name, variant, extra in (("tensor_core", nt.NTT_TC_FOURSTEP, 0),
                                 ("tensor_core_mma_sync", nt.NTT_TC_FOURSTEP, nt.NTT_TC_IMMA),
                                 ("butterfly", nt.NTT_FUSED, 0)):
        p = nt.ntt_plan_create(N, qs, variant, nt.NTT_ORDER_BITREV | extra)
        try:
            ms = _time_loop(torch, stream, lambda: nt.ntt_forward(p, d, B, sh), reps)
        finally:
            nt.ntt_plan_destroy(p)
        out[name] = {"value": B * 32 / (ms / 1e3), "unit": "NTT/s", "ms_per_call": ms}
    for name in ("tensor_core", "tensor_core_mma_sync"):
        out[name]["digit_tops"] = macs * 2 / (out[name]["ms_per_call"] / 1e3) / 1e12
    tp, tp_kind = tensor_peak()
    out["tensor_core"]["roofline"] = {
        "bound": "tensor", "achieved": out["tensor_core"]["digit_tops"], "peak": tp, "unit": "TFLOP/s",
        "frac": out["tensor_core"]["digit_tops"] / tp,
        "peak_source": "%s bf16_tflops (fp16 MMA, the kind used, runs at the bf16 rate)" % tp_kind}
    out["tensor_core"]["ratio_to_butterfly"] = out["tensor_core"]["ms_per_call"] / out["butterfly"]["ms_per_call"]
    out["tensor_core"]["instruction"] = "tcgen05.mma kind::f16 (balanced 8-bit digits, fp32 diagonals in TMEM)"
    out["tensor_core_mma_sync"]["instruction"] = "mma.sync m16n8k32 u8.u8.s32"
    return out


def variants_n1024(nt, torch, dev, reps=50):
    """The paper's comparison of dataflow variants on the N = 1024, q = 12289,
    64-polynomial workload: forward + inverse per variant (the per-stage
    variant kernels, and the fused path)."""
    N, B, qs = 1024, 64, [12289]
    host = ntt_synth.rns_batch(1001, qs, N, B, dtype=np.uint32)
    d = torch.from_numpy(host.view(np.int32).reshape(-1).copy()).to(dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    out = {"workload": "N=1024, q=12289, u32, 64 polys: forward + inverse (128 transforms)"}
    for name in ("dit", "dif", "flat", "pease", "pease_nc", "stockham", "sixstep", "fused"):
        p = nt.ntt_plan_create(N, qs, nt.VARIANTS[name], 0)
        try:
            nt.ntt_plan_reserve(p, B, sh)

            def step():
                nt.ntt_forward(p, d, B, sh)
                nt.ntt_inverse(p, d, B, sh)
            ms = _time_loop(torch, stream, step, reps)
        finally:
            nt.ntt_plan_destroy(p)
        out[name] = {"ms_per_step": ms, "value": 2 * B / (ms / 1e3), "unit": "NTT/s"}
    return out


def rns_n2p14(nt, torch, dev, reps=50):
    """N = 2^14, 8 primes q < 2^30 (= 1 mod 2^15), 128 polynomials: forward
    of all 128, 64 pointwise products fused into the inverse (single-pass
    fused kernels)."""
    qs = nt.ntt_find_primes(30, 15, 8)
    N, B = 1 << 14, 128
    host = ntt_synth.rns_batch(1002, qs, N, B, dtype=np.uint32)
    d = torch.from_numpy(host.view(np.int32).reshape(-1).copy()).to(dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    half = (B // 2) * 8 * N
    p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, nt.NTT_ORDER_BITREV)
    try:
        def step():
            nt.ntt_forward(p, d, B, sh)
            nt.ntt_pointwise_inverse(p, d, d, d[half:], B // 2, sh)
        ms = _time_loop(torch, stream, step, reps)
    finally:
        nt.ntt_plan_destroy(p)
    n = (B + B // 2) * 8
    return {"workload": "N=2^14, L=8, u32, 128 polys: forward x128, pointwise x64 + inverse x64",
            "ms_per_step": ms, "value": n / (ms / 1e3), "unit": "NTT/s"}


def tune_step_inverse_form(nt, torch, dev, N, qs, flags, inv_tuning, reps=50):
    """Time the step (forward of POLYS polynomials, then the product +
    inverse of PAIRS pairs, back to back) with each inverse form the
    autotuner found valid for the product batch; record the fastest in the
    tuning table.  Returns {form name: ms per step}."""
    names = {v: k for k, v in nt.FORMS.items()}
    fwd_form = inv_tuning["forward_form"]
    L = len(qs)
    half = PAIRS * L * N
    bufs = [torch.zeros(POLYS * L * N, dtype=torch.int32, device=dev) for _ in range(ROTATE)]
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    out = {}
    for form, ms in enumerate(inv_tuning["inverse_ms"]):
        if ms <= 0:
            continue
        nt.ntt_tune_set(N, L, flags, PAIRS, fwd_form, form)
        p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, flags)
        try:
            def step(b):
                nt.ntt_forward(p, b, POLYS, sh)
                nt.ntt_pointwise_inverse(p, b, b, b[half:], PAIRS, sh)
            turn = itertools.count()
            out[names[form]] = _time_loop(torch, stream, lambda: step(bufs[next(turn) % ROTATE]), reps)
        finally:
            nt.ntt_plan_destroy(p)
    best = min(out, key=out.get)
    nt.ntt_tune_set(N, L, flags, PAIRS, fwd_form, nt.FORMS[best])
    del bufs
    return out


def autotune_shapes(nt, torch, dev):
    """The autotuner on other two-pass shapes: which form wins per
    direction (0: one-warp chunk CTAs, 1: 16-chunk CTAs, 2: streamed)."""
    sh = torch.cuda.current_stream(dev).cuda_stream
    out = {}
    for name, n, w64, L, batch in (("u32_n2p15_L8_b32", 15, False, 8, 32), ("u32_n2p16_L32_b2", 16, False, 32, 2),
                                   ("u32_n2p17_L16_b8", 17, False, 16, 8), ("u64_n2p16_L24_b8", 16, True, 24, 8),
                                   ("u64_n2p14_L8_b64", 14, True, 8, 64)):
        qs = nt.ntt_find_primes(60 if w64 else 30, 18, L)
        flags = nt.NTT_ORDER_BITREV | (nt.NTT_WORD64 if w64 else 0)
        out[name] = nt.ntt_autotune(1 << n, qs, flags, batch, sh)
    nt.ntt_tune_clear()
    return out


def base_conv(nt, torch, dev, reps=50):
    """Fast RNS base conversion (ntt_bconv) of 8 polynomials, N = 2^16,
    from 32 primes q < 2^30 to 32 other primes: L x K = 1024 multiply-adds
    mod p per coefficient, on the integer pipes."""
    qs = nt.ntt_find_primes(30, 17, 32)
    ps = nt.ntt_find_primes(29, 17, 32)
    N, B, L, K = 1 << 16, 8, 32, 32
    host = ntt_synth.rns_batch(1006, qs, N, B, dtype=np.uint32)
    x = torch.from_numpy(host.view(np.int32).reshape(-1).copy()).to(dev)
    z = torch.empty(B * K * N, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    h = nt.ntt_bconv_create(qs, ps, N)
    try:
        ms = _time_loop(torch, stream, lambda: nt.ntt_bconv(h, z, x, B, sh), reps)
    finally:
        nt.ntt_bconv_destroy(h)
    coeffs = B * N
    byts = coeffs * (L + K) * 4
    return {"workload": "N=2^16, 8 polys, 32 primes q<2^30 -> 32 primes p<2^29",
            "ms_per_call": ms, "coefficients_per_s": coeffs / (ms / 1e3),
            "algorithmic_gbs": byts / (ms / 1e3) / 1e9,
            "mod_mults_per_s": coeffs * L * K / (ms / 1e3)}


def cluster_form(nt, torch, dev, reps=50):
    """N = 2^16, 32 primes q < 2^30, u32, 16 polys: forward and inverse as
    the two-pass split in two launches (default), in one streamed launch
    (NTT_STREAMED), and as one pass on eight-CTA clusters (NTT_CLUSTER),
    which reads and writes each word once."""
    qs = nt.ntt_find_primes(30, 17, 32)
    N, B = 1 << 16, 16
    host = ntt_synth.rns_batch(1005, qs, N, B, dtype=np.uint32)
    d = torch.from_numpy(host.view(np.int32).reshape(-1).copy()).to(dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    out = {"workload": "N=2^16, L=32 primes q<2^30, u32, 16 polys: forward, inverse"}
    for name, extra in (("two_pass_two_launches", 0), ("two_pass_one_streamed_launch", nt.NTT_STREAMED),
                        ("cluster_one_pass", nt.NTT_CLUSTER)):
        p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, nt.NTT_ORDER_BITREV | extra)
        try:
            ms_f = _time_loop(torch, stream, lambda: nt.ntt_forward(p, d, B, sh), reps)
            ms_i = _time_loop(torch, stream, lambda: nt.ntt_inverse(p, d, B, sh), reps)
        finally:
            nt.ntt_plan_destroy(p)
        out[name] = {"forward_ms": ms_f, "inverse_ms": ms_i,
                     "forward_value": B * 32 / (ms_f / 1e3), "unit": "NTT/s"}
    return out


def tw_otf(nt, torch, dev, reps=50):
    """The chunk-pass twiddles read from the per-chunk tables (default) or
    made on the fly from 8 seeds per chunk and 256 roots per limb
    (NTT_TW_OTF), on the headline data: forward of 16 polynomials and the
    pointwise product fused into the inverse of 8, four rotating copies of
    the input (512 MiB > L2), with each plan's device table bytes."""
    qs = nt.ntt_find_primes(30, 17, 32)
    N, B, L = 1 << 16, 16, 32
    host = ntt_synth.rns_batch(1005, qs, N, B, dtype=np.uint32)
    src = torch.from_numpy(host.view(np.int32).reshape(-1).copy()).to(dev)
    copies = [src.clone() for _ in range(4)]
    half = B // 2 * L * N
    c = torch.empty(half, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    out = {"workload": "N=2^16, L=32 primes q<2^30, u32, 16 polys: forward x16; pointwise x8 + inverse x8"}
    for name, extra in (("tables", 0), ("on_the_fly", nt.NTT_TW_OTF)):
        # each plan in its fastest forms for these batches (autotuned, the
        # product + inverse form on the step itself, as for the headline)
        nt.ntt_autotune(N, qs, nt.NTT_ORDER_BITREV | extra, B, sh)
        inv = nt.ntt_autotune(N, qs, nt.NTT_ORDER_BITREV | extra, B // 2, sh)
        tune_step_inverse_form(nt, torch, dev, N, qs, nt.NTT_ORDER_BITREV | extra, inv)
        p = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, nt.NTT_ORDER_BITREV | extra)
        names = {v: k for k, v in nt.FORMS.items()}
        forms = {"forward": names[nt.ntt_plan_form(p, B)], "product_inverse": names[nt.ntt_plan_form(p, B // 2, True)]}
        try:
            it = iter(range(1 << 30))
            ms_f = _time_loop(torch, stream, lambda: nt.ntt_forward(p, copies[next(it) % 4], B, sh), reps)
            ms_p = _time_loop(torch, stream, lambda: nt.ntt_pointwise_inverse(
                p, c, copies[next(it) % 4][:half], copies[next(it) % 4][half:], B // 2, sh), reps)
            status = nt.ntt_get_device_status(p)
            out[name] = {"forward_ms": ms_f, "pointwise_inverse_ms": ms_p,
                         "forward_value": B * L / (ms_f / 1e3), "unit": "NTT/s",
                         "table_bytes": nt.ntt_plan_table_bytes(p), "two_pass_forms": forms,
                         "device_status": status}
        finally:
            nt.ntt_plan_destroy(p)
    return out


# ------------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="nttgb", choices=["nttgb", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ragged and wide-word side measurements")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (default two-pass forms), e.g. for launch lists under ncu")
    ap.add_argument("--extra", default=None,
                    choices=["ragged", "wide_word_u64", "tc_fourstep", "cluster_form", "base_conv",
                             "variants_n1024", "rns_n2p14", "autotune_shapes", "tw_otf"],
                    help="run only this side measurement and print its JSON (for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import __graft_entry__
    import paper_2405_11353_gb300 as nt

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0 or not os.path.exists(nt.LIB_PATH):
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    nt.lib()
    if args.extra:
        fn = {"ragged": ragged_vs_plain, "wide_word_u64": wide_word, "tc_fourstep": tc_fourstep,
              "cluster_form": cluster_form, "base_conv": base_conv, "variants_n1024": variants_n1024,
              "rns_n2p14": rns_n2p14, "autotune_shapes": autotune_shapes, "tw_otf": tw_otf}[args.extra]
        print(json.dumps({args.extra: fn(nt, torch, dev)}), flush=True)
        return 0
    from paper_2405_11353_gb300 import build as nb
    digest = nb.kernel_digest(nb.FORWARD_U32_SOURCES)

    # limb sharding across ranks: the job is 16 polynomials of L x world
    # limbs and each rank transforms its slice of L limbs (its own primes),
    # so the work per GPU is fixed as ranks are added; one rank: all L limbs
    qs_all = nt.ntt_find_primes(BITS, M, L * world)
    first, count = nt.ntt_limb_shard(L * world, world, rank)
    qs = qs_all[first:first + count]
    flags = nt.NTT_ORDER_BITREV | nt.NTT_RED_SHOUP
    # the autotuner picks the two-pass form of each direction for the two
    # batch sizes of the step (forward of 16 polynomials, product + inverse
    # of 8) before the plan is made
    tuning = None
    if not args.no_tune:
        tuning = {"forward_batch%d" % POLYS: nt.ntt_autotune(N, qs, flags, POLYS),
                  "inverse_batch%d" % PAIRS: nt.ntt_autotune(N, qs, flags, PAIRS)}
        # The autotuner times each call alone.  Back to back, the product +
        # inverse follows the forward's chunk pass (a programmatic dependent
        # launch), and inverse forms that time alike alone can differ in
        # the step: time the step itself with each inverse form of the
        # product batch and keep the fastest.
        tuning["step_inverse_form_ms"] = tune_step_inverse_form(nt, torch, dev, N, qs, flags,
                                                                tuning["inverse_batch%d" % PAIRS])
    plan = nt.ntt_plan_create(N, qs, nt.NTT_FUSED, flags)
    form_names = {v: k for k, v in nt.FORMS.items()}
    forms = {"forward": form_names.get(nt.ntt_plan_form(plan, POLYS)),
             "product_inverse": form_names.get(nt.ntt_plan_form(plan, PAIRS, True))}
    split = nt.ntt_plan_chunk_log2(plan)
    radix = nt.ntt_plan_radix_log2(plan)
    host = ntt_synth.rns_batch(1005 + 7919 * rank, qs, N, POLYS, dtype=np.uint32)
    words = POLYS * L * N
    half = PAIRS * L * N
    pinned = torch.from_numpy(host.view(np.int32).reshape(-1).copy()).pin_memory()
    bufs = []
    for _ in range(ROTATE):
        b = torch.empty(words, dtype=torch.int32, device=dev)
        b.copy_(pinned, non_blocking=False)
        bufs.append(b)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream

    def step(b):
        nt.ntt_forward(plan, b, POLYS, sh)
        nt.ntt_pointwise_inverse(plan, b, b, b[half:], PAIRS, sh)

    def launches_per_step():
        nt.ntt_forward(plan, bufs[0], POLYS, sh)
        n = nt.ntt_plan_last_launches(plan)
        nt.ntt_pointwise_inverse(plan, bufs[0], bufs[0], bufs[0][half:], PAIRS, sh)
        n += nt.ntt_plan_last_launches(plan)
        return n

    lps = launches_per_step()
    for i in range(args.warmup):
        step(bufs[i % ROTATE])
    torch.cuda.synchronize()

    # ---------------- timed region: K steps back to back (the metric), then
    # K calls of each of the step's two calls back to back (their per-call
    # times, for the roofline).  Events sit only at the ends of each run:
    # an event between two launches would end their programmatic overlap.
    K = args.steps
    sampler = ClockSampler(dev.index) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    for i in range(K):
        step(bufs[i % ROTATE])
    ev[1].record(stream)
    for i in range(K):
        nt.ntt_forward(plan, bufs[i % ROTATE], POLYS, sh)
    ev[2].record(stream)
    for i in range(K):
        b = bufs[i % ROTATE]
        nt.ntt_pointwise_inverse(plan, b, b, b[half:], PAIRS, sh)
    ev[3].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    elapsed_ms = ev[0].elapsed_time(ev[1])
    fwd_ms = ev[1].elapsed_time(ev[2]) / K
    pwinv_ms = ev[2].elapsed_time(ev[3]) / K
    elapsed_ms = max_over_ranks(elapsed_ms, dist if world > 1 else None, dev)
    ms_per_step = elapsed_ms / K
    value = job_rate(NTT_PER_STEP, world, K, elapsed_ms)

    # ---------------- end to end through the host-buffer entry point
    h_in = pinned
    h_out = torch.empty(half, dtype=torch.int32).pin_memory()
    work = bufs[0]
    Ke = max(3, min(K, 200))
    for _ in range(3):
        nt.ntt_polymul_host(plan, h_out, h_in, work, PAIRS, sh)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(Ke):
        nt.ntt_polymul_host(plan, h_out, h_in, work, PAIRS, sh)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist if world > 1 else None, dev)
    e2e_value = job_rate(NTT_PER_STEP, world, Ke, e2e_ms)

    # ---------------- roofline of the forward transform (dominant call)
    peak, peak_kind = peaks()
    n_fwd = POLYS * L
    fwd_bytes = 2 * N * WORD * n_fwd + L * N * 2 * WORD      # data r+w, twiddle pairs once per prime
    achieved = fwd_bytes / (fwd_ms / 1000.0) / 1e9
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": achieved / peak, "traffic": traffic_from_profiles(digest),
        "kernel": "ntt_forward: %d-pt cols + %d-word chunks, %s, radix %d, %d NTTs" % (
            N >> split, 1 << split, forms["forward"], 1 << radix, n_fwd),
        "algorithmic_bytes_per_call": fwd_bytes, "avg_ms": fwd_ms,
        "peak_source": "measured hbm_gbs" if peak_kind == "measured" else "fallback 6.8 TB/s",
    }

    # the same call against the integer multiply pipe: every butterfly of the
    # Shoup form takes three 32-bit multiplies (one mad.hi, two mad.lo); the
    # peak is measured here (ntt_measure_int_mad_rate) for that mix
    muls = 3 * n_fwd * (N // 2) * 16
    lo_rate, hi_rate = measure_int_mad_rate(nt, torch, dev, stream)
    int_peak = 3.0 / (1.0 / hi_rate + 2.0 / lo_rate)
    int_roofline = {"bound": "alu", "achieved": muls / (fwd_ms / 1e3) / 1e12, "peak": int_peak / 1e12,
                    "unit": "T int32 multiplies/s", "frac": muls / (fwd_ms / 1e3) / int_peak,
                    "multiplies_per_call": muls,
                    "peak_source": "measured mad.lo %.2f, mad.hi %.2f T/s (1 hi : 2 lo)"
                                   % (lo_rate / 1e12, hi_rate / 1e12)}

    extras = {}
    if not args.no_extras:
        for name, fn in (("ragged", ragged_vs_plain), ("wide_word_u64", wide_word),
                         ("tc_fourstep", tc_fourstep), ("cluster_form", cluster_form),
                         ("base_conv", base_conv), ("variants_n1024", variants_n1024),
                         ("rns_n2p14", rns_n2p14), ("autotune_shapes", autotune_shapes), ("tw_otf", tw_otf)):
            try:
                extras[name] = fn(nt, torch, dev)
            except Exception as exc:     # a side measurement never hides the main line
                extras[name] = {"error": repr(exc)[:300]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, desc = oracle_sample(qs)
        cpu = {"value": v, "unit": "NTT/s", "cores": cores, "kind": "oracle", "sample": desc}
        extras["cpu_naive"] = {"n1024": oracle_naive_n1024(), "n65536": oracle_naive_n65536()}

    nt.ntt_plan_destroy(plan)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "NTT/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic (seeded SplitMix64 residues, uniform in [0,q))",
            "config": {"workload": WORKLOAD, "N": N, "L": L, "polys": POLYS, "word": "u32",
                       "variant": "fused", "reduction": "shoup", "order": "bitrev",
                       "two_pass_forms": forms, "chunk_log2": split, "radix_log2": radix,
                       "l2": "4 rotating input copies (512 MiB) > 129 MB L2",
                       "parallelism": ("limb-sharded x%d: %d limbs per rank of %d" % (world, count, L * world))
                       if world > 1 else "1 GPU"},
            "per_call_ms": {"forward_16polys": fwd_ms, "pointwise_inverse_8pairs": pwinv_ms},
            "roofline": roofline,
            "int_roofline": int_roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "NTT/s",
                    "h2d_bytes_per_step": POLYS * L * N * WORD,
                    "d2h_bytes_per_step": PAIRS * L * N * WORD, "steps": Ke},
            "gpu_launches": lps * K,
            "clocks": clocks,
        }
        # the side measurements in full, one line each, before the main line
        if tuning:
            print(json.dumps({"detail": "autotune", **tuning}), flush=True)
        for name, v in extras.items():
            print(json.dumps({"detail": name, **(v if isinstance(v, dict) else {"value": v})}), flush=True)
        # their headline figures close the main line (printed last)
        line["side"] = side_summary(extras)
        if "cpu_naive" in extras:
            line["side"]["cpu_oracle_naive_n65536_s"] = _pick(extras, "cpu_naive", "n65536", "seconds_per_transform")
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
