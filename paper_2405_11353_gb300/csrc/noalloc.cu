// noalloc.cu -- forward transform that allocates nothing.
//
// Some callers cannot let a library allocate device memory: a host
// framework that owns every byte of device memory through its own pool
// (a hidden cudaMalloc fragments it or breaks its budget), a latency-bound
// loop where cudaMalloc's implicit device synchronisation is not
// acceptable, or a plugin running under a fixed memory budget.  The regular
// entry points grow a plan-owned scratch buffer on demand; this one runs the
// Stockham dataflow with its ping-pong buffer in a fixed array of device
// memory that the library declares at file scope, so the call itself makes
// no cudaMalloc, cudaFree or other allocating call.
//
// The array (kNoAllocScratchBytes) is part of the library image: every GPU
// that loads the library holds it until the process exits.  All calls in the
// process share it and it keeps whatever the last call left there; nothing
// in it has to start at zero, because every Stockham stage writes the whole
// used range before the next stage reads it.  Calls whose work overlaps on
// the GPU (for example on two streams) race on the array.
//
// Host code cannot use the array's name as a device address: in host code
// it names a host-side stand-in.  The first call on each device therefore
// looks up the array's device address with cudaGetSymbolAddress (with that
// device current) and keeps it, with the device's SM count; later calls
// reuse both.  That first call should come before any stream capture.  The
// address belongs to the CUDA context it was looked up in: after
// cudaDeviceReset the device gets a new primary context, the library's
// module is loaded again and the array may sit elsewhere, so the cache is
// keyed on the current context and the address is looked up again when the
// context changes (that next call, too, should come before any capture).
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <type_traits>

#include "modarith.cuh"
#include "plan.hpp"

namespace {

using namespace nttgb;

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
struct DevCache {
    CUcontext ctx;     // the context the address was looked up in
    void *addr;        // device address of g_noalloc_scratch there
    unsigned max_grid; // 32 CTAs of kThreads per SM
};
DevCache g_cache[kMaxDevices] = {};

constexpr int kThreads = 256;

// The driver's cuCtxGetCurrent, reached through the runtime (the library
// does not link the driver library, so it loads on machines without one).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &f, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(f);
    }
    return fn;
}

// Device address of g_noalloc_scratch on the current device, and the grid
// limit for its kernels (looked up once per device and context).
cudaError_t scratch_address(void **out, unsigned *max_grid) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    CtxGetCurrentFn get_ctx = ctx_get_current();
    if (!get_ctx) return cudaErrorNotSupported;
    // the context the kernels will run in (none is current before the
    // runtime's first call on this thread: the symbol lookup below makes the
    // device's primary context current)
    CUcontext ctx = nullptr;
    if (get_ctx(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    DevCache &c = g_cache[dev];
    if (!ctx || !c.addr || c.ctx != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        c.ctx = ctx;
        c.addr = p;
        c.max_grid = (unsigned)(sms > 0 ? sms : 1) * 32u;
    }
    *out = c.addr;
    *max_grid = c.max_grid;
    return cudaSuccess;
}

unsigned grid_for(uint64_t work, unsigned max_grid) {
    uint64_t g = (work + kThreads - 1) / kThreads;
    if (g > max_grid) g = max_grid;
    return g ? (unsigned)g : 1u;
}

// x[t][n] *= psi^n (the twist of the forward transform)
template <class W, int RED>
__global__ void k_twist_na(W *__restrict__ x, const Tw<W> *__restrict__ tab, const LimbConst *__restrict__ lc,
                           uint32_t logN, uint32_t L, uint64_t total) {
    const uint32_t N = 1u << logN;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t t = g >> logN;
        uint32_t l = (uint32_t)(t % L);
        Lc<W> k;
        k.load(lc + l);
        x[g] = mul_full<RED>(x[g], ldtw(tab + (size_t)l * N + ((uint32_t)g & (N - 1))), k);
    }
}

// One Stockham stage (same dataflow as the plan path's Stockham kernel).
template <class W, int RED>
__global__ void k_stockham_na(W *__restrict__ dst, const W *__restrict__ src, const Tw<W> *__restrict__ wt,
                              const LimbConst *__restrict__ lc, uint32_t logN, uint32_t L, uint32_t s,
                              uint64_t total_bf) {
    const uint32_t N = 1u << logN;
    const uint32_t stride = 1u << (s - 1);
    const uint32_t m = N >> s;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total_bf;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t t = g >> (logN - 1);
        uint32_t b = (uint32_t)g & (N / 2 - 1);
        uint32_t tt = b & (stride - 1);
        uint32_t p = b >> (s - 1);
        Lc<W> k;
        k.load(lc + (uint32_t)(t % L));
        const W *st = src + t * N;
        W *dt = dst + t * N;
        W a = st[tt + stride * p];
        W c = st[tt + stride * (p + m)];
        Tw<W> tw = ldtw(wt + (size_t)(t % L) * N + (size_t)p * stride);
        dt[tt + stride * (2 * p)] = add_mod<W>(a, c, k.q);
        dt[tt + stride * (2 * p + 1)] = mul_full<RED>(sub_mod<W>(a, c, k.q), tw, k);
    }
}

template <class W>
__global__ void k_copy_na(W *__restrict__ dst, const W *__restrict__ src, uint64_t total) {
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x)
        dst[g] = src[g];
}

template <class W>
__global__ void k_bitrev_na(W *__restrict__ x, uint32_t logN, uint64_t total) {
    const uint32_t N = 1u << logN;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t i = (uint32_t)g & (N - 1);
        uint32_t j = __brev(i) >> (32 - logN);
        if (i < j) {
            W *base = x + (g - i);
            W a = base[i];
            base[i] = base[j];
            base[j] = a;
        }
    }
}

// Counts its launches in p.last_launches.
template <class W, int RED>
cudaError_t run_noalloc(ntt_plan_s &p, W *data, W *scr, uint32_t batch, unsigned mg, cudaStream_t st) {
    const uint32_t logN = p.logN, L = p.L, N = p.N;
    const uint64_t total = (uint64_t)batch * L * N;
    const uint64_t total_bf = total / 2;
    const Tw<W> *wt = reinterpret_cast<const Tw<W> *>(p.d_w_fwd);
    const Tw<W> *twist = reinterpret_cast<const Tw<W> *>(p.d_twist);
    k_twist_na<W, RED><<<grid_for(total, mg), kThreads, 0, st>>>(data, twist, p.d_limb, logN, L, total);
    ++p.last_launches;
    W *src = data, *dst = scr;
    for (uint32_t s = 1; s <= logN; ++s) {
        k_stockham_na<W, RED><<<grid_for(total_bf, mg), kThreads, 0, st>>>(dst, src, wt, p.d_limb, logN, L, s,
                                                                            total_bf);
        ++p.last_launches;
        W *t = src; src = dst; dst = t;
    }
    if (src != data) {
        k_copy_na<W><<<grid_for(total, mg), kThreads, 0, st>>>(data, src, total);
        ++p.last_launches;
    }
    if (p.bitrev_order) {
        k_bitrev_na<W><<<grid_for(total, mg), kThreads, 0, st>>>(data, logN, total);
        ++p.last_launches;
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" ntt_status ntt_forward_noalloc(ntt_plan_t plan, void *d_data, uint32_t batch, ntt_stream_t stream) {
    if (!plan || !d_data || batch == 0) return NTT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_data) & 15u) != 0) return NTT_ERR_ALIGNMENT;
    ntt_plan_s &p = *plan;
    // the Stockham dataflow needs the per-stage tables, which every plan
    // builds except the fused ones with N >= 16 (tensor-core four-step
    // plans build them too)
    if (!p.d_w_fwd || !p.d_twist) return NTT_ERR_UNSUPPORTED;
    const size_t bytes = (size_t)batch * p.L * p.N * p.word_bytes();
    if (bytes > kNoAllocScratchBytes) return NTT_ERR_SCRATCH_LIMIT;
    void *scr = nullptr;
    unsigned mg = 0;
    if (scratch_address(&scr, &mg) != cudaSuccess) { cudaGetLastError(); return NTT_ERR_CUDA; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    p.last_launches = 0;
    cudaError_t e = cudaSuccess;
    // NTT_CHECK: record input words >= q in the plan's status word, as
    // ntt_forward does (the check writes only that existing word)
    if (p.check) e = nttgb::launch_check_range(p, d_data, batch, st);
    if (e != cudaSuccess) { cudaGetLastError(); return NTT_ERR_CUDA; }
    if (p.word64) {
        switch (p.red) {
        case RED_SHOUP: e = run_noalloc<uint64_t, RED_SHOUP>(p, (uint64_t *)d_data, (uint64_t *)scr, batch, mg, st); break;
        case RED_BARRETT: e = run_noalloc<uint64_t, RED_BARRETT>(p, (uint64_t *)d_data, (uint64_t *)scr, batch, mg, st); break;
        default: e = run_noalloc<uint64_t, RED_MONTGOMERY>(p, (uint64_t *)d_data, (uint64_t *)scr, batch, mg, st); break;
        }
    } else {
        switch (p.red) {
        case RED_SHOUP: e = run_noalloc<uint32_t, RED_SHOUP>(p, (uint32_t *)d_data, (uint32_t *)scr, batch, mg, st); break;
        case RED_BARRETT: e = run_noalloc<uint32_t, RED_BARRETT>(p, (uint32_t *)d_data, (uint32_t *)scr, batch, mg, st); break;
        default: e = run_noalloc<uint32_t, RED_MONTGOMERY>(p, (uint32_t *)d_data, (uint32_t *)scr, batch, mg, st); break;
        }
    }
    if (e != cudaSuccess) { cudaGetLastError(); return NTT_ERR_CUDA; }
    return NTT_OK;
}
