// stage.cu -- the seven dataflow variants of Sec. II as per-stage kernels,
// plus the elementwise kernels shared by every path (pointwise product,
// psi twist, bit-reversal permutation, input range check).
//
// Each variant runs the cyclic N-point transform with root omega = psi^2 on
// the twisted input a[n] psi^n (forward), or with omega^-1 followed by the
// N^-1 psi^-n untwist (inverse), exactly as its dataflow is described in the
// paper; one launch is one stage (one pass over global memory), so the
// memory-access pattern of each variant is what the hardware sees:
//
//   DIT       Algorithm 1: in-place bit reversal, then stages s = 1..log N;
//             the k-outer / j-inner loop nest maps consecutive threads to
//             butterflies m apart (the stride pattern Sec. III-A discusses).
//   DIF       Algorithm 2: stages s = log N..1 with the same loop nest, then
//             the bit reversal.
//   Flat      Sec. II Flat-NTT: DIT with the k and j loops fused into one
//             index i < N/2, so consecutive threads touch consecutive words.
//   Pease     Eq. 7 / Algorithm 3 (constant geometry): every stage reads the
//             pair (2r, 2r+1) and writes (r, r + N/2) into a second buffer,
//             which is then copied back.  Algorithm 3 as printed omits the
//             twiddle; the stage s twiddle is omega^(r with its low
//             (log N - s) bits cleared), which reproduces the DIT result.
//   Pease_nc  Sec. II / III-B: Pease with the two buffers swapped after
//             each stage instead of copied (one final copy when log N is odd).
//   Stockham  Sec. II: self-sorting radix-2 ping-pong, natural order in and
//             out, no bit reversal.
//   Six-step  Sec. II: N = N1 N2; transpose, N1-point row transforms,
//             twiddle omega^(n2 k1), transpose, N2-point row transforms,
//             transpose.  The row transforms run in shared memory.
//
// Values are kept fully reduced to [0, q) after every stage (Algorithm 4).
#include <cuda_runtime.h>

#include <type_traits>

#include "modarith.cuh"
#include "plan.hpp"

namespace nttgb {

namespace {

constexpr int kThreads = 256;

// Programmatic dependent launch (as in the fused kernels): every kernel
// here lets the next launch on the stream be scheduled once all its CTAs
// have started, then waits for the previous launch's results before it
// touches data, so the launch latency of one stage hides behind the
// previous one.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void dep_begin() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
void launch_dep(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);   // errors surface through cudaGetLastError
}

inline unsigned grid_for(uint64_t work, int threads = kThreads) {
    uint64_t g = (work + threads - 1) / threads;
    if (g > 152ull * 32) g = 152ull * 32;
    if (g == 0) g = 1;
    return (unsigned)g;
}

__device__ __forceinline__ uint32_t brv(uint32_t x, uint32_t bits) {
    return bits ? (__brev(x) >> (32 - bits)) : 0u;
}

template <class W> __device__ __forceinline__ Lc<W> limb_k(const LimbConst *lc, uint32_t l) {
    Lc<W> k;
    k.load(lc + l);
    return k;
}

// ---------------------------------------------------------- elementwise
// x[t][n] = x[t][n] * tab[l][n] mod q  (psi twist / N^-1 psi^-n untwist)
template <class W, int RED>
__global__ void k_scale(W *__restrict__ x, const Tw<W> *__restrict__ tab, const LimbConst *__restrict__ lc,
                        uint32_t logN, uint32_t L, uint64_t total) {
    dep_begin();
    const uint32_t N = 1u << logN;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t t = g >> logN;
        uint32_t n = (uint32_t)g & (N - 1);
        uint32_t l = (uint32_t)(t % L);
        Lc<W> k = limb_k<W>(lc, l);
        x[g] = mul_full<RED>(x[g], ldtw(tab + (size_t)l * N + n), k);
    }
}

// in-place bit-reversal permutation of every transform
template <class W>
__global__ void k_bitrev(W *__restrict__ x, uint32_t logN, uint64_t total) {
    dep_begin();
    const uint32_t N = 1u << logN;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t i = (uint32_t)g & (N - 1);
        uint32_t j = brv(i, logN);
        if (i < j) {
            W *base = x + (g - i);
            W a = base[i], b = base[j];
            base[i] = b;
            base[j] = a;
        }
    }
}

template <class W>
__global__ void k_copy(W *__restrict__ dst, const W *__restrict__ src, uint64_t total) {
    dep_begin();
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x)
        dst[g] = src[g];
}

// c = a * b mod q, 16-byte vectors (V words per vector, all in one limb)
template <class W, int RED>
__global__ void k_pointwise_vec(W *c, const W *a, const W *b, const LimbConst *__restrict__ lc,
                                uint32_t logN, uint32_t L, uint64_t nvec) {
    dep_begin();
    constexpr int V = 16 / sizeof(W);
    using Vec = typename std::conditional<sizeof(W) == 4, uint4, ulonglong2>::type;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < nvec;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t e0 = g * V;
        uint32_t l = (uint32_t)((e0 >> logN) % L);
        Lc<W> k = limb_k<W>(lc, l);
        Vec va = reinterpret_cast<const Vec *>(a)[g];
        Vec vb = reinterpret_cast<const Vec *>(b)[g];
        W *pa = reinterpret_cast<W *>(&va);
        W *pb = reinterpret_cast<W *>(&vb);
#pragma unroll
        for (int i = 0; i < V; ++i) pa[i] = mul_var<RED>(pa[i], pb[i], k);
        reinterpret_cast<Vec *>(c)[g] = va;
    }
}

template <class W, int RED>
__global__ void k_pointwise_scalar(W *c, const W *a, const W *b, const LimbConst *__restrict__ lc,
                                   uint32_t logN, uint32_t L, uint64_t total) {
    dep_begin();
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t l = (uint32_t)((g >> logN) % L);
        Lc<W> k = limb_k<W>(lc, l);
        c[g] = mul_var<RED>(a[g], b[g], k);
    }
}

template <class W>
__global__ void k_check_range(const W *__restrict__ x, const LimbConst *__restrict__ lc, uint32_t logN,
                              uint32_t L, uint64_t total, uint32_t *status) {
    dep_begin();
    bool bad = false;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t l = (uint32_t)((g >> logN) % L);
        if ((uint64_t)x[g] >= lc[l].q) bad = true;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 1u);
}

// ------------------------------------------------------ in-place stages
enum { ST_DIT = 0, ST_DIF = 1, ST_FLAT = 2 };

// One stage s (m = 2^s) of Algorithm 1 / 2; tw = omega^((N/m) k).
template <class W, int RED, int KIND>
__global__ void k_stage_inplace(W *__restrict__ x, const Tw<W> *__restrict__ wt, const LimbConst *__restrict__ lc,
                                uint32_t logN, uint32_t L, uint32_t s, uint64_t total_bf) {
    dep_begin();
    const uint32_t N = 1u << logN;
    const uint32_t half = 1u << (s - 1);
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total_bf;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t t = g >> (logN - 1);
        uint32_t b = (uint32_t)g & (N / 2 - 1);
        uint32_t k, j;
        if (KIND == ST_FLAT) {
            k = b & (half - 1);
            j = (b >> (s - 1)) << s;
        } else {
            // k outer, j inner: consecutive b walk j = 0, m, 2m, ...
            k = b >> (logN - s);
            j = (b & ((N >> s) - 1)) << s;
        }
        uint32_t l = (uint32_t)(t % L);
        Lc<W> kk = limb_k<W>(lc, l);
        Tw<W> tw = ldtw(wt + (size_t)l * N + ((size_t)k << (logN - s)));
        W *xt = x + t * N;
        W f1 = xt[j + k], f2 = xt[j + k + half];
        if (KIND == ST_DIF) {
            xt[j + k] = add_mod<W>(f1, f2, kk.q);
            xt[j + k + half] = mul_full<RED>(sub_mod<W>(f1, f2, kk.q), tw, kk);
        } else {
            W v = mul_full<RED>(f2, tw, kk);
            xt[j + k] = add_mod<W>(f1, v, kk.q);
            xt[j + k + half] = sub_mod<W>(f1, v, kk.q);
        }
    }
}

// Constant-geometry stage s (Pease / Pease_nc): read (2r, 2r+1), write
// (r, r + N/2); twiddle omega^(r & ~(2^(logN-s) - 1)).
template <class W, int RED>
__global__ void k_stage_cg(W *__restrict__ dst, const W *__restrict__ src, const Tw<W> *__restrict__ wt,
                           const LimbConst *__restrict__ lc, uint32_t logN, uint32_t L, uint32_t s,
                           uint64_t total_bf) {
    dep_begin();
    const uint32_t N = 1u << logN;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total_bf;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t t = g >> (logN - 1);
        uint32_t r = (uint32_t)g & (N / 2 - 1);
        uint32_t l = (uint32_t)(t % L);
        Lc<W> kk = limb_k<W>(lc, l);
        uint32_t e = r & ~((1u << (logN - s)) - 1u);
        Tw<W> tw = ldtw(wt + (size_t)l * N + e);
        const W *st = src + t * N;
        W *dt = dst + t * N;
        W a = st[2 * r];
        W v = mul_full<RED>(st[2 * r + 1], tw, kk);
        dt[r] = add_mod<W>(a, v, kk.q);
        dt[r + N / 2] = sub_mod<W>(a, v, kk.q);
    }
}

// Stockham stage s: len = N / 2^(s-1), stride = 2^(s-1), m = len / 2;
// y[t + stride 2p] = a + c, y[t + stride (2p+1)] = (a - c) omega^(p stride).
template <class W, int RED>
__global__ void k_stage_stockham(W *__restrict__ dst, const W *__restrict__ src, const Tw<W> *__restrict__ wt,
                                 const LimbConst *__restrict__ lc, uint32_t logN, uint32_t L, uint32_t s,
                                 uint64_t total_bf) {
    dep_begin();
    const uint32_t N = 1u << logN;
    const uint32_t stride = 1u << (s - 1);
    const uint32_t m = N >> s;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total_bf;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t t = g >> (logN - 1);
        uint32_t b = (uint32_t)g & (N / 2 - 1);
        uint32_t tt = b & (stride - 1);
        uint32_t p = b >> (s - 1);
        uint32_t l = (uint32_t)(t % L);
        Lc<W> kk = limb_k<W>(lc, l);
        const W *st = src + t * N;
        W *dt = dst + t * N;
        W a = st[tt + stride * p];
        W c = st[tt + stride * (p + m)];
        Tw<W> tw = ldtw(wt + (size_t)l * N + (size_t)p * stride);
        dt[tt + stride * (2 * p)] = add_mod<W>(a, c, kk.q);
        dt[tt + stride * (2 * p + 1)] = mul_full<RED>(sub_mod<W>(a, c, kk.q), tw, kk);
    }
}

// ------------------------------------------------------------ six-step
// dst[t][c][r] = src[t][r][c] for an R x C matrix per transform.
template <class W>
__global__ void k_transpose(W *__restrict__ dst, const W *__restrict__ src, uint32_t logR, uint32_t logC,
                            uint64_t ntrans) {
    dep_begin();
    __shared__ W tile[32][33];
    const uint32_t R = 1u << logR, C = 1u << logC;
    const uint32_t tilesC = (C + 31) / 32, tilesR = (R + 31) / 32;
    const uint64_t tiles_per = (uint64_t)tilesC * tilesR;
    for (uint64_t tb = blockIdx.x; tb < ntrans * tiles_per; tb += gridDim.x) {
        uint64_t t = tb / tiles_per;
        uint32_t rem = (uint32_t)(tb % tiles_per);
        uint32_t r0 = (rem / tilesC) * 32, c0 = (rem % tilesC) * 32;
        const W *s = src + (t << (logR + logC));
        W *d = dst + (t << (logR + logC));
        for (uint32_t i = threadIdx.y; i < 32; i += blockDim.y) {
            uint32_t r = r0 + i, c = c0 + threadIdx.x;
            if (r < R && c < C) tile[i][threadIdx.x] = s[(size_t)r * C + c];
        }
        __syncthreads();
        for (uint32_t i = threadIdx.y; i < 32; i += blockDim.y) {
            uint32_t c = c0 + i, r = r0 + threadIdx.x;
            if (r < R && c < C) d[(size_t)c * R + r] = tile[threadIdx.x][i];
        }
        __syncthreads();
    }
}

// Cyclic transforms of every row (length 2^logRow, root omega^(N / row)) in
// shared memory: bit-reversed load, DIT stages, natural store; optionally
// multiplied by omega^(row * col) afterwards (six-step twiddle step).
template <class W, int RED>
__global__ void k_rows(W *__restrict__ x, const Tw<W> *__restrict__ wt, const LimbConst *__restrict__ lc,
                       uint32_t logN, uint32_t L, uint32_t logRow, uint64_t nrows_total, int twiddle) {
    dep_begin();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    W *sm = reinterpret_cast<W *>(smem_raw);
    const uint32_t N = 1u << logN, Rl = 1u << logRow;
    const uint32_t rows_per_t = N >> logRow;
    for (uint64_t row = blockIdx.x; row < nrows_total; row += gridDim.x) {
        uint64_t t = row / rows_per_t;
        uint32_t ri = (uint32_t)(row % rows_per_t);
        uint32_t l = (uint32_t)(t % L);
        Lc<W> kk = limb_k<W>(lc, l);
        const Tw<W> *wl = wt + (size_t)l * N;
        W *xr = x + row * Rl;
        for (uint32_t i = threadIdx.x; i < Rl; i += blockDim.x) sm[brv(i, logRow)] = xr[i];
        __syncthreads();
        for (uint32_t s = 1; s <= logRow; ++s) {
            uint32_t half = 1u << (s - 1);
            for (uint32_t b = threadIdx.x; b < Rl / 2; b += blockDim.x) {
                uint32_t k = b & (half - 1);
                uint32_t j = (b >> (s - 1)) << s;
                // omega_row^(k Rl / 2^s) = omega^(k N / 2^s)
                Tw<W> tw = ldtw(wl + ((size_t)k << (logN - s)));
                W f1 = sm[j + k];
                W v = mul_full<RED>(sm[j + k + half], tw, kk);
                sm[j + k] = add_mod<W>(f1, v, kk.q);
                sm[j + k + half] = sub_mod<W>(f1, v, kk.q);
            }
            __syncthreads();
        }
        for (uint32_t i = threadIdx.x; i < Rl; i += blockDim.x) {
            W v = sm[i];
            if (twiddle) v = mul_full<RED>(v, ldtw(wl + (size_t)ri * i), kk);
            xr[i] = v;
        }
        __syncthreads();
    }
}

template <class W, int RED>
cudaError_t run_variant_t(ntt_plan_s &p, ntt_variant variant, void *data_v, uint32_t batch, bool inverse,
                          cudaStream_t st) {
    W *data = reinterpret_cast<W *>(data_v);
    W *scr = reinterpret_cast<W *>(p.d_scratch);
    const uint32_t logN = p.logN, L = p.L, N = p.N;
    const uint64_t ntrans = (uint64_t)batch * L;
    const uint64_t total = ntrans * N;
    const uint64_t total_bf = ntrans * (N / 2);
    const Tw<W> *wt = reinterpret_cast<const Tw<W> *>(inverse ? p.d_w_inv : p.d_w_fwd);
    const Tw<W> *twist = reinterpret_cast<const Tw<W> *>(p.d_twist);
    const Tw<W> *untwist = reinterpret_cast<const Tw<W> *>(p.d_untwist);
    const LimbConst *lc = p.d_limb;
    uint32_t &nl = p.last_launches;
    const unsigned ge = grid_for(total), gb = grid_for(total_bf);

    // inverse input in bit-reversed order -> natural first
    if (inverse && p.bitrev_order) { launch_dep(k_bitrev<W>, ge, kThreads, 0, st, data, logN, total); ++nl; }
    if (!inverse) { launch_dep(k_scale<W, RED>, ge, kThreads, 0, st, data, twist, lc, logN, L, total); ++nl; }

    switch (variant) {
    case NTT_DIT:
    case NTT_FLAT:
        launch_dep(k_bitrev<W>, ge, kThreads, 0, st, data, logN, total); ++nl;
        for (uint32_t s = 1; s <= logN; ++s) {
            if (variant == NTT_DIT)
                launch_dep(k_stage_inplace<W, RED, ST_DIT>, gb, kThreads, 0, st, data, wt, lc, logN, L, s, total_bf);
            else
                launch_dep(k_stage_inplace<W, RED, ST_FLAT>, gb, kThreads, 0, st, data, wt, lc, logN, L, s, total_bf);
            ++nl;
        }
        break;
    case NTT_DIF:
        for (uint32_t s = logN; s >= 1; --s) {
            launch_dep(k_stage_inplace<W, RED, ST_DIF>, gb, kThreads, 0, st, data, wt, lc, logN, L, s, total_bf); ++nl;
        }
        launch_dep(k_bitrev<W>, ge, kThreads, 0, st, data, logN, total); ++nl;
        break;
    case NTT_PEASE:
    case NTT_PEASE_NC: {
        launch_dep(k_bitrev<W>, ge, kThreads, 0, st, data, logN, total); ++nl;
        W *src = data, *dst = scr;
        for (uint32_t s = 1; s <= logN; ++s) {
            launch_dep(k_stage_cg<W, RED>, gb, kThreads, 0, st, dst, src, wt, lc, logN, L, s, total_bf); ++nl;
            if (variant == NTT_PEASE) {
                // Algorithm 3: the new values are copied back before the next stage
                launch_dep(k_copy<W>, ge, kThreads, 0, st, src, dst, total); ++nl;
            } else {
                W *t = src; src = dst; dst = t;   // Pease_nc: swap the roles
            }
        }
        if (variant == NTT_PEASE_NC && src != data) { launch_dep(k_copy<W>, ge, kThreads, 0, st, data, src, total); ++nl; }
        break;
    }
    case NTT_STOCKHAM: {
        W *src = data, *dst = scr;
        for (uint32_t s = 1; s <= logN; ++s) {
            launch_dep(k_stage_stockham<W, RED>, gb, kThreads, 0, st, dst, src, wt, lc, logN, L, s, total_bf); ++nl;
            W *t = src; src = dst; dst = t;
        }
        if (src != data) { launch_dep(k_copy<W>, ge, kThreads, 0, st, data, src, total); ++nl; }
        break;
    }
    case NTT_SIXSTEP: {
        const uint32_t l1 = (logN + 1) / 2, l2 = logN / 2;   // N1 = 2^l1 rows, N2 = 2^l2 cols
        dim3 tb(32, 8);
        unsigned gt = grid_for(total, 256);
        auto rows = [&](W *x, uint32_t logRow, int tw) {
            uint64_t nrows = ntrans << (logN - logRow);
            unsigned thr = (1u << logRow) / 2 < 32 ? 32 : ((1u << logRow) / 2 > 256 ? 256 : (1u << logRow) / 2);
            unsigned g = nrows > 152ull * 32 ? 152u * 32 : (unsigned)nrows;
            launch_dep(k_rows<W, RED>, g, thr, sizeof(W) << logRow, st, x, wt, lc, logN, L, logRow, nrows, tw);
            ++nl;
        };
        // 1. A[n1][n2] (N1 x N2) -> T1[n2][n1]
        launch_dep(k_transpose<W>, gt, tb, 0, st, scr, data, l1, l2, ntrans); ++nl;
        // 2-3. N1-point transforms of the N2 rows, times omega^(n2 k1)
        rows(scr, l1, 1);
        // 4. T1 (N2 x N1) -> T2[k1][n2]
        launch_dep(k_transpose<W>, gt, tb, 0, st, data, scr, l2, l1, ntrans); ++nl;
        // 5. N2-point transforms of the N1 rows
        rows(data, l2, 0);
        // 6. T2 (N1 x N2) -> X[k2][k1] = X[k1 + N1 k2]
        launch_dep(k_transpose<W>, gt, tb, 0, st, scr, data, l1, l2, ntrans); ++nl;
        launch_dep(k_copy<W>, ge, kThreads, 0, st, data, scr, total); ++nl;
        break;
    }
    default:
        return cudaErrorInvalidValue;
    }

    if (inverse) { launch_dep(k_scale<W, RED>, ge, kThreads, 0, st, data, untwist, lc, logN, L, total); ++nl; }
    if (!inverse && p.bitrev_order) { launch_dep(k_bitrev<W>, ge, kThreads, 0, st, data, logN, total); ++nl; }
    return cudaGetLastError();
}

template <class F> cudaError_t dispatch(const ntt_plan_s &p, F &&f) {
    if (p.word64) {
        switch (p.red) {
        case RED_SHOUP: return f(uint64_t{}, std::integral_constant<int, RED_SHOUP>{});
        case RED_BARRETT: return f(uint64_t{}, std::integral_constant<int, RED_BARRETT>{});
        default: return f(uint64_t{}, std::integral_constant<int, RED_MONTGOMERY>{});
        }
    } else {
        switch (p.red) {
        case RED_SHOUP: return f(uint32_t{}, std::integral_constant<int, RED_SHOUP>{});
        case RED_BARRETT: return f(uint32_t{}, std::integral_constant<int, RED_BARRETT>{});
        default: return f(uint32_t{}, std::integral_constant<int, RED_MONTGOMERY>{});
        }
    }
}

}  // namespace

cudaError_t launch_variant(ntt_plan_s &p, ntt_variant v, void *data, uint32_t batch, bool inverse,
                           cudaStream_t st) {
    return dispatch(p, [&](auto w, auto r) {
        using W = decltype(w);
        return run_variant_t<W, decltype(r)::value>(p, v, data, batch, inverse, st);
    });
}

cudaError_t launch_fused(ntt_plan_s &p, void *data, uint32_t batch, bool inverse, cudaStream_t st) {
    if (p.fused_mode == FUSED_CLUSTER) {
        switch (p.red) {
        case RED_SHOUP: return run_cluster<RED_SHOUP>(p, data, batch, inverse, st);
        case RED_BARRETT: return run_cluster<RED_BARRETT>(p, data, batch, inverse, st);
        default: return run_cluster<RED_MONTGOMERY>(p, data, batch, inverse, st);
        }
    }
    return dispatch(p, [&](auto w, auto r) {
        using W = decltype(w);
        return run_fused_t<W, decltype(r)::value>(p, data, batch, inverse, st);
    });
}

cudaError_t launch_fused_pwinv(ntt_plan_s &p, void *c, const void *a, const void *b, uint32_t batch,
                               cudaStream_t st) {
    return dispatch(p, [&](auto w, auto r) {
        using W = decltype(w);
        return run_fused_pwinv_t<W, decltype(r)::value>(p, c, a, b, batch, st);
    });
}

cudaError_t launch_pointwise(ntt_plan_s &p, void *c, const void *a, const void *b, uint32_t batch, cudaStream_t st) {
    return dispatch(p, [&](auto w, auto r) {
        using W = decltype(w);
        constexpr int RED = decltype(r)::value;
        const uint64_t total = (uint64_t)batch * p.L * p.N;
        constexpr int V = 16 / sizeof(W);
        if (p.N % V == 0) {
            uint64_t nvec = total / V;
            launch_dep(k_pointwise_vec<W, RED>, grid_for(nvec), kThreads, 0, st, 
                (W *)c, (const W *)a, (const W *)b, p.d_limb, p.logN, p.L, nvec);
        } else {
            launch_dep(k_pointwise_scalar<W, RED>, grid_for(total), kThreads, 0, st, 
                (W *)c, (const W *)a, (const W *)b, p.d_limb, p.logN, p.L, total);
        }
        ++p.last_launches;
        return cudaGetLastError();
    });
}

cudaError_t launch_bitrev_permute(ntt_plan_s &p, void *data, uint32_t batch, cudaStream_t st) {
    const uint64_t total = (uint64_t)batch * p.L * p.N;
    if (p.word64) launch_dep(k_bitrev<uint64_t>, grid_for(total), kThreads, 0, st, (uint64_t *)data, p.logN, total);
    else launch_dep(k_bitrev<uint32_t>, grid_for(total), kThreads, 0, st, (uint32_t *)data, p.logN, total);
    ++p.last_launches;
    return cudaGetLastError();
}

cudaError_t launch_check_range(ntt_plan_s &p, const void *data, uint32_t batch, cudaStream_t st) {
    const uint64_t total = (uint64_t)batch * p.L * p.N;
    if (p.word64)
        launch_dep(k_check_range<uint64_t>, grid_for(total), kThreads, 0, st, (const uint64_t *)data, p.d_limb, p.logN,
                                                                     p.L, total, p.d_status);
    else
        launch_dep(k_check_range<uint32_t>, grid_for(total), kThreads, 0, st, (const uint32_t *)data, p.d_limb, p.logN,
                                                                     p.L, total, p.d_status);
    ++p.last_launches;
    return cudaGetLastError();
}

}  // namespace nttgb
