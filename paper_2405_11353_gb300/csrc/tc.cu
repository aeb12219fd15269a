// tc.cu -- four-step transform for N = 2^16 with the 256-point sub-transforms
// as exact split-integer products on the tensor cores.
//
// Four-step split (Sec. II, "Six-step": a large transform as smaller ones)
// of the negacyclic forward transform, with the data viewed as A[n1][n2],
// n = 256 n1 + n2, and the output in the bit-reversed order of the fused
// path (position 256 u + v holds X[bitrev16(256 u + v)], i.e. X[k1 + 256 k2]
// with k1 = bitrev8(u), k2 = bitrev8(v)):
//   C[u][n2] = T[u][n2] * sum_n1 M1[u][n1] A[n1][n2]
//   Y[u][v]  = sum_n2 C[u][n2] M2[v][n2]
//   M1[u][n1] = psi^(256 (2 k1 + 1) n1),  T[u][n2] = psi^(n2 (2 k1 + 1)),
//   M2[v][n2] = psi^(512 k2 n2)       (all mod q).
// The inverse runs the same two kinds of pass backwards with the inverse
// matrices (each carrying 1/256) and T^-1.
//
// Each 256 x 256 x 256 product mod q is exact on the integer tensor cores:
// both operands are split into four 8-bit digits, x = sum_i x_i 2^(8 i), and
// the 16 digit products are accumulated by diagonal s = i + j in 32-bit
// integers (at most 4 * 256 * 255^2 < 2^26 per entry, so nothing overflows
// or rounds), then recombined as sum_s S_s (2^(8 s) mod q) in 64 bits
// (< 2^59) and reduced (Barrett).  The digit products use the warp-level
// mma.sync m16n8k32 u8 x u8 -> s32 instruction: on sm_103a this is the
// integer tensor-core path (the tcgen05 MMA has no 8-bit integer kind on
// this target).
#include <cuda_runtime.h>

#include "modarith.cuh"
#include "plan.hpp"

namespace nttgb {
namespace {

// bytes per digit-plane row: 256 + 16, so the 8 rows x 4 words a fragment
// load touches fall on 32 distinct banks
constexpr int kPitch = 272;
constexpr int kPlane = 32 * kPitch;

__device__ __forceinline__ void imma(int (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t digits_of(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3, int j) {
    const int sh = 8 * j;
    return ((x0 >> sh) & 255u) | (((x1 >> sh) & 255u) << 8) | (((x2 >> sh) & 255u) << 16) |
           (((x3 >> sh) & 255u) << 24);
}

struct TcArgs {
    uint32_t *data;
    const uint8_t *mat;            // [L][4 digits][256][256]: row = output index, column = sum index
    const Tw<uint32_t> *tw;        // [L][256][256] twiddles of the epilogue (or null)
    const LimbConst *lc;
    const uint32_t *pow8;          // [L][8]: 2^(8 s) mod q
    uint32_t L;
};

// The warp's 32 x 32 output block over a sum of length 256: per diagonal s,
// the digit pairs (i, j = s - i) accumulate into 32-bit integers, then the
// diagonal is added into the 64-bit combination with weight 2^(8 s) mod q.
// A_SMEM: the A operand (rows) comes from the shared digit planes and B from
// the constant matrix; otherwise A is the constant matrix.
template <bool A_SMEM>
__device__ __forceinline__ void warp_product(uint64_t (&comb)[2][4][4], const uint8_t *planes, const uint8_t *mat,
                                             uint32_t a_row0, uint32_t b_col0, const uint32_t *pow8) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) comb[mt][nt][r] = 0;
#pragma unroll 1
    for (int s = 0; s < 7; ++s) {
        int acc[2][4][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[mt][nt][r] = 0;
        const int i_lo = s > 3 ? s - 3 : 0, i_hi = s < 3 ? s : 3;
#pragma unroll 1
        for (int i = i_lo; i <= i_hi; ++i) {
            const int j = s - i;
            const uint8_t *pa, *pb;
            if (A_SMEM) { pa = planes + i * kPlane; pb = mat + (size_t)j * 65536; }
            else { pa = mat + (size_t)i * 65536; pb = planes + j * kPlane; }
#pragma unroll 2
            for (int k0 = 0; k0 < 256; k0 += 32) {
                uint32_t a[2][4], b[4][2];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const uint32_t r0 = a_row0 + 16 * mt + g;
                    if (A_SMEM) {
                        const uint8_t *p = pa + r0 * kPitch + k0 + 4 * t;
                        a[mt][0] = *reinterpret_cast<const uint32_t *>(p);
                        a[mt][1] = *reinterpret_cast<const uint32_t *>(p + 8 * kPitch);
                        a[mt][2] = *reinterpret_cast<const uint32_t *>(p + 16);
                        a[mt][3] = *reinterpret_cast<const uint32_t *>(p + 8 * kPitch + 16);
                    } else {
                        const uint32_t *p = reinterpret_cast<const uint32_t *>(pa + r0 * 256 + k0 + 4 * t);
                        a[mt][0] = __ldg(p);
                        a[mt][1] = __ldg(p + 8 * 64);
                        a[mt][2] = __ldg(p + 4);
                        a[mt][3] = __ldg(p + 8 * 64 + 4);
                    }
                }
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const uint32_t c = b_col0 + 8 * nt + g;
                    if (A_SMEM) {
                        const uint32_t *p = reinterpret_cast<const uint32_t *>(pb + c * 256 + k0 + 4 * t);
                        b[nt][0] = __ldg(p);
                        b[nt][1] = __ldg(p + 4);
                    } else {
                        const uint8_t *p = pb + c * kPitch + k0 + 4 * t;
                        b[nt][0] = *reinterpret_cast<const uint32_t *>(p);
                        b[nt][1] = *reinterpret_cast<const uint32_t *>(p + 16);
                    }
                }
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt) imma(acc[mt][nt], a[mt], b[nt][0], b[nt][1]);
            }
        }
        const uint64_t w = pow8[s];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int r = 0; r < 4; ++r) comb[mt][nt][r] += (uint64_t)(uint32_t)acc[mt][nt][r] * w;
    }
}

// Column pass: out[u][c0 + c] = (T[u][c0 + c]) * sum_k mat[u][k] data[k][c0 + c]
// for one transform and a strip of 32 columns (all 256 rows).
template <bool TWEPI>
__global__ void __launch_bounds__(256) k_tc_cols(TcArgs a) {
    __shared__ __align__(16) uint8_t planes[4 * kPlane];
    const uint64_t t = blockIdx.x >> 3;
    const uint32_t c0 = (blockIdx.x & 7) * 32;
    const uint32_t l = (uint32_t)(t % a.L);
    uint32_t *x = a.data + t * 65536;
    // digit planes, transposed: plane[j][c][k] = digit j of data[k][c0 + c]
    for (uint32_t task = threadIdx.x; task < 2048; task += 256) {
        const uint32_t c = task & 31, k = (task >> 5) * 4;
        const uint32_t x0 = x[(k + 0) * 256 + c0 + c], x1 = x[(k + 1) * 256 + c0 + c];
        const uint32_t x2 = x[(k + 2) * 256 + c0 + c], x3 = x[(k + 3) * 256 + c0 + c];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            *reinterpret_cast<uint32_t *>(planes + j * kPlane + c * kPitch + k) = digits_of(x0, x1, x2, x3, j);
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    uint64_t comb[2][4][4];
    warp_product<false>(comb, planes, a.mat + (size_t)l * 4 * 65536, 32 * w, 0, a.pow8 + 8 * l);
    Lc<uint32_t> kk;
    kk.load(a.lc + l);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint32_t u = 32 * w + 16 * mt + g + 8 * (r >> 1);
                const uint32_t c = c0 + 8 * nt + 2 * tq + (r & 1);
                uint32_t v = csub<uint32_t>(barrett_lazy(comb[mt][nt][r], kk), kk.q);
                if (TWEPI) v = mul_full<RED_SHOUP>(v, ldtw(a.tw + (size_t)l * 65536 + u * 256 + c), kk);
                x[u * 256 + c] = v;
            }
}

// Row pass: out[r0 + r][n] = (T[r0 + r][n]) * sum_k data[r0 + r][k] mat[n][k]
// for one transform and a block of 32 rows (all 256 columns).
template <bool TWEPI>
__global__ void __launch_bounds__(256) k_tc_rows(TcArgs a) {
    __shared__ __align__(16) uint8_t planes[4 * kPlane];
    const uint64_t t = blockIdx.x >> 3;
    const uint32_t r0 = (blockIdx.x & 7) * 32;
    const uint32_t l = (uint32_t)(t % a.L);
    uint32_t *x = a.data + t * 65536;
    for (uint32_t task = threadIdx.x; task < 2048; task += 256) {
        const uint32_t r = task >> 6, k = (task & 63) * 4;
        const uint4 v = *reinterpret_cast<const uint4 *>(x + (r0 + r) * 256 + k);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            *reinterpret_cast<uint32_t *>(planes + j * kPlane + r * kPitch + k) = digits_of(v.x, v.y, v.z, v.w, j);
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    uint64_t comb[2][4][4];
    warp_product<true>(comb, planes, a.mat + (size_t)l * 4 * 65536, 0, 32 * w, a.pow8 + 8 * l);
    Lc<uint32_t> kk;
    kk.load(a.lc + l);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint32_t u = r0 + 16 * mt + g + 8 * (r >> 1);
                const uint32_t n = 32 * w + 8 * nt + 2 * tq + (r & 1);
                uint32_t v = csub<uint32_t>(barrett_lazy(comb[mt][nt][r], kk), kk.q);
                if (TWEPI) v = mul_full<RED_SHOUP>(v, ldtw(a.tw + (size_t)l * 65536 + u * 256 + n), kk);
                x[u * 256 + n] = v;
            }
}

}  // namespace

// TC table layout (plan->d_tc): matrices [4][L][4 digits][256][256] u8
// (0: forward column matrix, 1: forward row matrix, 2: inverse row matrix,
// 3: inverse column matrix; row = output index, column = sum index), then
// twiddles [2][L][256][256] Shoup pairs (0: forward column epilogue, 1:
// inverse row epilogue), then [L][8] u32 powers 2^(8 s) mod q.
cudaError_t launch_tc(ntt_plan_s &p, void *data, uint32_t batch, bool inverse, cudaStream_t st) {
    const uint64_t ntrans = (uint64_t)batch * p.L;
    const uint8_t *mats = reinterpret_cast<const uint8_t *>(p.d_tc);
    const Tw<uint32_t> *tws = reinterpret_cast<const Tw<uint32_t> *>(mats + (size_t)p.L * 16 * 65536);
    const uint32_t *pow8 = reinterpret_cast<const uint32_t *>(tws + (size_t)p.L * 2 * 65536);
    TcArgs a;
    a.data = reinterpret_cast<uint32_t *>(data);
    a.lc = p.d_limb;
    a.pow8 = pow8;
    a.L = p.L;
    const unsigned grid = (unsigned)(ntrans * 8);
    // kernels add l * 4 * 65536 (one limb's four digit planes) to `mat`
    auto mat = [&](int m) { return mats + (size_t)m * p.L * 4 * 65536; };
    if (!inverse) {
        a.mat = mat(0); a.tw = tws;
        k_tc_cols<true><<<grid, 256, 0, st>>>(a);
        a.mat = mat(1); a.tw = nullptr;
        k_tc_rows<false><<<grid, 256, 0, st>>>(a);
    } else {
        a.mat = mat(2); a.tw = tws + (size_t)p.L * 65536;
        k_tc_rows<true><<<grid, 256, 0, st>>>(a);
        a.mat = mat(3); a.tw = nullptr;
        k_tc_cols<false><<<grid, 256, 0, st>>>(a);
    }
    p.last_launches += 2;
    return cudaGetLastError();
}

}  // namespace nttgb
