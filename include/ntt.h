/*
 * ntt.h -- C ABI of libnttgb, a batched negacyclic number theoretic
 * transform library for NVIDIA GB300 (sm_103a).
 *
 * What is computed.  For a prime q, N = 2^n and psi a primitive 2N-th root of
 * unity mod q, the forward transform of one limb a[0..N) is
 *
 *     X[k] = sum_{n<N} a[n] * psi^((2k+1) n)  mod q,      k = 0..N-1,
 *
 * the cyclic transform of Eq. 3 (Sec. II, "Twiddle Factors") with the input
 * twisted by psi^n so that it evaluates a(x) at the N roots of x^N + 1.  The
 * inverse maps X back to a: a[n] = N^-1 psi^-n sum_k X[k] psi^(-2nk).  The
 * pointwise product c[k] = a[k] b[k] mod q turns a negacyclic polynomial
 * product into O(N) work (Sec. I).  psi defaults to g^((q-1)/(2N)) with g the
 * smallest generator of Z_q^*.
 *
 * Data layout.  A batch is `batch` polynomials of L RNS limbs each, stored
 * [batch][L][N] contiguously; limb l is reduced modulo q[l].  Words are
 * uint32_t (q < 2^30) or, with NTT_WORD64, uint64_t (q < 2^60).  Inputs must
 * lie in [0, q); outputs are fully reduced to [0, q).
 *
 * Ownership.  The caller owns every data buffer.  A plan owns its twiddle
 * tables, its scratch buffer (grown on demand, see ntt_plan_reserve) and a
 * device status word.  Device pointers must be 16-byte aligned.
 *
 * Streams and errors.  Calls that take a stream only enqueue work on it and
 * return at once; their return value covers argument validation and launch
 * errors.  Errors found on the device (NTT_CHECK input violations, the
 * ragged kernel's wait limit) are recorded in the plan's status word and
 * returned by ntt_get_device_status.  No kernel ever traps.  A plan may be
 * used from one host thread at a time.
 */
#ifndef NTTGB_NTT_H
#define NTTGB_NTT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ntt_plan_s *ntt_plan_t;
typedef struct ntt_ragged_s *ntt_ragged_t;
/* A cudaStream_t passed as an opaque pointer; NULL is the legacy stream. */
typedef void *ntt_stream_t;

typedef enum {
    NTT_OK = 0,
    NTT_ERR_INVALID_ARG = 1,        /* null pointer, L = 0, batch = 0, bad enum */
    NTT_ERR_N_NOT_POW2 = 2,         /* N is not a power of two */
    NTT_ERR_N_RANGE = 3,            /* N outside 2^1 .. 2^17 */
    NTT_ERR_Q_NOT_PRIME = 4,        /* some q[l] is composite */
    NTT_ERR_Q_NOT_NTT_FRIENDLY = 5, /* some q[l] != 1 (mod 2N) */
    NTT_ERR_Q_WIDTH = 6,            /* q >= 2^30 (u32) or q >= 2^60 (u64) */
    NTT_ERR_ALIGNMENT = 7,          /* device pointer not 16-byte aligned */
    NTT_ERR_CUDA = 8,               /* a CUDA runtime call failed */
    NTT_ERR_OOM = 9,                /* device allocation failed */
    NTT_ERR_INPUT_RANGE = 10,       /* NTT_CHECK: an input word was >= q */
    NTT_ERR_TIMEOUT = 11,           /* a bounded device wait ran out */
    NTT_ERR_UNSUPPORTED = 12,       /* valid request this build cannot serve */
    NTT_ERR_PSI = 13,               /* caller psi is not a primitive 2N-th root */
    NTT_ERR_SCRATCH_LIMIT = 14      /* ntt_forward_noalloc: batch needs more
                                       than its fixed scratch array */
} ntt_status;

/* Dataflow variants of Sec. II.  All produce bit-identical results. */
typedef enum {
    NTT_DIT = 0,      /* Algorithm 1: bit reversal, then log2 N in-place stages */
    NTT_DIF = 1,      /* Algorithm 2: log2 N in-place stages, then bit reversal */
    NTT_FLAT = 2,     /* Sec. II "Flat-NTT": DIT with the two inner loops fused */
    NTT_PEASE = 3,    /* Eq. 7 / Algorithm 3: constant geometry + copy back */
    NTT_PEASE_NC = 4, /* Sec. II/III-B "Pease_nc": constant geometry, buffer swap */
    NTT_STOCKHAM = 5, /* Sec. II "Stockham": self-sorting ping-pong */
    NTT_SIXSTEP = 6,  /* Sec. II "Six-step": transposes + small sub-transforms */
    NTT_FUSED = 7,    /* fast path: stages fused per CTA in registers (Sec. II
                         twiddle precompute, Sec. III-C reductions) */
    NTT_TC_FOURSTEP = 8 /* four-step with tensor-core sub-transforms */
} ntt_variant;

/* plan flags */
#define NTT_WORD64 0x1u            /* uint64_t words, q < 2^60 */
#define NTT_ORDER_BITREV 0x2u      /* forward output / inverse input in
                                      bit-reversed order: position p holds
                                      X[bitrev_n(p)] */
#define NTT_RED_SHOUP 0x00u        /* twiddle products: Algorithm 5 (Shoup) */
#define NTT_RED_BARRETT 0x10u      /* Barrett reduction */
#define NTT_RED_MONTGOMERY 0x20u   /* Montgomery reduction */
#define NTT_RED_MASK 0x30u
#define NTT_CHECK 0x100u           /* record input words >= q on the device */
#define NTT_CLUSTER 0x200u         /* NTT_FUSED, N = 2^16, 4-byte words: one
                                      pass per transform on a cluster of eight
                                      CTAs (each word through DRAM once, the
                                      exchange in distributed shared memory)
                                      instead of the two-pass split; results
                                      identical, kept for comparison (on
                                      GB300 it moves half the DRAM bytes but
                                      takes longer: a cluster barrier per
                                      transform and single-buffered tiles) */
#define NTT_STREAMED 0x400u        /* NTT_FUSED, two-pass sizes (N > 2^14 with
                                      4-byte words, N > 2^13 with 8-byte): run
                                      both passes in one launch that streams
                                      limb by limb, so each limb's
                                      intermediate is read back while still
                                      in L2 (about a quarter less DRAM
                                      traffic), instead of the default two
                                      launches with the whole batch written
                                      to memory between them; results
                                      identical (NTT_FORM_STREAMED below).
                                      Calls in the streamed form use one of
                                      16 counter sets of the plan in turn:
                                      at most 16 such calls of one plan may
                                      overlap on the GPU */
#define NTT_TC_IMMA 0x800u         /* NTT_TC_FOURSTEP: the digit products on
                                      the warp-level integer MMA (mma.sync
                                      u8 x u8 -> s32) instead of tcgen05
                                      (fp16 digits, fp32 accumulators in
                                      tensor memory); results identical, kept
                                      for comparison */
#define NTT_TW_OTF 0x2000u         /* NTT_FUSED, 4-byte words, Shoup
                                      twiddles (else NTT_ERR_UNSUPPORTED):
                                      the second pass of a two-pass plan
                                      (N > 2^14) makes its twiddles on the
                                      fly instead of reading the per-chunk
                                      tables.  Entry 2^s + i of chunk r is
                                      psi^bitrev(2^s (N1 + r) + i) =
                                      A_s(r) * B_s(i), A_s(r) =
                                      psi^(2^(7-s) (1 + 2 bitrev(r))) (8
                                      words per chunk), B_s(i) =
                                      psi^(2^(n-s) bitrev_s(i)) (255 pairs
                                      per limb): one modular product and
                                      its Shoup quotient per entry, when a
                                      CTA stages a chunk's table.  The
                                      chunk tables (N + N/32 pairs per limb
                                      and direction) are not built; results
                                      identical.  No effect on single-pass
                                      sizes; not with NTT_STREAMED */
#define NTT_TEST_STALL 0x8000u     /* test hook, fused and tensor-core
                                      plans: in every forward call one CTA's
                                      first tile (or first matrix copy)
                                      waits for 16 bytes that never arrive,
                                      so its bounded wait runs out (about a
                                      second) and ntt_get_device_status then
                                      reports NTT_ERR_TIMEOUT; the results of
                                      that call are not valid.  Ragged sets
                                      (ntt_ragged_create, not with
                                      NTT_RAGGED_TUNE): in every launch CTA 0
                                      leaves before the first grid barrier,
                                      the other CTAs' bounded barrier wait
                                      runs out (about two seconds) and
                                      ntt_ragged_status reports
                                      NTT_ERR_TIMEOUT; the results are not
                                      valid */

/*
 * Create a plan for batches of L-limb polynomials of N coefficients.
 * q[0..L) are the limb primes (copied).  Validates N (power of two,
 * 2 <= N <= 2^17), every q (prime, q = 1 mod 2N, below the word limit),
 * then builds the bit-reversed psi / psi^-1 twiddle tables of Sec. II
 * ("Twiddle Factors": all twiddles precomputed) with the companions the
 * selected reduction needs, and copies them to the current CUDA device.
 * On error *plan is set to NULL and nothing is allocated.
 */
ntt_status ntt_plan_create(ntt_plan_t *plan, uint32_t N, const uint64_t *q,
                           uint32_t L, ntt_variant variant, uint32_t flags);

/* As ntt_plan_create, with the caller's roots psi[0..L) (NULL = default).
 * Each psi[l] must satisfy psi^N = -1 (mod q[l]); else NTT_ERR_PSI. */
ntt_status ntt_plan_create_ex(ntt_plan_t *plan, uint32_t N, const uint64_t *q,
                              uint32_t L, ntt_variant variant, uint32_t flags,
                              const uint64_t *psi);

/* Release the plan's device memory (after synchronising its last stream). */
void ntt_plan_destroy(ntt_plan_t plan);

/* Pre-size the plan's scratch buffer for batches up to max_batch
 * polynomials, so that later calls allocate nothing.  Variants that work in
 * place (DIT, DIF, Flat, and Fused with NTT_ORDER_BITREV) need none. */
ntt_status ntt_plan_reserve(ntt_plan_t plan, uint32_t max_batch,
                            ntt_stream_t stream);

/*
 * Forward negacyclic NTT of `batch` polynomials in place: d_data holds
 * [batch][L][N] words on the device; afterwards position k holds X[k]
 * (natural order) or X[bitrev(k)] (NTT_ORDER_BITREV).  Eq. 3 with the psi
 * twist; the butterfly dataflow is the plan's variant (Algorithms 1-3,
 * Sec. II).
 */
ntt_status ntt_forward(ntt_plan_t plan, void *d_data, uint32_t batch,
                       ntt_stream_t stream);

/* Inverse negacyclic NTT in place (input order as ntt_forward's output). */
ntt_status ntt_inverse(ntt_plan_t plan, void *d_data, uint32_t batch,
                       ntt_stream_t stream);

/* As ntt_forward / ntt_inverse for polynomials of only the plan's first
 * `limbs` primes (1 <= limbs <= L): d_data holds [batch][limbs][N] words.
 * RNS schemes drop limbs as they rescale; one plan serves every level. */
ntt_status ntt_forward_prefix(ntt_plan_t plan, void *d_data, uint32_t batch,
                              uint32_t limbs, ntt_stream_t stream);
ntt_status ntt_inverse_prefix(ntt_plan_t plan, void *d_data, uint32_t batch,
                              uint32_t limbs, ntt_stream_t stream);

/*
 * c[k] = a[k] * b[k] mod q[l] for [batch][L][N] arrays (Sec. I: the product
 * step of NTT-based polynomial multiplication).  d_c may alias d_a or d_b.
 * Uses Barrett reduction (Montgomery under NTT_RED_MONTGOMERY).
 */
ntt_status ntt_pointwise_mul(ntt_plan_t plan, void *d_c, const void *d_a,
                             const void *d_b, uint32_t batch,
                             ntt_stream_t stream);

/*
 * c = INTT(a (.) b): the pointwise product followed by the inverse
 * transform (Sec. I: the last two steps of NTT-based polynomial
 * multiplication), for [batch][L][N] arrays of forward outputs; c then holds
 * the coefficients of the negacyclic products.  Same result as
 * ntt_pointwise_mul(c, a, b) then ntt_inverse(c).  For fused plans of the
 * two-pass size range (N > 2^14 with 4-byte words, N > 2^13 with 8-byte)
 * in bit-reversed order without NTT_CHECK, the product is taken inside the
 * first inverse pass (b is read beside a), saving a write and a read of c;
 * other plans run the two steps.  d_c may alias d_a or d_b, or be disjoint
 * from both; partial overlaps are not allowed.
 */
ntt_status ntt_pointwise_inverse(ntt_plan_t plan, void *d_c, const void *d_a,
                                 const void *d_b, uint32_t batch,
                                 ntt_stream_t stream);

/*
 * End-to-end negacyclic products from host memory, for `pairs` products:
 * h_in holds [2][pairs][L][N] words (all first factors, then all second
 * factors), h_out receives [pairs][L][N] words of a_i * b_i mod
 * (x^N + 1, q).  d_work is a device buffer of at least 2*pairs*L*N words
 * (its contents are overwritten).  The products are computed as up to 8
 * chunks of pairs (fused plans with one or two pairs: windows of limbs of
 * each pair, about 4 chunks in all) in a pipeline: each chunk's
 * host-to-device copy, its forward NTTs, pointwise product and inverse NTT,
 * and its device-to-host copy, with the copies on two streams the plan
 * owns and the transforms on
 * `stream`, so copies of one chunk overlap the arithmetic of others.  The
 * call is ordered after earlier work on `stream`, and later work on `stream`
 * after all of it; the caller synchronises `stream` before reading h_out.
 * Host buffers should be pinned (pageable memory serialises the copies).
 * The first call on a plan creates its streams and events: make it outside
 * stream capture.  Calls on one plan must not run concurrently from several
 * host threads.
 */
ntt_status ntt_polymul_host(ntt_plan_t plan, void *h_out, const void *h_in,
                            void *d_work, uint32_t pairs, ntt_stream_t stream);

/*
 * Forward transform that allocates nothing (the paper has no counterpart;
 * this is a deployment aid).  For callers that must not allocate device
 * memory -- a framework that owns all device memory through its own pool, a
 * latency-bound loop that cannot afford cudaMalloc's implicit device
 * synchronisation, a plugin under a fixed memory budget -- it runs the
 * forward transform with the Stockham dataflow using, as its ping-pong
 * buffer, a fixed 8 MiB device array that is part of the library (held by
 * every GPU that loads the library until the process exits).  The caller
 * passes the data; no cudaMalloc, cudaFree or other allocating call is
 * made.  Same result, order and NTT_CHECK behaviour as ntt_forward on the
 * same plan; ntt_plan_last_launches counts its launches.
 *   - Plans of the fused variant with N >= 16 have no per-stage tables:
 *     NTT_ERR_UNSUPPORTED.  (Tensor-core four-step plans carry them and are
 *     served.)
 *   - batch * L * N * word bytes must not exceed 8 MiB, else
 *     NTT_ERR_SCRATCH_LIMIT (e.g. at most one 32-limb polynomial of 2^16
 *     u32 words per call).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it per CUDA context; make that first
 *     call, and the first call after a cudaDeviceReset, before any stream
 *     capture.
 *   - All calls share the array and it keeps the last call's contents
 *     (nothing in it needs to start at zero); calls whose work overlaps on
 *     the GPU race on it.
 */
ntt_status ntt_forward_noalloc(ntt_plan_t plan, void *d_data, uint32_t batch,
                               ntt_stream_t stream);

/* Synchronise `stream`, then return and clear the plan's sticky device
 * status (NTT_OK, NTT_ERR_INPUT_RANGE or NTT_ERR_TIMEOUT). */
ntt_status ntt_get_device_status(ntt_plan_t plan, ntt_stream_t stream);

/* Copy the plan's roots psi[0..L) to host memory. */
ntt_status ntt_plan_get_psi(ntt_plan_t plan, uint64_t *psi_out);

/* Number of kernels the last ntt_forward / ntt_inverse / ntt_pointwise_mul
 * call on this plan launched (for launch accounting). */
uint32_t ntt_plan_last_launches(ntt_plan_t plan);

/* Bytes of device memory the plan holds for its tables (twiddles, limb
 * constants, tensor-core matrices), without the scratch buffer, its status
 * word and progress counters; 0 for a null plan. */
uint64_t ntt_plan_table_bytes(ntt_plan_t plan);

/* Human-readable name of a status code (static string). */
const char *ntt_status_string(ntt_status s);

/* ------------------------------------------------ host-only number theory
 * These touch no GPU and may be called on a machine without one. */

/* Same checks as ntt_plan_create, without building anything. */
ntt_status ntt_validate(uint32_t N, const uint64_t *q, uint32_t L,
                        uint32_t flags);

/* Default root psi = g^((q-1)/(2N)) (g = smallest generator of Z_q^*). */
ntt_status ntt_default_psi(uint64_t q, uint32_t N, uint64_t *psi_out);

/* The first `count` primes q = 2^bits - k 2^m + 1 (k = 1, 2, ...) with
 * 2^(bits-1) < q < 2^bits, in descending order; NTT_ERR_INVALID_ARG if
 * fewer exist or bits is outside 3..62. */
ntt_status ntt_find_primes(uint32_t bits, uint32_t m, uint32_t count,
                           uint64_t *out);

/* Limb sharding across processes (one GPU each).  Every limb of an RNS
 * polynomial is transformed modulo its own prime, independently of the
 * others (the per-limb transform of Eq. 3), so L limbs split into `world`
 * contiguous slices with no exchange on the transform path: rank r holds
 * limbs [*first, *first + *count) of every polynomial, as [batch][count][N]
 * words, and makes its plan over q[*first .. *first + *count).  The slices
 * are balanced (the first L mod world ranks hold one limb more) and in rank
 * order, so gathering them in rank order restores [batch][L][N] -- the one
 * exchange a sharded pipeline needs, before a step that reads every limb of
 * a coefficient (ntt_bconv).  Host-only.  NTT_ERR_INVALID_ARG for a null
 * pointer, world = 0, rank >= world or L < world. */
ntt_status ntt_limb_shard(uint32_t L, uint32_t world, uint32_t rank,
                          uint32_t *first, uint32_t *count);

/* ------------------------------------------------------------ autotuner
 * The two-pass fused path (N > 2^14 with 4-byte words, N > 2^13 with
 * 8-byte) leaves three things open.  The split N = 2^s1 x 2^s2: the first
 * pass runs the first s1 stages on columns of 2^s1 points, the second the
 * last s2 stages on chunks of 2^s2 consecutive words (the four-step split
 * of Sec. II); s2 is 7, 8 or 9 with 5 <= s1 <= 9, default 8.  The radix of
 * the register rounds inside each pass: radix_log2 = 4 (rounds of four
 * radix-2 stages on 16 words a thread, the default) or 3 (three stages on
 * 8 words).  The plan's twiddle tables are laid out for both at creation.
 * (NTT_STREAMED and NTT_TW_OTF plans keep s2 = 8, radix_log2 = 4.)  And
 * each direction's form: */
#define NTT_FORM_SMALL 0      /* chunk pass on one-warp CTAs */
#define NTT_FORM_WIDE 1       /* chunk pass on 256-thread CTAs */
#define NTT_FORM_STREAMED 2   /* both passes in one streamed launch (s2 = 8) */
#define NTT_FORM_SMALL_SHFL 3 /* NTT_FORM_SMALL with the chunk pass's
                                 exchanges between register rounds by warp
                                 shuffles instead of shared memory */
#define NTT_FORM_WIDE_SHFL 4  /* the same for NTT_FORM_WIDE */
/* Defaults: NTT_FORM_SMALL forward, NTT_FORM_WIDE inverse (NTT_FORM_STREAMED
 * both ways under NTT_STREAMED).  Chunk tiles hold the same chunk of
 * several polynomials (one twiddle table a tile) when their count divides
 * the batch and chunks have at least 256 words, else several chunks of one
 * polynomial.  The shuffle forms exist for 4-byte words with twiddle
 * tables (a plan with NTT_WORD64 or NTT_TW_OTF runs them as their
 * shared-memory forms); a chunk's threads are lanes of one warp except for
 * 512-word chunks in radix 8, whose exchanges stay in shared memory.
 * Results are identical in every split, form and tiling. */
typedef struct {
    float forward_ms[5];      /* per form, ms per call, at the chosen
                                 radix and split */
    float inverse_ms[5];
    int32_t forward_form;     /* the fastest */
    int32_t inverse_form;
    int32_t chunk_log2;       /* the chosen split s2 */
    int32_t radix_log2;       /* the chosen radix (3 or 4) */
    float config_ms[2][3];    /* [radix_log2 - 3][s2 - 7]: fastest forward +
                                 fastest inverse, ms; -1 where not valid */
} ntt_tune_result;

/* Time every valid (radix, split), and in each every form of both
 * directions, for (N, q[0..L), flags, batch) on the current device (a
 * scratch buffer of batch x L x N zero words, allocated and freed here);
 * record per (radix, split) the fastest form per direction in the
 * process-wide tuning table, keyed by (N, word size, L, reduction, order,
 * NTT_TW_OTF or not, s2, radix, floor(log2 batch)), and for the shape the
 * (radix, split) with the smallest forward + inverse time.  Plans created
 * afterwards with that shape take that radix and split and use the
 * recorded forms for calls in that batch bucket (NTT_STREAMED plans keep
 * theirs).  Forms that do not exist (streamed with s2 != 8, radix 3 or
 * NTT_TW_OTF; the shuffle forms with NTT_WORD64 or NTT_TW_OTF) are
 * reported as -1 and never chosen.  If the environment
 * variable NTT_TUNE_DB names a file, the tables are read from it at first
 * use and rewritten after each tuning (one JSON object per line).  flags:
 * as ntt_plan_create, without NTT_STREAMED, NTT_CHECK or NTT_TEST_STALL.
 * NTT_ERR_UNSUPPORTED for sizes outside the two-pass range.  result may be
 * NULL. */
ntt_status ntt_autotune(uint32_t N, const uint64_t *q, uint32_t L,
                        uint32_t flags, uint32_t batch, ntt_stream_t stream,
                        ntt_tune_result *result);

/* The form a plan uses for calls with this batch (0: forward, else
 * inverse), or -1 when the plan is not on the two-pass fused path. */
int32_t ntt_plan_form(ntt_plan_t plan, uint32_t batch, int inverse);

/* The plan's split s2 (chunks of 2^s2 words) and radix (3 or 4), or -1
 * when the plan is not on the two-pass fused path. */
int32_t ntt_plan_chunk_log2(ntt_plan_t plan);
int32_t ntt_plan_radix_log2(ntt_plan_t plan);

/* Host-only access to the tuning tables (no GPU needed): record forms for a
 * shape by hand, for the shape's current radix and split (saved to
 * NTT_TUNE_DB like a tuning; NTT_ERR_INVALID_ARG for a form outside 0..2 or
 * batch 0); read the form recorded for a shape's radix, split and
 * direction (-1: none); record a shape's split and radix
 * (NTT_ERR_INVALID_ARG for a pair the shape cannot take); read them (the
 * split is returned, the radix stored in *radix_log2 if not NULL; -1 for
 * both: none recorded, plans use s2 = 8, radix 4); empty the in-memory
 * tables (the file is not read again in this process).  Plans copy the
 * tables at creation. */
ntt_status ntt_tune_set(uint32_t N, uint32_t L, uint32_t flags, uint32_t batch,
                        int32_t forward_form, int32_t inverse_form);
int32_t ntt_tune_get(uint32_t N, uint32_t L, uint32_t flags, uint32_t batch,
                     int inverse);
ntt_status ntt_tune_set_split(uint32_t N, uint32_t L, uint32_t flags,
                              uint32_t chunk_log2, uint32_t radix_log2);
int32_t ntt_tune_get_split(uint32_t N, uint32_t L, uint32_t flags,
                           int32_t *radix_log2);
void ntt_tune_clear(void);

/* ------------------------------------------------ integer roofline
 * Measures the rate of 32-bit integer multiply-adds (the denominator the
 * butterfly kernels are reported against; not part of the paper's method):
 * launches blocks x 256 threads (blocks = 8 per SM, written to *blocks_out),
 * each running 8 independent chains of `iters` mad.lo.u32 (high = 0) or
 * mad.hi.u32 (high = 1) steps, i.e. blocks x 256 x 8 x iters operations;
 * the caller times the launch on `stream`.  d_scratch receives one word per
 * thread (scratch_bytes >= blocks x 1 KiB, else NTT_ERR_INVALID_ARG). */
ntt_status ntt_measure_int_mad_rate(int high, uint32_t iters, void *d_scratch,
                                    size_t scratch_bytes, uint32_t *blocks_out,
                                    ntt_stream_t stream);

/* ------------------------------------------------ RNS base conversion
 * Fast base conversion of coefficient residues (the basis-extension step
 * that follows the inverse transform in RNS homomorphic schemes, the
 * setting Sec. I motivates the NTT with; the paper defines no conversion).
 * For every coefficient with residues x_i = x mod q_i (i < L), Q = prod q_i,
 * qhat_i = Q / q_i:
 *     y_i = x_i qhat_i^-1 mod q_i,
 *     z_j = (sum_i y_i qhat_i) mod p_j                      (j < K),
 * so z_j = (x + alpha Q) mod p_j for one integer 0 <= alpha < L (the fast,
 * approximate conversion; no correction of alpha is made).  4-byte words:
 * every q_i and p_j prime, 3 <= prime < 2^30; the q_i distinct;
 * 1 <= L, K <= 64; N >= 1 coefficients per polynomial (any N). */
typedef struct ntt_bconv_s *ntt_bconv_t;

/* Build the conversion tables (host arithmetic, one device upload).
 * NTT_ERR_INVALID_ARG (null, L or K out of range, N = 0, repeated q_i),
 * NTT_ERR_Q_WIDTH, NTT_ERR_Q_NOT_PRIME, NTT_ERR_OOM. */
ntt_status ntt_bconv_create(ntt_bconv_t *out, const uint64_t *q, uint32_t L,
                            const uint64_t *p, uint32_t K, uint32_t N);

/* d_in: [batch][L][N] uint32_t residues (x_i < q_i), d_out: [batch][K][N]
 * uint32_t, fully reduced; device pointers, 4-byte aligned, not
 * overlapping.  Enqueued on `stream`, one launch. */
ntt_status ntt_bconv(ntt_bconv_t plan, void *d_out, const void *d_in,
                     uint32_t batch, ntt_stream_t stream);

/* Free the tables (after synchronising the device). */
void ntt_bconv_destroy(ntt_bconv_t plan);

/* ------------------------------------------------------- ragged batches
 * One persistent kernel, captured in a CUDA graph, runs every job of a
 * heterogeneous set (different N, L, word width, direction). */
typedef struct {
    void *d_data;         /* [batch][L][N] words on the device */
    const uint64_t *q;    /* L host primes (copied at create) */
    uint32_t N;           /* 2^12 .. 2^17 */
    uint32_t L;           /* limbs */
    uint32_t batch;       /* polynomials */
    uint32_t word64;      /* 0: uint32_t words (q < 2^30), 1: uint64_t */
    int32_t inverse;      /* 0 forward, 1 inverse */
    uint32_t reserved;
} ntt_job;

/* Validate the jobs (2^12 <= N <= 2^17), build twiddle tables once per
 * (N, word size, prime list) -- a job whose primes are a prefix of another
 * job's list shares its tables -- cut the passes of every transform into
 * work items, and capture one cooperative launch of the persistent kernel
 * into a CUDA graph.  All forward jobs complete before any inverse job
 * starts, so a set holding a forward and an inverse job on the same buffer
 * is a round trip.  flags: NTT_ORDER_BITREV (required: the ragged kernel
 * works in bit-reversed evaluation order), NTT_RED_*, NTT_RAGGED_TUNE
 * and the test hook NTT_TEST_STALL.  The job array and its q arrays are copied; the data
 * buffers must stay valid (their contents are not touched here). */
#define NTT_RAGGED_TUNE 0x1000u   /* autotune the work-item size: time items
                                     of 2, 4, 8 and 16 tiles (three launches
                                     each) on zeroed scratch copies of the
                                     jobs' buffers, allocated and freed here,
                                     and capture the fastest; default 8 */
ntt_status ntt_ragged_create(ntt_ragged_t *out, const ntt_job *jobs,
                             uint32_t n_jobs, uint32_t flags);

/* Tiles per work item the ragged set was captured with. */
uint32_t ntt_ragged_item_tiles(ntt_ragged_t r);

/* Replay the captured graph on `stream`. */
ntt_status ntt_ragged_launch(ntt_ragged_t r, ntt_stream_t stream);

/* Synchronise `stream` and return the ragged kernel's device status. */
ntt_status ntt_ragged_status(ntt_ragged_t r, ntt_stream_t stream);

void ntt_ragged_destroy(ntt_ragged_t r);

#ifdef __cplusplus
}
#endif

#endif /* NTTGB_NTT_H */
