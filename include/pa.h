/*
 * pa.h - C ABI of the GB300 privacy-amplification hash library (libpa_gb300.so).
 *
 * The library computes the modular-arithmetic universal_2 hash of
 * arXiv 1910.04429 (Sec. 2.3, Definition 5, Eq. 6 and Eq. 7):
 *
 *     g_{c,d}(x) = floor( ((c * x + d) mod 2^n) / 2^(n - m) )
 *
 * which compresses an n-bit reconciled key x to an m-bit final key using the
 * public seed (c, d) (Sec. 2.2: Alice and Bob publicly pick one g from the
 * family and apply it to their identical strings). Here c is called seed_a
 * and d seed_b. The product is exact: an NTT over the Goldilocks prime
 * 2^64 - 2^32 + 1 on 16- to 20-bit digits (Algorithm 1, Sec. 3.2.2, with GF(p) in
 * place of GMP's Fermat ring), then carry resolve, + d, mod 2^n and
 * extraction of the m most significant bits of the n-bit field (Sec. 3.2.3-
 * 3.2.5).
 *
 * Data layout (all entry points): an integer of w bits is an array of
 * ceil(w/64) uint64_t limbs, least significant limb first; integer bit i is bit
 * (i mod 64) of limb floor(i/64) (the least-significant-word-first import of
 * Sec. 3.2.1). Input bits at positions >= n are ignored (operands are elements
 * of Z_{2^n}); output bits at positions >= m are written as zero.
 *
 * Ownership: every buffer passed in is owned by the caller and must stay
 * valid until the work queued on `stream` has finished. Device pointers must
 * point to memory of the current CUDA device. The library owns its transform
 * workspace (stream-ordered allocations from its own memory pool) and its
 * twiddle tables (one set per device and transform size, kept until
 * pa_shutdown or process exit).
 *
 * Streams: `stream` is a cudaStream_t passed as void*; NULL means the legacy
 * default stream. Calls are asynchronous unless stated otherwise. The first
 * call for a new transform size on a device builds that size's twiddle tables
 * with a synchronous upload, so make that first call (or pa_prepare) before
 * any stream capture.
 *
 * Errors: every entry point returns an int status. On PA_EINVAL nothing has
 * been queued. A CUDA error while queueing returns PA_ECUDA (the message is
 * available from pa_last_error()).
 */
#ifndef PA_GB300_H
#define PA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PA_OK 0
#define PA_EINVAL (-1)   /* bad size, null pointer, m > n, or n beyond PA_MAX_BITS */
#define PA_ENOMEM (-2)   /* device or host allocation failed */
#define PA_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define PA_EAGAIN (-4)   /* serving: queue full / result not ready yet */
#define PA_ETIMEOUT (-5) /* a bounded device wait expired */

/* Largest key length: 2^31 bits (transform length 2^28, two 2 GiB buffers). */
#define PA_MAX_BITS (1ull << 31)

/*
 * pa_hash: out = floor(((seed_a * key + seed_b) mod 2^n) / 2^(n-m)).
 *   key, seed_a, seed_b : device pointers, ceil(n/64) limbs each (read only)
 *   n                   : key length in bits, 1 <= n <= PA_MAX_BITS
 *   m                   : output length in bits, 1 <= m <= n (the final-key
 *                         length r of Sec. 2.2 Eq. 1 and Sec. 3.2.5)
 *   out                 : device pointer, ceil(m/64) limbs (written)
 *   stream              : cudaStream_t or NULL
 * seed_a need not be odd: the formula is evaluated for any value (the family
 * of Eq. 6 draws odd c; that is the caller's choice of seed).
 * Returns PA_OK once all kernels are queued (asynchronous).
 *
 * Only bits [n-m, n) of the product mod 2^n reach the output, so where it is
 * shorter the product runs as a cyclic convolution of length N < 2L - 1
 * (L = ceil(n/w) digits of w bits, see pa_digit_width) whose wrapped-around part lands on the lowest
 * coefficients; those are dropped. The carry step then checks the limb of the
 * exact remaining sum just below bit n - m: unless all 64 of its bits are one,
 * the dropped part cannot reach the output and the result is exact. If they
 * are all one, an exact recomputation queued behind (one launch that returns
 * at once otherwise) computes the full product at a power-of-two length and
 * overwrites the output. With uniform seed_b this happens with probability
 * 2^-64 per hash; results are identical either way (see pa_plan_info,
 * pa_wrap_mode).
 */
int pa_hash(const uint64_t* key, const uint64_t* seed_a, const uint64_t* seed_b, uint64_t n,
            uint64_t m, uint64_t* out, void* stream);

/*
 * pa_hash_host: pa_hash on HOST buffers (same shapes); returns with `out`
 * filled (it waits for `stream`). key and seed_a are copied into device
 * staging buffers from the library's pool on the library's copy stream, and
 * seed_b behind them, so b's copy overlaps the transforms; the hash waits on
 * each copy with an event; the result is copied back on `stream`. Pinned
 * (page-locked) buffers make the copies asynchronous; pageable memory also
 * works. For n <= 2^21 with all four buffers in page-locked host memory that
 * the device can address (mapped: cudaHostAlloc'd or registered), there are no
 * copies: the kernels read the inputs and write `out` in place over the
 * host link, which saves the copy path's host work on blocks this small.
 *
 * pa_hash_host_async: the same, returning once everything is queued. The
 * copy stream runs at most two calls ahead of the hashes (staging memory is
 * bounded to three calls' inputs), so back-to-back calls overlap one call's
 * input copies with the previous call's transforms; each queued hash starts
 * once all three of its inputs are in (pa_hash_host starts the product once
 * key and seed_a are in and copies seed_b meanwhile). The caller must keep key,
 * seed_a, seed_b and out valid, leave the inputs unmodified and not read out
 * until `stream` has passed the call (e.g. cudaStreamSynchronize). With
 * pageable buffers the copies block the host and nothing overlaps.
 */
int pa_hash_host(const uint64_t* key, const uint64_t* seed_a, const uint64_t* seed_b,
                 uint64_t n, uint64_t m, uint64_t* out, void* stream);
int pa_hash_host_async(const uint64_t* key, const uint64_t* seed_a, const uint64_t* seed_b,
                       uint64_t n, uint64_t m, uint64_t* out, void* stream);

/*
 * pa_convolve16: the digit product of Algorithm 1 steps 1-5 (zero fill,
 * split into 16-bit digits, forward NTTs, pointwise product, inverse NTT),
 * before any carry:
 *   coef[k] = sum_{i+j=k} x_i a_j,  k < L = ceil(n/16),
 * where x_i, a_j are the 16-bit digits of key and seed_a reduced mod 2^n.
 *   key, seed_a : device, ceil(n/64) limbs;  coef : device, L words (written)
 * Each coef[k] < L * 2^32 < 2^64.
 */
int pa_convolve16(const uint64_t* key, const uint64_t* seed_a, uint64_t n, uint64_t* coef,
                  void* stream);

/*
 * pa_carry_extract: Algorithm 1 steps 6-7 plus Sec. 3.2.2-3.2.5 on given
 * digits: out = floor(((sum_{k<L} coef[k] 2^(16k) + seed_b) mod 2^n) / 2^(n-m)).
 *   coef : device, L words, each < 2^64, digit k weighing 2^(16k); digits at
 *          k >= L count as zero (L = ceil(n/16) covers every digit below 2^n)
 *   L    : number of words in coef (may be smaller than ceil(n/16))
 *   seed_b : device, ceil(n/64) limbs;  out : device, ceil(m/64) limbs
 */
int pa_carry_extract(const uint64_t* coef, uint64_t L, const uint64_t* seed_b, uint64_t n,
                     uint64_t m, uint64_t* out, void* stream);

/*
 * Seed reuse. Alice and Bob apply the same publicly chosen g = g_{c,d} to their
 * strings X and X' (Sec. 2.2), and a system may keep one seed for several
 * blocks of the same length: the transform of c can then be computed once.
 * pa_seed_create transforms seed_a (device, ceil(n/64) limbs, read during the
 * call's stream work only) into a handle that owns its spectrum (one
 * transform of N words, allocated with cudaMalloc, synchronous). It queues the
 * transform on `stream`; later calls that use the handle on other streams must
 * be ordered after it. pa_hash_seeded(seed, key, seed_b, m, out, stream) then
 * equals pa_hash(key, seed_a, seed_b, n, m, out, stream) for the handle's n
 * and skips the seed's transform. pa_seed_destroy frees the handle; no work
 * that uses it may be in flight.
 */
typedef struct pa_seed_s* pa_seed;
int pa_seed_create(const uint64_t* seed_a, uint64_t n, void* stream, pa_seed* out);
int pa_hash_seeded(pa_seed seed, const uint64_t* key, const uint64_t* seed_b, uint64_t m,
                   uint64_t* out, void* stream);
int pa_seed_destroy(pa_seed seed);

/* One hash problem for the batched call (all pointers device pointers). */
typedef struct {
    const uint64_t* key;
    const uint64_t* seed_a;
    const uint64_t* seed_b;
    uint64_t n;
    uint64_t m;
    uint64_t* out;
} pa_block;

/*
 * pa_hash_batched: hash `count` independent blocks of any sizes on `stream`.
 * `blocks` is a host array read during the call only. Each result equals the
 * result of pa_hash on that block alone. All blocks are validated before any
 * work is queued (PA_EINVAL if any is invalid).
 */
int pa_hash_batched(const pa_block* blocks, uint32_t count, void* stream);

/*
 * pa_batch_mode: how pa_hash_batched (and pa_batch_create) run the transforms.
 *   1: every block whose product has one or two strided passes before the
 *     4096-point tile pass (up to about 2^24 points) and whose key and seed_a
 *     are 16-byte aligned runs in one persistent cooperative kernel: two CTAs
 *     per SM take the tiles of all those blocks' passes from one work counter
 *     (first forward pass, radix-64 pass, tile pass with the pointwise
 *     product, inverse passes, in that order), each tile waiting only for its
 *     own block's previous pass (bounded waits), up to 256 blocks and 16
 *     transform lengths per launch; the other blocks run by size class on
 *     forked streams at the same time.
 *   0: every block by size class (one launch per pass and length).
 *   2 (default): mode 1 when the blocks the persistent kernel would take have
 *     at most 8 tiles (4096 points each) per SM in all, else mode 0: the single
 *     kernel is faster where launches dominate (small batches), the per-pass
 *     kernels where the work does.
 * The carry steps of all blocks follow in one batched launch either way.
 * Returns the previous mode, or PA_EINVAL. Results are identical in every mode.
 */
int pa_batch_mode(int mode);

/* ------------------------------------------------------------------------
 * Serving: blocks arrive one at a time (as error reconciliation emits them,
 * Sec. 2.2) and are hashed by a background loop that forms batches
 * continuously: a request is admitted once a device stream slot is free and
 * the sum of in-flight footprints (transform workspace + the block's I/O,
 * pa_workspace_bytes(n) + 8 * (3 ceil(n/64) + ceil(m/64)) bytes) stays within
 * the HBM budget; admitted batches run concurrently on `streams` device
 * streams. Requests are taken in arrival order (the head waits for memory
 * rather than being overtaken). Each result equals pa_hash on that block
 * alone. The block's buffers must stay valid until its ticket completes.
 * ------------------------------------------------------------------------ */
typedef struct {
    uint32_t max_batch;        /* blocks per device batch (0 = 64) */
    uint32_t streams;          /* concurrent device batches (0 = 2, at most 8) */
    uint32_t max_pending;      /* queue length before pa_submit returns PA_EAGAIN (0 = 65536) */
    uint32_t idle_poll_us;     /* how long the loop keeps polling (for new requests and for
                                  completions) after its last event before it sleeps until
                                  the next pa_submit; 0 = always poll (lowest latency; the
                                  loop then keeps one host core busy while it runs) */
    uint64_t hbm_budget_bytes; /* admission budget (0 = half of the free device memory) */
} pa_config;

/*
 * pa_init: start the serving loop on CUDA device `device` (-1 = the calling
 * thread's current device) with `cfg` (NULL = defaults). Optional: the first
 * pa_submit starts it with defaults on the current device. PA_EINVAL if it is
 * already running (stop it first) or device is not a valid device number.
 * Completion: the loop polls an event recorded behind each batch; a ticket
 * completes when the loop has seen its batch's event, and its status is that
 * of the batch's stream (PA_ETIMEOUT if a bounded wait of the library's
 * kernels ran out in that batch, PA_ECUDA on a CUDA error).
 */
int pa_init(int device, const pa_config* cfg);

/*
 * pa_submit: queue one block (device pointers, as in pa_block) and return its
 * ticket. Non-blocking. PA_EINVAL for bad sizes or pointers, or if the block's
 * footprint alone exceeds the budget; PA_EAGAIN if the queue is full.
 */
int pa_submit(const pa_block* blk, uint64_t* ticket);

/*
 * pa_poll: wait up to timeout_us for the ticket. PA_OK when it has completed
 * (*status = the hashing status, PA_OK on success; the ticket is then
 * released), PA_EAGAIN if it is still queued or running, PA_EINVAL for an
 * unknown or already released ticket.
 */
int pa_poll(uint64_t ticket, uint32_t timeout_us, int* status);

/* Serving counters since the loop started. Latency = submit to device completion. */
typedef struct {
    uint64_t completed, pending, batches, bits;
    uint64_t peak_inflight_bytes, peak_inflight_blocks, hbm_budget_bytes;
    double p50_us, p99_us, max_us;
    double mbps;               /* key bits completed / (last completion - first submit) */
} pa_serve_stats_t;

int pa_serve_stats(pa_serve_stats_t* out);

/* pa_serve_stop: finish queued and running work, stop the loop, reset the counters. */
int pa_serve_stop(void);

/*
 * Captured batches: for a fixed set of blocks (the same buffers hashed again
 * and again, e.g. the slots of a post-processing pipeline), pa_batch_create
 * runs pa_hash_batched once eagerly (building every table it needs) and then
 * captures the same launch sequence, including its forked streams, into a CUDA
 * graph with its own workspace (cudaMalloc, synchronous). pa_batch_run
 * replays the graph on `stream` with one launch: every block is rehashed from
 * the current contents of its buffers. pa_batch_destroy frees it (no replay
 * may be in flight). Buffers must stay valid for the life of the handle.
 */
typedef struct pa_batch_s* pa_batch;
int pa_batch_create(const pa_block* blocks, uint32_t count, pa_batch* out);
int pa_batch_run(pa_batch batch, void* stream);
int pa_batch_destroy(pa_batch batch);

/*
 * pa_prepare: build the twiddle tables of the transform that serves keys of
 * n bits on the current device, for the plan currently in effect for that
 * length (synchronous; after pa_autotune picks another plan, call it again).
 * It also builds those of every shorter length a wrapped product of n bits
 * may run (which depends on m; see pa_plan_info). Besides a few small tables
 * per length, every strided pass of a plan keeps 2 M words of inter-pass
 * twiddles (M its sub-problem size): about 205 MB for the full length at
 * n = 10^8 (and about 140 MB for its wrapped length), 2.3 GB at n = 10^9, kept until
 * pa_shutdown. Optional: pa_hash builds them lazily. Call it for every key
 * size before capturing a stream into a CUDA graph.
 */
int pa_prepare(uint64_t n);

/*
 * Autotuning. Every transform length has a few equivalent plans (PA_PLAN_*
 * bits: the odd first radix run last instead of first; forward or inverse
 * strided passes loading their tiles directly instead of staging them with
 * asynchronous copies; for transforms of at most 64 tiles with one strided
 * pass, single-block tiles of a quarter of the columns, four times the CTAs;
 * for single blocks, the staged word tiles of the strided passes copied by one
 * bulk copy per tile row (cp.async.bulk completing on an mbarrier) instead of
 * per-thread 16-byte asynchronous copies; for single blocks whose transform
 * has at most 64 tiles of 4096 words, each tile's pass run by a cluster of four
 * CTAs on four SMs, exchanging the tile's rows and columns through distributed
 * shared memory, instead of by one CTA). Variants are 0 .. 63. pa_autotune times the applicable plans for the
 * transform length that keys of n bits use (the fastest of three runs of reps
 * hashes each, on synthetic data, synchronous; it allocates with cudaMalloc)
 * and keeps the fastest for
 * that length on the current device; later calls (single, batched, seeded,
 * served) use it. With the environment variable PA_TUNE_CACHE naming a file,
 * choices are saved there per GPU name and loaded on first use.
 * pa_plan_override forces a variant for the length of the full-length
 * (unwrapped) product of n-bit keys at the current digit width (-1 clears; for
 * tests). Results are identical under every plan.
 */
#define PA_PLAN_R0_LAST 1
#define PA_PLAN_DIRECT_FWD 2
#define PA_PLAN_DIRECT_INV 4
#define PA_PLAN_NARROW 8
#define PA_PLAN_BULK 16
#define PA_PLAN_CLUSTER 32
int pa_autotune(uint64_t n, int reps, int* variant_out);
int pa_plan_override(uint64_t n, int variant);
/* pa_plan_override_length: the same for the transform length N itself (a length
 * pa_plan_info reports); PA_EINVAL if N is not one of the library's lengths. */
int pa_plan_override_length(uint64_t N, int variant);

/* pa_workspace_bytes: device workspace one pa_hash of n bits draws from the pool
 * (two buffers of the recomputation's power-of-two length, which also hold the
 * wrapped and the full-length product, and the carry states). */
uint64_t pa_workspace_bytes(uint64_t n);

/*
 * Wrapped products (see pa_hash).
 * pa_plan_info: host only, needs no device. For keys of n bits and m output
 *   bits, under the current pa_wrap_mode: info[0] = the length of the
 *   transform the hash runs first, info[1] =
 *   the full-length product's (N >= 2L - 1, used when not wrapped), info[2] =
 *   how many low coefficients the wrapped product drops (0: not wrapped,
 *   info[0] == info[1]).
 *   PA_EINVAL for sizes pa_hash rejects.
 * pa_wrap_mode: 1 (default) wrapped products where shorter and the full
 *   product has at least 2^19 points (below that the transforms fill a
 *   fraction of the GPU and the recomputation's launch outweighs the saving);
 *   0 always the full-length product; 2 wrapped wherever shorter; 3 as 2 with
 *   the check forced to fail, so every hash also runs the recomputation (tests
 *   of that path). Returns the
 *   previous mode, or PA_EINVAL. Applies to later pa_hash / pa_hash_host calls
 *   on every thread.
 * pa_wrap_flags: waits for the device, then stores in *count how many checks
 *   have failed (each ran the recomputation) since the counter was last
 *   cleared; clear != 0 clears it.
 */
int pa_plan_info(uint64_t n, uint64_t m, uint64_t info[3]);
int pa_wrap_mode(int mode);
int pa_wrap_flags(uint64_t* count, int clear);

/*
 * Digit width. Algorithm 1 (Sec. 3.2.2) splits the operands into pieces; here
 * a piece (digit) has w bits, 16 <= w <= 20, and the product of the pieces is
 * exact in GF(p) when ceil(n/w) (2^w - 1)^2 < p. Wider digits mean a shorter
 * transform (at n = 10^8, m = n/4: 3 * 2^21 points with 20-bit digits against
 * 2^23 with 16-bit ones). By default each hash takes, among the exact widths,
 * the one whose product (wrapped where the wrapping rule allows) is shortest,
 * the narrowest of equals. The wrapped product's rule of pa_hash holds for w-bit
 * digits with L = ceil(n/w) and the dropped part below lo * 2^(w (lo + 1)). The
 * exact recomputation behind a wrapped product always uses 16-bit digits.
 * pa_plan_digits: host only; stores the width a hash of n bits with m output
 *   bits uses under the current modes (pa_plan_info gives its lengths).
 * pa_digit_width: 0 (default) chooses as above; 16 .. 20 forces that width
 *   where it is exact (else 16). Returns the previous setting, or PA_EINVAL.
 *   Applies to later calls on every thread (tests of each width).
 */
int pa_plan_digits(uint64_t n, uint64_t m, uint32_t* width);
int pa_digit_width(int width);

/*
 * Toeplitz-hash privacy amplification on the same NTT engine: the hash family
 * the paper surveys (Sec. 1) as the usual PA choice, there computed by FFT or
 * NTT, and the comparison workload for the modular hash. The paper does not
 * restate the family; these calls use the usual random-Toeplitz-matrix form:
 * an (n + m - 1)-bit seed s defines the m x n matrix over GF(2)
 *     T[i][j] = s[i - j + n - 1],      0 <= i < m, 0 <= j < n,
 * and the hash of an n-bit key x is the m-bit vector y = T x,
 *     y[i] = XOR_{j<n} s[i + n - 1 - j] AND x[j].
 * Bit vectors use the limb layout above (bit i of a vector = bit i mod 64 of
 * limb i/64); key bits >= n and seed bits >= n + m - 1 are ignored and output
 * bits >= m are written as zero.
 *
 * pa_toeplitz(key, seed, n, m, out, stream):
 *   key  : device, ceil(n/64) limbs          seed : device, ceil((n+m-1)/64) limbs
 *   out  : device, ceil(m/64) limbs (written)
 *   1 <= m <= n and n + m - 1 <= PA_TOEPLITZ_MAX_BITS, else PA_EINVAL.
 * Method: the integer convolution of the seed's and the key's bits (one bit per
 * GF(p) coefficient, every count <= n < p, cyclic length N >= n + m - 1), whose
 * coefficient n - 1 + i has the parity y[i]. Workspace: pa_toeplitz_workspace_bytes
 * from the library's pool, stream-ordered as for pa_hash.
 *
 * Seed reuse (both parties hash with one public seed): pa_toeplitz_seed_create
 * transforms the seed once into a pa_seed handle (ownership, streams and
 * pa_seed_destroy as for pa_seed_create); pa_toeplitz_seeded(seed, key, out,
 * stream) then equals pa_toeplitz for the handle's n and m. A Toeplitz handle
 * passed to pa_hash_seeded, or a modular-hash handle passed to
 * pa_toeplitz_seeded, is rejected with PA_EINVAL.
 */
#define PA_TOEPLITZ_MAX_BITS (1ull << 28) /* bound on n + m - 1 */
int pa_toeplitz(const uint64_t* key, const uint64_t* seed, uint64_t n, uint64_t m, uint64_t* out,
                void* stream);
uint64_t pa_toeplitz_workspace_bytes(uint64_t n, uint64_t m);
int pa_toeplitz_seed_create(const uint64_t* seed, uint64_t n, uint64_t m, void* stream, pa_seed* out);
int pa_toeplitz_seeded(pa_seed seed, const uint64_t* key, uint64_t* out, void* stream);
/* pa_toeplitz_autotune: pa_autotune for the transform length pa_toeplitz(n, m) uses
 * (timed through modular hashes of that length; the kernels are the same). */
int pa_toeplitz_autotune(uint64_t n, uint64_t m, int reps, int* variant_out);

/* Per-kernel device time, aggregated by kernel name (see pa_profile). */
typedef struct {
    char name[32];
    uint32_t launches;
    double total_ms;
} pa_kernel_stat;

/*
 * pa_profile: on != 0 starts recording a CUDA event pair around every kernel
 * launch the library queues (on the launching stream); 0 stops recording.
 * Recording adds two event records per launch.
 */
int pa_profile(int on);

/*
 * pa_profile_collect: wait for the recorded events, aggregate the elapsed
 * time per kernel name into stats[0 .. cap), clear the records, and return the
 * number of entries written (or a negative status).
 */
int pa_profile_collect(pa_kernel_stat* stats, int cap);

/* ------------------------------------------------------------------------
 * Bit-string adapters (device). The reconciled key X arrives as a bit string
 * and the final key Y leaves as one (Sec. 2.2); Sec. 3.2.1 packs the string
 * into words for mpz_import with word order most- or least-significant first,
 * and Sec. 3.2.5 exports the r most significant bits. String bit i (reading
 * order, i < nbits) is bit (i mod 8) of byte i/8 (msb_bytes = 0) or bit
 * 7 - (i mod 8) (msb_bytes = 1). With msb_string = 0 string bit i is integer
 * bit i; with msb_string = 1 it is integer bit nbits - 1 - i (the first bit is
 * the most significant).
 *   pa_bits_to_limbs: bits (device, ceil(nbits/8) bytes) -> limbs (device,
 *     ceil(nbits/64) words, bits >= nbits zero).
 *   pa_limbs_to_bits: limbs (device, ceil(nbits/64) words) -> bits (device,
 *     ceil(nbits/8) bytes, padding bits zero).
 * PA_EINVAL for null pointers, nbits outside [1, PA_MAX_BITS], flags not 0/1.
 * ------------------------------------------------------------------------ */
int pa_bits_to_limbs(const uint8_t* bits, uint64_t nbits, int msb_string, int msb_bytes,
                     uint64_t* limbs, void* stream);
int pa_limbs_to_bits(const uint64_t* limbs, uint64_t nbits, int msb_string, int msb_bytes,
                     uint8_t* bits, void* stream);

/*
 * pa_final_key_length: Eq. 1 (Sec. 2.2), the largest integer
 * r <= hmin_bits - 2 log2(1/eps), where hmin_bits is the smooth min-entropy
 * H_min^{eps/2}(rho_SE | E) of the reconciled key (an estimate supplied by the
 * caller; the paper obtains r from GLLP theory and system parameters).
 * PA_EINVAL if eps is not in (0, 1) or no positive r exists.
 */
int pa_final_key_length(double hmin_bits, double eps, uint64_t* r);

/*
 * pa_leftover_epsilon: Definition 2 (quantum leftover hash lemma), the bound
 * eps_bar = 1/2 * 2^(-(hmin_bits - r) / 2) + eps on the distance of an r-bit
 * key hashed with a universal_2 family from an ideal key.
 */
int pa_leftover_epsilon(double hmin_bits, uint64_t r, double eps, double* eps_bar);

/* Largest key pa_hash_noalloc accepts: 2^20 bits (its fixed scratch size). */
#define PA_NOALLOC_MAX_BITS (1ull << 20)

/*
 * pa_hash_noalloc: the same result as pa_hash, for callers that cannot
 * allocate device memory (this entry point has no counterpart in the paper;
 * it exists for integration). Some callers must not let a library call
 * cudaMalloc, or allocate from a stream-ordered pool: code that builds CUDA
 * graphs without allocation nodes, real-time post-processing loops that
 * reserve all device memory up front and may not stall in an allocator, and
 * programs whose device memory belongs to another framework's allocator.
 * This entry point calls no cudaMalloc, cudaFree or other allocating routine:
 * its device scratch (two transform buffers, twiddle tables for every
 * transform size it serves, carry-scan bytes; about 3 MB) is a set of
 * fixed-size arrays compiled into the library, which every GPU that loads the
 * library holds until the process exits.
 *   key, seed_a, seed_b, n, m, out, stream: as for pa_hash (device pointers,
 *   caller-owned), with n <= PA_NOALLOC_MAX_BITS.
 * Returns PA_EINVAL (nothing queued) if n > PA_NOALLOC_MAX_BITS, for bad
 * sizes or null pointers; PA_ECUDA if set-up or a launch fails. The message
 * is available from pa_last_error().
 * The first call on a device does the set-up: it looks up the arrays' device
 * addresses, fills the twiddle tables on `stream` and waits for them. Make that
 * first call before any stream capture: a first call on a capturing stream
 * returns PA_EINVAL and leaves the capture as it was. Later calls only queue
 * kernels. pa_shutdown forgets the set-up; call it before a device reset
 * (cudaDeviceReset), so that the next call sets up again on the new context.
 * All calls share the one scratch area and it keeps the previous call's
 * contents: the transform buffers are rewritten before they are read, and the
 * carry step's tile states, which must start at zero, are cleared by a
 * cudaMemsetAsync on `stream` before each carry launch. Calls whose work
 * overlaps on the GPU (different streams, or unordered use from several
 * threads) race on the scratch and give wrong results: order them on one
 * stream or with events. A bounded-wait timeout in this call is reported by
 * pa_device_status only (the per-stream words of pa_stream_status are library
 * allocations, which this entry point does not make).
 */
int pa_hash_noalloc(const uint64_t* key, const uint64_t* seed_a, const uint64_t* seed_b,
                    uint64_t n, uint64_t m, uint64_t* out, void* stream);

/*
 * pa_shutdown: free tables, pooled memory and status words of all devices, stop
 * nothing else (no work may be in flight). Call it before resetting a device
 * that the library has used (cudaDeviceReset): the next call then sets up
 * again, including pa_hash_noalloc's scratch addresses.
 */
int pa_shutdown(void);

/*
 * pa_device_status: waits for all work on the current device, then returns
 * PA_ETIMEOUT if any kernel of this library has given up a bounded wait since
 * the last clear (the carry look-back waits at most ~2^20 polls for an earlier
 * tile; on timeout that call's output is wrong but the kernel finishes and the
 * context stays usable), else PA_OK. clear != 0 resets the flag.
 */
int pa_device_status(int clear);

/*
 * pa_stream_status: the status of the library's work queued on `stream` so far
 * (cudaStream_t as void*, NULL = the legacy default stream), without waiting for
 * other streams: it queues a copy of the stream's status word behind that work
 * (and, with clear != 0, a reset of the word), waits for `stream` alone, and
 * returns PA_ETIMEOUT if a kernel of this library on that stream has given up a
 * bounded wait since the word was last cleared (that call's output is wrong; the
 * context stays usable), PA_ECUDA if the stream reports a CUDA error, else
 * PA_OK. The library keeps one word per stream handle for the first 4096
 * handles it sees on a device (later ones share the last word); a stream
 * created after another was destroyed may get the same handle, and then its
 * word: clear it (clear != 0) before relying on it. Work replayed from a
 * pa_batch graph marks the word of the stream it was captured on, and
 * pa_hash_noalloc marks none: their timeouts are reported by pa_device_status.
 */
int pa_stream_status(void* stream, int clear);

/* Fault injection for tests of the timeout path (faults nothing on the GPU). */
#define PA_FAULT_CARRY_WAIT 1 /* the next carry launch never processes its first tile,
                                 so the second tile's bounded wait runs out (short limit) */
int pa_fault_inject(int what);

/* Human-readable text of the last error on the calling thread ("" if none). */
const char* pa_last_error(void);

/* Library version string. */
const char* pa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PA_GB300_H */
