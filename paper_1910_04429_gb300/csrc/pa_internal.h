// Internal interfaces between the translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ntt_tile.cuh"
#include "plan.h"

namespace pa {

// One operand pair's transform work: the key x (operand 0) and the seed a
// (operand 1), both N-element GF(p) buffers.
struct NttJob {
    Geom geom;
    Twiddles tw;
    u64* buf_x;   // N words: transform of x, then the product digits
    u64* buf_a;   // N words: transform of a (with a stored seed: its spectrum in tile
                  // register order, times N^-1)
    Digits dx, da;
    u64 L;        // live product digits kept by the last inverse pass
    u32* zero = nullptr;  // words the first kernel clears (the carry states), or null
    u32 zero_words = 0;
};

// Launches: digits of x and a -> convolution digits c_k (k < L) in buf_x.
cudaError_t launch_convolution(const NttJob& job, cudaStream_t st);

// Seed reuse: a's spectrum alone into buf_a; then x's transform against it.
cudaError_t launch_seed_spectrum(const NttJob& job, cudaStream_t st);
cudaError_t launch_convolution_seeded(const NttJob& job, cudaStream_t st);

// One block of a batch of transforms that share a geometry.
struct BlockIO {
    u64* buf_x;   // N words: x, then the product digits
    u64* buf_a;   // N words: a, then its spectrum (tile register order, times N^-1)
    Digits dx, da;
    u64 L;        // digits kept by the last inverse pass
};
constexpr int MAX_BATCH = 32;  // blocks per launch (kernel parameter array)
template <int B>
struct NttBatch {
    int count;
    u32* zero;        // words the launch's CTA (0, 0) clears first (the carry states that
    u32 zero_words;   // the carry step reads after the transforms), or 0 words
    BlockIO io[B];
};
// Launches the transforms of `count` blocks of geometry G, MAX_BATCH blocks per launch.
cudaError_t launch_convolution_batch(const Geom& G, const Twiddles& tw, const BlockIO* io,
                                     int count, cudaStream_t st);

// Carry resolve, + b, mod 2^n and extraction of bits [n-m, n) (Algorithm 1
// steps 6-7, Sec. 3.2.2-3.2.5), one kernel over the output tiles (carry-in from
// a halo, else bounded look-back).
struct CarryJob {
    const u64* coef;  // convolution digits, coefficient k weighs 2^(width k)
    u64 L;            // digits present (coef[k] = 0 for k >= L)
    const u64* b;     // addend limbs, ceil(n/64)
    u64 n, m;
    u64* out;         // ceil(m/64) limbs
    u32* state;       // scratch, carry_state_words(n) words, 4-byte aligned
    bool zeroed;      // state already cleared earlier on the stream; else the launch clears it
    u64 lo;           // coefficients k < lo read as zero (a wrapped product's folded ones)
    u32* flag;        // non-null: set to 1 when limb floor((n-m)/64) - 1 of the sum is all
                      // ones (the dropped coefficients could carry into the output)
    bool force_flag;  // set the flag whatever the limb holds (tests of the fallback)
    u32 width = 16;   // digit width W: coefficient k weighs 2^(W k) (16 .. 20)
};
template <int B>
struct CarryBatch {
    int count;
    u32* status;      // the launching stream's status word (PA_STATUS_* bits), or null
    CarryJob job[B];
};
constexpr int CARRY_THREADS = 128;
constexpr int CARRY_LIMBS = 2;  // limbs per thread (4 measured slower: longer per-thread chains)
// (tiles of 256 limbs: 128 x 2 measured ahead of 256 x 2 and 256 x 1)
constexpr u64 CARRY_TILE_LIMBS = (u64)CARRY_THREADS * CARRY_LIMBS;
constexpr u32 CARRY_SPIN_LIMIT = 1u << 20;  // polls of a predecessor tile before giving up (~0.1-1 s)
constexpr u64 CARRY_FIXED_MAX_CTAS = 256;   // carry grids up to this size take their tiles by block index
constexpr u32 PA_STATUS_TIMEOUT = 1u;       // device status bit: a bounded wait ran out
GL_HD u64 carry_tiles(u64 n) { return ((n + 63) / 64 + CARRY_TILE_LIMBS - 1) / CARRY_TILE_LIMBS; }
// tile states, the ticket counter, the wrapped product's flag
GL_HD u64 carry_state_words(u64 n) { return carry_tiles(n) + 2; }
GL_HD u64 carry_flag_word(u64 n) { return carry_tiles(n) + 1; }
// the first carry tile holding output limbs (limb (n - m) / 64 onwards), or
// with check the limb below them too
GL_HD u64 first_out_tile(u64 n, u64 m, bool check = false) {
    u64 q = (n - m) / 64;
    return (check && q ? q - 1 : q) / CARRY_TILE_LIMBS;
}
// status: the stream's status word, which a launch that gives up a bounded wait
// marks with PA_STATUS_TIMEOUT (as well as the device-wide sticky word), or null.
cudaError_t launch_carry(const CarryJob& job, cudaStream_t st, u32* status = nullptr);
// Carry steps of `count` independent blocks (any sizes), MAX_BATCH per launch.
cudaError_t launch_carry_batch(const CarryJob* jobs, int count, cudaStream_t st, u32* status = nullptr);
// The next carry launch leaves its first tile unprocessed, so the wait of the
// second tile on it runs out (bounded, short limit): a host-armed test of the
// timeout path that faults nothing.
void fault_inject_carry();
// Sticky device status bits (PA_STATUS_*); synchronous.
cudaError_t read_device_status(u32* out, bool clear);
// How many carry launches have set their wrapped-product flag; synchronous.
cudaError_t read_flag_count(unsigned long long* out, bool clear);

// Exact recomputation of one hash behind a wrapped product, run only when the
// wrapped product's carry step set its flag: the full product by a radix-2
// transform of length N = 2^logN >= 2L - 1, then the carry step over every limb.
struct FallbackJob {
    Digits dx, da;      // the key's and the seed's 16-bit digits (dx.L = L = ceil(n/16))
    const u64* b;       // addend limbs
    u64 n, m;
    u64* out;           // overwritten when the flag is set
    const u32* flag;    // the wrapped product's carry flag
    u64* X;             // N words each
    u64* A;
    int logN;
    const u64 *wlo, *wloi, *whi, *whii;  // w_N^t, w_N^-t (t < 4096), w_N^(4096 t), inverse
    u64 ninv;           // N^-1
    u32* state;         // carry_state_words(n) words, zeroed
};
template <int B>
struct FallbackBatch {
    int count;
    u32* barrier;       // zeroed word: the grid barrier's counter
    u32* status;        // the launching stream's status word, or null
    FallbackJob job[B];
};
// One cooperative launch per 64 jobs; it returns at once unless a flag is set.
cudaError_t launch_fallback(const FallbackJob* jobs, int count, cudaStream_t st, u32* status = nullptr);
cudaError_t read_fallback_status(u32* out, bool clear);

// Persistent batched transforms (pa_persist.cu): the products of many blocks in
// one cooperative launch. A block's plan must be persist_eligible: one or two
// strided passes with the odd radix first (the second, if any, radix 64), its
// digit sources 16-byte aligned. scratch: PERSIST_SCRATCH_WORDS per job, zeroed
// (each launch's ticket and per-block tile counters). The carry steps follow
// separately.
struct PersistJob {
    u64* buf_x;
    u64* buf_a;
    const uint64_t* key;
    const uint64_t* seed;
    u64 n;
    int w;         // digit width
    Geom G;        // the plan of its first product
    Twiddles tw;   // G's tables (get_tables)
};
constexpr u32 PERSIST_SCRATCH_WORDS = 6;
bool persist_eligible(const Geom& G);
cudaError_t launch_persistent(const PersistJob* jobs, int count, u32* scratch, cudaStream_t st, u32* status);
cudaError_t read_persist_status(u32* out, bool clear);
// Sticky status of the single-block transform kernels' bulk-copy waits
// (plan variant PLAN_BULK); synchronous.
cudaError_t read_bulk_status(u32* out, bool clear);

// Inter-pass twiddle tables of a strided pass (M = sub-problem size, S =
// stride): out[0 .. M) = w_M^(j k) at k S + j, out[M .. 2M) = w_M^-(j k).
cudaError_t launch_pass_twiddles(const Twiddles& tw, u64 N, u64 M, u64 S, u64* out, cudaStream_t st);

// Toeplitz hash, last step: out bit i = coef[first + i] mod 2 for i < m,
// ceil(m/64) little-endian limbs (bits >= m zero).
cudaError_t launch_parity_extract(const u64* coef, u64 first, u64 m, u64* out, cudaStream_t st);

// Per-kernel timing with CUDA events on the launching stream (off unless
// pa_profile(1) was called). prof_begin/prof_end bracket one launch.
void prof_begin(cudaStream_t st, const char* name);
void prof_end(cudaStream_t st);

// Sets the text pa_last_error() returns on the calling thread.
void set_error(const char* msg);

// Per-stream status words (pa_stream_status). status_word: the device word
// the library's kernels on stream st mark when a bounded wait runs out (a slot
// of a per-device slab; null if the slab could not be set up). The caller
// holds the library lock. queue_status_read: queues on st a copy of st's word
// into pinned host memory (then, with clear, a reset of the word) and returns
// the host word's address, valid once st has passed the copy; PA_OK or a
// status code.
u32* status_word(int dev, cudaStream_t st);
int queue_status_read(cudaStream_t st, bool clear, const volatile u32** host_word);

// pa_hash_noalloc's per-device set-up is forgotten (pa_shutdown): the next
// call looks its scratch up again.
void noalloc_reset();

}  // namespace pa
