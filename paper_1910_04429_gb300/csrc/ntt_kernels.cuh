// NTT multiply kernels: zero fill + split into 16-bit digits, forward
// transforms, pointwise product and inverse transform (Algorithm 1, steps
// 1-5, Sec. 3.2.2), as tile kernels over GF(p), p = 2^64 - 2^32 + 1, and the
// launch sequence of one plan (templates; pa_ntt.cu instantiates them for
// single blocks, pa_ntt_batch.cu for batches, in parallel builds).
//
// Every kernel serves a batch of independent blocks that share one transform
// geometry: blockIdx.x is the tile, blockIdx.y the block, and the per-block
// buffers and digit sources arrive in a __grid_constant__ parameter array.
#pragma once
#include <cooperative_groups.h>

#include <mutex>
#include <unordered_set>

#include "bulk_copy.cuh"
#include "cp_async.cuh"
#include "pdl.cuh"
#include "pa_internal.h"

namespace pa {

// The first kernel of a product clears the carry states in CTA (0, 0), after
// the dependent-launch wait, in place of a memset before it: the carry step
// runs after every transform kernel has completed.
template <int B>
__device__ __forceinline__ void clear_states(const NttBatch<B>& nb, int nthreads) {
    if (nb.zero_words && blockIdx.x == 0 && blockIdx.y == 0)
        for (u32 i = threadIdx.x; i < nb.zero_words; i += nthreads) nb.zero[i] = 0u;
}

// ---------------------------------------------------------------------------
// asynchronous staging of tile inputs (cp.async, 16-byte chunks)
// ---------------------------------------------------------------------------
// Words of a tile (R rows at stride S, C columns) into stage[d * C + c]. Tile
// bases and strides are even, so every 16-byte chunk is aligned.
template <int R, int C>
__device__ __forceinline__ void stage_words(u64* stage, const u64* buf, const StridedGeom& g,
                                            const TilePos& tp) {
    constexpr int CH = R * C / 2;
    for (int ch = threadIdx.x; ch < CH; ch += NT) {
        int d = ch / (C / 2), c = (ch % (C / 2)) * 2;
        cp_async16(stage + d * C + c, buf + tp.base + c + g.S * (u64)d, 16);
    }
}

// 16-bit digits of a tile into stage[d * C + c]; digits at positions >= L are
// zero-filled by the copy (and never read from memory). The caller checks
// that the digit source is 16-byte aligned.
template <int R, int C>
__device__ __forceinline__ void stage_digits(uint16_t* stage, const Digits& dig, const StridedGeom& g,
                                             const TilePos& tp, bool upper_zero) {
    // rows >= R/2 are all zero on the first pass of at most N/2 digits: not staged
    const int CH = (upper_zero ? R / 2 : R) * C / 8;
    for (int ch = threadIdx.x; ch < CH; ch += NT) {
        int d = ch / (C / 8), c = (ch % (C / 8)) * 8;
        u64 pos = tp.base + c + g.S * (u64)d;
        u64 live = pos < dig.L ? dig.L - pos : 0;
        int n = live >= 8 ? 8 : (int)live;
        cp_async16(stage + d * C + c, n ? dig.src + pos : dig.src, 2 * n);
    }
}

// Wider digits (width > 16): each row's 16-byte limb chunks, from the chunk that
// holds the row's first digit bit, into its slot of wide_row_chunks(C) chunks;
// chunks past the end of the limbs are zero-filled (never read from memory).
// After the chunks, per row: x = its first digit's bit offset in the slot
// (w P mod 128) | (its live digits, min(L - P, C) or 0) << 7, y = the column of
// digit L - 1 if the row holds it, else C (the reads then need no 64-bit
// position arithmetic per digit).
template <int R, int C>
__device__ __forceinline__ void stage_wide(u64* stage, const Digits& dig, const StridedGeom& g,
                                           const TilePos& tp, bool upper_zero) {
    constexpr int CHR = wide_row_chunks(C);
    const int rows = upper_zero ? R / 2 : R;
    const int CH = rows * CHR;
    const u64 bytes = dig.nlimbs * 8;
    const char* src = reinterpret_cast<const char*>(dig.src);
    for (int ch = threadIdx.x; ch < CH; ch += NT) {
        int d = ch / CHR, k = ch - d * CHR;
        u64 P = tp.base + g.S * (u64)d;
        u64 off = (((P * dig.width) >> 7) + (u64)k) * 16;
        int live = off >= bytes ? 0 : (bytes - off >= 16 ? 16 : (int)(bytes - off));
        cp_async16(reinterpret_cast<char*>(stage) + (size_t)ch * 16, live ? src + off : src, live);
    }
    uint2* rinfo = reinterpret_cast<uint2*>(stage + R * CHR * 2);
    for (int d = threadIdx.x; d < rows; d += NT) {
        const u64 P = tp.base + g.S * (u64)d;
        const u64 live = P >= dig.L ? 0 : (dig.L - P < (u64)C ? dig.L - P : (u64)C);
        const u64 top = dig.L - 1 - P;  // wraps (no match) when the row starts past L - 1
        rinfo[d] = make_uint2((u32)((P * dig.width) & 127) | ((u32)live << 7), top < (u64)C ? (u32)top : (u32)C);
    }
}

// Plan variant PLAN_BULK: a tile's R rows of C words by one bulk copy each,
// issued by warp 0 and completing on `bar` (armed here with the tile's bytes).
// Row d starts at word base + S d: bases and strides are even and the rows
// C >= 16 words long, so every copy is 16-byte aligned and sized.
template <int R, int C>
__device__ __forceinline__ void stage_rows_bulk(u64* stage, const u64* buf, const StridedGeom& g,
                                                const TilePos& tp, uint64_t* bar) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) mbar_arrive_expect(bar, (uint32_t)(R * C * sizeof(u64)));
    __syncwarp();
    for (int d = lane; d < R; d += 32)
        bulk_g2s(stage + d * C, buf + tp.base + g.S * (u64)d, (uint32_t)(C * sizeof(u64)), bar);
}

// polls of a bulk copy's barrier before the kernel gives up on it (seconds)
constexpr uint32_t BULK_WAIT_LIMIT = 1u << 22;
// sticky: a bulk-copy wait ran out (this translation unit's kernels; pa_device_status)
static __device__ u32 g_bulk_status;

template <int R, int C, bool PACK, bool WIDE = false>
struct StageSize {
    // one staged tile, in 8-byte words: a [R][C] tile of words, of 16-bit digits,
    // or (WIDE) R rows of limb chunks and a word of row facts per row; even, so
    // that the second operand's tile stays 16-byte aligned for cp.async
    static constexpr int WORDS = !PACK ? R * C : WIDE ? (R * wide_row_chunks(C) * 2 + R + 1) & ~1 : R * C / 4;
    static_assert(WORDS % 2 == 0, "staged tiles must keep 16-byte alignment");
    static constexpr size_t BYTES = (size_t)(TILE + 2 * WORDS) * sizeof(u64);
};

// Strided pass over one tile of both operands (OPS = 2: x and a; OPS = 1: x
// only, when a's spectrum is reused): the twiddles computed for x are kept in
// registers and reused for a. STAGED: the operands' tiles are copied into
// shared memory asynchronously first, so a's loads overlap x's arithmetic.
// (the body: one tile of block io, dynamic shared memory dsm; the kernel below
// and the persistent batched kernel run it)
template <int RA, int RB, int C, bool PACK, bool STAGED, int OPS, bool WIDE, bool BULK = false>
__device__ __forceinline__ void fwd_strided_tile(const StridedGeom& g, const BlockIO& io, const Twiddles& tw,
                                                 u64 tile, u64* dsm) {
    using S = Strided<RA, RB, C>;
    using SZ = StageSize<S::R, C, PACK, WIDE>;
    constexpr bool BULK_ROWS = STAGED && BULK && !PACK;  // words staged by bulk copies
    u64* sm = dsm;
    u64* st[2] = {dsm + TILE, dsm + TILE + SZ::WORDS};
    TilePos tp = S::tile(g, tile);
    __shared__ __align__(8) uint64_t bars[BULK_ROWS ? 2 : 1];
    if (BULK_ROWS) {
        if (threadIdx.x == 0)
            for (int op = 0; op < OPS; op++) mbar_init(&bars[op]);
        __syncthreads();
        if (threadIdx.x < 32)
            for (int op = 0; op < OPS; op++) stage_rows_bulk<S::R, C>(st[op], op ? io.buf_a : io.buf_x, g, tp, &bars[op]);
    } else if (STAGED) {
#pragma unroll
        for (int op = 0; op < OPS; op++) {
            if (PACK) {
                const Digits& dg = op ? io.da : io.dx;
                const bool uz = S::template upper_rows_zero<PACK>(g, dg);
                if (WIDE) stage_wide<S::R, C>(st[op], dg, g, tp, uz);
                else stage_digits<S::R, C>((uint16_t*)st[op], dg, g, tp, uz);
            }
            else stage_words<S::R, C>(st[op], op ? io.buf_a : io.buf_x, g, tp);
            cp_async_commit();
        }
    }
    if constexpr (OPS == 2 && 2 * S::NA <= NT && 2 * S::NB <= NT && 2 * S::R * C <= TILE) {
        // few columns per tile (narrow tiles): x in threads [0, NT/2), a in
        // [NT/2, NT), both operands at once, each half with its own twiddles
        // and its own [R][C] exchange area
        const int op = threadIdx.x >= NT / 2 ? 1 : 0;
        const int it = (int)threadIdx.x - op * (NT / 2);
        u64* buf = op ? io.buf_a : io.buf_x;
        const Digits& d = op ? io.da : io.dx;
        u64* smo = sm + op * (S::R * C);
        u64* sto = dsm + TILE + op * SZ::WORDS;  // st[op], without indexing an array at run time
        u64 wv[RA];
        if (it < S::NB) S::twiddles(g, tp, it, tw, wv);
        if (BULK_ROWS) {
            for (int o = 0; o < 2; o++)
                if (!mbar_wait(&bars[o], 0, BULK_WAIT_LIMIT)) atomicOr(&g_bulk_status, PA_STATUS_TIMEOUT);
        } else if (STAGED) {
            cp_async_wait<0>();
        }
        __syncthreads();  // both staged tiles complete
        if (it < S::NA) {
            if (STAGED) S::template fwd_a_staged<PACK, WIDE>(g, tp, it, sto, (const uint16_t*)sto, d, smo);
            else S::template fwd_a<PACK, WIDE>(g, tp, it, buf, d, smo);
        }
        __syncthreads();
        if (it < S::NB) S::fwd_b(g, tp, it, buf, smo, wv);
        return;
    }
    u64 w[S::ITEMS_B][RA];
#pragma unroll
    for (int i = 0; i < S::ITEMS_B; i++) {
        int it = threadIdx.x + i * NT;
        if (S::NB % NT == 0 || it < S::NB) S::twiddles(g, tp, it, tw, w[i]);
    }
#pragma unroll
    for (int op = 0; op < OPS; op++) {
        u64* buf = op ? io.buf_a : io.buf_x;
        const Digits& d = op ? io.da : io.dx;
        if (BULK_ROWS) {
            if (!mbar_wait(&bars[op], 0, BULK_WAIT_LIMIT)) atomicOr(&g_bulk_status, PA_STATUS_TIMEOUT);
        } else if (STAGED) {
            if (op || OPS == 1) cp_async_wait<0>();
            else cp_async_wait<1>();
        }
        __syncthreads();  // staged tile complete; the previous tile is out of sm
#pragma unroll
        for (int i = 0; i < S::ITEMS_A; i++) {
            int it = threadIdx.x + i * NT;
            if (S::NA % NT == 0 || it < S::NA) {
                if (STAGED)
                    S::template fwd_a_staged<PACK, WIDE>(g, tp, it, st[op], (const uint16_t*)st[op], d, sm);
                else
                    S::template fwd_a<PACK, WIDE>(g, tp, it, buf, d, sm);
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < S::ITEMS_B; i++) {
            int it = threadIdx.x + i * NT;
            if (S::NB % NT == 0 || it < S::NB) S::fwd_b(g, tp, it, buf, sm, w[i]);
        }
    }
}

template <int RA, int RB, int C, bool PACK, int B, bool STAGED, int OPS, bool WIDE = false, bool BULK = false>
__global__ void __launch_bounds__(NT, 2) k_fwd_strided(StridedGeom g, const __grid_constant__ NttBatch<B> nb,
                                                       Twiddles tw) {
    pdl_begin();
    clear_states(nb, NT);
    extern __shared__ __align__(16) u64 dsm[];
    fwd_strided_tile<RA, RB, C, PACK, STAGED, OPS, WIDE, BULK>(g, nb.io[blockIdx.y], tw, blockIdx.x, dsm);
}

// Inverse strided pass over one tile. STAGED: the tile is copied into shared
// memory asynchronously while the inverse twiddles are read; otherwise the
// first phase loads it directly (the autotuner picks per transform length).
// Three CTAs per SM (40 registers): the extra warps hide the global-load latency
// this one-operand pass is exposed to.
template <int RA, int RB, int C, bool LAST, bool STAGED, bool BULK = false>
__device__ __forceinline__ void inv_strided_tile(const StridedGeom& g, const BlockIO& io, const Twiddles& tw,
                                                 u64 tile, u64* dsm) {
    using S = Strided<RA, RB, C>;
    u64* sm = dsm;
    u64* st = dsm + TILE;
    TilePos tp = S::tile(g, tile);
    __shared__ __align__(8) uint64_t bar;
    if (STAGED) {
        if (BULK) {
            if (threadIdx.x == 0) mbar_init(&bar);
            __syncthreads();
            if (threadIdx.x < 32) stage_rows_bulk<S::R, C>(st, io.buf_x, g, tp, &bar);
        } else {
            stage_words<S::R, C>(st, io.buf_x, g, tp);
            cp_async_commit();
        }
        u64 w[S::ITEMS_B][RA];
#pragma unroll
        for (int i = 0; i < S::ITEMS_B; i++) {
            int it = threadIdx.x + i * NT;
            if (S::NB % NT == 0 || it < S::NB) S::inv_twiddles(g, tp, it, tw, w[i]);
        }
        if (BULK) {
            if (!mbar_wait(&bar, 0, BULK_WAIT_LIMIT)) atomicOr(&g_bulk_status, PA_STATUS_TIMEOUT);
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < S::ITEMS_B; i++) {
            int it = threadIdx.x + i * NT;
            if (S::NB % NT == 0 || it < S::NB) S::inv_b_staged(g, tp, it, st, sm, w[i]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < S::ITEMS_B; i++) {
            int it = threadIdx.x + i * NT;
            if (S::NB % NT == 0 || it < S::NB) S::inv_b(g, tp, it, io.buf_x, sm, tw);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < S::ITEMS_A; i++) {
        int it = threadIdx.x + i * NT;
        if (S::NA % NT == 0 || it < S::NA) S::template inv_a<LAST>(g, tp, it, io.buf_x, sm, io.L);
    }
}

template <int RA, int RB, int C, bool LAST, int B, bool STAGED, bool BULK = false>
__global__ void __launch_bounds__(NT, 3) k_inv_strided(StridedGeom g, const __grid_constant__ NttBatch<B> nb,
                                                       Twiddles tw) {
    pdl_begin();
    extern __shared__ __align__(16) u64 dsm[];
    inv_strided_tile<RA, RB, C, LAST, STAGED, BULK>(g, nb.io[blockIdx.y], tw, blockIdx.x, dsm);
}

// Forward contiguous pass of one tile; leaves the spectrum in registers.
// w4096: the middle twiddles (times N^-1 when the result is to be scaled).
template <bool PACK>
__device__ __forceinline__ void contig_forward(const u64* src, const Digits& d, u64 base,
                                               const u64* w4096, u64* sm, u64* v, int t) {
    c_fwd_col_a<PACK>(t, src, d, base, sm);
    __syncthreads();
    c_fwd_col_b_load(t, sm, w4096, v);
    __syncthreads();
    c_fwd_col_b_store(t, sm, v);
    __syncthreads();
    c_fwd_row_a_load(t, sm, v);
    __syncthreads();
    c_fwd_row_a_store(t, sm, v);
    __syncthreads();
    c_fwd_row_b_load(t, sm, v);
}

// Spectrum of a, scaled by N^-1 (the inverse transform's normalisation),
// stored over buf_a in register order: thread t of tile T owns words
// T*4096 + 8t .. +7. Each tile is read completely before it is overwritten.
template <bool PACK, int B>
__global__ void __launch_bounds__(NT) k_contig_seed(const __grid_constant__ NttBatch<B> nb, u64 ninv,
                                                    Twiddles tw) {
    pdl_begin();
    __shared__ u64 sm[TILE_SM];
    const BlockIO& io = nb.io[blockIdx.y];
    u64 base = (u64)blockIdx.x * TILE;
    u64 v[8];
    // with the scaled middle twiddles every word is multiplied by N^-1 once there
    const bool scaled = tw.w4096s != nullptr;
    contig_forward<PACK>(io.buf_a + base, io.da, base, scaled ? tw.w4096s : tw.w4096, sm, v, threadIdx.x);
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(io.buf_a + base + 8 * threadIdx.x);
    if (scaled) {
#pragma unroll
        for (int k = 0; k < 4; k++) dst[k] = make_ulonglong2(v[2 * k], v[2 * k + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++)
            dst[k] = make_ulonglong2(gl::mul(v[2 * k], ninv), gl::mul(v[2 * k + 1], ninv));
    }
}

// Forward contiguous pass of x, pointwise product with a's spectrum (Algorithm 1
// step 4) and the inverse contiguous pass, in one tile-resident kernel. With
// PACK (a single-tile transform) this is also the last inverse pass, which keeps
// only the digits below io.L.
template <bool PACK, int B>
__global__ void __launch_bounds__(NT) k_contig_fused(const __grid_constant__ NttBatch<B> nb, Twiddles tw) {
    pdl_begin();
    clear_states(nb, NT);
    __shared__ u64 sm[TILE_SM];
    const BlockIO& io = nb.io[blockIdx.y];
    u64 base = (u64)blockIdx.x * TILE;
    int t = threadIdx.x;
    u64 v[8];
    contig_forward<PACK>(io.buf_x + base, io.dx, base, tw.w4096, sm, v, threadIdx.x);
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(io.buf_a + base + 8 * t);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        ulonglong2 w = src[k];
        v[2 * k] = gl::mul(v[2 * k], w.x);
        v[2 * k + 1] = gl::mul(v[2 * k + 1], w.y);
    }
    __syncthreads();
    c_inv_row_b_store(t, sm, v);
    __syncthreads();
    c_inv_row_a_load(t, sm, v);
    __syncthreads();
    c_inv_row_a_store(t, sm, v);
    __syncthreads();
    c_inv_col_b_load(t, sm, tw, v);
    __syncthreads();
    c_inv_col_b_store(t, sm, v);
    __syncthreads();
    c_inv_col_a<PACK>(t, sm, io.buf_x + base, base, io.L);
}

// Both operands of one tile in one CTA: a's forward contiguous pass (times N^-1)
// parked in shared memory, then x's forward pass, the pointwise product and the
// inverse contiguous pass, as k_contig_seed followed by k_contig_fused but
// without a's spectrum going through global memory. Dynamic shared memory: the
// working tile, then a's spectrum word-interleaved by thread ([k * NT + t]).
template <bool PACK>
__device__ __forceinline__ void contig_both_tile(const BlockIO& io, u64 ninv, const Twiddles& tw, u64 tile,
                                                 u64* dsm) {
    u64* sm = dsm;
    u64* ah = dsm + TILE_SM;
    u64 base = tile * TILE;
    int t = threadIdx.x;
    u64 v[8];
    const bool scaled = tw.w4096s != nullptr;
    contig_forward<PACK>(io.buf_a + base, io.da, base, scaled ? tw.w4096s : tw.w4096, sm, v, threadIdx.x);
#pragma unroll
    for (int k = 0; k < 8; k++) ah[k * NT + t] = scaled ? v[k] : gl::mul(v[k], ninv);
    __syncthreads();  // every thread is done reading sm
    contig_forward<PACK>(io.buf_x + base, io.dx, base, tw.w4096, sm, v, threadIdx.x);
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = gl::mul(v[k], ah[k * NT + t]);
    __syncthreads();
    c_inv_row_b_store(t, sm, v);
    __syncthreads();
    c_inv_row_a_load(t, sm, v);
    __syncthreads();
    c_inv_row_a_store(t, sm, v);
    __syncthreads();
    c_inv_col_b_load(t, sm, tw, v);
    __syncthreads();
    c_inv_col_b_store(t, sm, v);
    __syncthreads();
    c_inv_col_a<PACK>(t, sm, io.buf_x + base, base, io.L);
}

template <bool PACK, int B>
__global__ void __launch_bounds__(NT, 2) k_contig_both(const __grid_constant__ NttBatch<B> nb, u64 ninv,
                                                    Twiddles tw) {
    pdl_begin();
    clear_states(nb, NT);
    extern __shared__ __align__(16) u64 dsm[];
    contig_both_tile<PACK>(nb.io[blockIdx.y], ninv, tw, blockIdx.x, dsm);
}

__device__ __forceinline__ void bar_sync_half() {  // named barrier 1 over NT threads
    asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory");
}

// k_contig_both for transforms of few tiles: 2 NT threads per tile, the first
// NT transform a (scaled by N^-1, parked in shared memory) while the second NT
// transform x; then the second half alone forms the product and runs the
// inverse tile pass (named barrier 1). The forward phases of both halves meet
// at the same block barriers. Shared memory: two working tiles, a's spectrum.
static __global__ void __launch_bounds__(2 * NT, 1) k_contig_pair(const __grid_constant__ NttBatch<1> nb, u64 ninv,
                                                          Twiddles tw) {
    pdl_begin();
    clear_states(nb, 2 * NT);
    extern __shared__ __align__(16) u64 dsm[];
    const int h = threadIdx.x / NT, t = threadIdx.x % NT;  // half 0: a, half 1: x
    u64* sm = dsm + h * TILE_SM;
    u64* ah = dsm + 2 * TILE_SM;
    const BlockIO& io = nb.io[0];
    u64 base = (u64)blockIdx.x * TILE;
    const bool scaled = tw.w4096s != nullptr;
    u64 v[8];
    if (h == 0)
        contig_forward<false>(io.buf_a + base, io.da, base, scaled ? tw.w4096s : tw.w4096, sm, v, t);
    else
        contig_forward<false>(io.buf_x + base, io.dx, base, tw.w4096, sm, v, t);
    if (h == 0) {
#pragma unroll
        for (int k = 0; k < 8; k++) ah[k * NT + t] = scaled ? v[k] : gl::mul(v[k], ninv);
    }
    __syncthreads();
    if (h == 0) return;
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = gl::mul(v[k], ah[k * NT + t]);
    c_inv_row_b_store(t, sm, v);
    bar_sync_half();
    c_inv_row_a_load(t, sm, v);
    bar_sync_half();
    c_inv_row_a_store(t, sm, v);
    bar_sync_half();
    c_inv_col_b_load(t, sm, tw, v);
    bar_sync_half();
    c_inv_col_b_store(t, sm, v);
    bar_sync_half();
    c_inv_col_a<false>(t, sm, io.buf_x + base, base, io.L);
}

// ---------------------------------------------------------------------------
// The tile pass on a cluster of four CTAs per tile (plan variant PLAN_CLUSTER:
// single blocks of at most CLUSTER_MAX_TILES tiles, both operands): the
// arithmetic of contig_both_tile spread over four SMs. CTA q of the cluster
// takes tile columns 16q .. 16q + 15 for the column half of a's and x's
// forward transforms, tile rows 16q .. 16q + 15 for the row half, the product
// and the row half of the inverse, and its columns again for the column half
// of the inverse. The two transposes between the halves store into the owning
// CTA's shared memory through the cluster (distributed shared memory), each
// followed by a cluster barrier. Every 64-point DFT runs as three radix-4
// steps on 16 threads (one per warp, 4 values each), so that a thread's chain
// of dependent instructions is short: a small transform is bound by that
// latency, not by throughput. Lanes 0-15 hold a's columns or rows, lanes
// 16-31 x's; after the product the a lanes run the inverse steps on their own
// (dead) data, so that no warp diverges, and store nothing.
// ---------------------------------------------------------------------------
constexpr int CL_Q = 4;                          // CTAs per tile
constexpr int CL_THREADS = 512;                  // 16 warps: w = warp
constexpr int CL_LINES = 64 / CL_Q;              // columns (rows) per CTA
constexpr int CL_CP = CL_LINES + 1;              // column-buffer pitch: lanes on 16 rows hit 16 banks
constexpr int CL_COLBUF = 64 * CL_CP;            // one operand's 64 rows x 16 columns
constexpr int CL_ROWBUF = CL_LINES * TILE_PITCH; // one operand's 16 rows x 64 columns

// Forward length-64 DFT over the 16 warps of a CTA, 4 values a thread, for
// one line per lane, with b (the line's 64 words at stride s) for the two
// exchanges. In: warp w holds x[w + 16 j] in v[j]. Out: warp w = 4 kh + th
// holds X[kh + 4 th + 16 t] in v[t]. Position p of the line is 64 = 4 x 16
// (p = r + 16 j), then 16 = 4 x 4 (r = sl + 4 sh): a DFT over j with roots
// w_64^(r kh), a DFT over sh with roots w_16^(sl th), a DFT over sl. The
// stores in the first step go to the words the thread's own loads came from,
// if they came from b.
__device__ __forceinline__ void dft64_fwd_r4(u64* v, u64* b, int s, int w) {
    gl::dft<4, false>(v);
    gl::RowRoots<64, false, 4, 16>::apply(v, w);
#pragma unroll
    for (int kh = 0; kh < 4; kh++) b[(16 * kh + w) * s] = v[kh];
    __syncthreads();
    const int kh = w >> 2, sl = w & 3;
#pragma unroll
    for (int sh = 0; sh < 4; sh++) v[sh] = b[(16 * kh + sl + 4 * sh) * s];
    gl::dft<4, false>(v);
    gl::RowRoots<16, false, 4, 4>::apply(v, sl);
#pragma unroll
    for (int th = 0; th < 4; th++) b[(16 * kh + 4 * th + sl) * s] = v[th];  // the words it read
    __syncthreads();
    const int th = w & 3;
#pragma unroll
    for (int i = 0; i < 4; i++) v[i] = b[(16 * kh + 4 * th + i) * s];
    gl::dft<4, false>(v);
}

// The inverse of dft64_fwd_r4 (without the 1/64): in, warp w = 4 kh + th holds
// Y[kh + 4 th + 16 t] in v[t]; out, warp w holds 64 x[w + 16 j] in v[j]. The
// first stores go to the words dft64_fwd_r4's last loads read in this thread.
__device__ __forceinline__ void dft64_inv_r4(u64* v, u64* b, int s, int w) {
    const int kh = w >> 2, th = w & 3;
    gl::dft<4, true>(v);
#pragma unroll
    for (int i = 0; i < 4; i++) b[(16 * kh + 4 * th + i) * s] = v[i];
    __syncthreads();
    const int sl = w & 3;
#pragma unroll
    for (int t = 0; t < 4; t++) v[t] = b[(16 * kh + 4 * t + sl) * s];
    gl::RowRoots<16, true, 4, 4>::apply(v, sl);
    gl::dft<4, true>(v);
#pragma unroll
    for (int sh = 0; sh < 4; sh++) b[(16 * kh + sl + 4 * sh) * s] = v[sh];  // the words it read
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; k++) v[k] = b[(16 * k + w) * s];
    gl::RowRoots<64, true, 4, 16>::apply(v, w);
    gl::dft<4, true>(v);
}

template <bool PACK>
__global__ void __cluster_dims__(CL_Q, 1, 1) __launch_bounds__(CL_THREADS)
    k_contig_cluster(const __grid_constant__ NttBatch<1> nb, u64 ninv, Twiddles tw) {
    namespace cg = cooperative_groups;
    __shared__ u64 colbuf[2 * CL_COLBUF];
    __shared__ u64 rowbuf[2 * CL_ROWBUF];
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    const BlockIO& io = nb.io[0];
    const u64 base = (u64)(blockIdx.x / CL_Q) * TILE;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, op = lane >> 4, li = lane & 15;
    const int c = CL_LINES * q + li;        // the lane's tile column in the column halves
    const int kk = (w >> 2) + 4 * (w & 3);  // the frequencies kk + 16 t the warp ends with
    const bool scaled = tw.w4096s != nullptr;
    u64* cb = colbuf + op * CL_COLBUF + li;               // column c of operand op, stride CL_CP
    u64* rb = rowbuf + op * CL_ROWBUF + li * TILE_PITCH;  // row 16 q + li of operand op
    // the twiddles w_4096^(+-c k) of the column halves, k = kk + 16 t (a's forward
    // ones times N^-1 when the table has them): read before the wait for the
    // previous kernel (the tables never change once built), so that no read of
    // them sits behind a barrier
    u64 twf[4], twi[4];
    {
        const u64* tws = (op == 0 && scaled) ? tw.w4096s : tw.w4096;
#pragma unroll
        for (int t = 0; t < 4; t++) {
            twf[t] = tws[c * (kk + 16 * t)];
            twi[t] = tw.w4096i[c * (kk + 16 * t)];
        }
    }
    pdl_begin();
    clear_states(nb, CL_THREADS);
    u64 v[4];

    // forward column half of operand op, column c: rows w + 16 j in
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int off = (w + 16 * j) * 64 + c;
        v[j] = PACK ? digit_at(op ? io.dx : io.da, base + off) : (op ? io.buf_x : io.buf_a)[base + off];
    }
    dft64_fwd_r4(v, cb, CL_CP, w);
    // times w_4096^(c k), then row k = kk + 16 t to the CTA that owns it (rank t, local row kk)
#pragma unroll
    for (int t = 0; t < 4; t++) {
        u64* dst = cluster.map_shared_rank(rowbuf + op * CL_ROWBUF, t);
        dst[kk * TILE_PITCH + c] = gl::mul(v[t], twf[t]);
    }
    cluster.sync();

    // forward row half of operand op, tile row 16 q + li
#pragma unroll
    for (int j = 0; j < 4; j++) v[j] = rb[w + 16 * j];
    dft64_fwd_r4(v, rb, 1, w);  // v[t]: the spectrum at (row 16 q + li, column kk + 16 t)
    // the product (Algorithm 1 step 4) in x's lanes, a's spectrum from lane - 16
#pragma unroll
    for (int t = 0; t < 4; t++) {
        const u64 av = __shfl_xor_sync(0xffffffffu, v[t], 16);
        if (op) v[t] = gl::mul(v[t], scaled ? av : gl::mul(av, ninv));
    }
    // inverse row half (x; the a lanes transform their own row and drop it)
    dft64_inv_r4(v, rb, 1, w);  // v[j]: row 16 q + li, column w + 16 j
    if (op) {
        // to the CTA owning column w + 16 j (rank j, local column w), x's column buffer
#pragma unroll
        for (int j = 0; j < 4; j++) {
            u64* dst = cluster.map_shared_rank(colbuf + CL_COLBUF, j);
            dst[(CL_LINES * q + li) * CL_CP + w] = v[j];
        }
    }
    cluster.sync();

    // inverse column half of x, column c (the a lanes again on dead data)
#pragma unroll
    for (int t = 0; t < 4; t++) v[t] = gl::mul(cb[(kk + 16 * t) * CL_CP], twi[t]);
    __syncthreads();  // every thread has read its rows before the buffer is reused
    dft64_inv_r4(v, cb, CL_CP, w);  // v[j]: row w + 16 j, column c
    if (op) {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const u64 p = base + (u64)((w + 16 * j) * 64 + c);
            if (!PACK) io.buf_x[p] = v[j];
            else if (p < io.L) io.buf_x[p] = gl::canon(v[j]);  // the transform's last pass: exact digits
        }
    }
}
// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------

// radix -> (RA, RB, columns per tile)
#define PA_RADIX_TABLE(X)                                                                  \
    X(2, 1, 2, 2048) X(4, 2, 2, 1024) X(8, 2, 4, 512) X(16, 4, 4, 256) X(32, 4, 8, 128)     \
    X(64, 8, 8, 64) X(3, 3, 1, 1024) X(6, 3, 2, 512) X(12, 3, 4, 256) X(24, 3, 8, 128)      \
    X(48, 6, 8, 64) X(5, 5, 1, 512) X(10, 5, 2, 256) X(20, 5, 4, 128) X(40, 5, 8, 64)

inline int strided_columns(int R) {
#define PA_COLS(r, a, b, c) if (R == r) return c;
    PA_RADIX_TABLE(PA_COLS)
#undef PA_COLS
    return 0;
}

// Opt a kernel into the dynamic shared memory it needs (once per kernel).
template <typename K>
static void allow_smem(K kernel, size_t bytes) {
    static std::mutex mu;
    static std::unordered_set<const void*> done;
    if (bytes <= 48 * 1024) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done.insert((const void*)kernel).second)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int B>
struct Launcher {
    const StridedGeom* g;
    const NttBatch<B>* nb;
    const Twiddles* tw;
    cudaStream_t st;
    bool stage_digits_ok;  // every digit source 16-byte aligned

    int ops;               // 2: transform x and a; 1: x only (a's spectrum reused)

    template <int RA, int RB, int C, bool PACK, bool STAGED, int OPS, bool WIDE = false, bool BULK = false>
    void fwd_k() const {
        dim3 grid((unsigned)(g->N / (RA * RB * C)), (unsigned)nb->count);
        size_t smem = STAGED ? StageSize<RA * RB, C, PACK, WIDE>::BYTES : TILE * sizeof(u64);
        auto k = k_fwd_strided<RA, RB, C, PACK, B, STAGED, OPS, WIDE, BULK>;
        allow_smem(k, smem);
        launch_pdl(k, grid, dim3(NT), smem, st, *g, *nb, *tw);
    }
    bool stage_fwd, stage_inv;  // plan variant: staged or direct tile loads

    template <int RA, int RB, int C, int OPS>
    void fwd_ops(bool pack) const {
        if (!pack) {
            if constexpr (B == 1) {
                if (stage_fwd && bulk) return fwd_k<RA, RB, C, false, true, OPS, false, true>();
            }
            if (stage_fwd) return fwd_k<RA, RB, C, false, true, OPS>();
            return fwd_k<RA, RB, C, false, false, OPS>();
        }
        if (wide) return fwd_k<RA, RB, C, true, true, OPS, true>();  // wider digits: staged only
        if (stage_digits_ok && stage_fwd) return fwd_k<RA, RB, C, true, true, OPS>();
        fwd_k<RA, RB, C, true, false, OPS>();
    }
    template <int RA, int RB, int C>
    void fwd(bool pack) const {
        if (ops == 1) return fwd_ops<RA, RB, C, 1>(pack);
        fwd_ops<RA, RB, C, 2>(pack);
    }
    template <int RA, int RB, int C, bool LAST, bool STAGED, bool BULK = false>
    void inv_k() const {
        dim3 grid((unsigned)(g->N / (RA * RB * C)), (unsigned)nb->count);
        size_t smem = (TILE + (STAGED ? RA * RB * C : 0)) * sizeof(u64);
        auto k = k_inv_strided<RA, RB, C, LAST, B, STAGED, BULK>;
        allow_smem(k, smem);
        launch_pdl(k, grid, dim3(NT), smem, st, *g, *nb, *tw);
    }
    template <int RA, int RB, int C>
    void inv(bool last) const {
        if constexpr (B == 1) {
            if (stage_inv && bulk) {
                if (last) return inv_k<RA, RB, C, true, true, true>();
                return inv_k<RA, RB, C, false, true, true>();
            }
        }
        if (last) {
            if (stage_inv) return inv_k<RA, RB, C, true, true>();
            return inv_k<RA, RB, C, true, false>();
        }
        if (stage_inv) return inv_k<RA, RB, C, false, true>();
        inv_k<RA, RB, C, false, false>();
    }
    // plan variant PLAN_NARROW (single blocks, single-pass plans): a quarter of
    // the columns per tile, four times the CTAs for transforms of few tiles
    bool narrow = false;
    // digits wider than 16 bits (every digit source then 16-byte aligned: the
    // wide first pass always stages its rows)
    bool wide = false;
    // plan variant PLAN_BULK (single blocks): staged word tiles by bulk row copies
    bool bulk = false;
    template <int RA, int RB, int C>
    void fwd_narrow() const {  // the only strided pass: digits in
        if (wide) {
            if (ops == 1) return fwd_k<RA, RB, C, true, true, 1, true>();
            return fwd_k<RA, RB, C, true, true, 2, true>();
        }
        if (ops == 1) {
            if (stage_digits_ok && stage_fwd) return fwd_k<RA, RB, C, true, true, 1>();
            return fwd_k<RA, RB, C, true, false, 1>();
        }
        if (stage_digits_ok && stage_fwd) return fwd_k<RA, RB, C, true, true, 2>();
        fwd_k<RA, RB, C, true, false, 2>();
    }
    template <int RA, int RB, int C>
    void inv_narrow() const {  // the only strided pass: digits out
        if (stage_inv && bulk) return inv_k<RA, RB, C, true, true, true>();
        if (stage_inv) return inv_k<RA, RB, C, true, true>();
        inv_k<RA, RB, C, true, false>();
    }
    void dispatch_fwd(int R, bool pack) const {
        if constexpr (B == 1) {
            if (narrow && pack) {
#define PA_FWDN(r, a, b, c) if (R == r) return fwd_narrow<a, b, c / 4>();
                PA_RADIX_TABLE(PA_FWDN)
#undef PA_FWDN
            }
        }
#define PA_FWD(r, a, b, c) if (R == r) return fwd<a, b, c>(pack);
        PA_RADIX_TABLE(PA_FWD)
#undef PA_FWD
    }
    void dispatch_inv(int R, bool last) const {
        if constexpr (B == 1) {
            if (narrow && last) {
#define PA_INVN(r, a, b, c) if (R == r) return inv_narrow<a, b, c / 4>();
                PA_RADIX_TABLE(PA_INVN)
#undef PA_INVN
            }
        }
#define PA_INV(r, a, b, c) if (R == r) return inv<a, b, c>(last);
        PA_RADIX_TABLE(PA_INV)
#undef PA_INV
    }
};

inline StridedGeom strided_geom(const Geom& G, const Twiddles& tw, int p, bool narrow = false) {
    u64 C = (u64)strided_columns(G.pass[p].R) / (narrow ? 4 : 1);
    return StridedGeom{G.N, G.pass[p].M, G.pass[p].S, (u32)(G.pass[p].S / C), tw.passf[p], tw.passi[p]};
}

// PLAN_NARROW applies to single blocks with one strided pass
template <int B>
inline bool narrow_plan(const Geom& G) {
    return B == 1 && (G.variant & PLAN_NARROW) && G.nstrided == 1;
}

// ops = 2: transform x and a and build a's spectrum; ops = 1: x only, each
// block's buf_a already holds a's spectrum (tile register order, times N^-1).
template <int B>
static cudaError_t launch_batch(const Geom& G, const Twiddles& tw, const NttBatch<B>& nb,
                                cudaStream_t st, int ops = 2) {
    bool stage_fwd = !(G.variant & PLAN_DIRECT_FWD), stage_inv = !(G.variant & PLAN_DIRECT_INV);
    bool narrow = narrow_plan<B>(G);
    const bool bulk = B == 1 && (G.variant & PLAN_BULK);
    bool aligned = true;
    for (int i = 0; i < nb.count; i++)
        aligned = aligned && ((uintptr_t)nb.io[i].dx.src % 16 == 0) && ((uintptr_t)nb.io[i].da.src % 16 == 0) &&
                  !nb.io[i].dx.one_bit && !nb.io[i].da.one_bit;
    // digits wider than 16 bits: every block of the launch, staged (aligned) sources
    const bool wide = nb.io[0].dx.width > 16;
    for (int i = 0; i < nb.count; i++)
        if ((nb.io[i].dx.width > 16) != wide || (ops == 2 && (nb.io[i].da.width > 16) != wide))
            return cudaErrorInvalidValue;
    if (wide && !aligned && G.nstrided > 0) return cudaErrorInvalidValue;
    // only the first launch clears the carry states
    NttBatch<B> later = nb;
    later.zero = nullptr;
    later.zero_words = 0;
    const NttBatch<B>* cur = &nb;
    for (int p = 0; p < G.nstrided; p++) {
        StridedGeom g = strided_geom(G, tw, p, narrow);
        prof_begin(st, p == 0 ? "ntt_fwd_strided_first" : "ntt_fwd_strided_r64");
        Launcher<B>{&g, cur, &tw, st, aligned, ops, stage_fwd, stage_inv, narrow, wide, bulk}.dispatch_fwd(
            G.pass[p].R, p == 0);
        prof_end(st);
        cur = &later;
    }
    dim3 tiles((unsigned)(G.N / TILE), (unsigned)nb.count);
    bool pack = G.nstrided == 0;  // a single 4096-word tile reads the digits itself
    u64 ninv = n_inverse(G.logN, G.odd);
    bool paired = false;
    if constexpr (B == 1) {
        if (ops == 2 && (G.variant & PLAN_CLUSTER) && G.N / TILE <= CLUSTER_MAX_TILES) {
            // each tile's pass on a four-CTA cluster
            dim3 cgrid((unsigned)(CL_Q * (G.N / TILE)), 1);
            prof_begin(st, "ntt_contig_both");
            if (pack) launch_pdl(k_contig_cluster<true>, cgrid, dim3(CL_THREADS), 0, st, *cur, ninv, tw);
            else launch_pdl(k_contig_cluster<false>, cgrid, dim3(CL_THREADS), 0, st, *cur, ninv, tw);
            prof_end(st);
            paired = true;
        } else if (ops == 2 && narrow && !pack) {
            // few tiles: the two operands' forward tile passes side by side
            constexpr size_t smem = (2 * TILE_SM + TILE) * sizeof(u64);
            prof_begin(st, "ntt_contig_both");
            allow_smem(k_contig_pair, smem);
            launch_pdl(k_contig_pair, tiles, dim3(2 * NT), smem, st, *cur, ninv, tw);
            prof_end(st);
            paired = true;
        }
    }
    if (!paired && ops == 2) {
        // both operands' tile passes in one kernel (a's spectrum stays on chip)
        constexpr size_t smem = (TILE_SM + TILE) * sizeof(u64);
        prof_begin(st, "ntt_contig_both");
        if (pack) {
            allow_smem(k_contig_both<true, B>, smem);
            launch_pdl(k_contig_both<true, B>, tiles, dim3(NT), smem, st, *cur, ninv, tw);
        } else {
            allow_smem(k_contig_both<false, B>, smem);
            launch_pdl(k_contig_both<false, B>, tiles, dim3(NT), smem, st, *cur, ninv, tw);
        }
        prof_end(st);
    } else if (!paired) {
        prof_begin(st, "ntt_contig_fused");
        if (pack)
            launch_pdl(k_contig_fused<true, B>, tiles, dim3(NT), 0, st, *cur, tw);
        else
            launch_pdl(k_contig_fused<false, B>, tiles, dim3(NT), 0, st, *cur, tw);
        prof_end(st);
    }
    for (int p = G.nstrided - 1; p >= 0; p--) {
        StridedGeom g = strided_geom(G, tw, p, narrow);
        prof_begin(st, p == 0 ? "ntt_inv_strided_last" : "ntt_inv_strided_r64");
        Launcher<B>{&g, &later, &tw, st, aligned, ops, stage_fwd, stage_inv, narrow, wide, bulk}.dispatch_inv(
            G.pass[p].R, p == 0);
        prof_end(st);
    }
    return cudaGetLastError();
}

}  // namespace pa
