// Carry resolve, addition of d, reduction mod 2^n and extraction of the top m
// bits (Algorithm 1 steps 6-7 "combine" and "carry", the y = cx + d of
// Sec. 3.2.2, Sec. 3.2.3 mod 2^n, Sec. 3.2.4-3.2.5 export of the r most
// significant bits; Eq. 7). The per-limb sums u_j and their carry chain of
// generate / propagate pairs are defined in carry.cuh.
//
// Digit k of the product weighs 2^(W k) for the digit width W of the launch
// (16 .. 20, a template argument: the digits of a limb and their shifts are
// then multiply-and-shift arithmetic).
//
// One kernel over the tiles of 256 limbs that hold output limbs (from limb
// (n - m) / 64 up; the limbs below matter only through the carry into the
// first of them). Each CTA takes the next such tile from an atomic ticket (so
// every earlier tile has started), stages its digits and addend limbs in
// shared memory with coalesced loads, scans its (g, p) pairs and publishes the
// tile aggregate. The carry into a tile is decided by the last limbs before it
// unless they propagate (u = 2^64 - 1): a four-limb halo resolves it from the
// two limbs before the tile, with no wait on any other tile. Otherwise the
// first output tile composes the tiles below it, one whole-CTA tile at a time,
// until one does not propagate (or limb 0); a later tile has warp 0 read 32
// predecessor states per round, down to the first output tile at most,
// stopping at the latest one that fixes its carry out (an inclusive prefix,
// or an aggregate with P = 0). The tile then publishes its inclusive prefix
// and writes its output bits. Every wait on another tile is bounded: when the
// limit runs out the kernel records PA_STATUS_TIMEOUT in the device status word
// and carries on with a carry-in of 0, so it always terminates.
//
// Wrapped products: the coefficients below job.lo read as zero, and the kernel
// also resolves limb q - 1 (q = floor((n - m)/64), the limb just below the
// output) and sets job.flag when it is all ones: only then can the dropped
// coefficients change the output, and the exact recomputation queued behind
// this launch (pa_fallback.cu) runs.
#include <atomic>

#include "carry.cuh"
#include "pdl.cuh"

namespace pa {

__device__ u32 g_status;  // sticky device status (PA_STATUS_* bits), read by pa_device_status
__device__ unsigned long long g_flags;  // carry launches that set their wrapped-product flag

// Only the tiles that hold output limbs (bits [n - m, n)) are processed: the
// limbs below matter only through the carry into the first of them. Grid:
// carry_tiles(n) - first_out_tile(n, m) CTAs per block (the widest block's
// count along x). ticket_start > 0 (fault injection) leaves the first output
// tiles unprocessed and makes every tile take the look-back path, so that the
// wait on them runs out. FIXED (grids small enough to be resident at once, no
// fault injection): CTA x takes output tile x, with no ticket, and stages its
// b limbs before the wait for the previous kernel (b is the caller's input,
// which no kernel of this hash writes), two memory round trips off the
// critical path of a small hash.
template <int B, bool VEC, int W, bool FIXED>
__global__ void __launch_bounds__(CARRY_THREADS) k_carry(const __grid_constant__ CarryBatch<B> cb,
                                                         u32 ticket_start, u32 spin_limit) {
    __shared__ __align__(16) u64 cs[SM_COEF];
    __shared__ __align__(16) u64 bs[SM_LIMBS_PAD];
    __shared__ u32 tile_sh;
    __shared__ int decided_sh, carry_in_sh;
    if constexpr (FIXED) {
        const CarryJob& c = cb.job[blockIdx.y];
        const u64 t = first_out_tile(c.n, c.m, c.flag != nullptr) + blockIdx.x;
        if (t >= carry_tiles(c.n)) return;
        stage_b<VEC, W>(c, (c.n + 63) / 64, (long long)t, bs);
    }
    pdl_begin();
    const CarryJob& c = cb.job[blockIdx.y];
    const u64 Ly = (c.n + 63) / 64, tiles = carry_tiles(c.n);
    const u64 t0 = first_out_tile(c.n, c.m, c.flag != nullptr);
    u32* state = c.state;  // tiles words, then the ticket counter
    if constexpr (!FIXED) {
        if (threadIdx.x == 0) tile_sh = atomicAdd(&state[tiles], 1u) + ticket_start;
        __syncthreads();
    }
    const u64 t = t0 + (FIXED ? blockIdx.x : tile_sh);
    if (t >= tiles) return;

    const TileBase tb = stage_tile<VEC, W>(c, Ly, (long long)t, cs, bs, FIXED);
    __syncthreads();

    const int l0 = HALO_LO + CARRY_LIMBS * threadIdx.x;  // shared position of the thread's first limb
    const u64 j0 = t * TILE_LIMBS + CARRY_LIMBS * threadIdx.x;
    Limb u[CARRY_LIMBS + 1];
    limbs_u<CARRY_LIMBS + 1, W>(cs, bs, l0, tb, u);
    int acc = GP_IDENTITY;
#pragma unroll
    for (int i = 0; i < CARRY_LIMBS; i++)
        if (j0 + i < Ly) acc = compose(acc, u[i].gp);
    int total;
    int pre = block_exclusive(acc, &total);

    // publish the aggregate; the carry into the tile from the two limbs before
    // it when they decide it (the common case: no wait and no more reads)
    if (threadIdx.x == 0) {
        publish(&state[t], (t == 0 ? ST_INC : ST_AGG) | (u32)total);
        int decided = 0, cin = 0;
        if (ticket_start == 0) {
            Limb h[2];  // limbs TILE_LIMBS t - 2 and TILE_LIMBS t - 1 (zero below limb 0)
            limbs_u<2, W>(cs, bs, HALO_LO - 2, tb, h);
            if (!(h[1].gp & 2)) decided = 1, cin = h[1].gp & 1;  // generate or kill
            else if (!(h[0].gp & 2)) decided = 1, cin = h[0].gp & 1;
        }
        decided_sh = decided;
        carry_in_sh = cin;
    }
    __syncthreads();
    if (!decided_sh) {
        if (t == t0 && ticket_start == 0) {
            // the first output tile: compose the tiles below it, one whole-CTA
            // tile at a time, until one does not propagate (or limb 0)
            int later = GP_IDENTITY, cin = 0;
            for (long long tc = (long long)t0 - 1;; tc--) {
                if (tc < 0) {
                    cin = later & 1;  // the chain starts with carry 0
                    break;
                }
                __syncthreads();  // cs / bs free again
                const TileBase tbc = stage_tile<VEC, W>(c, Ly, tc, cs, bs);
                __syncthreads();
                Limb w[CARRY_LIMBS];
                limbs_u<CARRY_LIMBS, W>(cs, bs, l0, tbc, w);
                int a = GP_IDENTITY;
#pragma unroll
                for (int i = 0; i < CARRY_LIMBS; i++) a = compose(a, w[i].gp);  // below tile t: all < Ly
                int tot;
                block_exclusive(a, &tot);
                later = compose(tot, later);
                if (!(tot & 2)) {
                    cin = later & 1;
                    break;
                }
            }
            if (threadIdx.x == 0) carry_in_sh = cin;
        } else if (threadIdx.x < 32) {
            // a later output tile: look back over the published states 32 at a
            // time, down to the first output tile at most (which publishes a
            // state that fixes its carry out: an inclusive prefix, or P = 0)
            const int lane = threadIdx.x;
            long long base = (long long)t - 1;  // lane l looks at tile base - l
            int later = GP_IDENTITY;            // tiles after the current window, composed
            while (true) {
                long long i = base - lane;
                u32 s = ST_INC;  // below the first output tile: never reached (see above)
                if (i >= (long long)t0) {
                    s = observe(&state[i]);
                    u32 spins = 0;
                    while (!(i == (long long)t0 ? ((s & ST_INC) || ((s & ST_AGG) && !(s & 2u)))
                                                 : (s & (ST_AGG | ST_INC)) != 0)) {
                        if (++spins > spin_limit) {
                            atomicOr(&g_status, PA_STATUS_TIMEOUT);
                            if (cb.status) atomicOr(cb.status, PA_STATUS_TIMEOUT);
                            s = ST_INC;  // give up: treat as an inclusive prefix (0, 0)
                            break;
                        }
                        __nanosleep(64);
                        s = observe(&state[i]);
                    }
                }
                // a tile whose state fixes its carry out whatever comes before it: an
                // inclusive prefix, or an aggregate that does not propagate (P = 0)
                unsigned inc = __ballot_sync(0xffffffffu, (s & ST_INC) != 0 || !(s & 2u));
                int stop = inc ? __ffs(inc) - 1 : 31;  // lanes 0 .. stop take part
                int v = lane <= stop ? (int)(s & 3u) : GP_IDENTITY;
                // lane 0 ends with tiles (base - stop .. base) composed in tile order
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    int o = __shfl_down_sync(0xffffffffu, v, off);
                    if (lane + off < 32) v = compose(o, v);  // higher lanes are earlier tiles
                }
                v = __shfl_sync(0xffffffffu, v, 0);
                later = compose(v, later);
                if (inc) break;
                base -= 32;
            }
            if (lane == 0) carry_in_sh = later & 1;  // carry into the tile
        }
        __syncthreads();
    }
    // the inclusive prefix for tiles that look back past this one
    if (threadIdx.x == 0 && t > 0) publish(&state[t], ST_INC | (u32)compose(carry_in_sh, total));
    int carry = (pre & 1) | ((pre >> 1) & carry_in_sh);
    u64 y[CARRY_LIMBS + 1];
#pragma unroll
    for (int i = 0; i < CARRY_LIMBS + 1; i++) {
        y[i] = u[i].lo + (u64)carry;
        carry = (u[i].gp & 1) | ((u[i].gp >> 1) & carry);
        u64 j = j0 + i;
        if (j >= Ly) y[i] = 0;
        else if (j == Ly - 1 && (c.n & 63)) y[i] &= (1ull << (c.n & 63)) - 1;  // mod 2^n
    }
    const u64 q = (c.n - c.m) >> 6;
    if (c.flag) {
#pragma unroll
        for (int i = 0; i < CARRY_LIMBS; i++)  // limb q - 1, if it is this thread's
            if (j0 + i + 1 == q && (c.force_flag || y[i] == ~0ull)) {
                *c.flag = 1u;
                atomicAdd(&g_flags, 1ull);
            }
    }
    write_window(c, j0, y);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// armed by fault_inject_carry() from any host thread; taken (and cleared) by the next launch
static std::atomic<u32> g_inject_ticket{0};

void fault_inject_carry() { g_inject_ticket.store(1); }

template <int B>
static cudaError_t launch_carry_b(const CarryBatch<B>& cb, cudaStream_t st) {
    u64 tiles = 0;
    for (int i = 0; i < cb.count; i++) {
        u64 tt = carry_tiles(cb.job[i].n);
        u64 out_tiles = tt - first_out_tile(cb.job[i].n, cb.job[i].m, cb.job[i].flag != nullptr);
        tiles = out_tiles > tiles ? out_tiles : tiles;
        if (cb.job[i].zeroed) continue;  // the caller cleared the states earlier on the stream
        cudaError_t e = cudaMemsetAsync(cb.job[i].state, 0, (tt + 1) * sizeof(u32), st);
        if (e != cudaSuccess) return e;
    }
    u32 start = g_inject_ticket.exchange(0);
    u32 limit = start ? 1000u : CARRY_SPIN_LIMIT;
    // a grid this small is resident at once: fixed tiles need no ticket
    const bool fixed = start == 0 && tiles * (u64)cb.count <= CARRY_FIXED_MAX_CTAS;
    bool vec = true;
    for (int i = 0; i < cb.count; i++)
        vec = vec && (uintptr_t)cb.job[i].coef % 16 == 0 && (uintptr_t)cb.job[i].b % 16 == 0 &&
              cb.job[i].lo % 2 == 0;
    dim3 grid((unsigned)tiles, (unsigned)cb.count);
    prof_begin(st, "carry_lookback");
    cudaError_t e = cudaErrorInvalidValue;
    switch (cb.job[0].width) {  // every job of a launch has the same digit width
#define PA_CARRY_W(w)                                                                                    \
    case w:                                                                                              \
        e = fixed ? (vec ? launch_pdl(k_carry<B, true, w, true>, grid, dim3(CARRY_THREADS), 0, st, cb, start, limit)   \
                         : launch_pdl(k_carry<B, false, w, true>, grid, dim3(CARRY_THREADS), 0, st, cb, start, limit)) \
                  : (vec ? launch_pdl(k_carry<B, true, w, false>, grid, dim3(CARRY_THREADS), 0, st, cb, start, limit)  \
                         : launch_pdl(k_carry<B, false, w, false>, grid, dim3(CARRY_THREADS), 0, st, cb, start, limit)); \
        break;
        PA_CARRY_W(16) PA_CARRY_W(17) PA_CARRY_W(18) PA_CARRY_W(19) PA_CARRY_W(20)
#undef PA_CARRY_W
    }
    prof_end(st);
    return e;
}

cudaError_t launch_carry(const CarryJob& c, cudaStream_t st, u32* status) {
    CarryBatch<1> cb;
    cb.count = 1;
    cb.status = status;
    cb.job[0] = c;
    return launch_carry_b<1>(cb, st);
}

cudaError_t launch_carry_batch(const CarryJob* jobs, int count, cudaStream_t st, u32* status) {
    // one launch per digit width present, MAX_BATCH jobs at most each
    for (int w = 16; w <= 20; w++) {
        CarryBatch<MAX_BATCH> cb;
        cb.count = 0;
        cb.status = status;
        for (int i = 0; i <= count; i++) {
            if (i < count && jobs[i].width == (u32)w) cb.job[cb.count++] = jobs[i];
            if (cb.count == MAX_BATCH || (i == count && cb.count)) {
                cudaError_t e = launch_carry_b<MAX_BATCH>(cb, st);
                if (e != cudaSuccess) return e;
                cb.count = 0;
            }
        }
    }
    return cudaSuccess;
}

cudaError_t read_flag_count(unsigned long long* out, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_flags, sizeof(*out));
    if (e == cudaSuccess && clear) {
        unsigned long long zero = 0;
        e = cudaMemcpyToSymbol(g_flags, &zero, sizeof(zero));
    }
    return e;
}

cudaError_t read_device_status(u32* out, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_status, sizeof(u32));
    if (e == cudaSuccess && clear) {
        u32 zero = 0;
        e = cudaMemcpyToSymbol(g_status, &zero, sizeof(u32));
    }
    return e;
}

}  // namespace pa
