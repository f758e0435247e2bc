// Carry resolve, addition of d, reduction mod 2^n and extraction of the top m
// bits (Algorithm 1 steps 6-7 "combine" and "carry", the y = cx + d of
// Sec. 3.2.2, Sec. 3.2.3 mod 2^n, Sec. 3.2.4-3.2.5 export of the r most
// significant bits; Eq. 7).
//
// With c_k < 2^64 the convolution digits and b the addend, define per 64-bit
// limb j
//   V_j = sum_{i<4} c_{4j+i} 2^(16 i) + b_j            (< 2^115)
//   E_j = lo64(V_j) + hi64(V_{j-1}) = e_j + f_j 2^64   (f_j in {0, 1})
//   u_j = e_j + f_{j-1}                                (in [0, 2^64])
// so that y = sum_j u_j 2^(64 j) exactly. What remains is a one-bit carry
// chain: carry_{j+1} = [u_j + carry_j >= 2^64], whose generate / propagate
// pairs (g_j = [u_j = 2^64], p_j = [u_j = 2^64 - 1]) compose associatively.
//
// One kernel over the tiles of 1024 limbs that hold output limbs (from limb
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
#include "cp_async.cuh"
#include "pa_internal.h"
#include "pdl.cuh"

namespace pa {

__device__ u32 g_status;  // sticky device status (PA_STATUS_* bits), read by pa_device_status

// (G, P) packed in two bits: bit 0 generate, bit 1 propagate.
__device__ __forceinline__ int compose(int earlier, int later) {
    int G = (later & 1) | ((later >> 1) & earlier & 1);
    int P = (later >> 1) & (earlier >> 1) & 1;
    return G | (P << 1);
}
constexpr int GP_IDENTITY = 2;

// tile state word: 0 = nothing yet, (1 << 2 | gp) = aggregate of the tile,
// (2 << 2 | gp) = inclusive prefix from tile 0 through the tile
constexpr u32 ST_AGG = 1u << 2, ST_INC = 2u << 2;

constexpr int HALO_LO = 4, HALO_HI = 1;                       // extra limbs before / after a tile
constexpr int TILE_LIMBS = CARRY_THREADS * CARRY_LIMBS;       // 1024
constexpr int SM_LIMBS = TILE_LIMBS + HALO_LO + HALO_HI;      // 1029
constexpr int SM_COEF = 4 * SM_LIMBS;                         // 4116
constexpr int SM_LIMBS_PAD = SM_LIMBS + 1;                    // whole 16-byte chunks

struct Limb {
    u64 lo;   // u_j mod 2^64
    int gp;   // (g_j, p_j)
};

// V of the limb at shared-memory position l (limb J0 + l)
__device__ __forceinline__ void limb_v(const u64* cs, const u64* bs, int l, u64* vlo, u64* vhi) {
    u64 lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        u64 ck = cs[4 * l + i];
        u64 plo = i ? (ck << (16 * i)) : ck;
        u64 phi = i ? (ck >> (64 - 16 * i)) : 0;
        lo += plo;
        hi += phi + (lo < plo);
    }
    u64 bj = bs[l];
    lo += bj;
    hi += (lo < bj);
    *vlo = lo;
    *vhi = hi;
}

// u of CNT limbs starting at shared position l0 (needs V at l0-2 .. l0+CNT-1)
template <int CNT>
__device__ __forceinline__ void limbs_u(const u64* cs, const u64* bs, int l0, Limb* u) {
    u64 vlo[CNT + 2], vhi[CNT + 2];
#pragma unroll
    for (int i = 0; i < CNT + 2; i++) limb_v(cs, bs, l0 - 2 + i, &vlo[i], &vhi[i]);
    u64 e[CNT + 1];
    int f[CNT + 1];
#pragma unroll
    for (int i = 0; i < CNT + 1; i++) {
        e[i] = vlo[i + 1] + vhi[i];
        f[i] = e[i] < vhi[i];
    }
#pragma unroll
    for (int i = 0; i < CNT; i++) {
        u64 lo = e[i + 1] + (u64)f[i];
        bool wrap = f[i] && lo == 0;  // u_j = 2^64
        u[i].lo = lo;
        u[i].gp = wrap ? 1 : ((lo == ~0ull) ? 2 : 0);
    }
}

// Block-wide exclusive scan of (G, P) in thread order; returns the prefix of
// all earlier threads and writes the block total to *total.
__device__ __forceinline__ int block_exclusive(int v, int* total) {
    __shared__ int warp_tot[CARRY_THREADS / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int o = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc = compose(o, inc);
    }
    int exc = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) exc = GP_IDENTITY;
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    int wpre = GP_IDENTITY, tot = GP_IDENTITY;
    for (int w = 0; w < CARRY_THREADS / 32; w++) {
        if (w == warp) wpre = tot;
        tot = compose(tot, warp_tot[w]);
    }
    *total = tot;
    return compose(wpre, exc);
}

// tile states: release store / acquire load at GPU scope
__device__ __forceinline__ void publish(u32* p, u32 v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ u32 observe(const u32* p) {
    u32 v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Words [w0, w0 + 2 * chunks) of src (count words live) into dst with 16-byte
// copies; words outside [0, count) read as zero. Needs src 16-byte aligned and
// w0 even.
__device__ __forceinline__ void stage_pairs(u64* dst, const u64* src, long long w0, int chunks, u64 count) {
    for (int ch = threadIdx.x; ch < chunks; ch += CARRY_THREADS) {
        long long k = w0 + 2 * ch;
        int live = (k < 0 || (u64)k >= count) ? 0 : ((u64)k + 1 < count ? 2 : 1);
        cp_async16(dst + 2 * ch, live ? src + k : src, 8 * live);
    }
}

// VEC: coef and b are 16-byte aligned (staged with cp.async), else plain loads.
// Digits [4 J0, 4 J0 + SM_COEF) and limbs [J0, J0 + SM_LIMBS) of tile tt
// (J0 = 1024 tt - 4) into cs / bs; positions outside the operands read 0.
template <bool VEC>
__device__ __forceinline__ void stage_tile(const CarryJob& c, u64 Ly, long long tt, u64* cs, u64* bs) {
    const long long J0 = tt * TILE_LIMBS - HALO_LO;
    if (VEC) {
        stage_pairs(cs, c.coef, 4 * J0, SM_COEF / 2, c.L);
        stage_pairs(bs, c.b, J0, SM_LIMBS_PAD / 2, Ly);
        cp_async_commit();
        cp_async_wait<0>();
    } else {
        for (int i = threadIdx.x; i < SM_COEF; i += CARRY_THREADS) {
            long long k = 4 * J0 + i;
            cs[i] = (k >= 0 && (u64)k < c.L) ? c.coef[k] : 0;
        }
        for (int i = threadIdx.x; i < SM_LIMBS; i += CARRY_THREADS) {
            long long j = J0 + i;
            bs[i] = (j >= 0 && (u64)j < Ly) ? c.b[j] : 0;
        }
    }
}

// Only the tiles that hold output limbs (bits [n - m, n)) are processed: the
// limbs below matter only through the carry into the first of them. Grid:
// carry_tiles(n) - first_out_tile(n, m) CTAs per block (the widest block's
// count along x). ticket_start > 0 (fault injection) leaves the first output
// tiles unprocessed and makes every tile take the look-back path, so that the
// wait on them runs out.
template <int B, bool VEC>
__global__ void __launch_bounds__(CARRY_THREADS) k_carry(const __grid_constant__ CarryBatch<B> cb,
                                                         u32 ticket_start, u32 spin_limit) {
    __shared__ __align__(16) u64 cs[SM_COEF];
    __shared__ __align__(16) u64 bs[SM_LIMBS_PAD];
    __shared__ u32 tile_sh;
    __shared__ int decided_sh, carry_in_sh;
    pdl_begin();
    const CarryJob& c = cb.job[blockIdx.y];
    const u64 Ly = (c.n + 63) / 64, tiles = carry_tiles(c.n);
    const u64 t0 = first_out_tile(c.n, c.m);
    u32* state = c.state;  // tiles words, then the ticket counter
    if (threadIdx.x == 0) tile_sh = atomicAdd(&state[tiles], 1u) + ticket_start;
    __syncthreads();
    const u64 t = t0 + tile_sh;
    if (t >= tiles) return;

    stage_tile<VEC>(c, Ly, (long long)t, cs, bs);
    __syncthreads();

    const int l0 = HALO_LO + CARRY_LIMBS * threadIdx.x;  // shared position of the thread's first limb
    const u64 j0 = t * TILE_LIMBS + CARRY_LIMBS * threadIdx.x;
    Limb u[CARRY_LIMBS + 1];
    limbs_u<CARRY_LIMBS + 1>(cs, bs, l0, u);
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
            Limb h[2];  // limbs 1024 t - 2 and 1024 t - 1 (zero below limb 0)
            limbs_u<2>(cs, bs, HALO_LO - 2, h);
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
                stage_tile<VEC>(c, Ly, tc, cs, bs);
                __syncthreads();
                Limb w[CARRY_LIMBS];
                limbs_u<CARRY_LIMBS>(cs, bs, l0, w);
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
    u64 s = c.n - c.m, q = s >> 6;
    unsigned r = (unsigned)(s & 63);
    u64 Mo = (c.m + 63) >> 6;
#pragma unroll
    for (int i = 0; i < CARRY_LIMBS; i++) {
        u64 j = j0 + i;
        if (j < q || j >= q + Mo) continue;
        u64 o = r ? ((y[i] >> r) | (y[i + 1] << (64 - r))) : y[i];
        u64 oi = j - q;
        if (oi == Mo - 1 && (c.m & 63)) o &= (1ull << (c.m & 63)) - 1;
        c.out[oi] = o;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static u32 g_inject_ticket = 0;  // armed by fault_inject_carry(); consumed by the next launch

void fault_inject_carry() { g_inject_ticket = 1; }

template <int B>
static cudaError_t launch_carry_b(const CarryBatch<B>& cb, cudaStream_t st) {
    u64 tiles = 0;
    for (int i = 0; i < cb.count; i++) {
        u64 tt = carry_tiles(cb.job[i].n);
        u64 out_tiles = tt - first_out_tile(cb.job[i].n, cb.job[i].m);
        tiles = out_tiles > tiles ? out_tiles : tiles;
        if (cb.job[i].zeroed) continue;  // the caller cleared the states earlier on the stream
        cudaError_t e = cudaMemsetAsync(cb.job[i].state, 0, (tt + 1) * sizeof(u32), st);
        if (e != cudaSuccess) return e;
    }
    u32 start = g_inject_ticket;
    u32 limit = start ? 1000u : CARRY_SPIN_LIMIT;
    g_inject_ticket = 0;
    bool vec = true;
    for (int i = 0; i < cb.count; i++)
        vec = vec && (uintptr_t)cb.job[i].coef % 16 == 0 && (uintptr_t)cb.job[i].b % 16 == 0;
    dim3 grid((unsigned)tiles, (unsigned)cb.count);
    prof_begin(st, "carry_lookback");
    cudaError_t e = vec ? launch_pdl(k_carry<B, true>, grid, dim3(CARRY_THREADS), 0, st, cb, start, limit)
                        : launch_pdl(k_carry<B, false>, grid, dim3(CARRY_THREADS), 0, st, cb, start, limit);
    prof_end(st);
    return e;
}

cudaError_t launch_carry(const CarryJob& c, cudaStream_t st) {
    CarryBatch<1> cb;
    cb.count = 1;
    cb.job[0] = c;
    return launch_carry_b<1>(cb, st);
}

cudaError_t launch_carry_batch(const CarryJob* jobs, int count, cudaStream_t st) {
    for (int i = 0; i < count; i += MAX_BATCH) {
        CarryBatch<MAX_BATCH> cb;
        cb.count = count - i < MAX_BATCH ? count - i : MAX_BATCH;
        for (int k = 0; k < cb.count; k++) cb.job[k] = jobs[i + k];
        cudaError_t e = launch_carry_b<MAX_BATCH>(cb, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
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
