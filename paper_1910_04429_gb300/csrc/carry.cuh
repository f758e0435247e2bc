// Device helpers of the carry step (Algorithm 1 steps 6-7): per-limb sums of
// the convolution digits and the addend, their one-bit carry chain as
// generate / propagate pairs, a block-wide scan of those pairs, and the
// staging of one tile of digits and addend limbs in shared memory. Shared by
// the carry kernel and the exact recomputation behind a wrapped product.
//
// With c_k < 2^64 the convolution digits (digit k weighing 2^(W k), W the digit
// width, 16 .. 20) and b the addend, define per 64-bit limb j
//   V_j = sum of c_k 2^(W k - 64 j) over the digits k with floor(W k / 64) = j,
//         plus b_j                                      (< 2^128: at most four
//         digits, their shifts W k - 64 j distinct and below 64)
//   E_j = lo64(V_j) + hi64(V_{j-1}) = e_j + f_j 2^64    (f_j in {0, 1})
//   u_j = e_j + f_{j-1}                                 (in [0, 2^64])
// so that y = sum_j u_j 2^(64 j) exactly. (With W = 16 limb j holds digits
// 4j .. 4j + 3 at shifts 0, 16, 32, 48.) What remains is a one-bit carry
// chain: carry_{j+1} = [u_j + carry_j >= 2^64], whose generate / propagate
// pairs (g_j = [u_j = 2^64], p_j = [u_j = 2^64 - 1]) compose associatively.
#pragma once
#include "cp_async.cuh"
#include "pa_internal.h"

namespace pa {

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
constexpr int TILE_LIMBS = CARRY_THREADS * CARRY_LIMBS;       // 256
constexpr int SM_LIMBS = TILE_LIMBS + HALO_LO + HALO_HI;      // 261
constexpr int SM_COEF = 4 * SM_LIMBS;                         // 1044
constexpr int SM_LIMBS_PAD = SM_LIMBS + 1;                    // whole 16-byte chunks

struct Limb {
    u64 lo;   // u_j mod 2^64
    int gp;   // (g_j, p_j)
};

// The first digit of limb J, ceil(64 J / W) (J < 0: the halo below limb 0).
template <int W>
__device__ __forceinline__ long long first_digit(long long J) {
    const long long t = 64 * J;
    return t >= 0 ? (t + W - 1) / W : -((-t) / W);
}

// Where a staged carry tile starts: limb J0 = TILE_LIMBS tt - HALO_LO, digit k0
// (the first digit of limb J0, rounded down to even: whole 16-byte pairs).
struct TileBase {
    long long J0, k0;
};
template <int W>
__device__ __forceinline__ TileBase tile_base(long long tt) {
    const long long J0 = tt * TILE_LIMBS - HALO_LO;
    return TileBase{J0, W == 16 ? 4 * J0 : (first_digit<W>(J0) & ~1ll)};
}

// V of the limb at shared-memory position l (limb J0 + l), its digits staged
// from digit k0 on
template <int W>
__device__ __forceinline__ void limb_v(const u64* cs, const u64* bs, int l, const TileBase& tb, u64* vlo,
                                       u64* vhi) {
    u64 lo = 0, hi = 0;
    if constexpr (W == 16) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            u64 ck = cs[4 * l + i];
            u64 plo = i ? (ck << (16 * i)) : ck;
            u64 phi = i ? (ck >> (64 - 16 * i)) : 0;
            lo += plo;
            hi += phi + (lo < plo);
        }
    } else {
        const long long J = tb.J0 + l, kf = first_digit<W>(J);
        const int base = (int)(kf - tb.k0);
        const int s0 = (int)(W * kf - 64 * J);  // 0 .. W - 1
#pragma unroll
        for (int i = 0; i < (64 + W - 1) / W; i++) {
            const int sh = s0 + W * i;
            if (sh < 64) {
                u64 ck = cs[base + i];
                u64 plo = ck << sh;
                u64 phi = sh ? (ck >> (64 - sh)) : 0;
                lo += plo;
                hi += phi + (lo < plo);
            }
        }
    }
    u64 bj = bs[l];
    lo += bj;
    hi += (lo < bj);
    *vlo = lo;
    *vhi = hi;
}

// u of CNT limbs starting at shared position l0 (needs V at l0-2 .. l0+CNT-1)
template <int CNT, int W>
__device__ __forceinline__ void limbs_u(const u64* cs, const u64* bs, int l0, const TileBase& tb, Limb* u) {
    u64 vlo[CNT + 2], vhi[CNT + 2];
#pragma unroll
    for (int i = 0; i < CNT + 2; i++) limb_v<W>(cs, bs, l0 - 2 + i, tb, &vlo[i], &vhi[i]);
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

// Words [w0, w0 + 2 * chunks) of src (words [lo, count) live) into dst with
// 16-byte copies; words outside [lo, count) read as zero. Needs src 16-byte
// aligned, w0 and lo even.
__device__ __forceinline__ void stage_pairs(u64* dst, const u64* src, long long w0, int chunks, u64 count,
                                            u64 lo = 0) {
    for (int ch = threadIdx.x; ch < chunks; ch += CARRY_THREADS) {
        long long k = w0 + 2 * ch;
        int live = (k < (long long)lo || (u64)k >= count) ? 0 : ((u64)k + 1 < count ? 2 : 1);
        cp_async16(dst + 2 * ch, live ? src + k : src, 8 * live);
    }
}

// VEC: coef and b are 16-byte aligned (staged with cp.async), else plain loads.
// Digits [k0, k0 + SM_COEF) and limbs [J0, J0 + SM_LIMBS) of tile tt (tile_base)
// into cs / bs; positions outside the operands read 0. (SM_COEF covers the
// digits of SM_LIMBS limbs for every width W >= 16, plus the rounding of k0.)
// The b limbs of a tile alone (VEC: issued as their own group of async copies,
// not waited for).
template <bool VEC, int W>
__device__ __forceinline__ void stage_b(const CarryJob& c, u64 Ly, long long tt, u64* bs) {
    const long long J0 = tile_base<W>(tt).J0;
    if (VEC) {
        stage_pairs(bs, c.b, J0, SM_LIMBS_PAD / 2, Ly);
        cp_async_commit();
    } else {
        for (int i = threadIdx.x; i < SM_LIMBS; i += CARRY_THREADS) {
            long long j = J0 + i;
            bs[i] = (j >= 0 && (u64)j < Ly) ? c.b[j] : 0;
        }
    }
}

// The digits of a tile, and its b limbs unless have_b (staged by stage_b);
// returns with everything staged in shared memory by this thread complete.
template <bool VEC, int W>
__device__ __forceinline__ TileBase stage_tile(const CarryJob& c, u64 Ly, long long tt, u64* cs, u64* bs,
                                               bool have_b = false) {
    const TileBase tb = tile_base<W>(tt);
    if (VEC) {
        stage_pairs(cs, c.coef, tb.k0, SM_COEF / 2, c.L, c.lo);
        if (!have_b) stage_pairs(bs, c.b, tb.J0, SM_LIMBS_PAD / 2, Ly);
        cp_async_commit();
        cp_async_wait<0>();
    } else {
        for (int i = threadIdx.x; i < SM_COEF; i += CARRY_THREADS) {
            long long k = tb.k0 + i;
            cs[i] = (k >= (long long)c.lo && (u64)k < c.L) ? c.coef[k] : 0;
        }
        if (!have_b) stage_b<false, W>(c, Ly, tt, bs);
    }
    return tb;
}

// The output limbs among the carried limbs y[0 .. CARRY_LIMBS] of limbs
// j0 .. j0 + CARRY_LIMBS (y[CARRY_LIMBS] supplies the bits above the last):
// out limb j - q = bits [64 j + r, 64 j + r + 64) for q = floor((n-m)/64),
// r = (n - m) mod 64, limbs q .. q + ceil(m/64) - 1, the top one masked to m bits.
__device__ __forceinline__ void write_window(const CarryJob& c, u64 j0, const u64* y) {
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

}  // namespace pa
