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
// Three kernels: tile aggregates, one scan over tiles, then every tile
// re-derives its limbs with its carry-in and writes the output bits.
#include "pa_internal.h"

namespace pa {

// (G, P) packed in two bits: bit 0 generate, bit 1 propagate.
__device__ __forceinline__ int compose(int earlier, int later) {
    int G = (later & 1) | ((later >> 1) & earlier & 1);
    int P = (later >> 1) & (earlier >> 1) & 1;
    return G | (P << 1);
}
constexpr int GP_IDENTITY = 2;

struct Limb {
    u64 lo;   // u_j mod 2^64
    int gp;   // (g_j, p_j)
};

// V_j as (lo, hi); V_j = 0 outside [0, Ly)
__device__ __forceinline__ void limb_v(const CarryJob& c, long long j, u64 Ly, u64* vlo, u64* vhi) {
    if (j < 0 || (u64)j >= Ly) { *vlo = 0; *vhi = 0; return; }
    u64 lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        u64 k = 4 * (u64)j + i;
        u64 ck = k < c.L ? c.coef[k] : 0;
        u64 plo = i ? (ck << (16 * i)) : ck;
        u64 phi = i ? (ck >> (64 - 16 * i)) : 0;
        lo += plo;
        hi += phi + (lo < plo);
    }
    u64 bj = c.b[j];
    lo += bj;
    hi += (lo < bj);
    *vlo = lo;
    *vhi = hi;
}

// u_j for j = j0 .. j0 + CNT - 1, from V_{j0-2} .. V_{j0+CNT-1}
template <int CNT>
__device__ __forceinline__ void limbs_u(const CarryJob& c, long long j0, u64 Ly, Limb* u) {
    u64 vlo[CNT + 2], vhi[CNT + 2];
#pragma unroll
    for (int i = 0; i < CNT + 2; i++) limb_v(c, j0 - 2 + i, Ly, &vlo[i], &vhi[i]);
    // E_{j0-1+i} = lo(V_{j0-1+i}) + hi(V_{j0-2+i}), i = 0 .. CNT
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

template <int B>
struct CarryBatch {
    int count;
    CarryJob job[B];
};

template <int B>
__global__ void __launch_bounds__(CARRY_THREADS) k_carry_tiles(const __grid_constant__ CarryBatch<B> cb) {
    const CarryJob& c = cb.job[blockIdx.y];
    u64 Ly = (c.n + 63) / 64;
    if (blockIdx.x >= carry_tiles(c.n)) return;
    long long j0 = ((long long)blockIdx.x * CARRY_THREADS + threadIdx.x) * CARRY_LIMBS;
    Limb u[CARRY_LIMBS];
    limbs_u<CARRY_LIMBS>(c, j0, Ly, u);
    int acc = GP_IDENTITY;
#pragma unroll
    for (int i = 0; i < CARRY_LIMBS; i++)
        if ((u64)(j0 + i) < Ly) acc = compose(acc, u[i].gp);
    int total;
    block_exclusive(acc, &total);
    if (threadIdx.x == 0) c.agg[blockIdx.x] = (uint8_t)total;
}

// One CTA per block: carry into every tile from the tile aggregates.
template <int B>
__global__ void __launch_bounds__(1024) k_carry_scan(const __grid_constant__ CarryBatch<B> cb) {
    const CarryJob& c = cb.job[blockIdx.x];
    u64 ntiles = carry_tiles(c.n);
    __shared__ int part[1024];
    u64 per = (ntiles + 1023) / 1024;
    u64 lo = threadIdx.x * per, hi = lo + per < ntiles ? lo + per : ntiles;
    int acc = GP_IDENTITY;
    for (u64 t = lo; t < hi; t++) acc = compose(acc, c.agg[t]);
    part[threadIdx.x] = acc;
    __syncthreads();
    // exclusive prefix over the 1024 partials (simple, ordered, per thread)
    if (threadIdx.x == 0) {
        int run = GP_IDENTITY;
        for (int i = 0; i < 1024; i++) {
            int x = part[i];
            part[i] = run;
            run = compose(run, x);
        }
    }
    __syncthreads();
    int pre = part[threadIdx.x];
    for (u64 t = lo; t < hi; t++) {
        c.cin[t] = (uint8_t)(pre & 1);  // carry into tile t (chain starts at 0)
        pre = compose(pre, c.agg[t]);
    }
}

template <int B>
__global__ void __launch_bounds__(CARRY_THREADS) k_carry_out(const __grid_constant__ CarryBatch<B> cb) {
    const CarryJob& c = cb.job[blockIdx.y];
    u64 Ly = (c.n + 63) / 64;
    if (blockIdx.x >= carry_tiles(c.n)) return;
    long long j0 = ((long long)blockIdx.x * CARRY_THREADS + threadIdx.x) * CARRY_LIMBS;
    Limb u[CARRY_LIMBS + 1];
    limbs_u<CARRY_LIMBS + 1>(c, j0, Ly, u);
    int acc = GP_IDENTITY;
#pragma unroll
    for (int i = 0; i < CARRY_LIMBS; i++)
        if ((u64)(j0 + i) < Ly) acc = compose(acc, u[i].gp);
    int total;
    int pre = block_exclusive(acc, &total);
    int tile_in = c.cin[blockIdx.x];
    int carry = (pre & 1) | ((pre >> 1) & tile_in);
    u64 y[CARRY_LIMBS + 1];
#pragma unroll
    for (int i = 0; i < CARRY_LIMBS + 1; i++) {
        y[i] = u[i].lo + (u64)carry;
        carry = (u[i].gp & 1) | ((u[i].gp >> 1) & carry);
        u64 j = (u64)j0 + i;
        if (j >= Ly) y[i] = 0;
        else if (j == Ly - 1 && (c.n & 63)) y[i] &= (1ull << (c.n & 63)) - 1;  // mod 2^n
    }
    u64 s = c.n - c.m, q = s >> 6;
    unsigned r = (unsigned)(s & 63);
    u64 Mo = (c.m + 63) >> 6;
#pragma unroll
    for (int i = 0; i < CARRY_LIMBS; i++) {
        u64 j = (u64)j0 + i;
        if (j < q || j >= q + Mo) continue;
        u64 o = r ? ((y[i] >> r) | (y[i + 1] << (64 - r))) : y[i];
        u64 oi = j - q;
        if (oi == Mo - 1 && (c.m & 63)) o &= (1ull << (c.m & 63)) - 1;
        c.out[oi] = o;
    }
}

template <int B>
static cudaError_t launch_carry_b(const CarryBatch<B>& cb, cudaStream_t st) {
    u64 tiles = 0;
    for (int i = 0; i < cb.count; i++) {
        u64 t = carry_tiles(cb.job[i].n);
        tiles = t > tiles ? t : tiles;
    }
    dim3 grid((unsigned)tiles, (unsigned)cb.count);
    prof_begin(st, "carry_tiles");
    k_carry_tiles<B><<<grid, CARRY_THREADS, 0, st>>>(cb);
    prof_end(st);
    prof_begin(st, "carry_scan");
    k_carry_scan<B><<<cb.count, 1024, 0, st>>>(cb);
    prof_end(st);
    prof_begin(st, "carry_out");
    k_carry_out<B><<<grid, CARRY_THREADS, 0, st>>>(cb);
    prof_end(st);
    return cudaGetLastError();
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

}  // namespace pa
