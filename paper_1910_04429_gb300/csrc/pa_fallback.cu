// Exact recomputation behind a wrapped product. A wrapped product (a cyclic
// convolution shorter than the full product, whose folded low coefficients
// are dropped) is exact unless the carry step found limb floor((n-m)/64) - 1
// of the remaining sum all ones, which happens with probability 2^-64 for a
// uniform addend b. Then this kernel computes the whole hash again from the
// full product (Algorithm 1 steps 1-7: digits, forward NTTs, pointwise
// product, inverse NTT, carry, + b, mod 2^n, the top m bits) and overwrites
// the output.
//
// It is queued after the carry step of every wrapped hash and returns at once
// unless a flag of its batch is set, so it costs one launch in the common
// case. Its work when it runs is not tuned: one cooperative grid of a few CTAs
// per SM walks the phases with grid-wide barriers in between: a radix-2
// decimation-in-frequency forward transform of x and a of length N = 2^logN
// >= 2L - 1 (natural order in, bit-reversed out), the pointwise product times
// N^-1, a decimation-in-time inverse transform (bit-reversed in, natural out),
// then the carry step over every limb in three phases (tile aggregates of
// generate / propagate pairs; their serial scan into a carry-in per tile; the
// output tiles). Every barrier wait is bounded: when its limit runs out the
// kernel records PA_STATUS_TIMEOUT in its status word and goes on, so it
// always terminates (the cooperative launch makes every CTA resident, so the
// limit is not reached in normal operation).
#include <mutex>

#include "carry.cuh"
#include "grid_sync.cuh"

namespace pa {

__device__ u32 g_fb_status;  // sticky status bits of this kernel (PA_STATUS_*)

constexpr u32 FB_SPIN_LIMIT = 1u << 24;  // polls of a grid barrier before giving up (seconds)
constexpr int FB_BATCH = 64;             // jobs per launch (kernel parameter array, 11 KB)

__device__ __forceinline__ u64 fb_omega(const FallbackJob& f, bool inv, u64 e) {  // w_N^(+-e), e < N
    const u64* lo = inv ? f.wloi : f.wlo;
    const u64* hi = inv ? f.whii : f.whi;
    return gl::mul(lo[e & 4095], hi[e >> 12]);
}

// Steps 1-5: X <- the linear convolution of x's and a's digits (coefficients
// k < L canonical; N >= 2L - 1, so nothing wraps).
__device__ void fb_product(const FallbackJob& f, GridBarrier& bar) {
    const int logN = f.logN;
    const u64 N = 1ull << logN, half_n = N / 2;
    const u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x, nth = (u64)gridDim.x * blockDim.x;
    for (u64 i = tid; i < N; i += nth) {
        f.X[i] = digit_at(f.dx, i);
        f.A[i] = digit_at(f.da, i);
    }
    grid_sync(bar);
    // forward, decimation in frequency: span 2h = N .. 2, twiddle w_(2h)^j after the difference
    for (int s = logN - 1; s >= 0; s--) {
        const u64 h = 1ull << s;
        for (u64 t = tid; t < half_n; t += nth) {
            const u64 j = t & (h - 1), i0 = ((t >> s) << (s + 1)) | j, i1 = i0 + h;
            const u64 w = fb_omega(f, false, j << (logN - 1 - s));
            const u64 x0 = f.X[i0], x1 = f.X[i1], a0 = f.A[i0], a1 = f.A[i1];
            f.X[i0] = gl::add(x0, x1);
            f.X[i1] = gl::mul(gl::sub(x0, x1), w);
            f.A[i0] = gl::add(a0, a1);
            f.A[i1] = gl::mul(gl::sub(a0, a1), w);
        }
        grid_sync(bar);
    }
    for (u64 i = tid; i < N; i += nth) f.X[i] = gl::mul(gl::mul(f.X[i], f.A[i]), f.ninv);
    grid_sync(bar);
    // inverse, decimation in time: span 2h = 2 .. N, twiddle w_(2h)^-j before the sum
    for (int s = 0; s < logN; s++) {
        const u64 h = 1ull << s;
        for (u64 t = tid; t < half_n; t += nth) {
            const u64 j = t & (h - 1), i0 = ((t >> s) << (s + 1)) | j, i1 = i0 + h;
            const u64 u = f.X[i0], v = gl::mul(f.X[i1], fb_omega(f, true, j << (logN - 1 - s)));
            f.X[i0] = gl::add(u, v);
            f.X[i1] = gl::sub(u, v);
        }
        grid_sync(bar);
    }
    const u64 L = f.dx.L;
    for (u64 i = tid; i < L; i += nth) f.X[i] = gl::canon(f.X[i]);
    grid_sync(bar);
}

// Steps 6-7 over every limb (the recomputation's 16-bit digits): f.state[t]
// first holds tile t's aggregate, then the carry into tile t.
__device__ void fb_carry(const FallbackJob& f, GridBarrier& bar, u64* cs, u64* bs) {
    const CarryJob c{f.X, f.dx.L, f.b, f.n, f.m, f.out, f.state, true, 0, nullptr, false};
    const u64 Ly = (f.n + 63) / 64, tiles = carry_tiles(f.n), t0 = first_out_tile(f.n, f.m);
    const int l0 = HALO_LO + CARRY_LIMBS * threadIdx.x;
    for (u64 t = blockIdx.x; t < tiles; t += gridDim.x) {
        __syncthreads();  // cs, bs free again
        const TileBase tb = stage_tile<false, 16>(c, Ly, (long long)t, cs, bs);
        __syncthreads();
        const u64 j0 = t * TILE_LIMBS + CARRY_LIMBS * threadIdx.x;
        Limb u[CARRY_LIMBS];
        limbs_u<CARRY_LIMBS, 16>(cs, bs, l0, tb, u);
        int acc = GP_IDENTITY;
#pragma unroll
        for (int i = 0; i < CARRY_LIMBS; i++)
            if (j0 + i < Ly) acc = compose(acc, u[i].gp);
        int total;
        block_exclusive(acc, &total);
        if (threadIdx.x == 0) f.state[t] = (u32)total;
    }
    grid_sync(bar);
    if (blockIdx.x == 0 && threadIdx.x < 32) {  // carry into each tile, 32 tiles a round
        const int lane = threadIdx.x;
        int carry = 0;
        for (u64 base = 0; base < tiles; base += 32) {
            const u64 t = base + lane;
            const int v = t < tiles ? (int)f.state[t] : GP_IDENTITY;
            int inc = v;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                int o = __shfl_up_sync(0xffffffffu, inc, off);
                if (lane >= off) inc = compose(o, inc);  // lower lanes are earlier tiles
            }
            int exc = __shfl_up_sync(0xffffffffu, inc, 1);
            if (lane == 0) exc = GP_IDENTITY;
            if (t < tiles) f.state[t] = (u32)((exc & 1) | ((exc >> 1) & carry));
            const int all = __shfl_sync(0xffffffffu, inc, 31);
            carry = (all & 1) | ((all >> 1) & carry);
        }
    }
    grid_sync(bar);
    for (u64 t = t0 + blockIdx.x; t < tiles; t += gridDim.x) {
        __syncthreads();
        const TileBase tb = stage_tile<false, 16>(c, Ly, (long long)t, cs, bs);
        __syncthreads();
        const u64 j0 = t * TILE_LIMBS + CARRY_LIMBS * threadIdx.x;
        Limb u[CARRY_LIMBS + 1];
        limbs_u<CARRY_LIMBS + 1, 16>(cs, bs, l0, tb, u);
        int acc = GP_IDENTITY;
#pragma unroll
        for (int i = 0; i < CARRY_LIMBS; i++)
            if (j0 + i < Ly) acc = compose(acc, u[i].gp);
        int total;
        const int pre = block_exclusive(acc, &total);
        const int cin = (int)__ldcg(&f.state[t]);
        int carry = (pre & 1) | ((pre >> 1) & cin);
        u64 y[CARRY_LIMBS + 1];
#pragma unroll
        for (int i = 0; i < CARRY_LIMBS + 1; i++) {
            y[i] = u[i].lo + (u64)carry;
            carry = (u[i].gp & 1) | ((u[i].gp >> 1) & carry);
            const u64 j = j0 + i;
            if (j >= Ly) y[i] = 0;
            else if (j == Ly - 1 && (f.n & 63)) y[i] &= (1ull << (f.n & 63)) - 1;  // mod 2^n
        }
        write_window(c, j0, y);
    }
    grid_sync(bar);
}

template <int B>
__global__ void __launch_bounds__(CARRY_THREADS) k_fallback(const __grid_constant__ FallbackBatch<B> fb,
                                                            u32 spin_limit) {
    __shared__ __align__(16) u64 cs[SM_COEF];
    __shared__ __align__(16) u64 bs[SM_LIMBS_PAD];
    __shared__ int any_sh;
    if (threadIdx.x == 0) {
        int any = 0;
        for (int i = 0; i < fb.count; i++) any |= __ldcg(fb.job[i].flag) != 0;
        any_sh = any;
    }
    __syncthreads();
    if (!any_sh) return;  // the common case: every wrapped product was certified
    GridBarrier bar{fb.barrier, gridDim.x, 0, spin_limit, &g_fb_status, fb.status};
    for (int i = 0; i < fb.count; i++) {
        const FallbackJob& f = fb.job[i];
        if (__ldcg(f.flag) == 0) continue;  // the same answer in every CTA
        fb_product(f, bar);
        fb_carry(f, bar, cs, bs);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int fb_grid(int dev) {  // CTAs that can all be resident at once
    static std::mutex mu;
    static int cached[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return 0;
    if (!cached[dev]) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fallback<FB_BATCH>, CARRY_THREADS, 0) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        cached[dev] = (per_sm < 4 ? per_sm : 4) * sms;
    }
    return cached[dev];
}

cudaError_t launch_fallback(const FallbackJob* jobs, int count, cudaStream_t st, u32* status) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int grid = fb_grid(dev);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    for (int i = 0; i < count; i += FB_BATCH) {
        FallbackBatch<FB_BATCH> fb;
        fb.count = count - i < FB_BATCH ? count - i : FB_BATCH;
        fb.status = status;
        for (int k = 0; k < fb.count; k++) fb.job[k] = jobs[i + k];
        // the barrier counter: the (zeroed, otherwise unused) ticket word of the first job's states
        fb.barrier = fb.job[0].state + carry_tiles(fb.job[0].n);
        u32 limit = FB_SPIN_LIMIT;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(CARRY_THREADS);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        prof_begin(st, "fallback_check");
        e = cudaLaunchKernelEx(&cfg, k_fallback<FB_BATCH>, fb, limit);
        prof_end(st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t read_fallback_status(u32* out, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_fb_status, sizeof(u32));
    if (e == cudaSuccess && clear) {
        u32 zero = 0;
        e = cudaMemcpyToSymbol(g_fb_status, &zero, sizeof(u32));
    }
    return e;
}

}  // namespace pa
