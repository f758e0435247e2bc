// Persistent batched transforms: the products of many blocks of uneven sizes
// (Algorithm 1 steps 1-5 for each, Sec. 3.2.2) in one cooperative launch.
//
// One grid of two 512-thread CTAs per SM stays resident and walks the phases
// of the plans its blocks share the shape of (the odd radix R_0 first, then at
// most one radix-64 pass, then the 4096-point tile pass):
//   F1  every block's first forward strided pass (radix R_0, digits in, both
//       operands per tile),
//   F2  the radix-64 forward pass of the blocks whose plan has one,
//   T   every block's tile pass (a's and x's last forward pass, the pointwise
//       product, the first inverse pass),
//   I2  the radix-64 inverse pass where present,
//   I1  every block's last inverse pass (digits below L kept),
// as one stream of work items, the tiles of every phase in that order (4096
// words in the tile pass and the radix-64 passes; R_0 rows of the radix
// table's column count in the R_0 passes, 3072 or 2560 words for the odd
// radices). A CTA takes the next item from an atomic ticket, finds its block
// by binary search over the blocks' first-tile offsets (kept in shared
// memory), waits until that block has finished the phase before (per-block
// tile counters, a bounded wait), runs the tile and counts it done. No grid-
// wide barrier: one block's tile pass runs while other blocks are still in
// their first pass, so the phases' tails overlap. Blocks of different
// transform lengths and digit widths mix freely: each block names a class (its
// length's geometry and twiddle tables) and its own digit width. The carry step
// of every block follows as the usual batched carry launch.
#include <mutex>

#include "ntt_kernels.cuh"

namespace pa {

__device__ u32 g_pk_status;  // sticky status bits of this kernel (PA_STATUS_*)

constexpr int PK_BLOCKS = 256;   // blocks per launch
constexpr int PK_CLASSES = 16;   // transform lengths per launch
constexpr u32 PK_SPIN_LIMIT = 1u << 24;
// the largest tile footprint of the phases: the radix-64 pass staging both operands
constexpr size_t PK_SMEM = StageSize<64, 64, false>::BYTES;
static_assert(PK_SMEM >= (size_t)(TILE_SM + TILE) * sizeof(u64), "tile pass does not fit");
static_assert(PK_SMEM >= StageSize<64, 64, true, true>::BYTES, "wide first pass does not fit");

struct PkClass {
    StridedGeom g0, g1;  // the first strided pass (radix R_0) and the radix-64 pass, if any
    Twiddles tw;
    u64 ninv;
    u32 R0, nstr;        // first radix; strided passes (1 or 2)
};

struct PkBlock {
    u64* buf_x;
    u64* buf_a;
    const uint64_t* key;
    const uint64_t* seed;
    u64 n;
    u32 w;      // digit width
    u32 cls;    // index into PkBatch::cls
    u32 tiles;  // N / 4096: tiles of the tile pass and of the radix-64 passes
    u32 tiles0; // N / (R_0 C_0): tiles of the R_0 passes
};

struct PkBatch {
    int nblocks;
    u32 spin_limit;
    u32* ticket;   // zeroed word: the next work item
    u32* done;     // zeroed words: done[5 b + phase], the phase's finished tiles of block b
    u32* status;   // the launching stream's status word, or null
    PkClass cls[PK_CLASSES];
    PkBlock blk[PK_BLOCKS];
};

static_assert(sizeof(PkBatch) <= 32000, "kernel parameters beyond the 32 KB limit");

__device__ __forceinline__ BlockIO pk_io(const PkBlock& b) {
    Digits dx = make_digits(b.key, b.n, (int)b.w), da = make_digits(b.seed, b.n, (int)b.w);
    return BlockIO{b.buf_x, b.buf_a, dx, da, dx.L};
}

// the block that owns item t of a phase: the last b with pre[b] <= t (blocks
// without items in the phase share their successor's offset)
__device__ __forceinline__ int pk_find(const u32* pre, int nb, u32 t) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Each pass body is its own (not inlined) function, register-allocated on its
// own as in its per-pass kernel; the call costs once per tile.
template <int RA, int RB, int C, bool WIDE>
__device__ __noinline__ void pk_fwd_first_body(const StridedGeom& g, const BlockIO& io, const Twiddles& tw, u64 tile,
                                               u64* dsm) {
    fwd_strided_tile<RA, RB, C, true, true, 2, WIDE>(g, io, tw, tile, dsm);
}
template <int RA, int RB, int C>
__device__ __noinline__ void pk_inv_last_body(const StridedGeom& g, const BlockIO& io, const Twiddles& tw, u64 tile,
                                              u64* dsm) {
    inv_strided_tile<RA, RB, C, true, true>(g, io, tw, tile, dsm);
}
__device__ __noinline__ void pk_fwd64_body(const StridedGeom& g, const BlockIO& io, const Twiddles& tw, u64 tile,
                                           u64* dsm) {
    fwd_strided_tile<8, 8, 64, false, true, 2, false>(g, io, tw, tile, dsm);
}
__device__ __noinline__ void pk_inv64_body(const StridedGeom& g, const BlockIO& io, const Twiddles& tw, u64 tile,
                                           u64* dsm) {
    inv_strided_tile<8, 8, 64, false, true>(g, io, tw, tile, dsm);
}
__device__ __noinline__ void pk_tile_body(const BlockIO& io, u64 ninv, const Twiddles& tw, u64 tile, u64* dsm) {
    contig_both_tile<false>(io, ninv, tw, tile, dsm);
}

__device__ __forceinline__ void pk_fwd_first(const PkClass& c, const BlockIO& io, bool wide, u64 tile, u64* dsm) {
    switch (c.R0) {
#define PK_FWD(r, a, b, cc)                                                     \
    case r:                                                                     \
        if (wide) pk_fwd_first_body<a, b, cc, true>(c.g0, io, c.tw, tile, dsm); \
        else pk_fwd_first_body<a, b, cc, false>(c.g0, io, c.tw, tile, dsm);     \
        break;
        PA_RADIX_TABLE(PK_FWD)
#undef PK_FWD
    }
}

__device__ __forceinline__ void pk_inv_last(const PkClass& c, const BlockIO& io, u64 tile, u64* dsm) {
    switch (c.R0) {
#define PK_INV(r, a, b, cc) \
    case r:                 \
        pk_inv_last_body<a, b, cc>(c.g0, io, c.tw, tile, dsm); \
        break;
        PA_RADIX_TABLE(PK_INV)
#undef PK_INV
    }
}

// phases in the order their items are handed out
enum : int { PK_F1 = 0, PK_F2 = 1, PK_T = 2, PK_I2 = 3, PK_I1 = 4 };

// Items are taken from one ticket in phase-major order (all F1 tiles, then F2,
// T, I2, I1). An item waits, bounded, until its own block has finished the
// phase before it (per-block counters), not for the whole grid: every tile it
// waits for has a lower ticket, so it was taken earlier by a resident CTA that
// waits only on still earlier tiles, and every wait ends.
__global__ void __launch_bounds__(NT, 2) k_persist(const __grid_constant__ PkBatch pb) {
    extern __shared__ __align__(16) u64 dsm[];
    // first-tile offsets: R_0 passes, tile pass, radix-64 passes
    __shared__ u32 pre_r0[PK_BLOCKS + 1], pre_all[PK_BLOCKS + 1], pre_two[PK_BLOCKS + 1];
    __shared__ u32 item_sh;
    __shared__ BlockIO io_sh;  // the item's block, built once per item (not held in registers)
    const int nb = pb.nblocks;
    if (threadIdx.x == 0) {
        u32 r = 0, a = 0, b2 = 0;
        for (int i = 0; i < nb; i++) {
            pre_r0[i] = r;
            pre_all[i] = a;
            pre_two[i] = b2;
            r += pb.blk[i].tiles0;
            a += pb.blk[i].tiles;
            if (pb.cls[pb.blk[i].cls].nstr == 2) b2 += pb.blk[i].tiles;
        }
        pre_r0[nb] = r;
        pre_all[nb] = a;
        pre_two[nb] = b2;
    }
    __syncthreads();
    const u32 s_f2 = pre_r0[nb], s_t = s_f2 + pre_two[nb], s_i2 = s_t + pre_all[nb], s_i1 = s_i2 + pre_two[nb],
              s_end = s_i1 + pre_r0[nb];
    while (true) {
        if (threadIdx.x == 0) item_sh = atomicAdd(pb.ticket, 1u);
        __syncthreads();
        const u32 t = item_sh;
        if (t >= s_end) break;
        int phase;
        const u32* pre;
        u32 local;
        if (t < s_f2) phase = PK_F1, pre = pre_r0, local = t;
        else if (t < s_t) phase = PK_F2, pre = pre_two, local = t - s_f2;
        else if (t < s_i2) phase = PK_T, pre = pre_all, local = t - s_t;
        else if (t < s_i1) phase = PK_I2, pre = pre_two, local = t - s_i2;
        else phase = PK_I1, pre = pre_r0, local = t - s_i1;
        const int b = pk_find(pre, nb, local);
        const u64 tile = local - pre[b];
        const PkBlock& k = pb.blk[b];
        const PkClass& c = pb.cls[k.cls];
        if (threadIdx.x == 0) io_sh = pk_io(k);
        if (threadIdx.x == 0 && phase != PK_F1) {
            // the phase before this one for block b: its counter and tile count
            int dep = phase - 1;
            if (c.nstr == 1 && (phase == PK_T || phase == PK_I1)) dep = phase - 2;
            const u32 need = dep == PK_F1 ? k.tiles0 : k.tiles;
            const u32* ctr = pb.done + 5 * b + dep;
            u32 v, spins = 0;
            while (true) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
                if (v >= need) break;
                if (++spins > pb.spin_limit) {
                    atomicOr(&g_pk_status, PA_STATUS_TIMEOUT);
                    if (pb.status) atomicOr(pb.status, PA_STATUS_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __syncthreads();
        const BlockIO& io = io_sh;
        switch (phase) {
        case PK_F1: pk_fwd_first(c, io, k.w > 16, tile, dsm); break;
        case PK_F2: pk_fwd64_body(c.g1, io, c.tw, tile, dsm); break;
        case PK_T: pk_tile_body(io, c.ninv, c.tw, tile, dsm); break;
        case PK_I2: pk_inv64_body(c.g1, io, c.tw, tile, dsm); break;
        default: pk_inv_last(c, io, tile, dsm); break;
        }
        __syncthreads();  // the tile's writes done; shared memory free for the next item
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(pb.done + 5 * b + phase, 1u);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool persist_eligible(const Geom& G) {
    return (G.nstrided == 1 || (G.nstrided == 2 && G.pass[1].R == 64)) && !(G.variant & PLAN_R0_LAST);
}

static int pk_grid(int dev) {  // CTAs that are all resident at once (at most 2 per SM)
    static std::mutex mu;
    static int cached[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return 0;
    if (!cached[dev]) {
        int per_sm = 0, sms = 0;
        if (cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PK_SMEM) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist, NT, PK_SMEM) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
            return 0;
        cached[dev] = (per_sm < 2 ? per_sm : 2) * sms;
    }
    return cached[dev];
}

static cudaError_t pk_launch(const PkBatch& pb, int grid, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = PK_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    prof_begin(st, "ntt_persistent");
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_persist, pb);
    prof_end(st);
    return e;
}

cudaError_t launch_persistent(const PersistJob* jobs, int count, u32* scratch, cudaStream_t st, u32* status) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int grid = pk_grid(dev);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    static PkBatch pb;  // about 19 KB: kept off the stack (the library lock serialises callers)
    u64 off = 0;  // words of scratch taken: a ticket and 5 counters per block, per launch
    pb.nblocks = 0;
    int ncls = 0;
    u64 clsN[PK_CLASSES];
    for (int i = 0; i <= count; i++) {
        int c = -1;
        if (i < count) {
            for (int k = 0; k < ncls; k++)
                if (clsN[k] == jobs[i].G.N) c = k;
        }
        // launch what is gathered when the batch ends or the next block does not fit
        if (pb.nblocks && (i == count || pb.nblocks == PK_BLOCKS || (c < 0 && ncls == PK_CLASSES))) {
            pb.spin_limit = PK_SPIN_LIMIT;
            pb.ticket = scratch + off;
            pb.done = scratch + off + 1;
            off += 1 + 5 * (u64)pb.nblocks;
            pb.status = status;
            if ((e = pk_launch(pb, grid, st)) != cudaSuccess) return e;
            pb.nblocks = 0;
            ncls = 0;
            c = -1;
            if (i < count)  // its class in the new launch
                for (int k = 0; k < ncls; k++)
                    if (clsN[k] == jobs[i].G.N) c = k;
        }
        if (i == count) break;
        const PersistJob& j = jobs[i];
        if (!persist_eligible(j.G)) return cudaErrorInvalidValue;
        if (c < 0) {
            c = ncls++;
            clsN[c] = j.G.N;
            PkClass& k = pb.cls[c];
            k.g0 = strided_geom(j.G, j.tw, 0);
            k.g1 = j.G.nstrided == 2 ? strided_geom(j.G, j.tw, 1) : k.g0;
            k.tw = j.tw;
            k.ninv = n_inverse(j.G.logN, j.G.odd);
            k.R0 = (u32)j.G.pass[0].R;
            k.nstr = (u32)j.G.nstrided;
        }
        const u64 tile0 = (u64)j.G.pass[0].R * (u64)strided_columns(j.G.pass[0].R);  // words of an R_0 tile
        pb.blk[pb.nblocks++] = PkBlock{j.buf_x, j.buf_a, j.key,         j.seed,
                                       j.n,     (u32)j.w, (u32)c,        (u32)(j.G.N / TILE),
                                       (u32)(j.G.N / tile0)};
    }
    return cudaSuccess;
}

cudaError_t read_persist_status(u32* out, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_pk_status, sizeof(u32));
    if (e == cudaSuccess && clear) {
        u32 zero = 0;
        e = cudaMemcpyToSymbol(g_pk_status, &zero, sizeof(u32));
    }
    return e;
}

}  // namespace pa
