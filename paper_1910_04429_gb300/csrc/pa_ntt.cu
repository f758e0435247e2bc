// NTT multiply kernels: zero fill + split into 16-bit digits, forward
// transforms, pointwise product and inverse transform (Algorithm 1, steps
// 1-5, Sec. 3.2.2), as tile kernels over GF(p), p = 2^64 - 2^32 + 1.
#include "pa_internal.h"

namespace pa {

// Strided pass over one tile of both operands: the twiddles computed for x
// are kept in registers and reused for a.
template <int RA, int RB, int C, bool PACK>
__global__ void __launch_bounds__(NT, 2) k_fwd_strided(StridedGeom g, u64* buf0, u64* buf1,
                                                       Digits d0, Digits d1, Twiddles tw) {
    using S = Strided<RA, RB, C>;
    __shared__ u64 sm[TILE];
    TilePos tp = S::tile(g, blockIdx.x);
    u64 w[S::ITEMS_B][RA];
#pragma unroll
    for (int i = 0; i < S::ITEMS_B; i++) {
        int it = threadIdx.x + i * NT;
        if (S::NB % NT == 0 || it < S::NB) S::twiddles(g, tp, it, tw, w[i]);
    }
#pragma unroll
    for (int op = 0; op < 2; op++) {
        u64* buf = op ? buf1 : buf0;
        const Digits& d = op ? d1 : d0;
        if (op) __syncthreads();  // the tile of x is out of shared memory
#pragma unroll
        for (int i = 0; i < S::ITEMS_A; i++) {
            int it = threadIdx.x + i * NT;
            if (S::NA % NT == 0 || it < S::NA) S::template fwd_a<PACK>(g, tp, it, buf, d, sm);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < S::ITEMS_B; i++) {
            int it = threadIdx.x + i * NT;
            if (S::NB % NT == 0 || it < S::NB) S::fwd_b(g, tp, it, buf, sm, w[i]);
        }
    }
}

template <int RA, int RB, int C, bool LAST>
__global__ void __launch_bounds__(NT, 2) k_inv_strided(StridedGeom g, u64* buf, u64 keep,
                                                       Twiddles tw) {
    using S = Strided<RA, RB, C>;
    __shared__ u64 sm[TILE];
    TilePos tp = S::tile(g, blockIdx.x);
#pragma unroll
    for (int i = 0; i < S::ITEMS_B; i++) {
        int it = threadIdx.x + i * NT;
        if (S::NB % NT == 0 || it < S::NB) S::inv_b(g, tp, it, buf, sm, tw);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < S::ITEMS_A; i++) {
        int it = threadIdx.x + i * NT;
        if (S::NA % NT == 0 || it < S::NA) S::template inv_a<LAST>(g, tp, it, buf, sm, keep);
    }
}

// Forward contiguous pass of one tile; leaves the spectrum in registers.
template <bool PACK>
__device__ __forceinline__ void contig_forward(const u64* src, const Digits& d, u64 base,
                                               const Twiddles& tw, u64* sm, u64* v) {
    int t = threadIdx.x;
    c_fwd_col_a<PACK>(t, src, d, base, sm);
    __syncthreads();
    c_fwd_col_b_load(t, sm, tw, v);
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
// stored in register order: thread t of tile T owns words T*4096 + 8t .. +7.
template <bool PACK>
__global__ void __launch_bounds__(NT) k_contig_seed(u64* buf, Digits d, u64* ahat, u64 ninv,
                                                    Twiddles tw) {
    __shared__ u64 sm[TILE];
    u64 base = (u64)blockIdx.x * TILE;
    u64 v[8];
    contig_forward<PACK>(buf + base, d, base, tw, sm, v);
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(ahat + base + 8 * threadIdx.x);
#pragma unroll
    for (int k = 0; k < 4; k++)
        dst[k] = make_ulonglong2(gl::mul(v[2 * k], ninv), gl::mul(v[2 * k + 1], ninv));
}

// Forward contiguous pass of x, pointwise product with a's spectrum (Algorithm 1
// step 4) and the inverse contiguous pass, in one tile-resident kernel.
template <bool PACK>
__global__ void __launch_bounds__(NT) k_contig_fused(u64* buf, Digits d, const u64* ahat,
                                                     u64 keep, Twiddles tw) {
    __shared__ u64 sm[TILE];
    u64 base = (u64)blockIdx.x * TILE;
    int t = threadIdx.x;
    u64 v[8];
    contig_forward<PACK>(buf + base, d, base, tw, sm, v);
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(ahat + base + 8 * t);
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
    c_inv_col_a(t, sm, buf + base, base, keep);
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
template <int RA, int RB, int C>
static void fwd_pass(const StridedGeom& g, bool pack, const NttJob& j, cudaStream_t st) {
    unsigned grid = (unsigned)(g.N / (RA * RB * C));
    if (pack)
        k_fwd_strided<RA, RB, C, true><<<grid, NT, 0, st>>>(g, j.buf_x, j.buf_a, j.dx, j.da, j.tw);
    else
        k_fwd_strided<RA, RB, C, false><<<grid, NT, 0, st>>>(g, j.buf_x, j.buf_a, j.dx, j.da, j.tw);
}

template <int RA, int RB, int C>
static void inv_pass(const StridedGeom& g, bool last, const NttJob& j, cudaStream_t st) {
    unsigned grid = (unsigned)(g.N / (RA * RB * C));
    if (last)
        k_inv_strided<RA, RB, C, true><<<grid, NT, 0, st>>>(g, j.buf_x, j.L, j.tw);
    else
        k_inv_strided<RA, RB, C, false><<<grid, NT, 0, st>>>(g, j.buf_x, j.L, j.tw);
}

// radix -> (RA, RB, columns per tile)
#define PA_RADIX_TABLE(X)                                                                  \
    X(2, 1, 2, 2048) X(4, 2, 2, 1024) X(8, 2, 4, 512) X(16, 4, 4, 256) X(32, 4, 8, 128)     \
    X(64, 8, 8, 64) X(3, 3, 1, 1024) X(6, 3, 2, 512) X(12, 3, 4, 256) X(24, 3, 8, 128)      \
    X(48, 6, 8, 64)

int strided_columns(int R) {
#define PA_COLS(r, a, b, c) if (R == r) return c;
    PA_RADIX_TABLE(PA_COLS)
#undef PA_COLS
    return 0;
}

static void dispatch_fwd(int R, const StridedGeom& g, bool pack, const NttJob& j, cudaStream_t st) {
#define PA_FWD(r, a, b, c) if (R == r) return fwd_pass<a, b, c>(g, pack, j, st);
    PA_RADIX_TABLE(PA_FWD)
#undef PA_FWD
}

static void dispatch_inv(int R, const StridedGeom& g, bool last, const NttJob& j, cudaStream_t st) {
#define PA_INV(r, a, b, c) if (R == r) return inv_pass<a, b, c>(g, last, j, st);
    PA_RADIX_TABLE(PA_INV)
#undef PA_INV
}

static StridedGeom strided_geom(const Geom& G, int p) {
    u64 C = (u64)strided_columns(G.pass[p].R);
    int log_tpb = 0;
    while ((C << log_tpb) < G.pass[p].S) log_tpb++;
    return StridedGeom{G.N, G.pass[p].M, G.pass[p].S, log_tpb};
}

cudaError_t launch_convolution(const NttJob& j, cudaStream_t st) {
    const Geom& G = j.geom;
    for (int p = 0; p < G.nstrided; p++) {
        StridedGeom g = strided_geom(G, p);
        prof_begin(st, p == 0 ? "ntt_fwd_strided_first" : "ntt_fwd_strided_r64");
        dispatch_fwd(G.pass[p].R, g, p == 0, j, st);
        prof_end(st);
    }
    unsigned tiles = (unsigned)(G.N / TILE);
    bool pack = G.nstrided == 0;  // a single 4096-word tile reads the digits itself
    u64 ninv = n_inverse(G.logN, G.three);
    u64 keep = pack ? j.L : G.N;
    prof_begin(st, "ntt_contig_seed");
    if (pack)
        k_contig_seed<true><<<tiles, NT, 0, st>>>(j.buf_a, j.da, j.ahat, ninv, j.tw);
    else
        k_contig_seed<false><<<tiles, NT, 0, st>>>(j.buf_a, j.da, j.ahat, ninv, j.tw);
    prof_end(st);
    prof_begin(st, "ntt_contig_fused");
    if (pack)
        k_contig_fused<true><<<tiles, NT, 0, st>>>(j.buf_x, j.dx, j.ahat, keep, j.tw);
    else
        k_contig_fused<false><<<tiles, NT, 0, st>>>(j.buf_x, j.dx, j.ahat, keep, j.tw);
    prof_end(st);
    for (int p = G.nstrided - 1; p >= 0; p--) {
        StridedGeom g = strided_geom(G, p);
        prof_begin(st, p == 0 ? "ntt_inv_strided_last" : "ntt_inv_strided_r64");
        dispatch_inv(G.pass[p].R, g, p == 0, j, st);
        prof_end(st);
    }
    return cudaGetLastError();
}

}  // namespace pa
