// NTT multiply kernels: zero fill + split into 16-bit digits, forward
// transforms, pointwise product and inverse transform (Algorithm 1, steps
// 1-5, Sec. 3.2.2), as tile kernels over GF(p), p = 2^64 - 2^32 + 1.
#include "pa_internal.h"

namespace pa {

// Strided pass over one tile of both operands: the twiddles computed for x
// are kept in registers and reused for a.
template <int RA, int RB, bool PACK>
__global__ void __launch_bounds__(NT, 2) k_fwd_strided(StridedGeom g, u64* buf0, u64* buf1,
                                                    Digits d0, Digits d1, Twiddles tw) {
    using S = Strided<RA, RB>;
    __shared__ u64 sm[TILE];
    TilePos tp = S::tile(g, blockIdx.x);
    u64 w[S::ITEMS_B][RA];
#pragma unroll
    for (int i = 0; i < S::ITEMS_B; i++) S::twiddles(g, tp, threadIdx.x + i * NT, tw, w[i]);
#pragma unroll
    for (int op = 0; op < 2; op++) {
        u64* buf = op ? buf1 : buf0;
        const Digits& d = op ? d1 : d0;
        if (op) __syncthreads();  // the tile of x is out of shared memory
#pragma unroll
        for (int i = 0; i < S::ITEMS_A; i++)
            S::template fwd_a<PACK>(g, tp, threadIdx.x + i * NT, buf, d, sm);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < S::ITEMS_B; i++) S::fwd_b(g, tp, threadIdx.x + i * NT, buf, sm, w[i]);
    }
}

template <int RA, int RB, bool LAST>
__global__ void __launch_bounds__(NT, 2) k_inv_strided(StridedGeom g, u64* buf, u64 keep,
                                                    Twiddles tw) {
    using S = Strided<RA, RB>;
    __shared__ u64 sm[TILE];
    TilePos tp = S::tile(g, blockIdx.x);
#pragma unroll
    for (int i = 0; i < S::ITEMS_B; i++) S::inv_b(g, tp, threadIdx.x + i * NT, buf, sm, tw);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < S::ITEMS_A; i++)
        S::template inv_a<LAST>(g, tp, threadIdx.x + i * NT, buf, sm, keep);
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
template <int RA, int RB>
static void fwd_pass(const StridedGeom& g, bool pack, const NttJob& j, cudaStream_t st) {
    unsigned grid = (unsigned)(g.N / TILE);
    if (pack)
        k_fwd_strided<RA, RB, true><<<grid, NT, 0, st>>>(g, j.buf_x, j.buf_a, j.dx, j.da, j.tw);
    else
        k_fwd_strided<RA, RB, false><<<grid, NT, 0, st>>>(g, j.buf_x, j.buf_a, j.dx, j.da, j.tw);
}

template <int RA, int RB>
static void inv_pass(const StridedGeom& g, bool last, const NttJob& j, cudaStream_t st) {
    unsigned grid = (unsigned)(g.N / TILE);
    if (last)
        k_inv_strided<RA, RB, true><<<grid, NT, 0, st>>>(g, j.buf_x, j.L, j.tw);
    else
        k_inv_strided<RA, RB, false><<<grid, NT, 0, st>>>(g, j.buf_x, j.L, j.tw);
}

static void dispatch_fwd(int R, const StridedGeom& g, bool pack, const NttJob& j, cudaStream_t st) {
    switch (R) {
        case 2: fwd_pass<1, 2>(g, pack, j, st); break;
        case 4: fwd_pass<2, 2>(g, pack, j, st); break;
        case 8: fwd_pass<2, 4>(g, pack, j, st); break;
        case 16: fwd_pass<4, 4>(g, pack, j, st); break;
        case 32: fwd_pass<4, 8>(g, pack, j, st); break;
        default: fwd_pass<8, 8>(g, pack, j, st); break;
    }
}

static void dispatch_inv(int R, const StridedGeom& g, bool last, const NttJob& j, cudaStream_t st) {
    switch (R) {
        case 2: inv_pass<1, 2>(g, last, j, st); break;
        case 4: inv_pass<2, 2>(g, last, j, st); break;
        case 8: inv_pass<2, 4>(g, last, j, st); break;
        case 16: inv_pass<4, 4>(g, last, j, st); break;
        case 32: inv_pass<4, 8>(g, last, j, st); break;
        default: inv_pass<8, 8>(g, last, j, st); break;
    }
}

static StridedGeom strided_geom(const Geom& G, int p) {
    u64 C = TILE / G.pass[p].R;
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
    u64 ninv = n_inverse(G.logN);
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
