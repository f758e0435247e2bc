// Single-block entry points of the NTT multiply (Algorithm 1, steps 1-5,
// Sec. 3.2.2) and the per-pass twiddle tables; the kernels and the launch
// sequence are in ntt_kernels.cuh.
#include "ntt_kernels.cuh"

namespace pa {

// Inter-pass twiddle tables of one strided pass (sub-problem size M, stride S):
// fwd[k S + j] = w_M^(j k), inv[k S + j] = w_M^-(j k), from the transform's
// w_N tables (w_M = w_N^(N/M)).
__global__ void k_pass_twiddles(Twiddles tw, u64 N, u64 M, u64 S, u64* fwd, u64* inv) {
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (u64)gridDim.x * blockDim.x) {
        u64 k = i / S, j = i - k * S;
        u64 e = (N / M) * j * k;  // < N
        fwd[i] = omega_n<false>(tw, e);
        inv[i] = omega_n<true>(tw, e);
    }
}

cudaError_t launch_pass_twiddles(const Twiddles& tw, u64 N, u64 M, u64 S, u64* out, cudaStream_t st) {
    u64 blocks = (M + 255) / 256;
    k_pass_twiddles<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(tw, N, M, S, out, out + M);
    return cudaGetLastError();
}

// the sticky status of this file's kernels' bulk-copy waits (ntt_kernels.cuh)
cudaError_t read_bulk_status(u32* out, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_bulk_status, sizeof(u32));
    if (e == cudaSuccess && clear) {
        u32 zero = 0;
        e = cudaMemcpyToSymbol(g_bulk_status, &zero, sizeof(u32));
    }
    return e;
}

cudaError_t launch_convolution(const NttJob& j, cudaStream_t st) {
    NttBatch<1> nb;
    nb.count = 1;
    nb.zero = j.zero;
    nb.zero_words = j.zero_words;
    nb.io[0] = BlockIO{j.buf_x, j.buf_a, j.dx, j.da, j.L};
    return launch_batch<1>(j.geom, j.tw, nb, st);
}

// Forward transform of a alone into buf_a (its spectrum, register order, x N^-1):
// the strided passes run with x = a (the x half of each CTA is skipped by
// pointing both halves at a and running ops = 1 on buf_a), then contig_seed.
cudaError_t launch_seed_spectrum(const NttJob& j, cudaStream_t st) {
    NttBatch<1> nb;
    nb.count = 1;
    nb.zero = nullptr;
    nb.zero_words = 0;
    nb.io[0] = BlockIO{j.buf_a, j.buf_a, j.da, j.da, j.L};
    bool aligned = (uintptr_t)j.da.src % 16 == 0 && !j.da.one_bit;
    const Geom& G = j.geom;
    bool narrow = narrow_plan<1>(G);
    if (j.da.width > 16 && !aligned && G.nstrided > 0) return cudaErrorInvalidValue;  // wider digits: staged only
    for (int p = 0; p < G.nstrided; p++) {
        StridedGeom g = strided_geom(G, j.tw, p, narrow);
        prof_begin(st, "ntt_seed_strided");
        Launcher<1>{&g, &nb, &j.tw, st, aligned, 1, !(G.variant & PLAN_DIRECT_FWD), true, narrow, j.da.width > 16}
            .dispatch_fwd(G.pass[p].R, p == 0);
        prof_end(st);
    }
    dim3 tiles((unsigned)(G.N / TILE), 1);
    prof_begin(st, "ntt_contig_seed");
    if (G.nstrided == 0)
        launch_pdl(k_contig_seed<true, 1>, tiles, dim3(NT), 0, st, nb, n_inverse(G.logN, G.odd), j.tw);
    else
        launch_pdl(k_contig_seed<false, 1>, tiles, dim3(NT), 0, st, nb, n_inverse(G.logN, G.odd), j.tw);
    prof_end(st);
    return cudaGetLastError();
}

// x's transform, product with the stored spectrum in buf_a, inverse.
cudaError_t launch_convolution_seeded(const NttJob& j, cudaStream_t st) {
    NttBatch<1> nb;
    nb.count = 1;
    nb.zero = j.zero;
    nb.zero_words = j.zero_words;
    nb.io[0] = BlockIO{j.buf_x, j.buf_a, j.dx, j.da, j.L};
    return launch_batch<1>(j.geom, j.tw, nb, st, 1);
}

}  // namespace pa
