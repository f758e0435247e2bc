// Batched entry point of the NTT multiply: blocks of one transform geometry,
// MAX_BATCH per launch along gridDim.y (kernels in ntt_kernels.cuh).
#include "ntt_kernels.cuh"

namespace pa {

cudaError_t launch_convolution_batch(const Geom& G, const Twiddles& tw, const BlockIO* io,
                                     int count, cudaStream_t st) {
    for (int i = 0; i < count; i += MAX_BATCH) {
        NttBatch<MAX_BATCH> nb;
        nb.count = count - i < MAX_BATCH ? count - i : MAX_BATCH;
        nb.zero = nullptr;  // a batch clears its carry states with one memset
        nb.zero_words = 0;
        for (int k = 0; k < nb.count; k++) nb.io[k] = io[i + k];
        cudaError_t e = launch_batch<MAX_BATCH>(G, tw, nb, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pa
