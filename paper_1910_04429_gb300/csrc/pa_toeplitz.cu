// Toeplitz-hash privacy amplification on the NTT engine (the hash family the
// paper surveys in Sec. 1 as the usual PA choice, computed there by FFT or NTT).
//
// An n + m - 1 bit seed s gives the m x n Toeplitz matrix T[i][j] = s[i - j + n - 1]
// over GF(2), and y = T x. Row i of T against x is
//     y[i] = XOR_j s[i + n - 1 - j] x[j] = (sum_j s[i + n - 1 - j] x[j]) mod 2,
// the parity of coefficient n - 1 + i of the integer convolution of the seed's
// bits with the key's bits. The convolution runs on the Goldilocks NTT with one
// bit per coefficient (every count is at most n < p, so it is exact) and a
// cyclic length N >= n + m - 1 (wrap-around then only lands below index n - 1).
// This file holds the last step: the parity of m consecutive coefficients,
// packed into little-endian 64-bit limbs.
#include "pa_internal.h"
#include "pdl.cuh"

namespace pa {

// One warp per output limb: lane t takes coefficients 64q + t and 64q + 32 + t,
// and two ballots gather their low bits (coalesced 256-byte reads).
__global__ void k_parity_extract(const u64* __restrict__ coef, u64 first, u64 m, u64* __restrict__ out) {
    pdl_begin();
    const u64 limbs = (m + 63) / 64;
    const int lane = threadIdx.x & 31;
    const u64 warps = (u64)gridDim.x * (blockDim.x / 32);
    for (u64 q = ((u64)blockIdx.x * blockDim.x + threadIdx.x) / 32; q < limbs; q += warps) {
        u64 i0 = 64 * q + lane, i1 = i0 + 32;
        bool b0 = i0 < m && (coef[first + i0] & 1u);
        bool b1 = i1 < m && (coef[first + i1] & 1u);
        unsigned lo = __ballot_sync(0xffffffffu, b0), hi = __ballot_sync(0xffffffffu, b1);
        if (lane == 0) out[q] = (u64)lo | ((u64)hi << 32);
    }
}

cudaError_t launch_parity_extract(const u64* coef, u64 first, u64 m, u64* out, cudaStream_t st) {
    u64 limbs = (m + 63) / 64;
    constexpr int THREADS = 256, WARPS = THREADS / 32;
    u64 blocks = (limbs + WARPS - 1) / WARPS;
    unsigned grid = (unsigned)(blocks < 152 * 16 ? blocks : 152 * 16);
    prof_begin(st, "toeplitz_parity");
    cudaError_t e = launch_pdl(k_parity_extract, dim3(grid), dim3(THREADS), 0, st, coef, first, m, out);
    prof_end(st);
    return e;
}

}  // namespace pa
