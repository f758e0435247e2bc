// Bit-string adapters and the final-key-length helpers.
//
// The reconciled key arrives as a bit string and the final key leaves as one
// (Sec. 2.2: X, X' and Y, Y' are bit strings; Sec. 3.2.1 turns the string into
// words before mpz_import, whose word order may be most or least significant
// first; Sec. 3.2.5 exports the r most significant bits as a bit string).
// These kernels convert between packed bit strings and the library's
// little-endian 64-bit limbs, one output byte per thread.
//
// String bit i (reading order, i < nbits) is bit (i mod 8) of byte i/8, or bit
// 7 - (i mod 8) with most-significant-first packing. With a least-significant-
// first string, string bit i is integer bit i; with a most-significant-first
// string, string bit i is integer bit nbits - 1 - i.
#include <math.h>

#include "../../include/pa.h"
#include "pa_internal.h"

namespace pa {

__device__ __forceinline__ u32 string_bit(const uint8_t* s, u64 i, int msb_bytes) {
    return (s[i >> 3] >> (msb_bytes ? 7 - (int)(i & 7) : (int)(i & 7))) & 1u;
}

// one output byte of limbs (integer bits 8q .. 8q + 7)
__global__ void k_bits_to_limbs(const uint8_t* s, u64 nbits, int msb_string, int msb_bytes,
                                uint8_t* out, u64 out_bytes) {
    for (u64 q = (u64)blockIdx.x * blockDim.x + threadIdx.x; q < out_bytes;
         q += (u64)gridDim.x * blockDim.x) {
        u32 v = 0;
#pragma unroll
        for (int t = 0; t < 8; t++) {
            u64 b = 8 * q + t;  // integer bit
            if (b < nbits) v |= string_bit(s, msb_string ? nbits - 1 - b : b, msb_bytes) << t;
        }
        out[q] = (uint8_t)v;  // little-endian limbs: byte q holds integer bits 8q .. 8q + 7
    }
}

// one output byte of the string (string bits 8q .. 8q + 7)
__global__ void k_limbs_to_bits(const u64* limbs, u64 nbits, int msb_string, int msb_bytes,
                                uint8_t* out, u64 out_bytes) {
    for (u64 q = (u64)blockIdx.x * blockDim.x + threadIdx.x; q < out_bytes;
         q += (u64)gridDim.x * blockDim.x) {
        u32 v = 0;
#pragma unroll
        for (int t = 0; t < 8; t++) {
            u64 i = 8 * q + t;  // string bit
            if (i < nbits) {
                u64 b = msb_string ? nbits - 1 - i : i;
                u32 bit = (u32)(limbs[b >> 6] >> (b & 63)) & 1u;
                v |= bit << (msb_bytes ? 7 - t : t);
            }
        }
        out[q] = (uint8_t)v;
    }
}

}  // namespace pa

using namespace pa;

extern "C" {

int pa_bits_to_limbs(const uint8_t* bits, uint64_t nbits, int msb_string, int msb_bytes,
                     uint64_t* limbs, void* stream) {
    if (!bits || !limbs || nbits < 1 || nbits > PA_MAX_BITS || (msb_string & ~1) || (msb_bytes & ~1)) {
        set_error("pa_bits_to_limbs: need bits, limbs, 1 <= nbits <= PA_MAX_BITS, flags 0 or 1");
        return PA_EINVAL;
    }
    u64 out_bytes = ((nbits + 63) / 64) * 8;  // whole limbs, padding zero
    unsigned grid = (unsigned)((out_bytes + 255) / 256 < 4096 ? (out_bytes + 255) / 256 : 4096);
    k_bits_to_limbs<<<grid, 256, 0, (cudaStream_t)stream>>>(bits, nbits, msb_string, msb_bytes,
                                                           (uint8_t*)limbs, out_bytes);
    if (cudaGetLastError() != cudaSuccess) {
        set_error("pa_bits_to_limbs: launch failed");
        return PA_ECUDA;
    }
    return PA_OK;
}

int pa_limbs_to_bits(const uint64_t* limbs, uint64_t nbits, int msb_string, int msb_bytes,
                     uint8_t* bits, void* stream) {
    if (!bits || !limbs || nbits < 1 || nbits > PA_MAX_BITS || (msb_string & ~1) || (msb_bytes & ~1)) {
        set_error("pa_limbs_to_bits: need bits, limbs, 1 <= nbits <= PA_MAX_BITS, flags 0 or 1");
        return PA_EINVAL;
    }
    u64 out_bytes = (nbits + 7) / 8;
    unsigned grid = (unsigned)((out_bytes + 255) / 256 < 4096 ? (out_bytes + 255) / 256 : 4096);
    k_limbs_to_bits<<<grid, 256, 0, (cudaStream_t)stream>>>(limbs, nbits, msb_string, msb_bytes, bits,
                                                           out_bytes);
    if (cudaGetLastError() != cudaSuccess) {
        set_error("pa_limbs_to_bits: launch failed");
        return PA_ECUDA;
    }
    return PA_OK;
}

// Eq. 1: r <= H_min^{eps/2}(rho_SE | E) - 2 log2(1/eps); the largest such integer.
int pa_final_key_length(double hmin_bits, double eps, uint64_t* r) {
    if (!r || !(eps > 0.0 && eps < 1.0) || !isfinite(hmin_bits)) {
        set_error("pa_final_key_length: need 0 < eps < 1, finite min-entropy, r");
        return PA_EINVAL;
    }
    double v = floor(hmin_bits - 2.0 * log2(1.0 / eps));
    if (!(v >= 1.0) || v > 18446744073709551615.0) {
        set_error("pa_final_key_length: no positive key length for this min-entropy and eps");
        return PA_EINVAL;
    }
    *r = (uint64_t)v;
    return PA_OK;
}

// Definition 2 (quantum leftover hash lemma): the distance bound
// eps_bar = 1/2 * 2^(-(H_min^eps - r)/2) + eps of a key of r bits.
int pa_leftover_epsilon(double hmin_bits, uint64_t r, double eps, double* eps_bar) {
    if (!eps_bar || !(eps >= 0.0) || !isfinite(hmin_bits)) {
        set_error("pa_leftover_epsilon: need eps >= 0, finite min-entropy, eps_bar");
        return PA_EINVAL;
    }
    *eps_bar = 0.5 * exp2(-0.5 * (hmin_bits - (double)r)) + eps;
    return PA_OK;
}

}  // extern "C"
