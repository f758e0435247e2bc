// Host-side transform plan: pass factorisation and twiddle tables.
#pragma once
#include <stdint.h>

#include <vector>

#include "gl.cuh"

namespace pa {

constexpr int LOG_TILE = 12;
constexpr int MAX_LOGN = 28;  // 2^28 coefficients: keys up to 2^31 bits

struct PassDesc {
    int R;      // radix of the strided pass
    uint64_t M; // sub-problem size
    uint64_t S; // stride = M / R
};

struct Geom {
    int logN = 0;
    uint64_t N = 0;
    int nstrided = 0;
    PassDesc pass[8];
};

// N = 2^logN (logN >= 12) = R_0 * 64^q * 4096: one strided pass of radix
// 2^((logN-12) mod 6) if that is > 1, then q strided passes of radix 64, then
// the contiguous 4096-element pass.
inline Geom make_geom(int logN) {
    Geom g;
    g.logN = logN;
    g.N = 1ull << logN;
    int rem = (logN - LOG_TILE) % 6, q = (logN - LOG_TILE) / 6;
    uint64_t M = g.N;
    if (rem) {
        g.pass[g.nstrided++] = PassDesc{1 << rem, M, M >> rem};
        M >>= rem;
    }
    for (int i = 0; i < q; i++) {
        g.pass[g.nstrided++] = PassDesc{64, M, M >> 6};
        M >>= 6;
    }
    return g;
}

// Smallest logN >= 12 with 2^logN >= 2L - 1: the cyclic convolution of two
// L-digit operands then equals their linear convolution (no wrap-around into
// the low digits).
inline int logn_for_digits(uint64_t L) {
    uint64_t need = 2 * L - 1;
    int k = LOG_TILE;
    while ((1ull << k) < need) k++;
    return k;
}

// A primitive 2^32-th root of unity r with r^(2^26) = 8, so that every
// w_N = r^(2^32 / N) satisfies w_N^(N/64) = 8 = 2^3 and all length-64 DFT roots
// are powers of two. 7 generates GF(p)^*.
inline uint64_t root_2_32() {
    const uint64_t p1 = gl::P - 1;
    uint64_t r0 = gl::pow(7, p1 >> 32);
    uint64_t c = gl::pow(r0, 1ull << 26);  // a primitive 64-th root: 8^u for an odd u
    int u = -1;
    uint64_t e = 1;
    for (int i = 0; i < 64; i++) {
        if (e == c) { u = i; break; }
        e = gl::mul(e, 8);
    }
    if (u < 0) return 0;
    int v = 1;
    while ((u * v) % 64 != 1) v += 2;  // v = u^-1 mod 64
    return gl::pow(r0, (uint64_t)v);
}

inline uint64_t omega(int logN) { return gl::pow(root_2_32(), 1ull << (32 - logN)); }

// Table layout: w4096 | w4096^-1 | wlo | wlo^-1 | whi | whi^-1
inline size_t table_words(int logN) { return 4 * 4096 + 2 * ((1ull << logN) >> 12); }

inline void make_tables(int logN, std::vector<uint64_t>& t) {
    uint64_t N = 1ull << logN;
    uint64_t w = omega(logN), wi = gl::pow(w, gl::P - 2);
    uint64_t w4 = gl::pow(w, N >> 12), w4i = gl::pow(wi, N >> 12);
    uint64_t nh = N >> 12;
    t.assign(table_words(logN), 0);
    uint64_t* w4096 = t.data();
    uint64_t* w4096i = w4096 + 4096;
    uint64_t* wlo = w4096i + 4096;
    uint64_t* wloi = wlo + 4096;
    uint64_t* whi = wloi + 4096;
    uint64_t* whii = whi + nh;
    uint64_t a = 1, b = 1, c = 1, d = 1;
    for (int i = 0; i < 4096; i++) {
        w4096[i] = a; a = gl::mul(a, w4);
        w4096i[i] = b; b = gl::mul(b, w4i);
        wlo[i] = c; c = gl::mul(c, w);
        wloi[i] = d; d = gl::mul(d, wi);
    }
    uint64_t s = gl::pow(w, 4096), si = gl::pow(wi, 4096);
    a = b = 1;
    for (uint64_t i = 0; i < nh; i++) {
        whi[i] = a; a = gl::mul(a, s);
        whii[i] = b; b = gl::mul(b, si);
    }
}

inline uint64_t n_inverse(int logN) { return gl::P - ((gl::P - 1) >> logN); }

}  // namespace pa
