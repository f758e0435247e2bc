// Goldilocks prime field GF(p), p = 2^64 - 2^32 + 1.
//
// The exact multiply of the G_{c,d} hash (arXiv 1910.04429, Sec. 3.2.2,
// Algorithm 1) is done here with a number-theoretic transform over this prime
// instead of GMP's Fermat-ring Schonhage-Strassen. Reduction uses the shape of p:
// 2^64 = 2^32 - 1 (mod p) and 2^96 = -1 (mod p), so 2 is a 192-th root of unity
// and 8 = 2^3 a primitive 64-th root: DFTs of length <= 64 need no general
// multiplies, only the shift-multiplies below.
//
// Field values are kept in [0, p] (p may stand for 0 inside a transform; see
// sub below), and canon() maps them to [0, p) where an exact integer leaves
// the field.
#pragma once
#include <stdint.h>

typedef uint64_t u64;
typedef uint32_t u32;

#if defined(__CUDACC__)
#define GL_HD __host__ __device__ __forceinline__
#else
#define GL_HD inline
#endif

namespace gl {

constexpr u64 P = 0xFFFFFFFF00000001ull;
constexpr u64 EPS = 0xFFFFFFFFull;  // 2^64 mod p

// Values are kept in [0, p]: p itself may stand for 0 inside a transform
// (neg(0) = p); add, sub, mul and the shifts accept and return that range, and
// canon() maps p to 0 where an exact integer leaves the field.
GL_HD u64 sub(u64 a, u64 b);

// a + b = a - (p - b): the subtraction's borrow fix-up is cheaper than an add's
// compare-and-select (p - b stays in [0, p] for b in [0, p]).
GL_HD u64 add(u64 a, u64 b) { return sub(a, P - b); }

GL_HD u64 sub(u64 a, u64 b) {
#if defined(__CUDA_ARCH__)
    // a - b; on borrow the wrapped value is 2^64 too large and 2^64 = EPS + p
    u64 d;
    u32 m;
    asm("sub.cc.u64 %0, %2, %3;\n\t"
        "subc.u32 %1, 0, 0;"
        : "=l"(d), "=r"(m)
        : "l"(a), "l"(b));
    return d - (u64)m;
#else
    u64 d = a - b;
    if (a < b) d -= EPS;
    return d;
#endif
}

GL_HD u64 neg(u64 a) { return P - a; }

GL_HD u64 canon(u64 a) { return a == P ? 0 : a; }

// (hi:lo) mod p for any 128-bit value, using 2^64 = EPS and 2^96 = -1;
// result in [0, p).
#if defined(__CUDA_ARCH__)
// r - p when r >= p (r + EPS carries out exactly then); r < 2^64
__device__ __forceinline__ u64 canon_lt2p(u64 r) {
    u64 q;
    u32 c;
    asm("add.cc.u64 %0, %2, 4294967295;\n\t"
        "addc.u32 %1, 0, 0;"
        : "=l"(q), "=r"(c)
        : "l"(r));
    return c ? q : r;
}

// t + h0 * 2^64 (mod p) for t < 2^64 and h0 < 2^32, in [0, p): 2^64 = EPS,
// the product h0 * EPS and the carry's EPS go through the multiplier (FMA pipe)
__device__ __forceinline__ u64 fold_word(u64 t, u32 h0) {
    u64 u, r;
    u32 c;
    asm("mul.wide.u32 %0, %1, 4294967295;" : "=l"(u) : "r"(h0));
    asm("add.cc.u64 %0, %2, %3;\n\t"
        "addc.u32 %1, 0, 0;"
        : "=l"(r), "=r"(c)
        : "l"(t), "l"(u));
    asm("mad.wide.u32 %0, %1, 4294967295, %0;" : "+l"(r) : "r"(c));  // carry of 2^64 = EPS
    return canon_lt2p(r);
}
#endif

// (hi:lo) mod p for any 128-bit value, using 2^64 = EPS and 2^96 = -1;
// result in [0, p).
GL_HD u64 reduce128(u64 lo, u64 hi) {
#if defined(__CUDA_ARCH__)
    u32 h0 = (u32)hi, h1 = (u32)(hi >> 32);
    u64 t;
    u32 m;
    asm("sub.cc.u64 %0, %2, %3;\n\t"
        "subc.u32 %1, 0, 0;"
        : "=l"(t), "=r"(m)
        : "l"(lo), "l"((u64)h1));
    t -= (u64)m;  // lo - h1 (a borrow of 2^64 = EPS)
    return fold_word(t, h0);
#else
    u64 h0 = hi & 0xFFFFFFFFull, h1 = hi >> 32;
    u64 t = lo - h1;
    if (lo < h1) t -= EPS;
    u64 u = (h0 << 32) - h0;
    u64 r = t + u;
    if (r < u) r += EPS;
    if (r >= P) r -= P;
    return r;
#endif
}

GL_HD u64 mul(u64 a, u64 b) {
#if defined(__CUDA_ARCH__)
    // 64 x 64 -> 128 from four 32 x 32 products with one carry chain
    u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
    u32 r0, r1, r2, r3;
    asm("mul.lo.u32 %0, %4, %6;\n\t"
        "mul.hi.u32 %1, %4, %6;\n\t"
        "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
        "madc.hi.u32 %2, %4, %7, 0;\n\t"
        "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
        "madc.hi.u32 %3, %5, %7, 0;\n\t"
        "mad.lo.cc.u32 %2, %5, %7, %2;\n\t"
        "addc.u32 %3, %3, 0;"
        : "=&r"(r0), "=&r"(r1), "=&r"(r2), "=&r"(r3)
        : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
    return reduce128(((u64)r1 << 32) | r0, ((u64)r3 << 32) | r2);
#else
    unsigned __int128 t = (unsigned __int128)a * b;
    return reduce128((u64)t, (u64)(t >> 64));
#endif
}

GL_HD u64 pow(u64 b, u64 e) {
    u64 r = 1;
    while (e) {
        if (e & 1) r = mul(r, b);
        b = mul(b, b);
        e >>= 1;
    }
    return r;
}

}  // namespace gl

namespace gl {

GL_HD constexpr u64 pow2_mod(int s) {
    // 2^s for s < 64, folded with 2^64 = EPS, 2^96 = -1 (constexpr, host and device)
    u64 r = 1;
    for (int i = 0; i < s; i++) {
        u64 t = r << 1;
        bool carry = r >> 63;
        if (carry) t += EPS;            // t + 2^64 = t + EPS; t < 2^64 - 2 so no second carry
        if (t >= P) t -= P;
        r = t;
    }
    return r;
}

// x * 2^s mod p for s in (0, 32): the product spans 96 bits and its top word
// h0 < 2^32 folds in once.
GL_HD u64 shl_small(u64 x, int s) {
#if defined(__CUDA_ARCH__)
    u64 lo = x << s;
    u32 h0 = (u32)(x >> (64 - s));
    return fold_word(lo, h0);
#else
    return reduce128(x << s, x >> (64 - s));
#endif
}

// t * EPS = t * 2^64 mod p for t < 2^32: one 32 x 32 -> 64 product (FMA pipe),
// at most (2^32 - 1)^2 < p.
GL_HD u64 mul_eps(u32 t) {
#if defined(__CUDA_ARCH__)
    u64 r;
    asm("mul.wide.u32 %0, %1, 4294967295;" : "=l"(r) : "r"(t));
    return r;
#else
    return (u64)t * EPS;
#endif
}

// x * 2^s mod p for s in [32, 64). With k = 96 - s in (32, 64], x = q 2^k + r:
// x 2^s = q 2^96 + r 2^s = -q + u 2^32, u = r 2^(s-32) = x << (s - 32) (mod 2^64,
// the bits of q shift out). With u = uh 2^32 + ul, u 2^32 = uh 2^64 + ul 2^32
// = uh EPS + ul 2^32 = (uh + ul) 2^32 - uh, and a carry out of uh + ul is one
// more 2^64 = EPS. That value is below p and q < 2^31, so one field sub ends it.
GL_HD u64 shl_mid(u64 x, int s) {
    u64 u = x << (s - 32);
    u32 uh = (u32)(u >> 32), ul = (u32)u;
    u64 q = s == 32 ? 0 : x >> (96 - s);
#if defined(__CUDA_ARCH__)
    u32 w, c;
    asm("add.cc.u32 %0, %2, %3;\n\t"
        "addc.u32 %1, 0, 0;"
        : "=r"(w), "=r"(c)
        : "r"(uh), "r"(ul));
    u64 v = ((u64)w << 32) - uh;
    asm("mad.wide.u32 %0, %1, 4294967295, %0;" : "+l"(v) : "r"(c));
#else
    u64 wide = (u64)uh + ul;
    u64 v = ((wide & 0xFFFFFFFFull) << 32) - uh + ((wide >> 32) ? EPS : 0);
#endif
    return sub(v, q);
}

// x * 2^s mod p for s in [64, 96). With k = 96 - s in (0, 32], x = q 2^k + r:
// x 2^s = q 2^96 + r 2^s = -q + t 2^64 = t EPS - q, t = r 2^(s-64) < 2^32
// (the low 32 bits of x shifted by s - 64; bits above k shift out).
GL_HD u64 shl_hi(u64 x, int s) { return sub(mul_eps((u32)x << (s - 64)), x >> (96 - s)); }

// x * 2^s mod p for s in [160, 192): 2^s = -2^(s-96), the negation of shl_hi.
GL_HD u64 shl_top(u64 x, int s) { return sub(x >> (192 - s), mul_eps((u32)x << (s - 160))); }

// x * 2^s mod p for a run-time s in [0, 192), by range. The integer ALU pipe
// bounds the transforms while the multiplier (FMA) pipe has room, so where a
// chain of the multiplier-based routes (shl_hi: 1 ALU + 3 FMA instructions,
// shl_top: 2 + 3) costs fewer ALU instructions than a direct route it is used
// instead, with 2^192 = 1 (2 has order 192 mod p):
//   s < 32           shl_small                      5 + 5
//   32 <= s < 64     2^64 * 2^(s+128): hi, top       3 + 6  (shl_mid: 8 + 3)
//   64 <= s < 96     shl_hi                          1 + 3
//   s = 96           negation
//   96 < s < 128     2^64 * 2^64 * 2^(s+64)          4 + 9  (negated shl_small: 7 + 5)
//   128 <= s < 160   2^64 * 2^(s-64): hi, hi         2 + 6  (negated shl_mid: 10 + 3)
//   160 <= s < 192   shl_top                         2 + 3
// Inside fully unrolled loops s is a constant and the branches fold away; where
// s varies it is uniform across a warp in every caller.
GL_HD u64 shl_v(u64 x, int s) {
    if (s == 0) return x;
    if (s < 32) return shl_small(x, s);
    if (s < 64) return shl_top(shl_hi(x, 64), s + 128);
    if (s < 96) return shl_hi(x, s);
    if (s == 96) return neg(x);
    if (s < 128) return shl_top(shl_hi(shl_hi(x, 64), 64), s + 64);
    if (s < 160) return shl_hi(shl_hi(x, 64), s - 64);
    return shl_top(x, s);
}

// Shift for w^e where w = 2^(192/R) is the R-th root of unity used by every
// radix-R DFT here (R | 192; 2 has order 192 mod p); INV selects w^-e.
template <int R, bool INV>
GL_HD int root_shift(int e) {
    int s = ((192 / R) * e) % 192;
    return INV ? (192 - s) % 192 : s;
}

// v[k] <- v[k] * w^(j k) for 0 < k < K, w = 2^(192/R) (or its inverse), for a
// run-time row j < J that is uniform across a warp: one branch on j picks a
// copy in which every shift amount is a compile-time constant and takes its
// fixed route (a run-time amount would pay a range dispatch per shift).
template <int R, bool INV, int K, int J>
struct RowRoots {
    static GL_HD void apply(u64* v, int j) {
        if (j == J - 1) {
#pragma unroll
            for (int k = 1; k < K; k++) v[k] = shl_v(v[k], root_shift<R, INV>((J - 1) * k));
        } else {
            RowRoots<R, INV, K, J - 1>::apply(v, j);
        }
    }
};
template <int R, bool INV, int K>
struct RowRoots<R, INV, K, 1> {  // row 0: w^0 = 1
    static GL_HD void apply(u64*, int) {}
};

template <int R>
GL_HD void dft_fwd(u64* v);

// Forward DFT of length R in {2, 4, 8} whose inputs v[R/2 ..] are zero (the
// first decimation-in-frequency stage reduces to copies and roots).
template <int R>
GL_HD void dft_fwd_upper_zero(u64* v) {
    if constexpr (R == 2) {
        v[1] = v[0];
    } else if constexpr (R == 4) {
        u64 a = v[0], d = shl_v(v[1], root_shift<4, false>(1));
        v[2] = sub(a, v[1]);
        v[0] = add(a, v[1]);
        v[1] = add(a, d);
        v[3] = sub(a, d);
    } else {
        static_assert(R == 8, "upper-zero DFT of length 2, 4 or 8");
        u64 s[4], t[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            s[i] = v[i];
            t[i] = shl_v(v[i], root_shift<8, false>(i));
        }
        dft_fwd<4>(s);
        dft_fwd<4>(t);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            v[2 * k] = s[k];
            v[2 * k + 1] = t[k];
        }
    }
}

// Roots for the lengths 5 * 2^k. w40_pow(e) = w_40^e for the 40th root w_40 that
// every transform of length 5 * 2^k uses (w_N^(N/40); the transform roots come
// from a fixed (15 * 2^32)-th root W with W^(5 * 2^26) = 2, and w_40 =
// W^(3 * 2^29)); w_40^(5 i) = 2^(24 i), consistent with the power-of-two roots
// of the other steps. Values checked on the host against that construction.
GL_HD constexpr u64 w40_pow(int e) {
    constexpr u64 t[40] = {
        0x0000000000000001ull, 0xd850dddf7d0e7367ull, 0x8ee62dc0237ef6b1ull, 0x0cadbf02e30803a7ull,
        0xecf1f86a7562be2bull, 0x0000000001000000ull, 0xe0555f506627af23ull, 0xc0b26523b07119d3ull,
        0x02efb5c2a6f35241ull, 0x6b6254b62a130e08ull, 0x0001000000000000ull, 0x51467d0e221faaa1ull,
        0x2471237ed23f4d9bull, 0xc2a9e30740fd104bull, 0xb695756207949dacull, 0x000000ffffffff00ull,
        0x0e736627a0aeb983ull, 0x7ef6b0709adb8eddull, 0x0803a6f34a3d561dull, 0x62be2a12ab496a8bull,
        0xffffffff00000000ull, 0x27af221f82f18c9aull, 0x7119d23edc810950ull, 0xf35240fc1cf7fc5aull,
        0x130e07948a9d41d6ull, 0xfffffffeff000001ull, 0x1faaa0ae99d850deull, 0x3f4d9adb4f8ee62eull,
        0xfd104a3c590cadc0ull, 0x949dab48d5ecf1f9ull, 0xfffeffff00000001ull, 0xaeb982f0dde05560ull,
        0xdb8edc802dc0b266ull, 0x3d561cf7bf02efb6ull, 0x496a8a9cf86b6255ull, 0xfffffeff00000101ull,
        0xf18c99d75f51467eull, 0x81094f8e65247124ull, 0xf7fc590bb5c2a9e4ull, 0x9d41d5ec54b69576ull,
};
    return t[e];
}
// Constants of the 5-point DFT with w = w_5 = w40_pow(8): with alpha = (w + w^4)/2,
// beta = (w^2 + w^3)/2, gamma = (w - w^4)/2, delta = (w^2 - w^3)/2 (alpha + beta
// = -1/2): K1 = (alpha - beta)/2, and gamma, gamma + delta, delta - gamma.
constexpr u64 DFT5_K1 = 0xaf3f49212a5a0254ull;
constexpr u64 DFT5_GA = 0x13b06ca0bc994feeull;
constexpr u64 DFT5_GPD = 0x91631be9c7a20bc5ull;
constexpr u64 DFT5_DMG = 0x6a0242a84e6f6be9ull;

// x * w_40^e: a shift where w_40^e is a power of two (e a multiple of 5), else
// a product by the constant.
template <int E>
GL_HD u64 mul_w40(u64 x) {
    constexpr int e = ((E % 40) + 40) % 40;
    if constexpr (e % 5 == 0) return shl_v(x, 24 * (e / 5));
    else return mul(x, w40_pow(e));
}

// RowRoots for R in {10, 20, 40} (R not a divisor of 192): v[k] <- v[k] * w_R^(j k),
// w_R = w_40^(40/R), for a run-time row j < J uniform across a warp.
template <int R, bool INV, int K, int J>
struct RowRoots40 {
    template <int k>
    static GL_HD void one(u64* v) {
        constexpr int e = (40 / R) * (J - 1) * k;
        v[k] = mul_w40<INV ? -e : e>(v[k]);
        if constexpr (k + 1 < K) one<k + 1>(v);
    }
    static GL_HD void apply(u64* v, int j) {
        if (j == J - 1) {
            if constexpr (K > 1) one<1>(v);
        } else {
            RowRoots40<R, INV, K, J - 1>::apply(v, j);
        }
    }
};
template <int R, bool INV, int K>
struct RowRoots40<R, INV, K, 1> {  // row 0: w^0 = 1
    static GL_HD void apply(u64*, int) {}
};

// The middle roots of a radix-R step: power-of-two shifts when R divides 192,
// else products by the w_40 constants.
template <int R, bool INV, int K, int J>
GL_HD void row_roots(u64* v, int j) {
    if constexpr (192 % R == 0) RowRoots<R, INV, K, J>::apply(v, j);
    else RowRoots40<R, INV, K, J>::apply(v, j);
}

// In-register DFT of length R in {1, 2, 3, 4, 5, 6, 8}, natural order in and out:
// v[k] <- sum_j v[j] w^(jk), w = 2^(192/R) (or its inverse), no 1/R scaling.
// The inverse is the forward DFT read backwards (sum_j v[j] w^(-jk) is the
// forward output R - k), which keeps every root a cheap forward shift.
template <int R, bool INV>
GL_HD void dft(u64* v) {
    dft_fwd<R>(v);
    if constexpr (INV) {
#pragma unroll
        for (int k = 1; k < R - k; k++) {
            u64 t = v[k];
            v[k] = v[R - k];
            v[R - k] = t;
        }
    }
}

template <int R>
GL_HD void dft_fwd(u64* v) {
    if constexpr (R == 1) {
        (void)v;
    } else if constexpr (R == 2) {
        u64 a = v[0], b = v[1];
        v[0] = add(a, b);
        v[1] = sub(a, b);
    } else if constexpr (R == 4) {
        // w = 2^48 (forward); w^2 = -1
        u64 a = add(v[0], v[2]), b = sub(v[0], v[2]);
        u64 c = add(v[1], v[3]);
        u64 d = shl_v(sub(v[1], v[3]), root_shift<4, false>(1));
        v[0] = add(a, c);
        v[2] = sub(a, c);
        v[1] = add(b, d);
        v[3] = sub(b, d);
    } else if constexpr (R == 3) {
        // w = 2^64 (forward), w^2 = -1 - w:
        // X0 = a + b + c, X1 = (a - c) + w (b - c), X2 = (a - b) - w (b - c)
        u64 a = v[0], b = v[1], c = v[2];
        u64 t = shl_v(sub(b, c), root_shift<3, false>(1));
        v[0] = add(add(a, b), c);
        v[1] = add(sub(a, c), t);
        v[2] = sub(sub(a, b), t);
    } else if constexpr (R == 6) {
        // X[2k] = DFT3(v_i + v_{i+3}), X[2k+1] = DFT3((v_i - v_{i+3}) w^i), w = 2^32
        u64 s[3], t[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            s[i] = add(v[i], v[i + 3]);
            t[i] = shl_v(sub(v[i], v[i + 3]), root_shift<6, false>(i));
        }
        dft_fwd<3>(s);
        dft_fwd<3>(t);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            v[2 * k] = s[k];
            v[2 * k + 1] = t[k];
        }
    } else if constexpr (R == 5) {
        // Winograd's form: with a1 = v1 + v4, b1 = v1 - v4, a2 = v2 + v3,
        // b2 = v2 - v3, s = a1 + a2: X0 = v0 + s, and from base = v0 - s/4,
        // m1 = K1 (a1 - a2), P = gamma b1 + delta b2, Q = delta b1 - gamma b2
        // (three products): X1 = base + m1 + P, X4 = base + m1 - P,
        // X2 = base - m1 + Q, X3 = base - m1 - Q
        u64 a1 = add(v[1], v[4]), b1 = sub(v[1], v[4]), a2 = add(v[2], v[3]), b2 = sub(v[2], v[3]);
        u64 s = add(a1, a2), x0 = v[0];
        u64 m1 = mul(sub(a1, a2), DFT5_K1);
        u64 base = sub(x0, shl_v(s, 190));  // s * 2^-2
        u64 ma = mul(sub(b1, b2), DFT5_GA);
        u64 pp = add(ma, mul(b2, DFT5_GPD));
        u64 qq = add(mul(b1, DFT5_DMG), ma);
        u64 bp = add(base, m1), bm = sub(base, m1);
        v[0] = add(x0, s);
        v[1] = add(bp, pp);
        v[4] = sub(bp, pp);
        v[2] = add(bm, qq);
        v[3] = sub(bm, qq);
    } else if constexpr (R == 8) {
        // one radix-2 decimation-in-frequency step, then two length-4 DFTs:
        // X[2k] = DFT4(v_i + v_{i+4}), X[2k+1] = DFT4((v_i - v_{i+4}) w^i)
        u64 s[4], t[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            s[i] = add(v[i], v[i + 4]);
            t[i] = shl_v(sub(v[i], v[i + 4]), root_shift<8, false>(i));
        }
        dft_fwd<4>(s);
        dft_fwd<4>(t);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            v[2 * k] = s[k];
            v[2 * k + 1] = t[k];
        }
    }
}

}  // namespace gl
