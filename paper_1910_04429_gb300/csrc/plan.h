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
    int logN = 0;    // log2 of the power-of-two part of N
    int odd = 1;     // N = odd * 2^logN, odd in {1, 3, 5}
    uint64_t N = 0;
    int nstrided = 0;
    PassDesc pass[8];
    int variant = 0; // PLAN_* bits the plan was made with
};

// Plan variants the autotuner chooses between (any order of the strided
// radices factors the same transform; only the memory access pattern and the
// twiddle work per pass change).
constexpr int PLAN_R0_LAST = 1;     // the odd radix R_0 runs last among the strided passes
constexpr int PLAN_DIRECT_FWD = 2;  // forward strided passes load their tiles directly
constexpr int PLAN_DIRECT_INV = 4;  // inverse strided passes load their tiles directly
constexpr int PLAN_NARROW = 8;      // single-pass plans, single blocks: tiles of a quarter of the columns
constexpr int PLAN_BULK = 16;       // single blocks: staged word tiles by one bulk copy per row (cp.async.bulk)
constexpr int PLAN_CLUSTER = 32;    // single blocks of at most 64 tiles: the tile pass on four-CTA clusters
constexpr int PLAN_VARIANTS = 64;
constexpr uint64_t CLUSTER_MAX_TILES = 64;  // PLAN_CLUSTER: transforms of at most this many tiles

// N = R_0 * 64^q * 4096 with N = odd * 2^logN and R_0 = odd * 2^((logN-12) mod 6)
// (omitted when 1; at most 48 for odd = 3, 40 for odd = 5): one strided pass of
// radix R_0, then q strided passes of radix 64, then the contiguous
// 4096-element pass.
inline Geom make_geom(int logN, int odd = 1, int variant = 0) {
    Geom g;
    g.logN = logN;
    g.odd = odd;
    g.variant = variant;
    g.N = (uint64_t)odd << logN;
    int rem = (logN - LOG_TILE) % 6, q = (logN - LOG_TILE) / 6;
    int R0 = odd << rem;
    int radix[8], nr = 0;
    if (R0 > 1 && !(variant & PLAN_R0_LAST)) radix[nr++] = R0;
    for (int i = 0; i < q; i++) radix[nr++] = 64;
    if (R0 > 1 && (variant & PLAN_R0_LAST)) radix[nr++] = R0;
    uint64_t M = g.N;
    for (int i = 0; i < nr; i++) {
        g.pass[g.nstrided++] = PassDesc{radix[i], M, M / radix[i]};
        M /= radix[i];
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

// Whether odd * 2^j (j >= 12) is a transform length here: its first radix
// odd * 2^((j-12) mod 6) is at most 48 (odd = 3) or 40 (odd = 5).
inline bool length_ok(int odd, int j) {
    if (j < LOG_TILE) return false;
    int rem = (j - LOG_TILE) % 6;
    return odd == 1 || (odd == 3 && rem <= 4) || (odd == 5 && rem <= 3);
}

// The shortest transform, 2^k, 3 * 2^k or 5 * 2^k (with the first radix
// bounds above), of at least `need` points (and at least one 4096-point tile).
inline Geom choose_geom_len(uint64_t need) {
    int k = LOG_TILE;
    while ((1ull << k) < need) k++;
    Geom best = make_geom(k, 1);
    for (int odd : {3, 5})
        for (int j = LOG_TILE; j < k; j++)
            if (length_ok(odd, j) && ((uint64_t)odd << j) >= need && ((uint64_t)odd << j) < best.N) {
                best = make_geom(j, odd);
                break;
            }
    return best;
}

// ... that holds the linear convolution of two L-digit operands.
inline Geom choose_geom(uint64_t L) { return choose_geom_len(2 * L - 1); }

// Digit width. Algorithm 1 splits the operands into pieces of M bits; here a
// piece (digit) has w bits, 16 <= w <= 20. The product's coefficients
// t_k = sum_{i+j=k} x_i a_j are below L (2^w - 1)^2 (L = ceil(n/w) digits), and
// the transform over GF(p) is exact when that bound is below p. Wider digits
// mean fewer of them and a shorter transform: at n = 10^8 20-bit digits are
// exact (5 * 10^6 digits, bound < 2^62.3) and need 3/4 of the 16-bit length.
constexpr int DIGIT_MIN = 16, DIGIT_MAX = 20;

inline uint64_t digits_for(uint64_t n, int w) { return (n + (uint64_t)w - 1) / (uint64_t)w; }

// L (2^w - 1)^2 < p, i.e. L <= (p - 1) / (2^w - 1)^2
inline bool width_exact(uint64_t n, int w) {
    if (w < DIGIT_MIN || w > DIGIT_MAX) return false;
    uint64_t d = (1ull << w) - 1;
    return digits_for(n, w) <= (gl::P - 1) / (d * d);
}

// Wrapped product for the modular hash (the output is bits [n-m, n) of
// (a x + b) mod 2^n). A cyclic convolution of length N, L <= N < 2L - 1, gives
// c_k = t_k + t_{k+N}, where t_k is the linear coefficient; t_{k+N} = 0 for
// k >= W = 2L - 1 - N, so every c_k with k >= lo (lo >= W) is exact. (The
// folded terms t_{k+N} weigh 2^(w(k+N)) >= 2^(wL) >= 2^n: they vanish mod 2^n
// in the true product.) The coefficients below lo are dropped: what they would
// add, T = sum_{k<lo} t_k 2^(wk) <= lo (2^w - 1)(2^(w lo) - 1), is below
// lo * 2^(w(lo+1)) <= 2^wbits, wbits = w (lo + 1) + bit_length(lo). The exact
// Q = sum_{k>=lo} c_k 2^(wk) + b then differs from a x + b by T alone, and T
// changes the carry into bit n - m only if every bit of Q in [wbits, n - m)
// is one. The carry step checks limb q - 1 of Q (q = floor((n - m)/64)), which
// lies inside that range when wbits <= 64 (q - 1): if that limb is not all
// ones the result from Q is exact, otherwise the full-length product decides.
// (The rounding test of correctly rounded multiple-precision short products,
// carried over to a truncated product's carry.)
struct WrapPlan {
    bool on = false;  // false: the full-length product (N >= 2L - 1)
    Geom geom;        // the cyclic length
    uint64_t lo = 0;  // coefficients k < lo are dropped (even: whole 16-byte pairs)
};

inline int bit_length(uint64_t v) {
    int b = 0;
    while (v) b++, v >>= 1;
    return b;
}

// Whether a cyclic length N serves keys of n bits with m output bits (L digits
// of w bits).
inline bool wrap_ok(uint64_t N, uint64_t L, uint64_t n, uint64_t m, uint64_t* lo_out, int w = 16) {
    if (N < L || N >= 2 * L - 1) return false;
    uint64_t W = 2 * L - 1 - N, lo = W + (W & 1);
    uint64_t q = (n - m) / 64;
    uint64_t wbits = (uint64_t)w * (lo + 1) + (uint64_t)bit_length(lo);
    if (q < 1 || wbits > 64 * (q - 1)) return false;
    *lo_out = lo;
    return true;
}

// Full-product lengths below this run as they are by default: their
// transforms fill a fraction of the GPU, so a shorter one saves no time and the
// recomputation's launch costs a few microseconds.
constexpr uint64_t WRAP_MIN_FULL = 1ull << 19;

// The shortest transform length that is a valid wrapped length for w-bit
// digits; off when none is shorter than the full-length product's, or that one
// is below min_full.
inline WrapPlan wrap_plan(uint64_t n, uint64_t m, uint64_t min_full = WRAP_MIN_FULL, int w = 16) {
    WrapPlan wp;
    uint64_t L = digits_for(n, w);
    Geom full = choose_geom(L);
    if (full.N < min_full) return wp;
    for (Geom g = choose_geom_len(L); g.N < full.N; g = choose_geom_len(g.N + 1)) {
        uint64_t lo;
        if (wrap_ok(g.N, L, n, m, &lo, w)) {
            wp.on = true;
            wp.geom = g;
            wp.lo = lo;
            return wp;
        }
    }
    return wp;
}

// The product one hash runs: the digit width, the digit count, the wrapped
// plan (or off) and the full-length geometry at that width.
struct DigitPlan {
    int w = 16;
    uint64_t L = 0;
    WrapPlan wp;
    Geom full;
    uint64_t first_n() const { return wp.on ? wp.geom.N : full.N; }
};

// wrap: whether a wrapped product may run (min_full as for wrap_plan);
// width: 0 chooses, among the exact widths, the one whose product is shortest
// (of equals an unwrapped product, which needs no recomputation launch, then
// the narrowest width: its digit split and carry are the cheapest), else that
// width (16 when it is not exact for n).
inline DigitPlan digit_plan(uint64_t n, uint64_t m, bool wrap, uint64_t min_full, int width = 0) {
    DigitPlan best;
    bool have = false;
    for (int w = DIGIT_MIN; w <= DIGIT_MAX; w++) {
        if (width && w != width) continue;
        if (!width_exact(n, w)) continue;
        DigitPlan d;
        d.w = w;
        d.L = digits_for(n, w);
        d.full = choose_geom(d.L);
        if (wrap) d.wp = wrap_plan(n, m, min_full, w);
        if (!have || d.first_n() < best.first_n() || (d.first_n() == best.first_n() && best.wp.on && !d.wp.on))
            best = d, have = true;
    }
    if (!have) {  // a forced width that is not exact: 16-bit digits always are (n <= 2^31)
        best.w = 16;
        best.L = digits_for(n, 16);
        best.full = choose_geom(best.L);
        if (wrap) best.wp = wrap_plan(n, m, min_full, 16);
    }
    return best;
}

// A primitive (15 * 2^32)-th root W with W^(5 * 2^26) = 2, from which every
// transform length N (dividing 15 * 2^32) takes its root w_N = W^(15 * 2^32 / N).
// Then w_N^(N/192) = 2 when 192 | N and w_N^(N/64) = 8 when 64 | N, so all DFTs
// of length dividing 192 inside a transform have power-of-two roots (2 has
// order 192), and w_N^(N/40) = W^(3 * 2^29) is the 40th root the radix-5 steps
// use (the constants gl::w40_pow and the DFT-5 constants are derived from it).
// One root for all lengths also makes a strided pass's twiddle table depend on
// its (M, S) alone. 7 generates GF(p)^*.
inline uint64_t root_15_2_32() {
    const uint64_t p1 = gl::P - 1;
    uint64_t r0 = gl::pow(7, p1 / (15ull << 32));  // order 15 * 2^32
    uint64_t c = gl::pow(r0, 5ull << 26);          // order 192: c = 2^u, gcd(u, 192) = 1
    int u = -1;
    uint64_t e = 1;
    for (int i = 0; i < 192; i++) {
        if (e == c) { u = i; break; }
        e = gl::mul(e, 2);
    }
    if (u < 0) return 0;
    int v = 1;
    while ((u * v) % 192 != 1) v++;               // v = u^-1 mod 192
    while (v % 5 == 0) v += 192;                  // keep the order 15 * 2^32
    return gl::pow(r0, (uint64_t)v);
}

// primitive N-th root for N = odd * 2^logN, odd in {1, 3, 5}
inline uint64_t omega(int logN, int odd = 1) {
    return gl::pow(root_15_2_32(), (uint64_t)(15 / odd) << (32 - logN));
}

// Table layout: w4096 | w4096^-1 | wlo | wlo^-1 | whi | whi^-1
inline size_t table_words_n(uint64_t N) { return 4 * 4096 + 2 * (N >> 12); }
inline size_t table_words(int logN) { return table_words_n(1ull << logN); }

inline void make_tables(int logN, std::vector<uint64_t>& t, int odd = 1) {
    uint64_t N = (uint64_t)odd << logN;
    uint64_t w = omega(logN, odd), wi = gl::pow(w, gl::P - 2);
    uint64_t w4 = gl::pow(w, N >> 12), w4i = gl::pow(wi, N >> 12);
    uint64_t nh = N >> 12;
    t.assign(table_words_n(N), 0);
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

inline uint64_t n_inverse(int logN, int odd = 1) {
    return gl::pow((uint64_t)odd << logN, gl::P - 2);
}

}  // namespace pa
