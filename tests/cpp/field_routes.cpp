// Host check of the field helpers shared with the kernels (csrc/gl.cuh, host
// variants): every route of x * 2^s mod p (s in [0, 192), including the chains
// of multiplier-based routes), sub, add and mul, against 128-bit arithmetic
// reduced with the % operator. Inputs: 0, 1, p - 1, p (the transforms' stand-in
// for 0) and pseudo-random values in [0, p]. Then the roots and steps of the
// lengths 5 * 2^k: the constants w40_pow(e) against the fixed root of
// plan.h (W^(3 * 2^29 e)), the transform roots' orders and their 64th-power
// relation, the 5-point DFT (forward and inverse) and the radix-10/20/40
// middle roots against direct sums and powers. Prints "ok" and exits 0 on
// success.
#include <cstdint>
#include <cstdio>

#include "gl.cuh"
#include "plan.h"

using namespace gl;

static u64 mod_mul(u64 a, u64 b) { return (u64)((unsigned __int128)a * b % P); }

static u64 splitmix(u64& s) {
    u64 z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int main() {
    u64 state = 1;
    const int per_shift = 4000;
    long bad = 0;
    for (int s = 0; s < 192; s++) {
        u64 pw = 1;
        for (int i = 0; i < s; i++) pw = mod_mul(pw, 2);
        for (int t = 0; t < per_shift; t++) {
            u64 x = t == 0 ? P : t == 1 ? 0 : t == 2 ? P - 1 : t == 3 ? 1 : splitmix(state) % (P + 1);
            u64 got = shl_v(x, s);
            if (got > P || got % P != mod_mul(x % P, pw)) {
                if (bad++ < 5) printf("shl_v s=%d x=%llx -> %llx\n", s, (unsigned long long)x, (unsigned long long)got);
            }
        }
    }
    for (int t = 0; t < 200000; t++) {
        u64 a = t < 4 ? (t & 1 ? P : 0) : splitmix(state) % (P + 1);
        u64 b = t < 4 ? (t & 2 ? P : 1) : splitmix(state) % (P + 1);
        u64 am = a % P, bm = b % P;
        u64 s = sub(a, b), d = add(a, b), m = mul(a, b);
        if (s > P || s % P != (u64)(((unsigned __int128)am + P - bm) % P)) bad++;
        if (d > P || d % P != (u64)(((unsigned __int128)am + bm) % P)) bad++;
        if (m >= P || m != mod_mul(am, bm)) bad++;
    }
    // lengths 5 * 2^k
    const u64 W = pa::root_15_2_32();
    const u64 w40 = pow(W, 3ull << 29);
    for (int e = 0; e < 40; e++)
        if (w40_pow(e) != pow(w40, (u64)e)) bad++, printf("w40_pow(%d)\n", e);
    if (pow(w40, 40) != 1 || pow(w40, 20) == 1 || pow(w40, 8) == 1) bad++, printf("w40 order\n");
    for (int odd : {1, 3, 5})  // every length's root: exact order, the power-of-two relations
        for (int logN = 12; logN <= 28; logN++) {
            u64 N = (u64)odd << logN, w = pa::omega(logN, odd);
            if (pow(w, N) != 1 || pow(w, N / 2) == 1 || (odd > 1 && pow(w, N / odd) == 1))
                bad++, printf("order %d %d\n", odd, logN);
            if (pow(w, N / 64) != 8) bad++, printf("w_64 %d %d\n", odd, logN);
            if (odd == 3 && pow(w, N / 192) != 2) bad++, printf("w_192 %d\n", logN);
            if (odd == 5 && pow(w, N / 40) != w40) bad++, printf("w_40 %d\n", logN);
            // a root of a length and of its multiples agree: w_(2N)^2 = w_N
            if (logN < 28 && pow(pa::omega(logN + 1, odd), 2) != w) bad++, printf("nested %d %d\n", odd, logN);
        }
    const u64 w5 = w40_pow(8), w5i = pow(w5, P - 2);
    for (int t = 0; t < 20000; t++) {
        u64 x[5], f[5], g[5];
        for (int j = 0; j < 5; j++) x[j] = t < 5 ? (j == t ? P : 0) : splitmix(state) % (P + 1);
        for (int j = 0; j < 5; j++) f[j] = g[j] = x[j];
        dft<5, false>(f);
        dft<5, true>(g);
        for (int k = 0; k < 5; k++) {
            u64 sf = 0, sg = 0;
            for (int j = 0; j < 5; j++) {
                sf = (u64)(((unsigned __int128)sf + mod_mul(x[j] % P, pow(w5, (u64)(j * k)))) % P);
                sg = (u64)(((unsigned __int128)sg + mod_mul(x[j] % P, pow(w5i, (u64)(j * k)))) % P);
            }
            if (f[k] > P || f[k] % P != sf || g[k] > P || g[k] % P != sg) bad++;
        }
    }
    // row roots: v[k] * w_R^(j k) (and w_R^-(j k)) for R in {10, 20, 40}, j < 5, k < 8
    {
        const int Rs[3] = {10, 20, 40};
        for (int ri = 0; ri < 3; ri++) {
            const int R = Rs[ri];
            const u64 wR = pow(w40, (u64)(40 / R)), wRi = pow(wR, P - 2);
            for (int j = 0; j < 5; j++) {
                u64 x[8], v[8], u[8];
                for (int k = 0; k < 8; k++) x[k] = v[k] = u[k] = splitmix(state) % (P + 1);
                if (R == 10) row_roots<10, false, 8, 5>(v, j), row_roots<10, true, 8, 5>(u, j);
                if (R == 20) row_roots<20, false, 8, 5>(v, j), row_roots<20, true, 8, 5>(u, j);
                if (R == 40) row_roots<40, false, 8, 5>(v, j), row_roots<40, true, 8, 5>(u, j);
                for (int k = 0; k < 8; k++) {
                    u64 wf = pow(wR, (u64)(j * k)), wi = pow(wRi, (u64)(j * k));
                    if (v[k] > P || v[k] % P != mod_mul(x[k] % P, wf)) bad++, printf("rows R=%d j=%d k=%d\n", R, j, k);
                    if (u[k] > P || u[k] % P != mod_mul(x[k] % P, wi)) bad++, printf("inv rows R=%d j=%d k=%d\n", R, j, k);
                }
            }
        }
    }
    if (bad) {
        printf("mismatches: %ld\n", bad);
        return 1;
    }
    printf("ok\n");
    return 0;
}
