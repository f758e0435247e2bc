// Host check of the field helpers shared with the kernels (csrc/gl.cuh, host
// variants): every route of x * 2^s mod p (s in [0, 192), including the chains
// of multiplier-based routes), sub, add and mul, against 128-bit arithmetic
// reduced with the % operator. Inputs: 0, 1, p - 1, p (the transforms' stand-in
// for 0) and pseudo-random values in [0, p]. Prints "ok" and exits 0 on success.
#include <cstdint>
#include <cstdio>

#include "gl.cuh"

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
    if (bad) {
        printf("mismatches: %ld\n", bad);
        return 1;
    }
    printf("ok\n");
    return 0;
}
