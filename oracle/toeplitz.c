/*
 * CPU oracle for Toeplitz-hash privacy amplification.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or
 * call this file; only the test suite and the benchmark's CPU-baseline leg use
 * it. It shares no code with the CUDA path.
 *
 * arXiv 1910.04429 (Sec. 1) surveys Toeplitz-hash PA as the established
 * alternative to its modular-arithmetic hash, computed there by FFT or NTT.
 * The paper does not restate the family; this file takes the usual one
 * (Krawczyk's random Toeplitz matrices over GF(2)): an n+m-1 bit seed s
 * defines the m x n matrix T[i][j] = s[i - j + n - 1], constant along its
 * diagonals, and the hash of an n-bit key x is the m-bit vector
 *
 *     y[i] = XOR over j < n of ( s[i + n - 1 - j] AND x[j] ),   i < m.
 *
 * Bit i of a bit vector is bit (i mod 64) of 64-bit limb floor(i / 64), as for
 * the modular hash; key bits >= n and seed bits >= n + m - 1 are ignored and
 * output bits >= m are written as zero.
 *
 * pa_oracle_toeplitz is that definition column by column: for every set key
 * bit j, the m seed bits s[n - 1 - j .. n - 2 - j + m] (column j of T) are
 * XORed into y, 64 at a time. Threads split the output limbs. Cost about
 * (n / 2) * (m / 64) word operations.
 *
 * pa_oracle_toeplitz_bit is the definition of one output bit, row by row
 * (row i of T against x): cost n bit operations, for sampled checks of keys
 * too large for the full product.
 *
 * Plain C, no SIMD or intrinsics: builds and agrees on x86-64 and aarch64.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;

static int bit_of(const u64 *v, u64 i) { return (int)((v[i >> 6] >> (i & 63)) & 1u); }

/* 64 bits of s starting at bit position o; bits at positions >= len read 0 */
static u64 window64(const u64 *s, u64 len, u64 o) {
    if (o >= len) return 0;
    u64 w = o >> 6, sh = o & 63, nw = (len + 63) >> 6;
    u64 lo = s[w] >> sh;
    if (sh && w + 1 < nw) lo |= s[w + 1] << (64 - sh);
    u64 live = len - o; /* bits of the window inside the seed */
    if (live < 64) lo &= (1ull << live) - 1;
    return lo;
}

struct toe_job {
    const u64 *x, *s;
    u64 n, m, slen;
    u64 *out;
    u64 w0, w1; /* output limbs [w0, w1) */
};

static void *toe_columns(void *arg) {
    struct toe_job *j = (struct toe_job *)arg;
    u64 *y = j->out;
    for (u64 w = j->w0; w < j->w1; w++) y[w] = 0;
    for (u64 col = 0; col < j->n; col++) {
        if (!bit_of(j->x, col)) continue;
        u64 o = j->n - 1 - col; /* T[i][col] = s[o + i] */
        for (u64 w = j->w0; w < j->w1; w++) y[w] ^= window64(j->s, j->slen, o + 64 * w);
    }
    u64 last = (j->m - 1) >> 6;
    if (j->w0 <= last && last < j->w1 && (j->m & 63)) y[last] &= (1ull << (j->m & 63)) - 1;
    return NULL;
}

/* y = T x for the Toeplitz matrix of seed s (n + m - 1 bits). Returns 0, or -1
 * for invalid sizes (need 1 <= m <= n). */
int pa_oracle_toeplitz(const u64 *x, const u64 *s, u64 n, u64 m, u64 *out, int threads) {
    if (n < 1 || m < 1 || m > n) return -1;
    u64 nw = (m + 63) >> 6;
    if (threads < 1) threads = 1;
    if ((u64)threads > nw) threads = (int)nw;
    struct toe_job *jobs = (struct toe_job *)calloc((size_t)threads, sizeof *jobs);
    pthread_t *th = (pthread_t *)calloc((size_t)threads, sizeof *th);
    int *started = (int *)calloc((size_t)threads, sizeof *started);
    if (!jobs || !th || !started) {
        free(jobs), free(th), free(started);
        return -1;
    }
    for (int t = 0; t < threads; t++) {
        jobs[t] = (struct toe_job){x, s, n, m, n + m - 1, out, nw * (u64)t / (u64)threads,
                                   nw * (u64)(t + 1) / (u64)threads};
        started[t] = t > 0 && pthread_create(&th[t], NULL, toe_columns, &jobs[t]) == 0;
    }
    toe_columns(&jobs[0]);
    for (int t = 1; t < threads; t++) {
        if (started[t]) pthread_join(th[t], NULL);
        else toe_columns(&jobs[t]);
    }
    free(jobs), free(th), free(started);
    return 0;
}

/* Output bit i of the same hash: row i of T against x. Returns 0 or 1, or -1
 * for invalid arguments. */
int pa_oracle_toeplitz_bit(const u64 *x, const u64 *s, u64 n, u64 m, u64 i) {
    if (n < 1 || m < 1 || m > n || i >= m) return -1;
    int acc = 0;
    for (u64 j = 0; j < n; j++) acc ^= bit_of(s, i + n - 1 - j) & bit_of(x, j);
    return acc;
}
