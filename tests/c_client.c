/*
 * A plain C client of libpa_gb300.so: only include/pa.h and the library, no
 * CUDA or Python headers. It draws one block with SplitMix64 (x, then a with
 * bit 0 set, then b; bits >= n cleared, as the Python input generator does),
 * hashes it through the host-buffer entry point and prints the ceil(m/64)
 * output limbs as hexadecimal, one per line. Used by the GPU test suite.
 *
 *   c_client <n> <m> <seed>
 */
#include <inttypes.h>
#include <stdio.h>
#include <stdlib.h>

#include "pa.h"

static uint64_t splitmix64(uint64_t seed, uint64_t i) {  /* output i of the stream seeded with seed */
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int main(int argc, char** argv) {
    if (argc != 4) {
        fprintf(stderr, "usage: c_client <n> <m> <seed>\n");
        return 2;
    }
    uint64_t n = strtoull(argv[1], NULL, 10), m = strtoull(argv[2], NULL, 10);
    uint64_t seed = strtoull(argv[3], NULL, 10);
    uint64_t L = (n + 63) / 64, Mo = (m + 63) / 64;
    uint64_t* x = malloc(L * sizeof *x);
    uint64_t* a = malloc(L * sizeof *a);
    uint64_t* b = malloc(L * sizeof *b);
    uint64_t* out = calloc(Mo ? Mo : 1, sizeof *out);
    if (!x || !a || !b || !out) return 3;
    for (uint64_t i = 0; i < L; i++) {
        x[i] = splitmix64(seed, i);
        a[i] = splitmix64(seed, L + i);
        b[i] = splitmix64(seed, 2 * L + i);
    }
    if (n % 64) {
        uint64_t mask = (1ull << (n % 64)) - 1;
        x[L - 1] &= mask, a[L - 1] &= mask, b[L - 1] &= mask;
    }
    a[0] |= 1;
    int rc = pa_hash_host(x, a, b, n, m, out, NULL);
    if (rc != PA_OK) {
        fprintf(stderr, "pa_hash_host: %d %s\n", rc, pa_last_error());
        return 1;
    }
    /* no bounded wait of the library's kernels ran out on this stream */
    rc = pa_stream_status(NULL, 1);
    if (rc != PA_OK) {
        fprintf(stderr, "pa_stream_status: %d %s\n", rc, pa_last_error());
        return 1;
    }
    for (uint64_t i = 0; i < Mo; i++) printf("%016" PRIx64 "\n", out[i]);
    free(x), free(a), free(b), free(out);
    return pa_shutdown() == PA_OK ? 0 : 1;
}
