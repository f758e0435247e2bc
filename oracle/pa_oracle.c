/*
 * CPU oracle for the G_{c,d} privacy-amplification hash.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or
 * call this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it. It shares no code with the CUDA path.
 *
 * What it computes (arXiv 1910.04429, Sec. 2.3, Definition 5, Eq. 6 and
 * Eq. 7): for an alpha-bit input x and a seed (c, d) with c, d in Z_{2^alpha},
 *
 *     g_{c,d}(x) = floor( ((c*x + d) mod 2^alpha) / 2^(alpha-beta) ),
 *
 * i.e. the beta most significant bits of the alpha-bit field
 * y = (c*x + d) mod 2^alpha. In this library's names alpha = n, beta = m,
 * c = seed_a, d = seed_b, and Sec. 3.2.5 calls beta the final-key length r.
 *
 * The result has a plain definition, so the oracle is that definition
 * written out with schoolbook / Karatsuba limb arithmetic:
 *   1. P = (a*x) mod 2^(64*L), L = ceil(n/64)   (low-half product; Sec. 3.2.2
 *      forms the full product, whose low n bits are the same)
 *   2. y = (P + b) mod 2^n                       (Sec. 3.2.2 "y = cx + d",
 *                                                 Sec. 3.2.3 mod 2^n by masking)
 *   3. out = floor(y / 2^(n-m))                  (Eq. 7; Sec. 3.2.5 keeps the
 *                                                 most significant r bits)
 * Operands are little-endian arrays of 64-bit limbs: integer bit i is bit
 * (i mod 64) of limb floor(i/64) (the least-significant-word-first import of
 * Sec. 3.2.1). Input bits at positions >= n are ignored, since the operands
 * live in Z_{2^n}; output bits at positions >= m are written as zero.
 *
 * Plain C, no SIMD, no intrinsics: the same source builds on x86-64 and
 * aarch64. The only parallelism is an optional split of the top Karatsuba
 * levels over POSIX threads, which does not change any arithmetic.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;

#define KARA_MIN 48      /* below this many limbs the schoolbook product is used */
#define PAR_MIN 4096     /* sub-products at least this long may run on a thread */

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2 };

/* ------------------------------------------------------------------ */
/* limb helpers                                                        */
/* ------------------------------------------------------------------ */

/* r[0..n) += s[0..ns) (ns <= n); returns the carry out of limb n-1. */
static u64 add_into(u64 *r, size_t n, const u64 *s, size_t ns) {
    u64 c = 0;
    size_t i = 0;
    for (; i < ns; i++) {
        u128 t = (u128)r[i] + s[i] + c;
        r[i] = (u64)t;
        c = (u64)(t >> 64);
    }
    for (; i < n && c; i++) {
        u128 t = (u128)r[i] + c;
        r[i] = (u64)t;
        c = (u64)(t >> 64);
    }
    return c;
}

/* r[0..n) -= s[0..ns) (ns <= n); returns the borrow out of limb n-1. */
static u64 sub_from(u64 *r, size_t n, const u64 *s, size_t ns) {
    u64 bw = 0;
    size_t i = 0;
    for (; i < ns; i++) {
        u64 ri = r[i], si = s[i];
        u64 d = ri - si - bw;
        bw = (ri < si) || (ri - si < bw);
        r[i] = d;
    }
    for (; i < n && bw; i++) {
        u64 ri = r[i];
        r[i] = ri - 1;
        bw = (ri == 0);
    }
    return bw;
}

/* ------------------------------------------------------------------ */
/* full products                                                       */
/* ------------------------------------------------------------------ */

/* r[0..na+nb) = a[0..na) * b[0..nb), grade-school method. */
static void mul_school(const u64 *a, size_t na, const u64 *b, size_t nb, u64 *r) {
    memset(r, 0, (na + nb) * sizeof(u64));
    for (size_t i = 0; i < na; i++) {
        u64 c = 0;
        for (size_t j = 0; j < nb; j++) {
            u128 t = (u128)a[i] * b[j] + r[i + j] + c;
            r[i + j] = (u64)t;
            c = (u64)(t >> 64);
        }
        r[i + nb] = c;
    }
}

/* Scratch (in limbs) that kara() needs for an n-limb product. */
static size_t kara_scratch(size_t n) {
    size_t s = 0;
    while (n >= KARA_MIN) {
        size_t hh = n - n / 2;
        s += 4 * (hh + 1);
        n = hh + 1;
    }
    return s + 8;
}

struct kara_job {
    const u64 *a, *b;
    size_t n;
    u64 *r;
    int depth;
    int status;
};

static void kara(const u64 *a, const u64 *b, size_t n, u64 *r, u64 *scratch, int depth);

static void *kara_thread(void *arg) {
    struct kara_job *j = (struct kara_job *)arg;
    u64 *s = (u64 *)malloc(kara_scratch(j->n) * sizeof(u64));
    if (!s) { j->status = OR_ENOMEM; return NULL; }
    kara(j->a, j->b, j->n, j->r, s, j->depth);
    free(s);
    j->status = OR_OK;
    return NULL;
}

/*
 * r[0..2n) = a[0..n) * b[0..n), Karatsuba:
 *   a = a0 + a1 B^h, b = b0 + b1 B^h  (B = 2^64, h = floor(n/2)),
 *   a*b = z0 + (z1 - z0 - z2) B^h + z2 B^(2h),
 *   z0 = a0 b0, z2 = a1 b1, z1 = (a0 + a1)(b0 + b1).
 * depth > 0 lets the three sub-products run on their own threads.
 */
static void kara(const u64 *a, const u64 *b, size_t n, u64 *r, u64 *scratch, int depth) {
    if (n < KARA_MIN) {
        mul_school(a, n, b, n, r);
        return;
    }
    size_t h = n / 2, hh = n - h;           /* low part h limbs, high part hh >= h */
    u64 *sa = scratch;                       /* hh + 1 limbs */
    u64 *sb = sa + (hh + 1);                 /* hh + 1 limbs */
    u64 *z1 = sb + (hh + 1);                 /* 2 (hh + 1) limbs */
    u64 *rest = z1 + 2 * (hh + 1);

    memcpy(sa, a + h, hh * sizeof(u64));
    sa[hh] = 0;
    add_into(sa, hh + 1, a, h);
    memcpy(sb, b + h, hh * sizeof(u64));
    sb[hh] = 0;
    add_into(sb, hh + 1, b, h);

    if (depth > 0 && n >= PAR_MIN) {
        struct kara_job jobs[3] = {
            {a, b, h, r, depth - 1, OR_OK},                 /* z0 -> r[0, 2h)  */
            {a + h, b + h, hh, r + 2 * h, depth - 1, OR_OK}, /* z2 -> r[2h, 2n) */
            {sa, sb, hh + 1, z1, depth - 1, OR_OK},          /* z1             */
        };
        pthread_t th[3];
        int started[3] = {0, 0, 0};
        for (int i = 0; i < 3; i++)
            started[i] = pthread_create(&th[i], NULL, kara_thread, &jobs[i]) == 0;
        for (int i = 0; i < 3; i++) {
            if (started[i]) pthread_join(th[i], NULL);
            else kara(jobs[i].a, jobs[i].b, jobs[i].n, jobs[i].r, rest, 0);
        }
    } else {
        kara(a, b, h, r, rest, 0);
        kara(a + h, b + h, hh, r + 2 * h, rest, 0);
        kara(sa, sb, hh + 1, z1, rest, 0);
    }

    /* z1 <- z1 - z0 - z2, which is >= 0 and < 2^(64 (2hh + 1)) */
    sub_from(z1, 2 * (hh + 1), r, 2 * h);
    sub_from(z1, 2 * (hh + 1), r + 2 * h, 2 * hh);
    /* r += z1 B^h; limbs of z1 that fall beyond r are zero */
    size_t room = 2 * n - h;
    size_t used = 2 * (hh + 1) < room ? 2 * (hh + 1) : room;
    add_into(r + h, room, z1, used);
}

/* r[0..n) = (a[0..n) * b[0..n)) mod B^n, the low half of the product:
 *   a*b mod B^n = a0 b0 + (a0 b1 + a1 b0) B^h  (mod B^n),  h = ceil(n/2),
 * where a0 b0 is a full product and the two cross terms are needed only
 * modulo B^(n-h), so they recurse on this function. */
static void mullo(const u64 *a, const u64 *b, size_t n, u64 *r, int depth);

struct lo_job {
    const u64 *a, *b;
    size_t n;
    u64 *r;
    int depth;
};

static void *mullo_thread(void *arg) {
    struct lo_job *j = (struct lo_job *)arg;
    mullo(j->a, j->b, j->n, j->r, j->depth);
    return NULL;
}

static void mullo(const u64 *a, const u64 *b, size_t n, u64 *r, int depth) {
    if (n == 0) return;
    if (n < 2 * KARA_MIN) {
        memset(r, 0, n * sizeof(u64));
        for (size_t i = 0; i < n; i++) {
            u64 c = 0;
            for (size_t j = 0; i + j < n; j++) {
                u128 t = (u128)a[i] * b[j] + r[i + j] + c;
                r[i + j] = (u64)t;
                c = (u64)(t >> 64);
            }
        }
        return;
    }
    size_t h = n - n / 2, l = n - h; /* h = ceil(n/2), l = floor(n/2) <= h */
    u64 *full = (u64 *)malloc(2 * h * sizeof(u64));
    u64 *t1 = (u64 *)malloc(l * sizeof(u64));
    u64 *t2 = (u64 *)malloc(l * sizeof(u64));
    if (!full || !t1 || !t2) abort(); /* oracle: out of host memory is fatal */

    struct lo_job j1 = {a, b + h, l, t1, depth - 1};   /* a0 b1 mod B^l */
    struct lo_job j2 = {a + h, b, l, t2, depth - 1};   /* a1 b0 mod B^l */
    pthread_t th1, th2;
    int s1 = 0, s2 = 0;
    if (depth > 0 && n >= PAR_MIN) {
        s1 = pthread_create(&th1, NULL, mullo_thread, &j1) == 0;
        s2 = pthread_create(&th2, NULL, mullo_thread, &j2) == 0;
    }
    {
        u64 *scr = (u64 *)malloc(kara_scratch(h) * sizeof(u64));
        if (!scr) abort();
        kara(a, b, h, full, scr, depth > 0 ? depth : 0); /* a0 b0, 2h limbs */
        free(scr);
    }
    if (!s1) mullo(j1.a, j1.b, j1.n, j1.r, 0);
    if (!s2) mullo(j2.a, j2.b, j2.n, j2.r, 0);
    if (s1) pthread_join(th1, NULL);
    if (s2) pthread_join(th2, NULL);

    memcpy(r, full, n * sizeof(u64));
    add_into(r + h, l, t1, l);
    add_into(r + h, l, t2, l);
    free(full);
    free(t1);
    free(t2);
}

/* ------------------------------------------------------------------ */
/* public oracle entry points                                          */
/* ------------------------------------------------------------------ */

static int depth_for_threads(int threads) {
    int d = 0, t = 1;
    while (t * 3 <= threads && d < 6) { t *= 3; d++; }
    return d;
}

/* out[0..2k) = a[0..k) * b[0..k) (full product). Exposed so that the tests can
 * pin the multiplier on its own against independent arithmetic. */
int pa_oracle_mul_full(const u64 *a, const u64 *b, u64 k, u64 *out, int threads) {
    if (k == 0) return OR_OK;
    if (!a || !b || !out) return OR_EINVAL;
    u64 *s = (u64 *)malloc(kara_scratch((size_t)k) * sizeof(u64));
    if (!s) return OR_ENOMEM;
    kara(a, b, (size_t)k, out, s, depth_for_threads(threads));
    free(s);
    return OR_OK;
}

/* out[0..k) = (a[0..k) * b[0..k)) mod 2^(64 k). */
int pa_oracle_mul_low(const u64 *a, const u64 *b, u64 k, u64 *out, int threads) {
    if (k == 0) return OR_OK;
    if (!a || !b || !out) return OR_EINVAL;
    mullo(a, b, (size_t)k, out, depth_for_threads(threads));
    return OR_OK;
}

/*
 * The hash. x, a, b: ceil(n/64) limbs each; out: ceil(m/64) limbs.
 * Returns 0, or OR_EINVAL for n == 0, m == 0, m > n or a null pointer.
 * threads: host threads the product may use (1 = single-threaded).
 */
int pa_oracle_hash(const u64 *x, const u64 *a, const u64 *b, u64 n, u64 m, u64 *out,
                   int threads) {
    if (n == 0 || m == 0 || m > n || !x || !a || !b || !out) return OR_EINVAL;
    size_t L = (size_t)((n + 63) / 64), M = (size_t)((m + 63) / 64);
    u64 top = (n % 64) ? ((1ull << (n % 64)) - 1) : ~0ull; /* live bits of limb L-1 */

    u64 *xm = (u64 *)malloc(L * sizeof(u64));
    u64 *am = (u64 *)malloc(L * sizeof(u64));
    u64 *y = (u64 *)malloc(L * sizeof(u64));
    if (!xm || !am || !y) { free(xm); free(am); free(y); return OR_ENOMEM; }

    /* operands are elements of Z_{2^n}: drop bits >= n */
    memcpy(xm, x, L * sizeof(u64));
    memcpy(am, a, L * sizeof(u64));
    xm[L - 1] &= top;
    am[L - 1] &= top;

    /* step 1: low L limbs of a*x */
    mullo(am, xm, L, y, depth_for_threads(threads));

    /* step 2: + b, keeping L limbs (the carry out of limb L-1 is >= 2^n) */
    {
        u64 c = 0;
        for (size_t i = 0; i < L; i++) {
            u64 bi = b[i];
            if (i == L - 1) bi &= top;
            u128 t = (u128)y[i] + bi + c;
            y[i] = (u64)t;
            c = (u64)(t >> 64);
        }
    }
    /* mod 2^n: clear bits >= n */
    y[L - 1] &= top;

    /* step 3: out = floor(y / 2^(n - m)), i.e. bits [n-m, n) of y */
    {
        u64 s = n - m;
        size_t q = (size_t)(s / 64);
        unsigned r = (unsigned)(s % 64);
        for (size_t j = 0; j < M; j++) {
            u64 lo = (q + j < L) ? y[q + j] : 0;
            u64 hi = (q + j + 1 < L) ? y[q + j + 1] : 0;
            out[j] = r ? ((lo >> r) | (hi << (64 - r))) : lo;
        }
        if (m % 64) out[M - 1] &= (1ull << (m % 64)) - 1;
    }
    free(xm);
    free(am);
    free(y);
    return OR_OK;
}
