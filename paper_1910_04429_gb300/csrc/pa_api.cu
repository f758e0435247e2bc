// C ABI of the library (declared in include/pa.h): argument checks, plan and
// twiddle-table cache, stream-ordered workspace, and the launch sequence of
// the G_{c,d} hash (Sec. 2.3 Eq. 7; pipeline of Sec. 3.2).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/pa.h"
#include "pa_internal.h"

using namespace pa;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PA_ENOMEM : PA_ECUDA;
}

constexpr int SIDE_STREAMS = 4;  // concurrent size classes inside one batched call

struct Device {
    bool tune_loaded = false;
    std::unordered_map<u64, int> tuned;   // N -> plan variant chosen by pa_autotune
    std::unordered_map<u64, int> forced;  // N -> plan variant forced by pa_plan_override
    cudaMemPool_t pool = nullptr;
    std::unordered_map<u64, u64*> tables;  // transform length N -> device twiddle tables
    std::map<std::pair<u64, u64>, u64*> pass_tables;  // (M, S) -> a strided pass's twiddles
    cudaStream_t table_stream = nullptr;   // private stream of the table builds
    cudaStream_t side[SIDE_STREAMS] = {};  // forked from the caller's stream per batch
    cudaEvent_t fork = nullptr, join[SIDE_STREAMS] = {};
    // host-buffer calls: input copies run on `copy`, at most two calls ahead
    // of the hashes (done[i % 2] marks the end of call i's hash and frees)
    cudaStream_t copy = nullptr;
    cudaEvent_t xa_ready = nullptr, b_ready = nullptr, done[2] = {};
    u64 host_calls = 0;
    // per-stream status words (pa_stream_status): a device slab of STATUS_SLOTS
    // words, its pinned host mirror, and the slot of each stream seen (by stream id)
    u32* status_dev = nullptr;
    u32* status_host = nullptr;
    bool status_failed = false;
    std::unordered_map<const void*, int> status_slot;  // by stream handle
};

// Streams that get a status word of their own; later streams share the last
// slot (their bounded-wait timeouts are then reported for all of them).
constexpr int STATUS_SLOTS = 4096;

std::mutex g_mu;
std::unordered_map<int, Device> g_dev;

int current_device(int* dev) {
    cudaError_t e = cudaGetDevice(dev);
    return e == cudaSuccess ? PA_OK : cuda_fail(e, "cudaGetDevice");
}

// Pool with no release threshold: freed workspace stays reserved for reuse.
int get_pool(int dev, cudaMemPool_t* out) {
    Device& d = g_dev[dev];
    if (!d.pool) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaError_t e = cudaMemPoolCreate(&d.pool, &props);
        if (e != cudaSuccess) { d.pool = nullptr; return cuda_fail(e, "cudaMemPoolCreate"); }
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &thr);
        // reuse across streams only along event dependencies (or when the free has
        // completed): an allocation on the copy stream never gains a hidden wait
        // on a hash stream
        int no = 0;
        cudaMemPoolSetAttribute(d.pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
    *out = d.pool;
    return PA_OK;
}

// The tables every plan of length G.N shares (no per-pass tables).
int get_base_tables(int dev, const Geom& G, Twiddles* tw) {
    Device& d = g_dev[dev];
    auto it = d.tables.find(G.N);
    u64* p = nullptr;
    size_t base_words = table_words_n(G.N);
    if (it == d.tables.end()) {
        std::vector<u64> host;
        make_tables(G.logN, host, G.odd);
        // then w_4096^t * N^-1: the seed's tile pass scales by N^-1 through its twiddles
        u64 ninv = n_inverse(G.logN, G.odd);
        host.resize(base_words + 4096);
        for (size_t i = 0; i < 4096; i++) host[base_words + i] = gl::mul(host[i], ninv);
        cudaError_t e = cudaMalloc(&p, host.size() * sizeof(u64));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(twiddles)");
        e = cudaMemcpy(p, host.data(), host.size() * sizeof(u64), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(p); return cuda_fail(e, "cudaMemcpy(twiddles)"); }
        d.tables[G.N] = p;
    } else {
        p = it->second;
    }
    u64 nh = G.N >> 12;
    *tw = Twiddles{};
    tw->w4096 = p;
    tw->w4096i = p + 4096;
    tw->wlo = p + 8192;
    tw->wloi = p + 12288;
    tw->whi = p + 16384;
    tw->whii = p + 16384 + nh;
    tw->w4096s = p + base_words;
    return PA_OK;
}

int get_tables(int dev, const Geom& G, Twiddles* tw) {
    int rc = get_base_tables(dev, G, tw);
    if (rc) return rc;
    Device& d = g_dev[dev];
    // per strided pass: full tables of its inter-pass twiddles (2 M words),
    // built once on the device and waited for
    for (int i = 0; i < G.nstrided && i < MAX_PASSES; i++) {
        std::pair<u64, u64> key{G.pass[i].M, G.pass[i].S};
        auto pt = d.pass_tables.find(key);
        u64* q = nullptr;
        if (pt == d.pass_tables.end()) {
            cudaError_t e = cudaSuccess;
            if (!d.table_stream) e = cudaStreamCreateWithFlags(&d.table_stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaMalloc(&q, 2 * key.first * sizeof(u64));
            if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(pass twiddles)");
            e = launch_pass_twiddles(*tw, G.N, key.first, key.second, q, d.table_stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(d.table_stream);
            if (e != cudaSuccess) { cudaFree(q); return cuda_fail(e, "pass twiddles"); }
            d.pass_tables[key] = q;
        } else {
            q = pt->second;
        }
        tw->passf[i] = q;
        tw->passi[i] = q + key.first;
    }
    return PA_OK;
}

struct Scratch {
    cudaStream_t st;
    cudaMemPool_t pool;
    std::vector<void*> ptrs;
    Scratch(cudaStream_t s, cudaMemPool_t p) : st(s), pool(p) {}
    int get(size_t bytes, void** out) {
        cudaError_t e = cudaMallocFromPoolAsync(out, bytes ? bytes : 16, pool, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocFromPoolAsync");
        ptrs.push_back(*out);
        return PA_OK;
    }
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
};

bool check_sizes(uint64_t n, uint64_t m) { return n >= 1 && m >= 1 && m <= n && n <= PA_MAX_BITS; }

Geom geom_for_bits(uint64_t n) { return choose_geom((n + 15) / 16); }

// Plan variants that change anything for this transform length.
int applicable_variants(const Geom& g) {
    const int cluster = g.N / TILE <= CLUSTER_MAX_TILES ? PLAN_CLUSTER : 0;
    if (g.nstrided == 0) return cluster;
    int R0 = g.odd << ((g.logN - LOG_TILE) % 6);
    return (R0 > 1 && g.nstrided > 1 ? PLAN_R0_LAST : 0) | PLAN_DIRECT_FWD | PLAN_DIRECT_INV |
           (g.nstrided == 1 && g.N / TILE <= 64 ? PLAN_NARROW : 0) | PLAN_BULK | cluster;
}

// The plan for a transform length on device dev: base's length, with the
// variant forced for it, else the tuned one, else 0.
Geom plan_for_base(int dev, const Geom& base) {
    Device& d = g_dev[dev];
    int v = 0;
    auto f = d.forced.find(base.N);
    if (f != d.forced.end()) v = f->second;
    else {
        auto t = d.tuned.find(base.N);
        if (t != d.tuned.end()) v = t->second;
    }
    return make_geom(base.logN, base.odd, v & applicable_variants(base));
}

// ... for keys of n bits (the modular hash)
Geom plan_for(int dev, uint64_t n) { return plan_for_base(dev, geom_for_bits(n)); }

// ... for Toeplitz hashes of n key bits and m output bits
bool check_toeplitz(uint64_t n, uint64_t m) {
    return n >= 1 && m >= 1 && m <= n && n + m - 1 <= PA_TOEPLITZ_MAX_BITS;
}
Geom toeplitz_base(uint64_t n, uint64_t m) { return choose_geom_len(n + m - 1); }

// The key's (and seed's) bits as one-bit digits of the convolution.
Digits bit_digits(const uint64_t* v, uint64_t bits) {
    return Digits{reinterpret_cast<const uint16_t*>(v), bits, 0xFFFF, 1};
}

// Tuning cache file (PA_TUNE_CACHE): lines "<gpu name>\t<N>\t<variant>".
std::string device_name(int dev) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string s = prop.name;
    for (char& c : s)
        if (c == '\t' || c == '\n') c = ' ';
    return s;
}

void load_tune_cache(int dev) {
    Device& d = g_dev[dev];
    if (d.tune_loaded) return;
    d.tune_loaded = true;
    const char* path = getenv("PA_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    std::string name = device_name(dev);
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char* t1 = strchr(line, '\t');
        if (!t1) continue;
        *t1 = 0;
        unsigned long long N = 0;
        int v = 0;
        if (name == line && sscanf(t1 + 1, "%llu\t%d", &N, &v) == 2 && v >= 0 && v < PLAN_VARIANTS)
            d.tuned[(u64)N] = v;
    }
    fclose(f);
}

void save_tune_cache(int dev) {
    const char* path = getenv("PA_TUNE_CACHE");
    if (!path || !*path) return;
    std::string name = device_name(dev);
    std::vector<std::string> keep;
    if (FILE* f = fopen(path, "r")) {
        char line[512];
        while (fgets(line, sizeof line, f)) {
            const char* t1 = strchr(line, '\t');
            if (t1 && std::string((const char*)line, t1) != name) keep.push_back(line);
        }
        fclose(f);
    }
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return;
    for (auto& l : keep) fputs(l.c_str(), f);
    for (auto& kv : g_dev[dev].tuned)
        fprintf(f, "%s\t%llu\t%d\n", name.c_str(), (unsigned long long)kv.first, kv.second);
    fclose(f);
    rename(tmp.c_str(), path);
}

// Queue steps 1-5 of Algorithm 1; on success *coef points at the digits (k < L).
int queue_convolution(const uint64_t* key, const uint64_t* seed_a, uint64_t n, cudaStream_t st,
                      Scratch& scr, int dev, u64** coef) {
    u64 L = (n + 15) / 16;
    NttJob j;
    j.geom = plan_for(dev, n);
    j.L = L;
    int rc = get_tables(dev, j.geom, &j.tw);
    if (rc) return rc;
    void *bx, *ba;
    if ((rc = scr.get(j.geom.N * sizeof(u64), &bx))) return rc;
    if ((rc = scr.get(j.geom.N * sizeof(u64), &ba))) return rc;
    j.buf_x = (u64*)bx;
    j.buf_a = (u64*)ba;
    j.dx = make_digits(key, n, 16);
    j.da = make_digits(seed_a, n, 16);
    cudaError_t e = launch_convolution(j, st);
    if (e != cudaSuccess) return cuda_fail(e, "NTT launch");
    *coef = j.buf_x;
    return PA_OK;
}

// The carry step's scratch states, cleared on st now: queued before the
// transforms, so that no memset sits between the last transform kernel and the
// carry kernel (which then follows it by programmatic dependent launch).
int carry_states(uint64_t n, cudaStream_t st, Scratch& scr, u32** state) {
    void* p;
    int rc = scr.get(carry_state_words(n) * sizeof(u32), &p);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(p, 0, carry_state_words(n) * sizeof(u32), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(carry states)");
    *state = (u32*)p;
    return PA_OK;
}

int queue_carry(const u64* coef, u64 L, const uint64_t* seed_b, uint64_t n, uint64_t m,
                uint64_t* out, cudaStream_t st, Scratch& scr, u32* zeroed_state = nullptr) {
    u32* state = zeroed_state;
    int rc;
    if (!state) {
        void* p;
        if ((rc = scr.get(carry_state_words(n) * sizeof(u32), &p))) return rc;
        state = (u32*)p;
    }
    CarryJob c{coef, L, seed_b, n, m, out, state, zeroed_state != nullptr};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t e = launch_carry(c, st, status_word(dev, st));
    if (e != cudaSuccess) return cuda_fail(e, "carry launch");
    return PA_OK;
}

// Wrapped products: 0 never; 1 (default) where one is shorter and the full
// product has at least WRAP_MIN_FULL points; 2 wherever one is shorter; 3 as 2
// with the flag forced (every hash then also runs the exact recomputation: a
// test of that path).
int g_wrap_mode = 1;

// Digit width: 0 (default) the width whose product is shortest among the exact
// ones, 16 .. 20 that width where it is exact (tests; pa_digit_width).
int g_digit_width = 0;

// The product a single hash of n bits (m output bits) runs under the current
// modes. Digits wider than 16 bits are read by staged 16-byte copies, so they
// need 16-byte-aligned key and seed limbs; other operands take 16-bit digits.
DigitPlan plan_digits(uint64_t n, uint64_t m, bool aligned = true) {
    return digit_plan(n, m, g_wrap_mode != 0, g_wrap_mode == 1 ? WRAP_MIN_FULL : 0, aligned ? g_digit_width : 16);
}

bool aligned16(const void* a, const void* b) { return (uintptr_t)a % 16 == 0 && (uintptr_t)b % 16 == 0; }

// One hash's plans and scratch. Without wrapping: the full-length product.
// With it: the wrapped product, then its carry step (which sets the flag when
// the certificate fails), then the exact recomputation (one launch that does
// nothing unless the flag is set); the buffers are sized for the
// recomputation's power-of-two length, which the wrapped product's prefix of
// them precedes.
struct HashPlan {
    DigitPlan dp;     // digit width, digit count, wrapped plan
    WrapPlan wp;      // dp.wp
    NttJob prod;      // the product that runs first
    FallbackJob fb;   // with wp.on: the recomputation
    u32* state;       // carry states: one set, or two (wrapped, recomputation)
};

NttJob product_job(const Geom& G, u64* bx, u64* ba, const uint64_t* key, const uint64_t* seed_a, uint64_t n,
                   int w) {
    NttJob j;
    j.geom = G;
    j.dx = make_digits(key, n, w);
    j.da = make_digits(seed_a, n, w);
    j.L = j.dx.L;
    j.buf_x = bx;
    j.buf_a = ba;
    return j;
}

// The recomputation's power-of-two length (>= 2L - 1, at least one tile).
Geom fallback_geom(uint64_t n) { return make_geom(logn_for_digits((n + 15) / 16)); }

// Words of each transform buffer a hash of n bits may need, whatever m is.
u64 buffer_words(uint64_t n) {
    u64 full = geom_for_bits(n).N, fb = fallback_geom(n).N;
    return full > fb ? full : fb;
}

// The recomputation of one wrapped hash: the key's and the seed's limbs (read
// as 16-bit digits, whatever width the wrapped product used); buffers X, A of
// the power-of-two length's words; its own (zeroed) carry states; the wrapped
// product's flag. b and out are filled in when the carry step is queued.
int fallback_job(int dev, uint64_t n, uint64_t m, const uint64_t* key, const uint64_t* seed_a, u64* X, u64* A,
                 u32* state, const u32* flag, FallbackJob* f) {
    const Geom fg = fallback_geom(n);
    Twiddles t;
    int rc = get_base_tables(dev, fg, &t);
    if (rc) return rc;
    *f = FallbackJob{};
    f->dx = make_digits(key, n, 16);
    f->da = make_digits(seed_a, n, 16);
    f->n = n;
    f->m = m;
    f->flag = flag;
    f->X = X;
    f->A = A;
    f->logN = fg.logN;
    f->wlo = t.wlo;
    f->wloi = t.wloi;
    f->whi = t.whi;
    f->whii = t.whii;
    f->ninv = n_inverse(fg.logN, fg.odd);
    f->state = state;
    return PA_OK;
}

// Plans, twiddle tables, buffers and the carry states (cleared by the first
// transform kernel). fixed_ws: a caller-provided workspace of
// pa_workspace_bytes(n) (captured graphs), else one allocation from the pool.
int hash_prepare(const uint64_t* key, const uint64_t* seed_a, uint64_t n, uint64_t m, Scratch& scr, int dev,
                 HashPlan* hp, void* fixed_ws = nullptr) {
    hp->dp = plan_digits(n, m, aligned16(key, seed_a));
    hp->wp = hp->dp.wp;
    const Geom first = plan_for_base(dev, hp->wp.on ? hp->wp.geom : hp->dp.full);
    const Geom fg = fallback_geom(n);
    const u64 words = hp->wp.on ? (fg.N > first.N ? fg.N : first.N) : first.N;
    int rc;
    // one pool allocation per hash: both transform buffers, then the carry states
    const size_t state_words = (hp->wp.on ? 2 : 1) * carry_state_words(n);
    void* ws = fixed_ws;
    if (!ws && (rc = scr.get(2 * words * sizeof(u64) + state_words * sizeof(u32), &ws))) return rc;
    u64* bx = (u64*)ws;
    u64* ba = bx + words;
    hp->prod = product_job(first, bx, ba, key, seed_a, n, hp->dp.w);
    if ((rc = get_tables(dev, first, &hp->prod.tw))) return rc;
    hp->state = (u32*)(ba + words);
    if (hp->wp.on && (rc = fallback_job(dev, n, m, key, seed_a, bx, ba,
                                        hp->state + carry_state_words(n), hp->state + carry_flag_word(n),
                                        &hp->fb)))
        return rc;
    // no memset between this hash and the previous one on the stream: the
    // first transform kernel clears the states
    hp->prod.zero = hp->state;
    hp->prod.zero_words = (u32)state_words;
    return PA_OK;
}

// Steps 1-5 of Algorithm 1: the wrapped product, else the full-length one.
int hash_product(HashPlan& hp, cudaStream_t st) {
    cudaError_t e = launch_convolution(hp.prod, st);
    return e == cudaSuccess ? PA_OK : cuda_fail(e, "NTT launch");
}

// Steps 6-7: the carry step; after a wrapped product, the recomputation.
int hash_finish(HashPlan& hp, const uint64_t* seed_b, uint64_t n, uint64_t m, uint64_t* out, cudaStream_t st,
                int dev) {
    u32* flag = hp.wp.on ? hp.state + carry_flag_word(n) : nullptr;
    u32* sw = status_word(dev, st);
    CarryJob c{hp.prod.buf_x, hp.dp.L, seed_b, n, m, out, hp.state, true, hp.wp.lo, flag, g_wrap_mode == 3,
               (u32)hp.dp.w};
    cudaError_t e = launch_carry(c, st, sw);
    if (e != cudaSuccess) return cuda_fail(e, "carry launch");
    if (hp.wp.on) {
        hp.fb.b = seed_b;
        hp.fb.out = out;
        if ((e = launch_fallback(&hp.fb, 1, st, sw)) != cudaSuccess) return cuda_fail(e, "recomputation launch");
    }
    return PA_OK;
}

int hash_device(const uint64_t* key, const uint64_t* seed_a, const uint64_t* seed_b, uint64_t n,
                uint64_t m, uint64_t* out, cudaStream_t st, int dev, cudaMemPool_t pool, void* fixed_ws = nullptr) {
    Scratch scr(st, pool);
    HashPlan hp;
    int rc = hash_prepare(key, seed_a, n, m, scr, dev, &hp, fixed_ws);
    if (!rc) rc = hash_product(hp, st);
    if (!rc) rc = hash_finish(hp, seed_b, n, m, out, st, dev);
    return rc;
}

int side_streams(int dev) {
    Device& d = g_dev[dev];
    if (d.fork) return PA_OK;
    cudaError_t e = cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming);
    for (int i = 0; e == cudaSuccess && i < SIDE_STREAMS; i++) {
        e = cudaStreamCreateWithFlags(&d.side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&d.copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.xa_ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.b_ready, cudaEventDisableTiming);
    for (int i = 0; e == cudaSuccess && i < 2; i++) e = cudaEventCreateWithFlags(&d.done[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        d.fork = nullptr;
        return cuda_fail(e, "side stream set-up");
    }
    return PA_OK;
}

// Blocks grouped by the geometry of the product they run first: each group
// runs its passes as batched launches (blocks along gridDim.y), groups on side
// streams forked from and joined back into `st`, then one batched carry launch
// for every block and, when some block's product was wrapped, the exact
// recomputation's launches (which return at once unless a flag is set). A
// batch fills the GPU, so its blocks wrap wherever a shorter length exists
// (mode 1 as well as 2); mode 0 never wraps, mode 3 forces the recomputation.
// Batched calls (pa_batch_mode): 1 the blocks whose plan has one or two
// strided passes run their transforms in the persistent kernel (one
// cooperative launch), the rest by size class; 0 every block by size class;
// 2 (default) the persistent kernel when those blocks' tiles number at most
// PERSIST_AUTO_TILES_PER_SM per SM, else by size class. (Measured on the
// GB300: 16 blocks of 1e6..2e6 bits, about 770 tiles, 0.126 ms persistent
// against 0.169 ms by size class; 64 such blocks 0.413 against 0.372 ms; the
// 256-block workload of 1e6..1e7 bits 5.13 against 4.17 ms. Per-pass kernels
// keep their own occupancy and overlap across size classes, which a single
// kernel serving every pass cannot; it wins where launches dominate.)
int g_batch_mode = 2;
constexpr u64 PERSIST_AUTO_TILES_PER_SM = 8;

DigitPlan batch_digits(uint64_t n, uint64_t m, bool aligned) {
    return digit_plan(n, m, g_wrap_mode != 0, 0, aligned ? g_digit_width : 16);
}

u64 batch_workspace_bytes(const pa_block* blocks, uint32_t count) {
    u64 bytes = 0;
    for (uint32_t i = 0; i < count; i++)
        bytes += 2 * buffer_words(blocks[i].n) * sizeof(u64) + 2 * carry_state_words(blocks[i].n) * sizeof(u32);
    return bytes + count * PERSIST_SCRATCH_WORDS * sizeof(u32);  // the persistent launches' counters
}

// fixed_ws: a caller-provided workspace of batch_workspace_bytes() (used for
// captured graphs); otherwise it comes from the pool, stream-ordered.
int hash_batch_device(const pa_block* blocks, uint32_t count, cudaStream_t st, int dev,
                      cudaMemPool_t pool, void* fixed_ws = nullptr) {
    int rc = side_streams(dev);
    if (rc) return rc;
    Device& d = g_dev[dev];
    std::vector<DigitPlan> dps(count);
    std::vector<std::pair<u64, std::vector<uint32_t>>> groups;  // (first length, wide) -> block indices
    for (uint32_t i = 0; i < count; i++) {
        dps[i] = batch_digits(blocks[i].n, blocks[i].m, aligned16(blocks[i].key, blocks[i].seed_a));
        // a group shares one transform length and one kind of first pass (16-bit or wider digits)
        u64 N = dps[i].first_n() * 2 + (dps[i].w > 16 ? 1 : 0);
        size_t g = 0;
        while (g < groups.size() && groups[g].first != N) g++;
        if (g == groups.size()) groups.push_back({N, {}});
        groups[g].second.push_back(i);
    }
    // workspace: every block's two transform buffers, then the carry states, in one allocation
    u64 words = 0, carry_bytes = 0;
    for (uint32_t i = 0; i < count; i++) {
        words += 2 * buffer_words(blocks[i].n);
        carry_bytes += 2 * carry_state_words(blocks[i].n) * sizeof(u32);
    }
    u32* barriers = nullptr;  // the persistent launches' counters, after the carry states, cleared with them
    const u64 barrier_off = carry_bytes;
    carry_bytes += count * PERSIST_SCRATCH_WORDS * sizeof(u32);
    Scratch scr(st, pool);
    void* ws = fixed_ws;
    if (!ws && (rc = scr.get(words * sizeof(u64) + carry_bytes, &ws))) return rc;
    std::vector<u64*> wbuf(count);
    std::vector<u32*> sbuf(count);
    {
        u64* w = (u64*)ws;
        u32* cb = (u32*)((u64*)ws + words);
        for (uint32_t i = 0; i < count; i++) {
            wbuf[i] = w;
            w += 2 * buffer_words(blocks[i].n);
            sbuf[i] = cb;
            cb += 2 * carry_state_words(blocks[i].n);
        }
        barriers = (u32*)((char*)((u64*)ws + words) + barrier_off);
    }
    std::vector<PersistJob> pj;
    bool use_persist = g_batch_mode == 1;
    if (g_batch_mode == 2) {  // the tiles the persistent kernel would take
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        u64 tiles = 0;
        for (uint32_t i = 0; i < count; i++) {
            const Geom& base = dps[i].wp.on ? dps[i].wp.geom : dps[i].full;
            if (persist_eligible(make_geom(base.logN, base.odd, 0)) && aligned16(blocks[i].key, blocks[i].seed_a))
                tiles += base.N / TILE;
        }
        use_persist = tiles <= PERSIST_AUTO_TILES_PER_SM * (u64)sms;
    }
    std::vector<CarryJob> cj(count);
    std::vector<FallbackJob> fj;

    // every block's carry states cleared at once, before the transforms
    cudaError_t e = cudaMemsetAsync((u64*)ws + words, 0, carry_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(carry states)");
    e = cudaEventRecord(d.fork, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord(fork)");
    int used = 0;
    int sgroups = 0;  // groups run by size class, on the side streams
    for (size_t g = 0; g < groups.size(); g++) {
        const auto& idx = groups[g].second;
        const DigitPlan& d0 = dps[idx[0]];
        const Geom& base = d0.wp.on ? d0.wp.geom : d0.full;
        Geom G = plan_for_base(dev, base);
        Twiddles tw;
        if ((rc = get_tables(dev, G, &tw))) return rc;
        // the persistent kernel runs the plan with the odd radix first, staged
        const Geom P = make_geom(base.logN, base.odd, 0);
        const bool persist = use_persist && persist_eligible(P);
        Twiddles ptw;
        if (persist && (rc = get_tables(dev, P, &ptw))) return rc;
        std::vector<BlockIO> io;
        for (size_t k = 0; k < idx.size(); k++) {
            const uint32_t i = idx[k];
            const pa_block& b = blocks[i];
            const DigitPlan& dp = dps[i];
            const u64 L = dp.L, bw = buffer_words(b.n);
            Digits dx = make_digits(b.key, b.n, dp.w), da = make_digits(b.seed_a, b.n, dp.w);
            if (persist && aligned16(b.key, b.seed_a))
                pj.push_back(PersistJob{wbuf[i], wbuf[i] + bw, b.key, b.seed_a, b.n, dp.w, P, ptw});
            else
                io.push_back(BlockIO{wbuf[i], wbuf[i] + bw, dx, da, L});
            const WrapPlan& wp = dp.wp;
            u32* flag = wp.on ? sbuf[i] + carry_flag_word(b.n) : nullptr;
            cj[i] = CarryJob{wbuf[i], L, b.seed_b, b.n, b.m, b.out, sbuf[i], true, wp.lo, flag, g_wrap_mode == 3,
                             (u32)dp.w};
            if (wp.on) {
                FallbackJob f;
                if ((rc = fallback_job(dev, b.n, b.m, b.key, b.seed_a, wbuf[i], wbuf[i] + bw,
                                       sbuf[i] + carry_state_words(b.n), flag, &f)))
                    return rc;
                f.b = b.seed_b;
                f.out = b.out;
                fj.push_back(f);
            }
        }
        if (io.empty()) continue;
        cudaStream_t s = d.side[sgroups % SIDE_STREAMS];
        if (sgroups < SIDE_STREAMS) {
            if ((e = cudaStreamWaitEvent(s, d.fork, 0)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamWaitEvent(fork)");
            used++;
        }
        sgroups++;
        if ((e = launch_convolution_batch(G, tw, io.data(), (int)io.size(), s)) != cudaSuccess)
            return cuda_fail(e, "batched NTT launch");
    }
    // the persistent kernel on st, beside the size-class groups on the side streams
    if (!pj.empty() && (e = launch_persistent(pj.data(), (int)pj.size(), barriers, st, status_word(dev, st))) !=
                           cudaSuccess)
        return cuda_fail(e, "persistent transform launch");
    for (int i = 0; i < used; i++) {
        if ((e = cudaEventRecord(d.join[i], d.side[i])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st, d.join[i], 0)) != cudaSuccess)
            return cuda_fail(e, "join");
    }
    u32* sw = status_word(dev, st);
    if ((e = launch_carry_batch(cj.data(), (int)count, st, sw)) != cudaSuccess)
        return cuda_fail(e, "batched carry launch");
    if (!fj.empty() && (e = launch_fallback(fj.data(), (int)fj.size(), st, sw)) != cudaSuccess)
        return cuda_fail(e, "recomputation launch");
    return PA_OK;
}

// The device's status slab, allocated (and cleared) on the first call on the
// device, which is also when the pool and the first tables are made.
void status_slab(int dev) {
    Device& d = g_dev[dev];
    if (d.status_dev || d.status_failed) return;
    u32* p = nullptr;
    u32* h = nullptr;
    cudaError_t e = cudaMalloc(&p, STATUS_SLOTS * sizeof(u32));
    if (e == cudaSuccess) e = cudaMemset(p, 0, STATUS_SLOTS * sizeof(u32));
    if (e == cudaSuccess) e = cudaMallocHost(&h, STATUS_SLOTS * sizeof(u32));
    if (e != cudaSuccess) {
        if (p) cudaFree(p);
        d.status_failed = true;  // the kernels then report through the device-wide word only
        cudaGetLastError();
        return;
    }
    memset(h, 0, STATUS_SLOTS * sizeof(u32));
    d.status_dev = p;
    d.status_host = h;
}

int setup(int* dev, cudaMemPool_t* pool) {
    int rc = current_device(dev);
    if (rc) return rc;
    load_tune_cache(*dev);
    status_slab(*dev);
    return get_pool(*dev, pool);
}

// Slot of stream st on device dev (-1 without a slab). Streams are told apart
// by their handle, with no CUDA call (queries such as cudaStreamGetId are not
// allowed while a stream is being captured into a graph).
int status_slot_of(int dev, cudaStream_t st) {
    Device& d = g_dev[dev];
    if (!d.status_dev) return -1;
    auto it = d.status_slot.find((const void*)st);
    if (it != d.status_slot.end()) return it->second;
    int slot = (int)d.status_slot.size();
    if (slot >= STATUS_SLOTS) slot = STATUS_SLOTS - 1;
    d.status_slot[(const void*)st] = slot;
    return slot;
}

// Host buffers in, host buffer out, queued without waiting: x and a are copied
// on the device's copy stream (two calls at most ahead of the hashes, so the
// next call's copies overlap this call's transforms), b behind them, the hash
// runs on st after each copy's event, and the result is copied back on st.
// Host-buffer hashes of at most this many bits run in place on mapped memory.
constexpr u64 ZERO_COPY_MAX_BITS = 1ull << 21;

// The device address of host buffer [p, p + bytes) when all of it is host
// memory the device can address (page-locked and mapped: its first and last
// bytes both mapped, at device addresses bytes - 1 apart), else null.
const void* mapped_host(const void* p, size_t bytes) {
    cudaPointerAttributes a0, a1;
    const char* last = (const char*)p + bytes - 1;
    if (cudaPointerGetAttributes(&a0, p) != cudaSuccess || cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
        cudaGetLastError();  // an unregistered pointer is not an error here
        return nullptr;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
        return nullptr;
    if ((const char*)a1.devicePointer - (const char*)a0.devicePointer != (ptrdiff_t)(bytes - 1)) return nullptr;
    return a0.devicePointer;
}

int queue_hash_host(const uint64_t* key, const uint64_t* seed_a, const uint64_t* seed_b, uint64_t n,
                    uint64_t m, uint64_t* out, cudaStream_t st, bool queued) {
    std::lock_guard<std::mutex> lk(g_mu);
    int dev, rc;
    cudaMemPool_t pool;
    if ((rc = setup(&dev, &pool))) return rc;
    Device& d = g_dev[dev];
    size_t in_bytes = ((n + 63) / 64) * sizeof(u64), out_bytes = ((m + 63) / 64) * sizeof(u64);
    if (n <= ZERO_COPY_MAX_BITS) {
        // Small blocks in mapped page-locked memory: the kernels read the inputs
        // and write the result in place over the host link. The copy path's
        // staging, copies and events cost more host time than such a hash
        // takes on the device.
        const void* kx = mapped_host(key, in_bytes);
        const void* ka = kx ? mapped_host(seed_a, in_bytes) : nullptr;
        const void* kb = ka ? mapped_host(seed_b, in_bytes) : nullptr;
        void* ko = kb ? (void*)mapped_host(out, out_bytes) : nullptr;
        if (ko) return hash_device((const u64*)kx, (const u64*)ka, (const u64*)kb, n, m, (u64*)ko, st, dev, pool);
    }
    if ((rc = side_streams(dev))) return rc;
    cudaEvent_t done = d.done[d.host_calls & 1];  // recorded by the call two before this one
    cudaError_t e = cudaSuccess;
    if (d.host_calls >= 2) e = cudaStreamWaitEvent(d.copy, done, 0);
    void *dx = nullptr, *da = nullptr, *db = nullptr;
    if (!e) e = cudaMallocFromPoolAsync(&dx, in_bytes, pool, d.copy);
    if (!e) e = cudaMallocFromPoolAsync(&da, in_bytes, pool, d.copy);
    if (!e) e = cudaMallocFromPoolAsync(&db, in_bytes, pool, d.copy);
    if (!e) e = cudaMemcpyAsync(dx, key, in_bytes, cudaMemcpyHostToDevice, d.copy);
    if (!e) e = cudaMemcpyAsync(da, seed_a, in_bytes, cudaMemcpyHostToDevice, d.copy);
    if (!e) e = cudaEventRecord(d.xa_ready, d.copy);
    if (!e) e = cudaMemcpyAsync(db, seed_b, in_bytes, cudaMemcpyHostToDevice, d.copy);
    // b's event is recorded even after a failure, so that st can order the frees
    cudaError_t eb = cudaEventRecord(d.b_ready, d.copy);
    if (!e) e = eb;
    {
        Scratch scr(st, pool);  // frees the inputs and the workspace on st, in order
        for (void* p : {dx, da, db})
            if (p) scr.ptrs.push_back(p);
        if (e) {
            cudaStreamWaitEvent(st, d.b_ready, 0);
            return cuda_fail(e, "host-buffer copies");
        }
        void* mo = nullptr;
        HashPlan hp;
        rc = hash_prepare((const u64*)dx, (const u64*)da, n, m, scr, dev, &hp);
        // A queued call waits for all three inputs before its first kernel (their
        // copies ran during the hashes before it), so that nothing sits between
        // the product's last kernel and the carry kernel on st and the
        // programmatic launch joins them; a call that waits for its result starts
        // the product once x and a are in and copies b meanwhile.
        cudaEvent_t in_ready = queued ? d.b_ready : d.xa_ready;
        if (rc || (e = cudaStreamWaitEvent(st, in_ready, 0))) {
            cudaStreamWaitEvent(st, d.b_ready, 0);
            return rc ? rc : cuda_fail(e, "cudaStreamWaitEvent");
        }
        rc = hash_product(hp, st);
        if (!queued && (e = cudaStreamWaitEvent(st, d.b_ready, 0))) return cuda_fail(e, "cudaStreamWaitEvent");
        if (rc) return rc;
        // the result goes to device memory and is copied back (writing it into a
        // mapped pinned buffer from the carry kernel measured slower)
        if ((rc = scr.get(out_bytes, &mo))) return rc;
        if ((rc = hash_finish(hp, (const u64*)db, n, m, (u64*)mo, st, dev))) return rc;
        if ((e = cudaMemcpyAsync(out, mo, out_bytes, cudaMemcpyDeviceToHost, st)))
            return cuda_fail(e, "cudaMemcpyAsync(D2H)");
    }
    if ((e = cudaEventRecord(done, st))) return cuda_fail(e, "cudaEventRecord");
    d.host_calls++;
    return PA_OK;
}


// Times every applicable plan variant of transform length base.N through
// hashes of n bits (m output bits) on st and records the fastest in the tuned
// table: the fastest of three timed runs of reps hashes each (short hashes
// time noisily). *err receives a CUDA error, the return value a library one.
int tune_length(int dev, cudaMemPool_t pool, const Geom& base, uint64_t n, uint64_t m, int reps,
                cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, const u64* x, const u64* a, const u64* b,
                u64* out, int* best_out, cudaError_t* err) {
    Device& d = g_dev[dev];
    const int mask = applicable_variants(base);
    const bool had_force = d.forced.count(base.N) != 0;
    const int old_force = had_force ? d.forced[base.N] : 0;
    int best = 0, rc = PA_OK;
    float best_ms = 0;
    cudaError_t e = cudaSuccess;
    for (int v = 0; e == cudaSuccess && rc == PA_OK && v < PLAN_VARIANTS; v++) {
        if (v & ~mask) continue;
        d.forced[base.N] = v;
        for (int i = 0; i < 2 && rc == PA_OK; i++) rc = hash_device(x, a, b, n, m, out, st, dev, pool);
        float ms = 0;
        for (int trial = 0; trial < 3 && e == cudaSuccess && rc == PA_OK; trial++) {
            if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
            for (int i = 0; i < reps && rc == PA_OK; i++) rc = hash_device(x, a, b, n, m, out, st, dev, pool);
            if (rc) break;
            if ((e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess)
                break;
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            if (trial == 0 || t < ms) ms = t;
        }
        if (rc || e != cudaSuccess) break;
        if (v == 0 || ms < best_ms) {
            best = v;
            best_ms = ms;
        }
    }
    if (had_force) d.forced[base.N] = old_force;
    else d.forced.erase(base.N);
    if (rc == PA_OK && e == cudaSuccess) d.tuned[base.N] = best;
    *best_out = best;
    *err = e;
    return rc;
}

}  // namespace

// ---------------------------------------------------------------------------
// per-kernel CUDA-event profiling
// ---------------------------------------------------------------------------
namespace {
struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
}  // namespace

namespace pa {
void set_error(const char* msg) { g_err = msg; }

u32* status_word(int dev, cudaStream_t st) {
    int slot = status_slot_of(dev, st);
    return slot < 0 ? nullptr : g_dev[dev].status_dev + slot;
}

int queue_status_read(cudaStream_t st, bool clear, const volatile u32** host_word) {
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    int slot = status_slot_of(dev, st);
    if (slot < 0) {
        *host_word = nullptr;
        return PA_OK;
    }
    Device& d = g_dev[dev];
    cudaError_t e = cudaMemcpyAsync(d.status_host + slot, d.status_dev + slot, sizeof(u32),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && clear) e = cudaMemsetAsync(d.status_dev + slot, 0, sizeof(u32), st);
    if (e != cudaSuccess) return cuda_fail(e, "status word read");
    *host_word = d.status_host + slot;
    return PA_OK;
}

void prof_begin(cudaStream_t st, const char* name) {
    if (!g_prof_on) return;
    ProfRec r{name, nullptr, nullptr};
    if (cudaEventCreate(&r.a) != cudaSuccess) return;
    if (cudaEventCreate(&r.b) != cudaSuccess) { cudaEventDestroy(r.a); return; }
    cudaEventRecord(r.a, st);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back(r);
}
void prof_end(cudaStream_t st) {
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof.empty()) cudaEventRecord(g_prof.back().b, st);
}
}  // namespace pa

extern "C" {

int pa_profile(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return PA_OK;
}

int pa_profile_collect(pa_kernel_stat* stats, int cap) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::vector<pa_kernel_stat> agg;
    int rc = PA_OK;
    for (ProfRec& r : g_prof) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) rc = cuda_fail(e, "profile event");
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
        pa_kernel_stat* s = nullptr;
        for (auto& x : agg)
            if (!strncmp(x.name, r.name, sizeof(x.name))) s = &x;
        if (!s) {
            agg.push_back(pa_kernel_stat{});
            s = &agg.back();
            strncpy(s->name, r.name, sizeof(s->name) - 1);
        }
        s->launches += 1;
        s->total_ms += ms;
    }
    g_prof.clear();
    if (rc) return rc;
    int n = (int)agg.size() < cap ? (int)agg.size() : cap;
    for (int i = 0; i < n; i++) stats[i] = agg[i];
    return n;
}

int pa_hash(const uint64_t* key, const uint64_t* seed_a, const uint64_t* seed_b, uint64_t n,
            uint64_t m, uint64_t* out, void* stream) {
    if (!check_sizes(n, m)) return fail(PA_EINVAL, "pa_hash: need 1 <= m <= n <= PA_MAX_BITS");
    if (!key || !seed_a || !seed_b || !out) return fail(PA_EINVAL, "pa_hash: null pointer");
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    return hash_device(key, seed_a, seed_b, n, m, out, (cudaStream_t)stream, dev, pool);
}

int pa_hash_host(const uint64_t* key, const uint64_t* seed_a, const uint64_t* seed_b,
                 uint64_t n, uint64_t m, uint64_t* out, void* stream) {
    if (!check_sizes(n, m)) return fail(PA_EINVAL, "pa_hash_host: need 1 <= m <= n <= PA_MAX_BITS");
    if (!key || !seed_a || !seed_b || !out) return fail(PA_EINVAL, "pa_hash_host: null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = queue_hash_host(key, seed_a, seed_b, n, m, out, st, false);
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return PA_OK;
}

int pa_hash_host_async(const uint64_t* key, const uint64_t* seed_a, const uint64_t* seed_b,
                       uint64_t n, uint64_t m, uint64_t* out, void* stream) {
    if (!check_sizes(n, m)) return fail(PA_EINVAL, "pa_hash_host_async: need 1 <= m <= n <= PA_MAX_BITS");
    if (!key || !seed_a || !seed_b || !out) return fail(PA_EINVAL, "pa_hash_host_async: null pointer");
    return queue_hash_host(key, seed_a, seed_b, n, m, out, (cudaStream_t)stream, true);
}

int pa_convolve16(const uint64_t* key, const uint64_t* seed_a, uint64_t n, uint64_t* coef,
                  void* stream) {
    if (n < 1 || n > PA_MAX_BITS) return fail(PA_EINVAL, "pa_convolve16: need 1 <= n <= PA_MAX_BITS");
    if (!key || !seed_a || !coef) return fail(PA_EINVAL, "pa_convolve16: null pointer");
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch scr(st, pool);
    u64* c = nullptr;
    if ((rc = queue_convolution(key, seed_a, n, st, scr, dev, &c))) return rc;
    cudaError_t e = cudaMemcpyAsync(coef, c, ((n + 15) / 16) * sizeof(u64),
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(D2D)");
    return PA_OK;
}

int pa_carry_extract(const uint64_t* coef, uint64_t L, const uint64_t* seed_b, uint64_t n,
                     uint64_t m, uint64_t* out, void* stream) {
    if (!check_sizes(n, m)) return fail(PA_EINVAL, "pa_carry_extract: need 1 <= m <= n <= PA_MAX_BITS");
    if ((!coef && L) || !seed_b || !out) return fail(PA_EINVAL, "pa_carry_extract: null pointer");
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch scr(st, pool);
    u64 Lmax = (n + 15) / 16;
    return queue_carry(coef, L < Lmax ? L : Lmax, seed_b, n, m, out, st, scr);
}

int pa_hash_batched(const pa_block* blocks, uint32_t count, void* stream) {
    if (count && !blocks) return fail(PA_EINVAL, "pa_hash_batched: null block array");
    for (uint32_t i = 0; i < count; i++) {
        const pa_block& b = blocks[i];
        if (!check_sizes(b.n, b.m) || !b.key || !b.seed_a || !b.seed_b || !b.out)
            return fail(PA_EINVAL, "pa_hash_batched: invalid block " + std::to_string(i));
    }
    if (!count) return PA_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    return hash_batch_device(blocks, count, (cudaStream_t)stream, dev, pool);
}

}  // extern "C"

struct pa_batch_s {
    int dev;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    void* ws;
};

extern "C" {

int pa_batch_create(const pa_block* blocks, uint32_t count, pa_batch* out) {
    if (!out || !count || !blocks) return fail(PA_EINVAL, "pa_batch_create: need blocks, count > 0, out");
    for (uint32_t i = 0; i < count; i++) {
        const pa_block& b = blocks[i];
        if (!check_sizes(b.n, b.m) || !b.key || !b.seed_a || !b.seed_b || !b.out)
            return fail(PA_EINVAL, "pa_batch_create: invalid block " + std::to_string(i));
    }
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    if ((rc = side_streams(dev))) return rc;
    void* ws = nullptr;
    cudaError_t e = cudaMalloc(&ws, batch_workspace_bytes(blocks, count));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(batch workspace)");
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool prof = g_prof_on;
    auto cleanup = [&](int code) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        cudaFree(ws);
        g_prof_on = prof;
        return code;
    };
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaStreamCreate"));
    // A batch of one runs the single-block path (its own plan variants, the
    // programmatic launch chain between its kernels), into the same workspace.
    auto run = [&](cudaStream_t s) {
        const pa_block& b = blocks[0];
        return count == 1 ? hash_device(b.key, b.seed_a, b.seed_b, b.n, b.m, b.out, s, dev, pool, ws)
                          : hash_batch_device(blocks, count, s, dev, pool, ws);
    };
    // one eager run first: builds every twiddle table and kernel attribute the
    // capture will use (neither may happen during capture)
    if ((rc = run(cs))) return cleanup(rc);
    if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return cleanup(cuda_fail(e, "warm-up run"));
    g_prof_on = false;
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaStreamBeginCapture"));
    rc = run(cs);
    e = cudaStreamEndCapture(cs, &graph);
    if (rc) return cleanup(rc);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaStreamEndCapture"));
    if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaGraphInstantiate"));
    cudaStreamDestroy(cs);
    g_prof_on = prof;
    *out = new pa_batch_s{dev, graph, exec, ws};
    return PA_OK;
}

int pa_batch_run(pa_batch batch, void* stream) {
    if (!batch) return fail(PA_EINVAL, "pa_batch_run: null batch");
    cudaError_t e = cudaGraphLaunch(batch->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? PA_OK : cuda_fail(e, "cudaGraphLaunch");
}

int pa_batch_destroy(pa_batch batch) {
    if (!batch) return PA_OK;
    cudaGraphExecDestroy(batch->exec);
    cudaGraphDestroy(batch->graph);
    cudaError_t e = cudaFree(batch->ws);
    delete batch;
    return e == cudaSuccess ? PA_OK : cuda_fail(e, "cudaFree(batch workspace)");
}

}  // extern "C"

// A spectrum of the seed for one product (transform length and digit width),
// built on first use on the caller's stream; later uses on any stream wait for
// `ready`.
struct SeedSpectrum {
    Geom G;
    int w;
    u64* spec;
    cudaEvent_t ready;
};

struct pa_seed_s {
    int dev;
    uint64_t n;
    Geom G;
    u64* spec;  // Toeplitz handles: the seed's spectrum, N words (tile register order, times N^-1)
    uint64_t m = 0;         // Toeplitz handles: output bits
    bool toeplitz = false;  // a Toeplitz seed (one-bit digits, n + m - 1 bits)
    u64* limbs = nullptr;   // modular-hash handles: a copy of the seed's limbs (the digits of
                            // every spectrum and of the recomputation)
    std::vector<SeedSpectrum> spectra;  // modular-hash handles: one per (length, width) used
};

namespace {

// The handle's spectrum for a product of length G0.N on w-bit digits (plan for
// that length taken on first use).
int seed_spectrum(pa_seed seed, const Geom& G0, int w, cudaStream_t st, int dev, SeedSpectrum** out) {
    for (SeedSpectrum& s : seed->spectra)
        if (s.G.N == G0.N && s.w == w) {
            cudaError_t e = cudaStreamWaitEvent(st, s.ready, 0);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent(seed spectrum)");
            *out = &s;
            return PA_OK;
        }
    SeedSpectrum s{plan_for_base(dev, G0), w, nullptr, nullptr};
    NttJob j;
    j.geom = s.G;
    int rc = get_tables(dev, s.G, &j.tw);
    if (rc) return rc;
    cudaError_t e = cudaMalloc(&s.spec, s.G.N * sizeof(u64));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ready, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        j.buf_x = j.buf_a = s.spec;
        j.da = j.dx = make_digits(seed->limbs, seed->n, w);
        j.L = j.dx.L;
        e = launch_seed_spectrum(j, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(s.ready, st);
    if (e != cudaSuccess) {
        if (s.ready) cudaEventDestroy(s.ready);
        cudaFree(s.spec);
        return cuda_fail(e, "seed spectrum");
    }
    seed->spectra.push_back(s);
    *out = &seed->spectra.back();
    return PA_OK;
}

}  // namespace

extern "C" {

// The seed's limbs are copied into the handle (the spectra of the products it
// serves are built from them), and the spectrum of the full-length product at
// the width a hash of n bits uses when it does not wrap is built now.
int pa_seed_create(const uint64_t* seed_a, uint64_t n, void* stream, pa_seed* out) {
    if (n < 1 || n > PA_MAX_BITS) return fail(PA_EINVAL, "pa_seed_create: need 1 <= n <= PA_MAX_BITS");
    if (!seed_a || !out) return fail(PA_EINVAL, "pa_seed_create: null pointer");
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    u64* limbs = nullptr;
    const size_t limb_bytes = ((n + 63) / 64) * sizeof(u64);
    cudaError_t e = cudaMalloc(&limbs, limb_bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(limbs, seed_a, limb_bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        cudaFree(limbs);
        return cuda_fail(e, "seed limbs copy");
    }
    pa_seed_s* h = new pa_seed_s{dev, n, Geom{}, nullptr};
    h->limbs = limbs;
    const DigitPlan dp = digit_plan(n, n, false, 0, g_digit_width);
    SeedSpectrum* ss = nullptr;
    if ((rc = seed_spectrum(h, dp.full, dp.w, st, dev, &ss))) {
        cudaFree(limbs);
        delete h;
        return rc;
    }
    h->G = ss->G;
    *out = h;
    return PA_OK;
}

// x's transform at the product's length against the seed's spectrum there,
// the carry step (certified when the product is wrapped) and, behind a
// wrapped product, the recomputation (a's digits from the handle's copy).
int pa_hash_seeded(pa_seed seed, const uint64_t* key, const uint64_t* seed_b, uint64_t m,
                   uint64_t* out, void* stream) {
    if (!seed || !key || !seed_b || !out) return fail(PA_EINVAL, "pa_hash_seeded: null pointer");
    if (seed->toeplitz) return fail(PA_EINVAL, "pa_hash_seeded: a Toeplitz seed handle");
    if (m < 1 || m > seed->n) return fail(PA_EINVAL, "pa_hash_seeded: need 1 <= m <= n");
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    if (dev != seed->dev) return fail(PA_EINVAL, "pa_hash_seeded: seed made on another device");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch scr(st, pool);
    const uint64_t n = seed->n;
    const DigitPlan dp = plan_digits(n, m, aligned16(key, seed->limbs));
    const WrapPlan& wp = dp.wp;
    SeedSpectrum* ss = nullptr;
    if ((rc = seed_spectrum(seed, wp.on ? wp.geom : dp.full, dp.w, st, dev, &ss))) return rc;
    const Geom fg = fallback_geom(n);
    const u64 words = wp.on && fg.N > ss->G.N ? fg.N : ss->G.N;
    const size_t state_words = (wp.on ? 2 : 1) * carry_state_words(n);
    void *bx, *ba = nullptr, *sp;
    if ((rc = scr.get(words * sizeof(u64), &bx)) || (wp.on && (rc = scr.get(fg.N * sizeof(u64), &ba))) ||
        (rc = scr.get(state_words * sizeof(u32), &sp)))
        return rc;
    u32* state = (u32*)sp;
    NttJob j;
    j.zero = state;  // cleared by the first transform kernel
    j.zero_words = (u32)state_words;
    j.geom = ss->G;
    if ((rc = get_tables(dev, j.geom, &j.tw))) return rc;
    j.buf_x = (u64*)bx;
    j.buf_a = ss->spec;
    j.dx = make_digits(key, n, dp.w);
    j.da = make_digits(seed->limbs, n, dp.w);
    j.L = dp.L;
    cudaError_t e;
    if ((e = launch_convolution_seeded(j, st)) != cudaSuccess) return cuda_fail(e, "seeded NTT launch");
    u32* flag = wp.on ? state + carry_flag_word(n) : nullptr;
    u32* sw = status_word(dev, st);
    CarryJob c{j.buf_x, j.L, seed_b, n, m, out, state, true, wp.lo, flag, g_wrap_mode == 3, (u32)dp.w};
    if ((e = launch_carry(c, st, sw)) != cudaSuccess) return cuda_fail(e, "carry launch");
    if (!wp.on) return PA_OK;
    FallbackJob f;
    if ((rc = fallback_job(dev, n, m, key, seed->limbs, (u64*)bx, (u64*)ba, state + carry_state_words(n), flag,
                           &f)))
        return rc;
    f.b = seed_b;
    f.out = out;
    if ((e = launch_fallback(&f, 1, st, sw)) != cudaSuccess) return cuda_fail(e, "recomputation launch");
    return PA_OK;
}

int pa_toeplitz(const uint64_t* key, const uint64_t* seed, uint64_t n, uint64_t m, uint64_t* out,
                void* stream) {
    if (!check_toeplitz(n, m))
        return fail(PA_EINVAL, "pa_toeplitz: need 1 <= m <= n, n + m - 1 <= PA_TOEPLITZ_MAX_BITS");
    if (!key || !seed || !out) return fail(PA_EINVAL, "pa_toeplitz: null pointer");
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch scr(st, pool);
    NttJob j;
    j.geom = plan_for_base(dev, toeplitz_base(n, m));
    j.L = n + m - 1;  // the last inverse pass keeps coefficients below n + m - 1
    if ((rc = get_tables(dev, j.geom, &j.tw))) return rc;
    void *bx, *ba;
    if ((rc = scr.get(j.geom.N * sizeof(u64), &bx)) || (rc = scr.get(j.geom.N * sizeof(u64), &ba))) return rc;
    j.buf_x = (u64*)bx;
    j.buf_a = (u64*)ba;
    j.dx = bit_digits(key, n);
    j.da = bit_digits(seed, n + m - 1);
    cudaError_t e = launch_convolution(j, st);
    if (e != cudaSuccess) return cuda_fail(e, "Toeplitz NTT launch");
    if ((e = launch_parity_extract(j.buf_x, n - 1, m, out, st)) != cudaSuccess)
        return cuda_fail(e, "parity launch");
    return PA_OK;
}

uint64_t pa_toeplitz_workspace_bytes(uint64_t n, uint64_t m) {
    if (!check_toeplitz(n, m)) return 0;
    return 2 * toeplitz_base(n, m).N * sizeof(u64);
}

int pa_toeplitz_seed_create(const uint64_t* seed, uint64_t n, uint64_t m, void* stream, pa_seed* out) {
    if (!check_toeplitz(n, m))
        return fail(PA_EINVAL, "pa_toeplitz_seed_create: need 1 <= m <= n, n + m - 1 <= PA_TOEPLITZ_MAX_BITS");
    if (!seed || !out) return fail(PA_EINVAL, "pa_toeplitz_seed_create: null pointer");
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    NttJob j;
    j.geom = plan_for_base(dev, toeplitz_base(n, m));
    j.L = n + m - 1;
    if ((rc = get_tables(dev, j.geom, &j.tw))) return rc;
    u64* spec = nullptr;
    cudaError_t e = cudaMalloc(&spec, j.geom.N * sizeof(u64));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(seed spectrum)");
    j.buf_x = j.buf_a = spec;
    j.da = j.dx = bit_digits(seed, n + m - 1);
    if ((e = launch_seed_spectrum(j, (cudaStream_t)stream)) != cudaSuccess) {
        cudaFree(spec);
        return cuda_fail(e, "seed transform launch");
    }
    pa_seed_s* h = new pa_seed_s{dev, n, j.geom, spec};
    h->m = m;
    h->toeplitz = true;
    *out = h;
    return PA_OK;
}

int pa_toeplitz_seeded(pa_seed seed, const uint64_t* key, uint64_t* out, void* stream) {
    if (!seed || !key || !out) return fail(PA_EINVAL, "pa_toeplitz_seeded: null pointer");
    if (!seed->toeplitz) return fail(PA_EINVAL, "pa_toeplitz_seeded: a modular-hash seed handle");
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    if (dev != seed->dev) return fail(PA_EINVAL, "pa_toeplitz_seeded: seed made on another device");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch scr(st, pool);
    const uint64_t n = seed->n, m = seed->m;
    NttJob j;
    j.geom = seed->G;
    j.L = n + m - 1;
    if ((rc = get_tables(dev, j.geom, &j.tw))) return rc;
    void* bx;
    if ((rc = scr.get(j.geom.N * sizeof(u64), &bx))) return rc;
    j.buf_x = (u64*)bx;
    j.buf_a = seed->spec;
    j.dx = j.da = bit_digits(key, n);
    cudaError_t e = launch_convolution_seeded(j, st);
    if (e != cudaSuccess) return cuda_fail(e, "seeded Toeplitz NTT launch");
    if ((e = launch_parity_extract(j.buf_x, n - 1, m, out, st)) != cudaSuccess)
        return cuda_fail(e, "parity launch");
    return PA_OK;
}

int pa_seed_destroy(pa_seed seed) {
    if (!seed) return PA_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(seed->dev);
    cudaError_t e = seed->spec ? cudaFree(seed->spec) : cudaSuccess;
    if (seed->limbs) cudaFree(seed->limbs);
    for (SeedSpectrum& s : seed->spectra) {
        cudaError_t es = cudaFree(s.spec);
        if (e == cudaSuccess) e = es;
        cudaEventDestroy(s.ready);
    }
    if (prev >= 0) cudaSetDevice(prev);
    delete seed;
    return e == cudaSuccess ? PA_OK : cuda_fail(e, "cudaFree(seed spectrum)");
}

int pa_plan_override(uint64_t n, int variant) {
    if (n < 1 || n > PA_MAX_BITS || variant < -1 || variant >= PLAN_VARIANTS)
        return fail(PA_EINVAL, "pa_plan_override: need 1 <= n <= PA_MAX_BITS, -1 <= variant < 64");
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    // the length of the full-length product a hash of n bits runs at the current digit width
    u64 N = digit_plan(n, n, false, 0, g_digit_width).full.N;
    if (variant < 0) g_dev[dev].forced.erase(N);
    else g_dev[dev].forced[N] = variant;
    return PA_OK;
}

int pa_plan_override_length(uint64_t N, int variant) {
    if (variant < -1 || variant >= PLAN_VARIANTS)
        return fail(PA_EINVAL, "pa_plan_override_length: need -1 <= variant < 64");
    if (N < 4096 || N > (1ull << MAX_LOGN) || choose_geom_len(N).N != N)
        return fail(PA_EINVAL, "pa_plan_override_length: not a transform length of the library");
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    if (variant < 0) g_dev[dev].forced.erase(N);
    else g_dev[dev].forced[N] = variant;
    return PA_OK;
}

int pa_autotune(uint64_t n, int reps, int* variant_out) {
    if (n < 1 || n > PA_MAX_BITS) return fail(PA_EINVAL, "pa_autotune: need 1 <= n <= PA_MAX_BITS");
    if (reps < 1) reps = 5;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    u64 m = n / 4 ? n / 4 : 1;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    void *x = nullptr, *a = nullptr, *b = nullptr, *out = nullptr;
    size_t in_bytes = ((n + 63) / 64) * 8, out_bytes = ((m + 63) / 64) * 8;
    if (e == cudaSuccess) e = cudaMalloc(&x, in_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&a, in_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b, in_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&out, out_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(x, 0x5A, in_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a, 0xC3, in_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b, 0x3C, in_bytes, st);
    // The lengths a hash of n bits (m = n / 4) runs, at the digit width each
    // would use: the full-length product's, timed with wrapping off, and the
    // wrapped product's when there is one (the default mode's choice).
    const DigitPlan dfull = digit_plan(n, m, false, 0, g_digit_width);
    const DigitPlan dwrap = digit_plan(n, m, true, WRAP_MIN_FULL, g_digit_width);
    const WrapPlan& wp = dwrap.wp;
    const Geom lens[2] = {dfull.full, wp.geom};
    const int saved_mode = g_wrap_mode;
    int best_full = 0;
    for (int li = 0; li < (wp.on ? 2 : 1) && e == cudaSuccess && rc == PA_OK; li++) {
        g_wrap_mode = li;
        int best = 0;
        rc = tune_length(dev, pool, lens[li], n, m, reps, st, e0, e1, (const u64*)x, (const u64*)a,
                         (const u64*)b, (u64*)out, &best, &e);
        if (li == 0) best_full = best;
    }
    g_wrap_mode = saved_mode;
    if (st) cudaStreamSynchronize(st);
    cudaFree(x);
    cudaFree(a);
    cudaFree(b);
    cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "pa_autotune");
    save_tune_cache(dev);
    if (variant_out) *variant_out = best_full;
    return PA_OK;
}

// The plans of a transform length are the same kernels whatever feeds them, so
// the Toeplitz transform's length is tuned through a modular hash of that length
// (keys of 16 N / 2 bits: 2 L - 1 = N - 1 digits of product).
int pa_toeplitz_autotune(uint64_t n, uint64_t m, int reps, int* variant_out) {
    if (!check_toeplitz(n, m))
        return fail(PA_EINVAL, "pa_toeplitz_autotune: need 1 <= m <= n, n + m - 1 <= PA_TOEPLITZ_MAX_BITS");
    uint64_t N = toeplitz_base(n, m).N;
    return pa_autotune(16 * (N / 2), reps, variant_out);
}

int pa_prepare(uint64_t n) {
    if (n < 1 || n > PA_MAX_BITS) return fail(PA_EINVAL, "pa_prepare: need 1 <= n <= PA_MAX_BITS");
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    cudaMemPool_t pool;
    int rc = setup(&dev, &pool);
    if (rc) return rc;
    Twiddles tw;
    // the recomputation's length; for every digit width a hash of n bits may use
    // (all exact ones when the width is chosen), its full-length product and
    // every shorter length a wrapped product may run (which depends on m)
    if ((rc = get_base_tables(dev, fallback_geom(n), &tw))) return rc;
    for (int w = DIGIT_MIN; w <= DIGIT_MAX; w++) {
        if ((g_digit_width && w != g_digit_width) || !width_exact(n, w)) continue;
        const u64 L = digits_for(n, w);
        const Geom full = choose_geom(L);
        if ((rc = get_tables(dev, plan_for_base(dev, full), &tw))) return rc;
        for (Geom g = choose_geom_len(L); g.N < full.N; g = choose_geom_len(g.N + 1))
            if ((rc = get_tables(dev, plan_for_base(dev, g), &tw))) return rc;
    }
    if (g_digit_width && !width_exact(n, g_digit_width)) {  // the forced width falls back to 16
        const Geom full = choose_geom(digits_for(n, 16));
        if ((rc = get_tables(dev, plan_for_base(dev, full), &tw))) return rc;
        for (Geom g = choose_geom_len(digits_for(n, 16)); g.N < full.N; g = choose_geom_len(g.N + 1))
            if ((rc = get_tables(dev, plan_for_base(dev, g), &tw))) return rc;
    }
    return PA_OK;
}

uint64_t pa_workspace_bytes(uint64_t n) {
    if (n < 1 || n > PA_MAX_BITS) return 0;
    return 2 * buffer_words(n) * sizeof(u64) + 2 * carry_state_words(n) * sizeof(u32);
}

int pa_plan_info(uint64_t n, uint64_t m, uint64_t info[3]) {
    if (!check_sizes(n, m)) return fail(PA_EINVAL, "pa_plan_info: need 1 <= m <= n <= PA_MAX_BITS");
    if (!info) return fail(PA_EINVAL, "pa_plan_info: null pointer");
    DigitPlan dp, df;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        dp = plan_digits(n, m);
        df = digit_plan(n, m, false, 0, g_digit_width);
    }
    info[0] = dp.first_n();
    info[1] = df.full.N;
    info[2] = dp.wp.on ? dp.wp.lo : 0;
    return PA_OK;
}

int pa_plan_digits(uint64_t n, uint64_t m, uint32_t* width) {
    if (!check_sizes(n, m)) return fail(PA_EINVAL, "pa_plan_digits: need 1 <= m <= n <= PA_MAX_BITS");
    if (!width) return fail(PA_EINVAL, "pa_plan_digits: null pointer");
    std::lock_guard<std::mutex> lk(g_mu);
    *width = (uint32_t)plan_digits(n, m).w;
    return PA_OK;
}

int pa_batch_mode(int mode) {
    if (mode < 0 || mode > 2) return fail(PA_EINVAL, "pa_batch_mode: mode must be 0, 1 or 2");
    std::lock_guard<std::mutex> lk(g_mu);
    int prev = g_batch_mode;
    g_batch_mode = mode;
    return prev;
}

int pa_digit_width(int width) {
    if (width != 0 && (width < DIGIT_MIN || width > DIGIT_MAX))
        return fail(PA_EINVAL, "pa_digit_width: width must be 0 or 16 .. 20");
    std::lock_guard<std::mutex> lk(g_mu);
    int prev = g_digit_width;
    g_digit_width = width;
    return prev;
}

int pa_wrap_mode(int mode) {
    if (mode < 0 || mode > 3) return fail(PA_EINVAL, "pa_wrap_mode: mode must be 0, 1, 2 or 3");
    std::lock_guard<std::mutex> lk(g_mu);
    int prev = g_wrap_mode;
    g_wrap_mode = mode;
    return prev;
}

int pa_wrap_flags(uint64_t* count, int clear) {
    if (!count) return fail(PA_EINVAL, "pa_wrap_flags: null pointer");
    cudaError_t e = cudaDeviceSynchronize();
    unsigned long long c = 0;
    if (e == cudaSuccess) e = read_flag_count(&c, clear != 0);
    if (e != cudaSuccess) return cuda_fail(e, "pa_wrap_flags");
    *count = c;
    return PA_OK;
}

int pa_shutdown(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    int prev = -1;
    cudaGetDevice(&prev);
    for (auto& kv : g_dev) {
        cudaSetDevice(kv.first);
        for (auto& t : kv.second.tables) cudaFree(t.second);
        for (auto& t : kv.second.pass_tables) cudaFree(t.second);
        if (kv.second.table_stream) cudaStreamDestroy(kv.second.table_stream);
        if (kv.second.copy) {
            cudaStreamDestroy(kv.second.copy);
            cudaEventDestroy(kv.second.xa_ready);
            cudaEventDestroy(kv.second.b_ready);
            for (cudaEvent_t ev : kv.second.done) cudaEventDestroy(ev);
        }
        if (kv.second.pool) cudaMemPoolDestroy(kv.second.pool);
        if (kv.second.status_dev) cudaFree(kv.second.status_dev);
        if (kv.second.status_host) cudaFreeHost(kv.second.status_host);
        if (kv.second.fork) {
            cudaEventDestroy(kv.second.fork);
            for (int i = 0; i < SIDE_STREAMS; i++) {
                cudaStreamDestroy(kv.second.side[i]);
                cudaEventDestroy(kv.second.join[i]);
            }
        }
    }
    g_dev.clear();
    noalloc_reset();
    if (prev >= 0) cudaSetDevice(prev);
    return PA_OK;
}

int pa_device_status(int clear) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    u32 st = 0;
    if ((e = read_device_status(&st, clear != 0)) != cudaSuccess) return cuda_fail(e, "device status");
    u32 fst = 0, pst = 0;
    if ((e = read_fallback_status(&fst, clear != 0)) != cudaSuccess) return cuda_fail(e, "device status");
    if ((e = read_persist_status(&pst, clear != 0)) != cudaSuccess) return cuda_fail(e, "device status");
    u32 bst = 0;
    if ((e = read_bulk_status(&bst, clear != 0)) != cudaSuccess) return cuda_fail(e, "device status");
    if (bst & PA_STATUS_TIMEOUT) return fail(PA_ETIMEOUT, "a bounded device wait ran out (bulk tile copy)");
    if (pst & PA_STATUS_TIMEOUT) return fail(PA_ETIMEOUT, "a bounded device wait ran out (persistent transforms)");
    if (st & PA_STATUS_TIMEOUT) return fail(PA_ETIMEOUT, "a bounded device wait ran out (carry look-back)");
    if (fst & PA_STATUS_TIMEOUT) return fail(PA_ETIMEOUT, "a bounded device wait ran out (recomputation barrier)");
    return PA_OK;
}

int pa_stream_status(void* stream, int clear) {
    cudaStream_t st = (cudaStream_t)stream;
    const volatile u32* word = nullptr;
    int rc = queue_status_read(st, clear != 0, &word);
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (word && (*word & PA_STATUS_TIMEOUT))
        return fail(PA_ETIMEOUT, "a bounded device wait ran out on this stream");
    return PA_OK;
}

int pa_fault_inject(int what) {
    if (what != PA_FAULT_CARRY_WAIT) return fail(PA_EINVAL, "pa_fault_inject: unknown fault");
    std::lock_guard<std::mutex> lk(g_mu);
    fault_inject_carry();
    return PA_OK;
}

const char* pa_last_error(void) { return g_err.c_str(); }

const char* pa_version(void) { return "pa_gb300 0.1.0 (sm_103a)"; }

}  // extern "C"
