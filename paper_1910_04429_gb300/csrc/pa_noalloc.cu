// pa_hash_noalloc: the hash with every byte of device scratch taken from
// fixed-size arrays compiled into this library, for callers that cannot
// allocate device memory themselves or let a library do it: code running
// inside a CUDA graph that must not contain allocation nodes, hosts whose
// memory is fully reserved up front (real-time QKD post-processing loops that
// must not stall in the allocator), and environments where the device
// allocator is owned by another framework.
//
// Scratch lives in file-scope __device__ arrays sized for keys of up to
// PA_NOALLOC_MAX_BITS bits. Every GPU that loads the library holds them until
// process exit. Host code cannot use the array names as device addresses (in
// host code they are host-side stand-ins), so the set-up below looks the
// device addresses up with cudaGetSymbolAddress once per device, with that
// device current, and passes them to the kernels.
//
// The first call on a device performs that set-up and also fills the twiddle
// tables on the caller's stream and waits for them; make the first call before
// any stream capture (a first call on a capturing stream is refused, leaving
// the capture intact). pa_shutdown forgets the set-up, so that after a device
// reset the next call looks the arrays up again. All calls share the same
// arrays and the arrays keep the last call's contents: the transform buffers
// are written before they are read in a call, and the carry step's tile
// states, which must start at zero, are cleared on the stream by a memset
// before each carry launch (a memset allocates nothing). Calls that overlap on
// the GPU (on different streams, or on one stream from several threads
// without ordering) race on the scratch and give wrong results.
#include <mutex>

#include "../../include/pa.h"
#include "pa_internal.h"

using namespace pa;

namespace {

constexpr int NA_MAX_LOGN = 17;                          // 2^20-bit keys: 2^16 digits -> N = 2^17
constexpr u64 NA_MAX_N = 1ull << NA_MAX_LOGN;
constexpr int NA_LOGN0 = LOG_TILE;                       // smallest transform, 2^12
constexpr int NA_SIZES = NA_MAX_LOGN - NA_LOGN0 + 1;
constexpr u64 NA_TABLE_WORDS = 4 * 4096 + 2 * (NA_MAX_N >> 12);
constexpr u64 NA_CARRY_BYTES = 1024;                     // carry tile states, ticket, flag
static_assert(((PA_NOALLOC_MAX_BITS + 63) / 64 + CARRY_TILE_LIMBS - 1) / CARRY_TILE_LIMBS * 4 + 8 <= NA_CARRY_BYTES,
              "carry-state scratch too small for the cap");

static_assert(PA_NOALLOC_MAX_BITS <= 16 * (NA_MAX_N / 2), "transform too short for the cap");

// transform buffers (x and a), one twiddle table set per transform size, and
// the carry-scan bytes
__device__ __align__(256) u64 g_na_work[2 * NA_MAX_N];
__device__ __align__(256) u64 g_na_tables[NA_SIZES * NA_TABLE_WORDS];
__device__ __align__(256) uint8_t g_na_carry[NA_CARRY_BYTES];

constexpr int NA_MAX_DEVICES = 64;
struct NaDevice {
    bool ready = false;
    u64* work = nullptr;
    u64* tables = nullptr;
    uint8_t* carry = nullptr;
};
std::mutex g_na_mu;
NaDevice g_na_dev[NA_MAX_DEVICES];

// tables[t] for one transform size in the layout of make_tables():
// w4096 | w4096^-1 | wlo | wlo^-1 | whi | whi^-1, computed as powers
__global__ void k_na_tables(u64* tab, u64 nh, u64 w4, u64 w4i, u64 w, u64 wi, u64 s, u64 si) {
    u64 total = 4 * 4096 + 2 * nh;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        u64 v;
        if (i < 4096) v = gl::pow(w4, i);
        else if (i < 8192) v = gl::pow(w4i, i - 4096);
        else if (i < 12288) v = gl::pow(w, i - 8192);
        else if (i < 16384) v = gl::pow(wi, i - 12288);
        else if (i < 16384 + nh) v = gl::pow(s, i - 16384);
        else v = gl::pow(si, i - 16384 - nh);
        tab[i] = v;
    }
}

int na_setup(int dev, cudaStream_t st, NaDevice** out) {
    NaDevice& d = g_na_dev[dev];
    if (!d.ready) {
        // the set-up launches kernels and waits for them: on a capturing stream
        // that would end the caller's capture, so refuse and leave it intact
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
            set_error("pa_hash_noalloc: cudaStreamIsCapturing failed");
            return PA_ECUDA;
        }
        if (cap != cudaStreamCaptureStatusNone) {
            set_error("pa_hash_noalloc: the first call on a device (its set-up) must not be on a capturing stream");
            return PA_EINVAL;
        }
        cudaError_t e = cudaGetSymbolAddress((void**)&d.work, g_na_work);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&d.tables, g_na_tables);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&d.carry, g_na_carry);
        if (e != cudaSuccess) {
            set_error("pa_hash_noalloc: cudaGetSymbolAddress failed");
            return PA_ECUDA;
        }
        for (int logN = NA_LOGN0; logN <= NA_MAX_LOGN; logN++) {
            u64 N = 1ull << logN;
            u64 w = omega(logN), wi = gl::pow(w, gl::P - 2);
            k_na_tables<<<64, 256, 0, st>>>(d.tables + (logN - NA_LOGN0) * NA_TABLE_WORDS, N >> 12,
                                            gl::pow(w, N >> 12), gl::pow(wi, N >> 12), w, wi,
                                            gl::pow(w, 4096), gl::pow(wi, 4096));
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("pa_hash_noalloc: twiddle set-up failed");
            return PA_ECUDA;
        }
        d.ready = true;
    }
    *out = &d;
    return PA_OK;
}

}  // namespace

namespace pa {
void noalloc_reset() {
    std::lock_guard<std::mutex> lk(g_na_mu);
    for (NaDevice& d : g_na_dev) d = NaDevice{};
}
}  // namespace pa

extern "C" int pa_hash_noalloc(const uint64_t* key, const uint64_t* seed_a, const uint64_t* seed_b,
                               uint64_t n, uint64_t m, uint64_t* out, void* stream) {
    if (n < 1 || m < 1 || m > n) {
        set_error("pa_hash_noalloc: need 1 <= m <= n");
        return PA_EINVAL;
    }
    if (n > PA_NOALLOC_MAX_BITS) {
        set_error("pa_hash_noalloc: n exceeds PA_NOALLOC_MAX_BITS (fixed scratch size)");
        return PA_EINVAL;
    }
    if (!key || !seed_a || !seed_b || !out) {
        set_error("pa_hash_noalloc: null pointer");
        return PA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        set_error("pa_hash_noalloc: no usable current device");
        return PA_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    NaDevice* d = nullptr;
    int rc = na_setup(dev, st, &d);
    if (rc) return rc;

    u64 L = (n + 15) / 16;
    int logN = logn_for_digits(L);
    NttJob j;
    j.geom = make_geom(logN);
    j.L = L;
    const u64* tab = d->tables + (logN - NA_LOGN0) * NA_TABLE_WORDS;
    u64 nh = j.geom.N >> 12;
    j.tw = Twiddles{tab, tab + 4096, tab + 8192, tab + 12288, tab + 16384, tab + 16384 + nh};
    j.buf_x = d->work;
    j.buf_a = d->work + j.geom.N;
    j.dx = make_digits(key, n, 16);
    j.da = make_digits(seed_a, n, 16);
    if (launch_convolution(j, st) != cudaSuccess) {
        set_error("pa_hash_noalloc: NTT launch failed");
        return PA_ECUDA;
    }
    CarryJob c{j.buf_x, L, seed_b, n, m, out, reinterpret_cast<uint32_t*>(d->carry)};
    if (launch_carry(c, st) != cudaSuccess) {
        set_error("pa_hash_noalloc: carry launch failed");
        return PA_ECUDA;
    }
    return PA_OK;
}

