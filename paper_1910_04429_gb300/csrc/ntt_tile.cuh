// Per-thread phases of the NTT tile kernels.
//
// The exact product of Algorithm 1 (Sec. 3.2.2: zero fill and split, evaluate
// by NTT, pointwise multiply, interpolate by inverse NTT) is computed with a
// length-N transform over GF(p), N = 2^k. The transform is factored
// (Cooley-Tukey, decimation in frequency) into passes; each pass works on
// independent tiles of 4096 elements held by one 512-thread CTA:
//
//  * a strided pass of radix R (2..64) over stride S: for every column j < S of
//    a sub-problem of size M = R*S, a length-R DFT down the column, then the
//    inter-pass twiddle w_M^(j*k) on output k (in place, k replacing the digit);
//  * one contiguous pass over 4096 consecutive elements (64 x 64 tile: column
//    DFTs, the twiddle w_4096^(c*k), row DFTs).
// Every length-64 DFT is 8 x 8 with in-register length-8 DFTs; all their
// roots are powers of 2 (w_64 = 8), so only shift-multiplies occur inside.
// The spectrum ends up in a fixed digit-reversed order, identical for both
// operands, and the inverse passes run the same steps mirrored, so the
// pointwise product needs no reordering.
//
// Each phase is a function of (thread or work item, registers) so that the
// kernels are plain sequences of phases separated by __syncthreads().
#pragma once
#include "gl.cuh"

namespace pa {

constexpr int TILE = 4096;
constexpr int NT = 512;  // threads per tile CTA

// ---------------------------------------------------------------------------
// twiddles
// ---------------------------------------------------------------------------
constexpr int MAX_PASSES = 8;  // strided passes of a plan

struct Twiddles {
    const u64* w4096;   // w_4096^t, t < 4096
    const u64* w4096i;  // w_4096^-t
    const u64* wlo;     // w_N^t, t < 4096
    const u64* wloi;
    const u64* whi;     // w_N^(4096 t), t < N / 4096
    const u64* whii;
    // Strided pass p of the plan (sub-problem size M = R S): its inter-pass
    // twiddles w_M^(j k) at [k S + j] (j < S, k < R) and w_M^-(j k) likewise.
    // Null: computed from wlo / whi at run time.
    const u64* passf[MAX_PASSES];
    const u64* passi[MAX_PASSES];
    const u64* w4096s;  // w_4096^t * N^-1 (a forward tile pass that also scales), or null
};

template <bool INV>
GL_HD u64 omega_n(const Twiddles& tw, u64 e) {  // w_N^(+-e), e < N
    const u64* lo = INV ? tw.wloi : tw.wlo;
    const u64* hi = INV ? tw.whii : tw.whi;
    return gl::mul(lo[e & 4095], hi[e >> 12]);
}

// ---------------------------------------------------------------------------
// key digits: the w-bit coefficients of Algorithm 1's split step
// ---------------------------------------------------------------------------
struct Digits {
    const uint16_t* src;  // little-endian limbs (viewed as 16-bit digits when width is 16)
    u64 L;                // live digits: ceil(n / width), or n with one_bit
    u32 top_mask;         // mask of digit L-1 (bits >= n cleared); unused with one_bit
    uint16_t one_bit;     // 1: every bit is a digit (GF(2) vectors as 0/1 coefficients)
    uint16_t width;       // digit bits, 16 .. 20: digit k = bits [w k, w k + w) of the key
    u64 nlimbs;           // 64-bit limbs of the source (bits beyond them are never read)
};

// digits of w bits of an n-bit integer held in ceil(n/64) limbs
GL_HD Digits make_digits(const uint64_t* limbs, u64 n, int w) {
    u64 L = (n + (u64)w - 1) / (u64)w;
    u32 top = (u32)(n - (u64)w * (L - 1));  // live bits of the top digit, 1 .. w
    u32 mask = top >= 32 ? 0xFFFFFFFFu : (1u << top) - 1;
    return Digits{reinterpret_cast<const uint16_t*>(limbs), L, mask, 0, (uint16_t)w, (n + 63) / 64};
}

// 16-bit digits (or one-bit ones): the hot first pass reads these without the
// wider-digit code, which would cost its kernels registers
GL_HD u64 digit_at16(const Digits& d, u64 pos) {
    if (pos >= d.L) return 0;  // zero fill (Algorithm 1, step 1)
    if (d.one_bit) return (d.src[pos >> 4] >> (pos & 15)) & 1u;
    uint16_t v = d.src[pos];
    if (pos == d.L - 1) v &= (uint16_t)d.top_mask;
    return v;
}

// any width
GL_HD u64 digit_at(const Digits& d, u64 pos) {
    if (pos >= d.L) return 0;  // zero fill (Algorithm 1, step 1)
    if (d.one_bit) return (d.src[pos >> 4] >> (pos & 15)) & 1u;
    if (d.width == 16) {
        uint16_t v = d.src[pos];
        if (pos == d.L - 1) v &= (uint16_t)d.top_mask;
        return v;
    }
    const u64* limbs = reinterpret_cast<const u64*>(d.src);
    const u64 bit = pos * d.width, li = bit >> 6;
    const unsigned sh = (unsigned)(bit & 63);
    u64 v = limbs[li] >> sh;
    if (sh + d.width > 64 && li + 1 < d.nlimbs) v |= limbs[li + 1] << (64 - sh);
    v &= (1ull << d.width) - 1;
    if (pos == d.L - 1) v &= d.top_mask;
    return v;
}

// Staged wide digits (width > 16): row d of a strided tile (digits P_d .. P_d + C - 1)
// is staged as the 16-byte chunks of the limbs from chunk floor(w P_d / 128) on, in a
// slot of wide_row_chunks(C) chunks (enough for 20-bit digits, plus the misalignment
// and the second word of the last digit's read).
GL_HD constexpr int wide_row_chunks(int C) { return (20 * C + 127) / 128 + 2; }

// digit c of a staged row: bit offset r0 + w c, r0 = (w P_d) mod 128
GL_HD u64 wide_digit(const u32* row, u32 r0, int w, int c) {
    u32 o = r0 + (u32)(w * c);
    u32 lo = row[o >> 5], hi = row[(o >> 5) + 1];
#if defined(__CUDA_ARCH__)
    u32 v = __funnelshift_r(lo, hi, o & 31);
#else
    u32 v = (u32)((((u64)hi << 32) | lo) >> (o & 31));
#endif
    return v & ((1u << w) - 1);
}

// ---------------------------------------------------------------------------
// strided pass, radix R = RA * RB in {2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64}
// ---------------------------------------------------------------------------
struct StridedGeom {
    u64 N, M, S;     // transform length, sub-problem size, stride (= M / R)
    u32 tpb;         // tiles per sub-problem, S / C
    const u64* twf;  // this pass's twiddle tables (Twiddles::passf / passi), or null
    const u64* twi;
};

// Where tile t of a strided pass sits: sub-problem b, first column jl0.
struct TilePos {
    u64 base;  // b * M + jl0: position of (column 0, digit 0)
    u64 jl0;   // first column of the tile within its sub-problem
};

// Tile of a radix-R pass: R rows (digits) x C consecutive columns, R * C <= 4096.
template <int RA, int RB, int CC>
struct Strided {
    static constexpr int R = RA * RB;
    static constexpr int C = CC;
    static constexpr int NA = RA * C;                   // phase-A items (RB words each)
    static constexpr int NB = RB * C;                   // phase-B items (RA words each)
    static constexpr int ITEMS_A = (NA + NT - 1) / NT;  // per thread
    static constexpr int ITEMS_B = (NB + NT - 1) / NT;
    static_assert(R * C <= TILE, "tile larger than shared memory");

    static GL_HD TilePos tile(const StridedGeom& g, u64 t) {
        u32 b = (u32)t / g.tpb, cg = (u32)t - b * g.tpb;  // the grid has fewer than 2^31 tiles
        return TilePos{b * g.M + (u64)cg * C, (u64)cg * C};
    }

    // forward, step 1: length-RB DFT over j1 of digits j0 + RA*j1, twiddle w_R^(j0 kr)
    // first pass on digits of at most N/2 live positions: rows j0 + RA j1 with
    // j1 >= RB/2 lie at or above N/2, so they are zero
    template <bool PACK>
    static GL_HD bool upper_rows_zero(const StridedGeom& g, const Digits& dig) {
        return PACK && (RB == 2 || RB == 4 || RB == 8) && 2 * dig.L <= g.N;
    }
    // WIDE: digits wider than 16 bits (a separate instantiation)
    template <bool PACK, bool WIDE = false>
    static GL_HD void fwd_a(const StridedGeom& g, const TilePos& tp, int it, const u64* buf,
                            const Digits& dig, u64* sm) {
        int j0 = it / C, c = it % C;
        u64 v[RB];
        const bool half = upper_rows_zero<PACK>(g, dig);
#pragma unroll
        for (int j1 = 0; j1 < RB; j1++) {
            u64 p = tp.base + c + g.S * (u64)(j0 + RA * j1);
            v[j1] = (half && 2 * j1 >= RB) ? 0 : PACK ? (WIDE ? digit_at(dig, p) : digit_at16(dig, p)) : buf[p];
        }
        if constexpr (PACK && (RB == 2 || RB == 4 || RB == 8)) {
            if (half) gl::dft_fwd_upper_zero<RB>(v);
            else gl::dft<RB, false>(v);
        } else {
            gl::dft<RB, false>(v);
        }
        gl::row_roots<R, false, RB, RA>(v, j0);
#pragma unroll
        for (int kr = 0; kr < RB; kr++) sm[(kr * RA + j0) * C + c] = v[kr];
    }

    // fwd_a reading the tile from a [R][C] staging copy: words, or (PACK) 16-bit
    // digits already zero past the last live digit, or (PACK, wider digits) each
    // row's limb chunks (digits past the last live one read as zero here)
    template <bool PACK, bool WIDE = false>
    static GL_HD void fwd_a_staged(const StridedGeom& g, const TilePos& tp, int it, const u64* st64,
                                   const uint16_t* st16, const Digits& dig, u64* sm) {
        int j0 = it / C, c = it % C;
        u64 v[RB];
        const bool half = upper_rows_zero<PACK>(g, dig);  // those rows were not staged
#pragma unroll
        for (int j1 = 0; j1 < RB; j1++) {
            int d = j0 + RA * j1;
            if (half && 2 * j1 >= RB) {
                v[j1] = 0;
            } else if (PACK && !WIDE) {
                uint16_t x = st16[d * C + c];
                if (tp.base + c + g.S * (u64)d == dig.L - 1) x &= (uint16_t)dig.top_mask;
                v[j1] = x;
            } else if (PACK) {
                // the row's bit offset and live digits, worked out once when it was staged
                const uint2 ri = reinterpret_cast<const uint2*>(st64 + R * wide_row_chunks(C) * 2)[d];
                const u32* row = reinterpret_cast<const u32*>(st64) + d * wide_row_chunks(C) * 4;
                u64 x = wide_digit(row, ri.x & 127u, dig.width, c);
                if ((u32)c >= (ri.x >> 7)) x = 0;
                else if ((u32)c == ri.y) x &= dig.top_mask;
                v[j1] = x;
            } else {
                v[j1] = st64[d * C + c];
            }
        }
        if constexpr (PACK && (RB == 2 || RB == 4 || RB == 8)) {
            if (half) gl::dft_fwd_upper_zero<RB>(v);
            else gl::dft<RB, false>(v);
        } else {
            gl::dft<RB, false>(v);
        }
        gl::row_roots<R, false, RB, RA>(v, j0);
#pragma unroll
        for (int kr = 0; kr < RB; kr++) sm[(kr * RA + j0) * C + c] = v[kr];
    }

    // inter-pass twiddle w_M^(+-jl k) of column jl, digit k: the pass's table, or
    // w_N^(e k) with e = (N / M) jl from the transform's tables
    template <bool INV>
    static GL_HD u64 pass_twiddle(const StridedGeom& g, const Twiddles& tw, u64 jl, u64 k) {
        const u64* t = INV ? g.twi : g.twf;
        if (t) return t[k * g.S + jl];
        return omega_n<INV>(tw, (g.N / g.M) * jl * k);
    }

    // inverse inter-pass twiddles w_M^-(jl k) of one phase-B item, k = RB ks + kr
    static GL_HD void inv_twiddles(const StridedGeom& g, const TilePos& tp, int it, const Twiddles& tw,
                                   u64* w) {
        int kr = it / C, c = it % C;
#pragma unroll
        for (int ks = 0; ks < RA; ks++) w[ks] = pass_twiddle<true>(g, tw, tp.jl0 + c, (u64)(RB * ks + kr));
    }

    // inv_b reading the tile from a [R][C] staging copy, with its twiddles given
    static GL_HD void inv_b_staged(const StridedGeom& g, const TilePos& tp, int it, const u64* st64,
                                   u64* sm, const u64* tws) {
        int kr = it / C, c = it % C;
        u64 w[RA];
#pragma unroll
        for (int ks = 0; ks < RA; ks++) w[ks] = gl::mul(st64[(RB * ks + kr) * C + c], tws[ks]);
        gl::dft<RA, true>(w);
#pragma unroll
        for (int j0 = 0; j0 < RA; j0++) sm[(kr * RA + j0) * C + c] = w[j0];
    }

    // inter-pass twiddles w_M^(jl k) of one phase-B item, k = RB ks + kr
    static GL_HD void twiddles(const StridedGeom& g, const TilePos& tp, int it, const Twiddles& tw,
                               u64* w) {
        int kr = it / C, c = it % C;
#pragma unroll
        for (int ks = 0; ks < RA; ks++) w[ks] = pass_twiddle<false>(g, tw, tp.jl0 + c, (u64)(RB * ks + kr));
    }

    // forward, step 2: length-RA DFT over j0, times the twiddles, store digit k = RB ks + kr
    static GL_HD void fwd_b(const StridedGeom& g, const TilePos& tp, int it, u64* buf,
                            const u64* sm, const u64* w) {
        int kr = it / C, c = it % C;
        u64 v[RA];
#pragma unroll
        for (int j0 = 0; j0 < RA; j0++) v[j0] = sm[(kr * RA + j0) * C + c];
        gl::dft<RA, false>(v);
#pragma unroll
        for (int ks = 0; ks < RA; ks++)
            buf[tp.base + c + g.S * (u64)(RB * ks + kr)] = gl::mul(v[ks], w[ks]);
    }

    // inverse, mirror of fwd_b
    static GL_HD void inv_b(const StridedGeom& g, const TilePos& tp, int it, const u64* buf, u64* sm,
                            const Twiddles& tw) {
        int kr = it / C, c = it % C;
        u64 w[RA];
#pragma unroll
        for (int ks = 0; ks < RA; ks++) {
            u64 k = RB * ks + kr;
            w[ks] = gl::mul(buf[tp.base + c + g.S * k], pass_twiddle<true>(g, tw, tp.jl0 + c, k));
        }
        gl::dft<RA, true>(w);
#pragma unroll
        for (int j0 = 0; j0 < RA; j0++) sm[(kr * RA + j0) * C + c] = w[j0];
    }

    // inverse, mirror of fwd_a; LAST keeps only positions < keep, as exact digits
    template <bool LAST>
    static GL_HD void inv_a(const StridedGeom& g, const TilePos& tp, int it, u64* buf,
                            const u64* sm, u64 keep) {
        int j0 = it / C, c = it % C;
        u64 v[RB];
#pragma unroll
        for (int kr = 0; kr < RB; kr++) v[kr] = sm[(kr * RA + j0) * C + c];
        gl::row_roots<R, true, RB, RA>(v, j0);
        gl::dft<RB, true>(v);
#pragma unroll
        for (int j1 = 0; j1 < RB; j1++) {
            u64 p = tp.base + c + g.S * (u64)(j0 + RA * j1);
            if (!LAST) buf[p] = v[j1];
            else if (p < keep) buf[p] = gl::canon(v[j1]);  // p stands for 0 inside the field
        }
    }
};

// ---------------------------------------------------------------------------
// contiguous 4096-element pass: 64 x 64 tile, element (r, c) at offset 64 r + c
// ---------------------------------------------------------------------------
// The contiguous pass's 64 x 64 tile in shared memory, rows padded to 65 words:
// a column access (one row across a warp's lanes) and a row access (one column
// across lanes, rows 65 words apart, 65 = 1 mod 16) both touch 16 distinct
// 8-byte bank slots per half-warp, and every address is affine in the loop
// index, so the per-access offsets fold into the load and store instructions.
constexpr int TILE_PITCH = 65;
constexpr int TILE_SM = 64 * TILE_PITCH;  // words
GL_HD int sidx(int r, int c) { return r * TILE_PITCH + c; }

struct Lane {
    int u;    // warp & 7: j0 or kr of the current step (uniform in a warp)
    int idx;  // 32 * (warp >> 3) + lane: the column (or row) this thread owns
};
GL_HD Lane lane_of(int t) { return Lane{(t >> 5) & 7, 32 * (t >> 8) + (t & 31)}; }

// F1: column c = idx, digits u + 8 j1: length-8 DFT, twiddle w_64^(u kr) -> smem row kr*8+u
template <bool PACK>
GL_HD void c_fwd_col_a(int t, const u64* src, const Digits& dig, u64 base, u64* sm) {
    Lane ln = lane_of(t);
    u64 v[8];
#pragma unroll
    for (int j1 = 0; j1 < 8; j1++) {
        int off = (ln.u + 8 * j1) * 64 + ln.idx;
        v[j1] = PACK ? digit_at(dig, base + off) : src[off];
    }
    gl::dft<8, false>(v);
    gl::RowRoots<64, false, 8, 8>::apply(v, ln.u);
#pragma unroll
    for (int kr = 0; kr < 8; kr++) sm[sidx(kr * 8 + ln.u, ln.idx)] = v[kr];
}

// F3: kr = u: length-8 DFT over j0, twiddle w_4096^(c k) with k = 8 ks + kr (regs only)
// (w4096: the w_4096 powers, or those powers times N^-1 to scale the result)
GL_HD void c_fwd_col_b_load(int t, const u64* sm, const u64* w4096, u64* v) {
    Lane ln = lane_of(t);
#pragma unroll
    for (int j0 = 0; j0 < 8; j0++) v[j0] = sm[sidx(ln.u * 8 + j0, ln.idx)];
    gl::dft<8, false>(v);
#pragma unroll
    for (int ks = 0; ks < 8; ks++) v[ks] = gl::mul(v[ks], w4096[ln.idx * (8 * ks + ln.u)]);
}
// F4: row k of the tile receives column c's output k
GL_HD void c_fwd_col_b_store(int t, u64* sm, const u64* v) {
    Lane ln = lane_of(t);
#pragma unroll
    for (int ks = 0; ks < 8; ks++) sm[sidx(8 * ks + ln.u, ln.idx)] = v[ks];
}
// F5: row r = idx, columns u + 8 j1: length-8 DFT, twiddle w_64^(u kr)
GL_HD void c_fwd_row_a_load(int t, const u64* sm, u64* v) {
    Lane ln = lane_of(t);
#pragma unroll
    for (int j1 = 0; j1 < 8; j1++) v[j1] = sm[sidx(ln.idx, ln.u + 8 * j1)];
    gl::dft<8, false>(v);
    gl::RowRoots<64, false, 8, 8>::apply(v, ln.u);
}
// F6
GL_HD void c_fwd_row_a_store(int t, u64* sm, const u64* v) {
    Lane ln = lane_of(t);
#pragma unroll
    for (int kr = 0; kr < 8; kr++) sm[sidx(ln.idx, kr * 8 + ln.u)] = v[kr];
}
// F7: kr = u: length-8 DFT over j0; v[ks] is the spectrum at (r, 8 ks + kr)
GL_HD void c_fwd_row_b_load(int t, const u64* sm, u64* v) {
    Lane ln = lane_of(t);
#pragma unroll
    for (int j0 = 0; j0 < 8; j0++) v[j0] = sm[sidx(ln.idx, ln.u * 8 + j0)];
    gl::dft<8, false>(v);
}

// I1: inverse of F7
GL_HD void c_inv_row_b_store(int t, u64* sm, u64* v) {
    Lane ln = lane_of(t);
    gl::dft<8, true>(v);
#pragma unroll
    for (int j0 = 0; j0 < 8; j0++) sm[sidx(ln.idx, ln.u * 8 + j0)] = v[j0];
}
// I2: inverse of F5 (j0 = u)
GL_HD void c_inv_row_a_load(int t, const u64* sm, u64* v) {
    Lane ln = lane_of(t);
#pragma unroll
    for (int kr = 0; kr < 8; kr++) v[kr] = sm[sidx(ln.idx, kr * 8 + ln.u)];
    gl::RowRoots<64, true, 8, 8>::apply(v, ln.u);
    gl::dft<8, true>(v);
}
// I3
GL_HD void c_inv_row_a_store(int t, u64* sm, const u64* v) {
    Lane ln = lane_of(t);
#pragma unroll
    for (int j1 = 0; j1 < 8; j1++) sm[sidx(ln.idx, ln.u + 8 * j1)] = v[j1];
}
// I4: inverse of F3 (kr = u)
GL_HD void c_inv_col_b_load(int t, const u64* sm, const Twiddles& tw, u64* v) {
    Lane ln = lane_of(t);
#pragma unroll
    for (int ks = 0; ks < 8; ks++)
        v[ks] = gl::mul(sm[sidx(8 * ks + ln.u, ln.idx)], tw.w4096i[ln.idx * (8 * ks + ln.u)]);
    gl::dft<8, true>(v);
}
// I5
GL_HD void c_inv_col_b_store(int t, u64* sm, const u64* v) {
    Lane ln = lane_of(t);
#pragma unroll
    for (int j0 = 0; j0 < 8; j0++) sm[sidx(ln.u * 8 + j0, ln.idx)] = v[j0];
}
// I6: inverse of F1 (j0 = u): rows u + 8 j1 of column c go back to global.
// LAST (the transform's last pass): only positions below keep, as exact
// digits; otherwise field values for the next inverse pass (p may stand for 0).
template <bool LAST>
GL_HD void c_inv_col_a(int t, const u64* sm, u64* dst, u64 base, u64 keep) {
    Lane ln = lane_of(t);
    u64 v[8];
#pragma unroll
    for (int kr = 0; kr < 8; kr++) v[kr] = sm[sidx(kr * 8 + ln.u, ln.idx)];
    gl::RowRoots<64, true, 8, 8>::apply(v, ln.u);
    gl::dft<8, true>(v);
#pragma unroll
    for (int j1 = 0; j1 < 8; j1++) {
        int off = (ln.u + 8 * j1) * 64 + ln.idx;
        if (!LAST) dst[off] = v[j1];
        else if (base + off < keep) dst[off] = gl::canon(v[j1]);
    }
}

}  // namespace pa
