// Device pieces shared by the tensor-core kernels (MTTKRP, batched MTTKRP,
// fused TTMc): tile constants, the case-0 / case-1 row view of a 128 x 64
// chunk, and the converters that read a raw FP32 chunk and write its split
// BF16 hi / lo operand tiles in the 128-byte-swizzled K-major layout.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"
#include "sm100.cuh"

namespace deinsum {
namespace {

using namespace sm100;

constexpr int BM = DEINSUM_BM;
constexpr int BK = DEINSUM_BK;
constexpr int CONV_WARPS = 8;
constexpr int EPI_WARPS = 4;

// Case 0 rows of a tile: row l of tile t is the (p, i_n) pair with flat index
// rowbase + l in the P x I_n row space, where rowbase = t*G*I_n (narrow: the
// tile holds G consecutive p with all I_n rows) or t*I_n + col*128 (wide).
__device__ __forceinline__ int64_t tile_rowbase(const MttkrpGeom &g, int64_t col, int64_t t) {
    return g.narrow ? t * g.G * g.I : t * g.I + col * BM;
}
// opack tiles: row l = g * I_n + i_n of tile t holds outer index t*G + g (I_n <= 64,
// so the division is a 32-bit one).
__device__ __forceinline__ bool opack_row_valid(const MttkrpGeom &g, int64_t t, int l) {
    return l < int(g.G * g.I) && t * g.G + l / int(g.I) < g.O;
}
__device__ __forceinline__ bool row_valid(const MttkrpGeom &g, int64_t col, int64_t rowbase, int l) {
    if (g.kcase == 1) return col * BM + l < g.I;
    if (g.narrow) return l < g.G * g.I && rowbase + l < g.P * g.I;
    return col * BM + l < g.I;
}

// ---------------------------------------------------------------------------
// Converter inputs.  Each of the 256 converter threads owns 32 values of a chunk:
//   case 0: rows rsub + 16 j (j < 8), k = 4 k4 .. 4 k4 + 3   (pt = 16 rsub + k4)
//   case 1: row pt % 128, k = 32 (pt / 128) .. + 31
// ---------------------------------------------------------------------------

// From the raw tile the TMA wrote (out-of-bounds rows and k were zero-filled
// by the TMA; narrow rows beyond G*I_n, which the box does not cover, are zeroed here).
// OPACK: the tile packs outer indices (see MttkrpGeom::opack); a compile-time
// flag so that kernels without packing keep the plain case-1 read.
template <bool OPACK>
__device__ __forceinline__ void conv_read_smem_t(const MttkrpGeom &g, int pitch, const float *raw, int pt,
                                                 float4 (&v)[8]) {
    if (g.kcase == 0) {
        const int k4 = pt & 15, rsub = pt >> 4;
        const int nrows = g.narrow ? int(g.G * g.I) : BM;
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int row = rsub + 16 * j;
            v[j] = row < nrows ? *reinterpret_cast<const float4 *>(raw + row * BK + 4 * k4)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    } else if (!OPACK) {
        const int row = pt & (BM - 1), kh = pt >> 7;
        const bool rv = row < pitch;
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
            float e[4];
            #pragma unroll
            for (int q = 0; q < 4; ++q) e[q] = rv ? raw[(32 * kh + 4 * j + q) * pitch + row] : 0.f;
            v[j] = make_float4(e[0], e[1], e[2], e[3]);
        }
    } else {
        // opack: the box lands as [o][k][i] with G outer groups, tile row = gq * I_n + i
        const int row = pt & (BM - 1), kh = pt >> 7;
        const int gq = row / pitch, i = row - gq * pitch;
        const bool rv = gq < g.G;
        const float *rb = raw + gq * BK * pitch + i;
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
            float e[4];
            #pragma unroll
            for (int q = 0; q < 4; ++q) e[q] = rv ? rb[(32 * kh + 4 * j + q) * pitch] : 0.f;
            v[j] = make_float4(e[0], e[1], e[2], e[3]);
        }
    }
}

// Case 0 with a full 128-row tile (not narrow): plain float4 reads, rows 16 apart.
__device__ __forceinline__ void conv_read_smem_wide(const float *raw, int pt, float4 (&v)[8]) {
    const float4 *r = reinterpret_cast<const float4 *>(raw + (pt >> 4) * BK) + (pt & 15);
    #pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = r[j * (16 * BK / 4)];
}

// run-time choice (kernels that serve both kinds of tile)
__device__ __forceinline__ void conv_read_smem(const MttkrpGeom &g, int pitch, const float *raw, int pt,
                                               float4 (&v)[8]) {
    if (g.opack) conv_read_smem_t<true>(g, pitch, raw, pt, v);
    else conv_read_smem_t<false>(g, pitch, raw, pt, v);
}
__device__ __forceinline__ void conv_read_smem(const MttkrpArgs &a, const float *raw, int pt, float4 (&v)[8]) {
    conv_read_smem(a.g, a.raw_pitch, raw, pt, v);
}

// ---------------------------------------------------------------------------
// Case 1 with an MN-major A operand: the raw tile already runs along the tile
// rows for a fixed k, so the converters keep that order (no transpose).  The
// raw tile holds G groups (G = 1 without opack) of `pitch` rows: row
// m = gq * pitch + i at raw[gq * 64 * pitch + k * pitch + i]; rows past the
// groups read as zero.  Thread pt (warp w = pt / 32, lane) holds k = 8 w + j
// (j < 8) of rows 4 lane .. 4 lane + 3.  Its positions are fixed for a launch.
// ---------------------------------------------------------------------------
struct MnPos {
    int off[4];      // raw offsets of the four rows at k = 0
    uint32_t valid;  // bit q: row 4 lane + q is inside the groups
    bool vec;        // pitch % 4 == 0: the four rows are one aligned float4
    bool full;       // vec, and groups x pitch >= 128: every row of the tile is inside (same for all threads)
};
__device__ __forceinline__ MnPos mn_pos(int pitch, int groups, int pt) {
    MnPos p;
    p.valid = 0;
    p.vec = (pitch & 3) == 0;
    p.full = p.vec && groups * pitch >= BM;
    const int m0 = 4 * (pt & 31);
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int m = m0 + q, gq = m / pitch, i = m - gq * pitch;
        p.off[q] = gq * BK * pitch + i;
        if (gq < groups) p.valid |= 1u << q;
    }
    return p;
}
__device__ __forceinline__ void conv_read_smem_mn(const MnPos &p, int pitch, const float *raw, int pt,
                                                  float4 (&v)[8]) {
    const int kb0 = 8 * (pt >> 5);
    if (p.full) {
        // every row of the tile is inside a group: unconditional float4 reads
        const float *r = raw + p.off[0] + kb0 * pitch;
        #pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = *reinterpret_cast<const float4 *>(r + j * pitch);
    } else if (p.vec) {
        const bool rv = p.valid != 0;
        #pragma unroll
        for (int j = 0; j < 8; ++j)
            v[j] = rv ? *reinterpret_cast<const float4 *>(raw + p.off[0] + (kb0 + j) * pitch)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
            float e[4];
            #pragma unroll
            for (int q = 0; q < 4; ++q) e[q] = ((p.valid >> q) & 1u) ? raw[p.off[q] + (kb0 + j) * pitch] : 0.f;
            v[j] = make_float4(e[0], e[1], e[2], e[3]);
        }
    }
}
// The common case (one group of 128 rows: pitch 128, every row inside): plain
// float4 reads 512 bytes apart.
__device__ __forceinline__ void conv_read_smem_mn128(const float *raw, int pt, float4 (&v)[8]) {
    const float4 *r = reinterpret_cast<const float4 *>(raw + 8 * (pt >> 5) * BM) + (pt & 31);
    #pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = r[j * (BM / 4)];
}
// Split and store: lanes 0-15 fill one 128-byte k-row of the first 64-row atom,
// lanes 16-31 the same k-row of the second (two wavefronts per 8-byte store).
// The warp's eight k (one 8-k group) are one atom row each: offset = atom base
// + 128 j + 16 (c ^ j) + 8 (lane & 1), c the lane's 16-byte chunk.
__device__ __forceinline__ void conv_store_mn(int pt, uint32_t a_hi, uint32_t a_lo, const float4 (&v)[8]) {
    const int lane = pt & 31;
    const uint32_t base = uint32_t((pt >> 5) * 2 + (lane >> 4)) * 1024u + uint32_t(lane & 1) * 8u;
    const uint32_t c = uint32_t((lane & 15) >> 1);
    #pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t off = base + uint32_t(j) * 128u + ((c ^ uint32_t(j)) << 4);
        uint32_t h0, l0, h1, l1;
        split2(v[j].x, v[j].y, h0, l0);
        split2(v[j].z, v[j].w, h1, l1);
        sts64(a_hi + off, h0, h1);
        sts64(a_lo + off, l0, l1);
    }
}

// Split and store the thread's 32 values into the stage's A_hi / A_lo tiles.
__device__ __forceinline__ void conv_store(const MttkrpGeom &g, int pt, uint32_t a_hi, uint32_t a_lo,
                                           const float4 (&v)[8]) {
    if (g.kcase == 0) {
        // 16 lanes cover one 128-byte swizzled row: conflict-free 8-byte stores.  Rows
        // rsub + 16 j share row & 7, so sw128_offset(rsub + 16 j, 4 k4) = base + 2048 j.
        const int k4 = pt & 15, rsub = pt >> 4;
        const uint32_t base = uint32_t(rsub >> 3) * 1024u + uint32_t(rsub & 7) * 128u +
                              ((uint32_t((k4 >> 1) ^ (rsub & 7)) & 7u) << 4) + uint32_t(k4 & 1) * 8u;
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t off = base + 2048u * uint32_t(j);
            uint32_t h0, l0, h1, l1;
            split2(v[j].x, v[j].y, h0, l0);
            split2(v[j].z, v[j].w, h1, l1);
            sts64(a_hi + off, h0, h1);
            sts64(a_lo + off, l0, l1);
        }
    } else {
        // eight consecutive lanes hold eight consecutive rows: their 16-byte
        // stores land in distinct swizzled bank groups
        const int row = pt & (BM - 1), kh = pt >> 7;
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 x0 = v[2 * q], x1 = v[2 * q + 1];
            uint32_t h[4], lo[4];
            split2(x0.x, x0.y, h[0], lo[0]);
            split2(x0.z, x0.w, h[1], lo[1]);
            split2(x1.x, x1.y, h[2], lo[2]);
            split2(x1.z, x1.w, h[3], lo[3]);
            const uint32_t off = sw128_offset(uint32_t(row), uint32_t(32 * kh + 8 * q));
            sts128(a_hi + off, h[0], h[1], h[2], h[3]);
            sts128(a_lo + off, lo[0], lo[1], lo[2], lo[3]);
        }
    }
}

// ---------------------------------------------------------------------------
// Rows that are not 16-byte aligned: the row-class tensor maps (MTTKRP and TTMc)
// ---------------------------------------------------------------------------

// Raw tiles of rows that are not 16-byte aligned, loaded through the four row-class tensor
// maps (MttkrpArgs::xrow).  A chunk is four boxes, one per class c, each member row padded by
// 4 words so that the box can start at the 16-byte granule of the row's first element:
//   case 0: class c = rows of the tile with (global row) = c mod 4: 32 rows of BK + 4 words;
//           tile row l is row l / 4 of the box of class (rowbase + l) mod 4
//   case 1: class c = k lines with (o K_in + k) = c mod 4: 16 lines of BM + 4 words;
//           chunk line kl is line kl / 4 of the box of class (o K_in + k0 + kl) mod 4
// and a member's first element sits d words into its slot, d = its word address mod 4.
constexpr int kRcPitch0 = BK + 4, kRcRows0 = BM / 4;
constexpr int kRcPitch1 = BM + 4, kRcRows1 = BK / 4;
constexpr int kRcBox0 = kRcRows0 * kRcPitch0 * 4;   // bytes of one class box
constexpr int kRcBox1 = kRcRows1 * kRcPitch1 * 4;
constexpr int kRcRawBytes = 4 * kRcBox0;
static_assert(4 * kRcBox1 <= kRcRawBytes, "case-1 class boxes in a raw stage");
static_assert(kRcRawBytes % 1024 == 0 && kRcBox0 % 128 == 0 && kRcBox1 % 128 == 0, "box alignment");

__device__ __forceinline__ float4 lds128(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

// Words d .. d + 3 from the 16-byte aligned address `addr` on, d uniform across the warp (the
// switch does not diverge): one aligned load for d = 0, two otherwise.
__device__ __forceinline__ float4 lds_words(uint32_t addr, int d) {
    const float4 a = lds128(addr);
    if (d == 0) return a;
    const float4 b = lds128(addr + 16u);
    if (d == 1) return make_float4(a.y, a.z, a.w, b.x);
    if (d == 2) return make_float4(a.z, a.w, b.x, b.y);
    return make_float4(a.w, b.x, b.y, b.z);
}

__device__ __forceinline__ uint64_t word_index(const void *p) {
    return uint64_t(reinterpret_cast<uintptr_t>(p) >> 2);
}

// Converter thread -> rows for the row-class tiles of case 0: the two half-warps of warp w take
// rsub = (w mod 4) + 8 (w / 4) and rsub + 4, so that every row of a warp (rsub + 16 j) is in
// one class and starts at one word offset.  Returned in the packed form conv_store reads
// (16 rsub + k4); a bijection of 0..255.
__device__ __forceinline__ int rowcls_thread(int pt) {
    const int w = pt >> 5, h = (pt >> 4) & 1;
    return (((w & 3) + 8 * (w >> 2) + 4 * h) << 4) | (pt & 15);
}

// Case 0 from the four class boxes (thread layout: rows rsub + 16 j, k = 4 k4 .. + 3 with
// pt = 16 rsub + k4 from rowcls_thread).  Row rsub + 16 j is box row rsub / 4 + 4 j of class
// (rowbase + rsub) mod 4, and the class's word offset d is the same for the whole warp.
// Rows outside the tile and k >= K_in read as zero.
__device__ __forceinline__ void conv_read_rowcls(const MttkrpGeom &g, const void *X, int64_t col, int64_t tile,
                                                 int64_t o, int kb, const float *raw, int pt, float4 (&v)[8]) {
    const int k4 = pt & 15, rsub = pt >> 4;
    const int64_t rowbase = tile_rowbase(g, col, tile);
    const int64_t k0 = int64_t(kb) * BK;
    const uint64_t w0 = word_index(X) + uint64_t(rowbase + rsub) * uint64_t(g.Q) + uint64_t(o * g.K_in + k0);
    const int d = int(w0 & 3u);
    const int c = int(uint64_t(rowbase + rsub) & 3u);
    const uint32_t r = smem_u32(raw) + uint32_t(((c * kRcRows0 + (rsub >> 2)) * kRcPitch0 + 4 * k4) * 4);
    constexpr uint32_t JS = 4u * kRcPitch0 * 4u;   // bytes between box rows rsub / 4 + 4 j
    switch (d) {
        case 0:
            #pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = lds128(r + JS * j);
            break;
        case 1:
            #pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = lds_words(r + JS * j, 1);
            break;
        case 2:
            #pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = lds_words(r + JS * j, 2);
            break;
        default:
            #pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = lds_words(r + JS * j, 3);
            break;
    }
    // Values a box brings in beyond the tile's own elements need no mask here.  Past K_in
    // (the last chunk of a fiber group) they are the same row's next outer index, or zero
    // past the row's end (out of the class map), and the split factor tile is zero for
    // k >= K_in.  Past the tile's rows in a wide tile they are rows of the next leading index
    // (or zero past the tensor), which reach only TMEM lanes and partial rows that the
    // reduction never reads.  Narrow tiles do read every group's rows, so rows of leading
    // indices past P are cleared.  (X is assumed finite: a non-finite value times a zero
    // factor row would be NaN.)
    if (!g.narrow || rowbase + BM <= g.P * g.I) return;
    #pragma unroll
    for (int j = 0; j < 8; ++j)
        if (!row_valid(g, col, rowbase, rsub + 16 * j)) v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Case 0 from the four class boxes, one half row per thread, into a class-major A tile (the
// batched kernel's layout).  A row a holds tile row l = 4 (a mod 32) + a / 32: the rows of
// each residue l mod 4 form one 32-row block of A, a fixed permutation that the epilogue
// undoes (rowcls_tile_row), whatever the tile.  Warp w takes the residue e = w mod 4, i.e.
// class c = (rowbase + e) mod 4, whose box row b is tile row 4 b + e; lane b reads words
// 32 h .. 32 h + 31 of box row b (h = w / 4), so v[i] = words 32 h + 4 i .. + 3 of that row.
// A class's rows start at one word offset d within their 16-byte granule (the same for the
// warp): nine aligned 16-byte reads per half row (eight for d = 0), and the 68-word box pitch
// puts a warp's 32 rows on all banks.  Masking as in conv_read_rowcls.
__device__ __forceinline__ int rowcls_tile_row(int a) { return 4 * (a & 31) + (a >> 5); }
// Words D .. D + 31 from the 16-byte aligned address r on (nine aligned reads for D > 0).
template <int D>
__device__ __forceinline__ void half_row_read(uint32_t r, float4 (&v)[8]) {
    if constexpr (D == 0) {
        #pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = lds128(r + 16u * uint32_t(i));
    } else {
        float4 a0 = lds128(r);
        #pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 a1 = lds128(r + 16u * uint32_t(i + 1));
            if constexpr (D == 1) v[i] = make_float4(a0.y, a0.z, a0.w, a1.x);
            else if constexpr (D == 2) v[i] = make_float4(a0.z, a0.w, a1.x, a1.y);
            else v[i] = make_float4(a0.w, a1.x, a1.y, a1.z);
            a0 = a1;
        }
    }
}
__device__ __forceinline__ void conv_read_rowcls_half(const MttkrpGeom &g, const void *X, int64_t col,
                                                      int64_t tile, int64_t o, int kb, const float *raw, int pt,
                                                      float4 (&v)[8]) {
    const int w = pt >> 5, b = pt & 31;
    const int e = w & 3, h = w >> 2;
    const int64_t rowbase = tile_rowbase(g, col, tile);
    const int cls = int(uint64_t(rowbase + e) & 3u);
    const int64_t k0 = int64_t(kb) * BK;
    const uint64_t w0 = word_index(X) + uint64_t(rowbase + e) * uint64_t(g.Q) + uint64_t(o * g.K_in + k0);
    const int d = int(w0 & 3u);
    const uint32_t r = smem_u32(raw) + uint32_t(((cls * kRcRows0 + b) * kRcPitch0 + 32 * h) * 4);
    switch (d) {
        case 0: half_row_read<0>(r, v); break;
        case 1: half_row_read<1>(r, v); break;
        case 2: half_row_read<2>(r, v); break;
        default: half_row_read<3>(r, v); break;
    }
    if (!g.narrow || rowbase + BM <= g.P * g.I) return;
    if (!row_valid(g, col, rowbase, 4 * b + e)) {
        #pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}
// Split and store conv_read_rowcls_half's half rows: A row 32 e + b (the warp's 32 consecutive
// rows, all eight swizzle phases), k = 32 h .. 32 h + 31 = 16-byte chunks 4 h .. 4 h + 3 of the
// 128-byte-swizzled K-major row: four wavefronts per 512-byte warp store, the least possible.
__device__ __forceinline__ void conv_store_rowcls_half(int pt, uint32_t a_hi, uint32_t a_lo, const float4 (&v)[8]) {
    const int w = pt >> 5;
    const uint32_t arow = uint32_t(32 * (w & 3) + (pt & 31)), h = uint32_t(w >> 2);
    #pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t off = sw128_offset(arow, 32u * h + 8u * uint32_t(j));
        const float4 x0 = v[2 * j], x1 = v[2 * j + 1];
        uint32_t hi[4], lo[4];
        split2(x0.x, x0.y, hi[0], lo[0]);
        split2(x0.z, x0.w, hi[1], lo[1]);
        split2(x1.x, x1.y, hi[2], lo[2]);
        split2(x1.z, x1.w, hi[3], lo[3]);
        sts128(a_hi + off, hi[0], hi[1], hi[2], hi[3]);
        sts128(a_lo + off, lo[0], lo[1], lo[2], lo[3]);
    }
}

// Case 1 from the four class boxes.  Thread layout (warp w, lane): the warp holds the eight
// k lines kl = r + 4 (8 h + j), j < 8, of one residue r = w mod 4 (h = w / 4), rows
// m = 4 lane .. + 3 of each.  All of a warp's lines are members of one class, c = (L0 + r)
// mod 4 with L0 = o K_in + k0, so they start at one word offset d within their 16-byte
// granule: the offset is fixed for the chunk (one switch, as in case 0), and line kl is
// box line kl / 4 = 8 h + j of that class.  conv_store_mn_cls writes them.
__device__ __forceinline__ void conv_read_rowcls_mn(const MttkrpGeom &g, const void *X, int64_t col, int64_t o,
                                                    int kb, const float *raw, int pt, float4 (&v)[8]) {
    const int w = pt >> 5, lane = pt & 31;
    const int r = w & 3, h = w >> 2;
    const int64_t k0 = int64_t(kb) * BK;
    const uint64_t L0 = uint64_t(o * g.K_in + k0);
    const int c = int((L0 + uint64_t(r)) & 3u);
    const int d = int((word_index(X) + (L0 + uint64_t(r)) * uint64_t(g.I) + uint64_t(col * BM)) & 3u);
    const uint32_t p = smem_u32(raw) + uint32_t(((c * kRcRows1 + 8 * h) * kRcPitch1 + 4 * lane) * 4);
    constexpr uint32_t JS = kRcPitch1 * 4u;   // bytes between box lines
    switch (d) {
        case 0:
            #pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = lds128(p + JS * j);
            break;
        case 1:
            #pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = lds_words(p + JS * j, 1);
            break;
        case 2:
            #pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = lds_words(p + JS * j, 2);
            break;
        default:
            #pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = lds_words(p + JS * j, 3);
            break;
    }
    // No masks (as in conv_read_rowcls for wide tiles): lines past K_in belong to the next
    // outer index and meet the zero rows of the split factor tile; rows past I are zero past
    // the end of a line (out of the class map) and otherwise reach only TMEM lanes that the
    // reduction never reads.
}

// Split and store in the thread layout of conv_read_rowcls_mn: k line kl = r + 4 (8 h + j)
// of rows 4 lane .. + 3 goes to the MN-major tile at sw128_mn_offset(4 lane, kl) (8 bytes,
// hi and lo tiles).  Per store, lanes 0-15 fill one 128-byte k-row of the first 64-row atom
// and lanes 16-31 the same k-row of the second, as in conv_store_mn.
__device__ __forceinline__ void conv_store_mn_cls(int pt, uint32_t a_hi, uint32_t a_lo, const float4 (&v)[8]) {
    const int w = pt >> 5, lane = pt & 31;
    const uint32_t r = uint32_t(w & 3), h = uint32_t(w >> 2);
    const uint32_t cl = uint32_t((lane & 15) >> 1);
    const uint32_t base = uint32_t(lane >> 4) * 1024u + uint32_t(lane & 1) * 8u + h * 8192u;
    #pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t kr = r + 4u * uint32_t(j & 1);            // kl mod 8
        const uint32_t off = base + uint32_t(j >> 1) * 2048u + kr * 128u + ((cl ^ kr) << 4);
        uint32_t h0, l0, h1, l1;
        split2(v[j].x, v[j].y, h0, l0);
        split2(v[j].z, v[j].w, h1, l1);
        sts64(a_hi + off, h0, h1);
        sts64(a_lo + off, l0, l1);
    }
}

// One chunk through the row-class maps (one thread): the four boxes into raw stage `dst`.
// Box c starts at the class's first row (line) of the chunk and, along the row, at the chunk's
// first element rounded down to its 16-byte granule (a multiple of 4 words, as a tiled load
// requires); rows past the class's last member are zero-filled.
__device__ __forceinline__ void rowcls_load(const MttkrpGeom &g, const void *X, const CUtensorMap *xrow, int64_t col,
                                            int64_t tile, int64_t o, int kb, uint32_t dst, uint32_t bar) {
    const int64_t k0 = int64_t(kb) * BK;
    const uint64_t xw = word_index(X);
    if (g.kcase == 0) {
        mbar_arrive_expect_tx(bar, 4 * kRcBox0);
        const int64_t rowbase = tile_rowbase(g, col, tile);
        #pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t rc = rowbase + ((c - rowbase) & 3);        // first tile row of class c
            const uint64_t dc = (xw + uint64_t(c) * uint64_t(g.Q)) & 3u; // class offset in its granule
            const int64_t x = int64_t(dc) + o * g.K_in + k0;          // chunk start within the map row
            tma_load_2d(dst + uint32_t(c * kRcBox0), &xrow[c], int(x & ~int64_t(3)), int((rc - c) >> 2), bar);
        }
    } else {
        mbar_arrive_expect_tx(bar, 4 * kRcBox1);
        const int64_t L0 = o * g.K_in + k0;
        #pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t lc = L0 + ((c - L0) & 3);                  // first chunk line of class c
            tma_load_2d(dst + uint32_t(c * kRcBox1), &xrow[c], int(col * BM), int((lc - c) >> 2), bar);
        }
    }
}

}  // namespace
}  // namespace deinsum
