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

}  // namespace
}  // namespace deinsum
