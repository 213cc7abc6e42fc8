// Pieces of the split-BF16 MTTKRP pipeline shared by the single-instance kernel
// (mttkrp_tc.cu) and the batched kernel (mttkrp_tc_batched.cu): the tile configuration
// (shared-memory rings, TMEM accumulators, barrier counts), the chunk iterator of a
// CTA's units, the converters' per-thread global loads (rows that neither a tensor map
// nor the row-class maps serve), the weight tables and the weight-ring copy of a fiber
// group's Khatri-Rao weights.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"
#include "sm100.cuh"
#include "tc_common.cuh"

namespace deinsum {
namespace {

using namespace sm100;

constexpr int kFoldEvery = 64;  // fiber groups accumulated in registers before a flush

// Two MMAs per 16-k step with N = 2 RP (X_hi and X_lo against [U_hi; U_lo]) into an
// accumulator whose column r holds the U_hi products and column RP + r the U_lo products:
// all four split products, 8 MMAs per 64-k chunk.  Three products into one accumulator of
// RP columns (X_hi U_hi + X_hi U_lo + X_lo U_hi) halve the epilogue's TMEM reads but take a
// chain of 12 MMAs per chunk, which measured slower in both kernels (1024^3: 0.687 against
// 0.652 ms; the 512-instance batch: 4.97 against 4.80 ms, aligned instances 10 % slower).
// BATCHED: the persistent batched kernel's extra accumulators and ticket ring.
template <int RP, bool BATCHED = false> struct TcCfg {
    static constexpr int N = 2 * RP;                       // rows of the split factor tile: hi, then lo
    static constexpr int ACC = 2 * RP;                     // MMA N and accumulator columns
    static constexpr int RS = RP <= 32 ? 4 : 3;            // raw X stages
    static constexpr int AS = 2;                           // operand stages
    static constexpr int MMA_WARP = CONV_WARPS + EPI_WARPS;
    static constexpr int TMA_WARP = MMA_WARP + 1;
    static constexpr int WARPS = TMA_WARP + 1;
    static constexpr int THREADS = WARPS * 32;
    static constexpr int RAW_BYTES = BM * BK * 4;          // one box of the tensor map
    static constexpr int RAW_STAGE = kRcRawBytes;          // stage stride: also holds four class boxes
    static constexpr int A_BYTES = BM * BK * 2;            // one of hi / lo
    static constexpr int B_BYTES = N * BK * 2;
    static constexpr int ASTAGE_BYTES = 2 * A_BYTES + B_BYTES;
    // weight ring: one slot per fiber group in flight, holding its Ofac row
    // (RP floats) and then its L rows (one per p of the tile, at most GMAX)
    static constexpr int WSLOTS = 4;
    static constexpr int WSLOT_FLOATS = (DEINSUM_GMAX + 1) * RP;
    static constexpr int WBUF_BYTES = WSLOTS * WSLOT_FLOATS * 4;
    // TMEM accumulators in flight: four, so that short fiber groups (one or two chunks) do not
    // hold the MMAs up behind the epilogue
    static constexpr int NACC = 4;
    static constexpr int TMEM_COLS = NACC * ACC < 32 ? 32 : NACC * ACC;   // a power of two, >= 32
    static_assert(TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0, "TMEM allocation");
    // batched kernel: a ring of NQ unit tickets (the TMA thread takes each from the device
    // counter and hands it to the other roles: qfull / qempty)
    static constexpr int NQ = BATCHED ? 8 : 0;
    static constexpr int NBARS = 2 * RS + 3 * AS + 2 * NACC + 1 + 2 * WSLOTS + 2 * NQ;
    static constexpr size_t SMEM = size_t(RS) * RAW_STAGE + size_t(AS) * ASTAGE_BYTES + WBUF_BYTES + 1024 + 512;
    static_assert(SMEM <= 232448, "dynamic shared memory above the 227 KB per-CTA limit");
    static_assert(RAW_BYTES <= RAW_STAGE, "a tensor-map box fits a raw stage");
    static_assert(NBARS * 8 + 8 + NQ * 8 <= 512, "barrier area (+ TMEM holder, abort flag, ticket ring)");
};

// Product of the outer factors' entries at outer index o (row-major over the
// outer modes), column c.
__device__ __forceinline__ float outer_weight(const MttkrpArgs &a, int64_t o, int c) {
    float v = 1.f;
    for (int k = a.g.n_outer - 1; k >= 0; --k) {
        const int64_t d = a.g.outer_dim[k];
        const int64_t i = o % d;
        o /= d;
        v *= __ldg(static_cast<const float *>(a.U[a.g.outer_mode[k]]) + i * a.g.R + c);
    }
    return v;
}

// Product of the factors of modes 0..n-1 at p (row-major over those modes), column c.
__device__ __forceinline__ float row_weight(const MttkrpArgs &a, int64_t p, int c) {
    float v = 1.f;
    for (int k = a.g.n_lmodes - 1; k >= 0; --k) {
        const int64_t d = a.g.dims[k];
        const int64_t i = p % d;
        p /= d;
        v *= __ldg(static_cast<const float *>(a.U[k]) + i * a.g.R + c);
    }
    return v;
}

// Weight tables (one pass before the tensor-core kernel, so that its epilogue
// reads each fiber group's weights as whole rows, copied ahead by the TMA warp):
//   Lw[p, c] = row_weight(p, c)    (n_lmodes > 0), p < P
//   Ow[o, c] = outer_weight(o, c)  (n_outer > 0),  o < O
// for c < R_pad, zero for c >= R (the products in the same order as above).
__device__ __forceinline__ void weight_tables_body(const MttkrpArgs &a, int64_t t0, int64_t stride) {
    const MttkrpGeom &g = a.g;
    const int rp = g.R_pad;
    const int64_t nl = g.n_lmodes > 0 ? g.P * rp : 0;
    const int64_t no = g.n_outer > 0 ? g.O * rp : 0;
    for (int64_t t = t0; t < nl + no; t += stride) {
        if (t < nl) {
            const int64_t p = t / rp;
            const int c = int(t - p * rp);
            a.Lw[t] = c < g.R ? row_weight(a, p, c) : 0.f;
        } else {
            const int64_t u = t - nl;
            const int64_t o = u / rp;
            const int c = int(u - o * rp);
            a.Ow[u] = c < g.R ? outer_weight(a, o, c) : 0.f;
        }
    }
}

struct Iter {
    int64_t u, col, fg, fg1, tile, o;
    int seg, kb, kb_lo, kb_hi;   // kb: the chunk's index along the inner mode; [kb_lo, kb_hi): the group's
    bool done;
    __device__ __forceinline__ void set_fg(const MttkrpGeom &g) {
        const int64_t per_tile = g.O_iter * g.kseg;
        tile = fg / per_tile;
        const int64_t rem = fg - tile * per_tile;
        o = rem / g.kseg;
        seg = int(rem - o * g.kseg);
        kb_lo = seg * g.n_kb_seg;
        kb_hi = kb_lo + g.n_kb_seg < g.n_kb ? kb_lo + g.n_kb_seg : g.n_kb;
        kb = kb_lo;
    }
    __device__ __forceinline__ void load_unit(const MttkrpArgs &a) {
        while (u < a.n_units) {
            col = a.units[3 * u];
            fg = a.units[3 * u + 1];
            fg1 = a.units[3 * u + 2];
            if (fg < fg1) {
                set_fg(a.g);
                done = false;
                return;
            }
            u += gridDim.x;
        }
        done = true;
    }
    __device__ __forceinline__ void init(const MttkrpArgs &a) {
        u = blockIdx.x;
        load_unit(a);
    }
    // to the next fiber group
    __device__ __forceinline__ void next_fg(const MttkrpArgs &a) {
        if (++fg < fg1) {
            set_fg(a.g);
            return;
        }
        u += gridDim.x;
        load_unit(a);
    }
    // advance by one chunk
    __device__ __forceinline__ void next(const MttkrpArgs &a) {
        if (++kb < kb_hi) return;
        next_fg(a);
    }
};

// From global memory with per-element bounds checks (rows not 16-byte aligned).
template <bool OPACK>
__device__ __forceinline__ void conv_read_global(const MttkrpArgs &a, const Iter &it, int pt, float4 (&v)[8]) {
    const MttkrpGeom &g = a.g;
    const float *X = static_cast<const float *>(a.X);
    const int64_t k0 = int64_t(it.kb) * BK;
    if (OPACK && g.kcase == 0) {
        // row l = gq * I_n + i (P = 1): X[i, o0 + gq, k]
        const int k4 = pt & 15, rsub = pt >> 4;
        const int64_t kpos = k0 + 4 * k4;
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int l = rsub + 16 * j;
            float e[4] = {0.f, 0.f, 0.f, 0.f};
            if (opack_row_valid(g, it.tile, l)) {
                const int gq = l / int(g.I);
                const int64_t i = l - gq * int(g.I);
                const float *pr = X + i * g.Q + (it.tile * g.G + gq) * g.K_in + kpos;
                #pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (kpos + q < g.K_in) e[q] = __ldg(pr + q);
            }
            v[j] = make_float4(e[0], e[1], e[2], e[3]);
        }
    } else if (OPACK) {
        // case 1, row l = gq * I_n + i: X[o0 + gq, k, i]
        const int row = pt & (BM - 1), kh = pt >> 7;
        const bool rv = opack_row_valid(g, it.tile, row);
        const int gq = row / int(g.I);
        const int64_t i = row - gq * int(g.I);
        const int64_t kbase = k0 + 32 * kh;
        const float *base = X + ((it.tile * g.G + gq) * g.K_in + kbase) * g.I + i;
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
            float e[4];
            #pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int kk = 4 * j + q;
                e[q] = (rv && kbase + kk < g.K_in) ? __ldg(base + int64_t(kk) * g.I) : 0.f;
            }
            v[j] = make_float4(e[0], e[1], e[2], e[3]);
        }
    } else if (g.kcase == 0) {
        const int k4 = pt & 15, rsub = pt >> 4;
        const int64_t rowbase = tile_rowbase(g, it.col, it.tile);
        const int64_t kpos = k0 + 4 * k4;
        const float *p0 = X + (rowbase + rsub) * g.Q + it.o * g.K_in + kpos;
        const int64_t rstride = 16 * g.Q;
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
            float e[4] = {0.f, 0.f, 0.f, 0.f};
            if (row_valid(g, it.col, rowbase, rsub + 16 * j))
                #pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (kpos + q < g.K_in) e[q] = __ldg(p0 + j * rstride + q);
            v[j] = make_float4(e[0], e[1], e[2], e[3]);
        }
    } else {
        const int row = pt & (BM - 1), kh = pt >> 7;
        const bool rv = it.col * BM + row < g.I;
        const int64_t kbase = k0 + 32 * kh;
        const float *base = X + (it.o * g.K_in + kbase) * g.I + it.col * BM + row;
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
            float e[4];
            #pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int kk = 4 * j + q;
                e[q] = (rv && kbase + kk < g.K_in) ? __ldg(base + int64_t(kk) * g.I) : 0.f;
            }
            v[j] = make_float4(e[0], e[1], e[2], e[3]);
        }
    }
}

// Case 1 from global memory for the MN-major operand (the thread layout of
// conv_read_smem_mn): row m of the tile is i_n = col * 128 + m at outer index o,
// or with opack i_n = m - gq I_n at outer index tile * G + gq; X[o, k, i_n].
template <bool OPACK>
__device__ __forceinline__ void conv_read_global_mn(const MttkrpArgs &a, const Iter &it, int pt, float4 (&v)[8]) {
    const MttkrpGeom &g = a.g;
    const float *X = static_cast<const float *>(a.X);
    const int64_t kbase = int64_t(it.kb) * BK + 8 * (pt >> 5);
    const float *src[4];
    bool rv[4];
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int m = 4 * (pt & 31) + q;
        int64_t o, i;
        if (OPACK) {
            const int gq = m / int(g.I);
            i = m - gq * int(g.I);
            o = it.tile * g.G + gq;
            rv[q] = opack_row_valid(g, it.tile, m);
        } else {
            i = it.col * BM + m;
            o = it.o;
            rv[q] = i < g.I;
        }
        src[q] = X + (o * g.K_in + kbase) * g.I + i;
    }
    #pragma unroll
    for (int j = 0; j < 8; ++j) {
        const bool kv = kbase + j < g.K_in;
        float e[4];
        #pragma unroll
        for (int q = 0; q < 4; ++q) e[q] = (kv && rv[q]) ? __ldg(src[q] + int64_t(j) * g.I) : 0.f;
        v[j] = make_float4(e[0], e[1], e[2], e[3]);
    }
}

// Copy the weights of fiber group (tile, o) into a weight-ring slot (TMA warp,
// one thread): the row common to the tile at floats [0, rp), then one row per
// row group at [rp, ...) -- Ofac(o) and the L rows of the tile's p values, or,
// with opack, L(0) and the Ofac rows of the tile's outer indices -- completing
// on `bar` (a plain arrive when there are none).
__device__ __forceinline__ void load_fg_weights(const MttkrpGeom &g, const float *Lw, const float *Ow, int64_t tile,
                                                int64_t o, uint32_t dst, uint32_t bar) {
    const uint32_t rowb = uint32_t(g.R_pad) * 4u;
    if (g.opack) {
        const int64_t o0 = tile * g.G;
        const uint32_t no = uint32_t(g.O - o0 < g.G ? g.O - o0 : g.G);
        const uint32_t bytes = (g.n_lmodes > 0 ? rowb : 0u) + no * rowb;
        mbar_arrive_expect_tx(bar, bytes);
        if (g.n_lmodes > 0) bulk_g2s(dst, Lw, rowb, bar);
        bulk_g2s(dst + rowb, Ow + o0 * g.R_pad, no * rowb, bar);
        return;
    }
    uint32_t bytes = 0, nl = 0;
    int64_t p0 = 0;
    if (g.n_outer > 0) bytes += rowb;
    if (g.n_lmodes > 0) {
        p0 = g.narrow ? tile * g.G : tile;
        const int64_t rows = g.narrow ? (g.P - p0 < g.G ? g.P - p0 : g.G) : 1;
        nl = uint32_t(rows);
        bytes += nl * rowb;
    }
    if (bytes == 0) {
        mbar_arrive(bar);
        return;
    }
    mbar_arrive_expect_tx(bar, bytes);
    if (g.n_outer > 0) bulk_g2s(dst, Ow + o * g.R_pad, rowb, bar);
    if (nl) bulk_g2s(dst + rowb, Lw + p0 * g.R_pad, nl * rowb, bar);
}

}  // namespace
}  // namespace deinsum
