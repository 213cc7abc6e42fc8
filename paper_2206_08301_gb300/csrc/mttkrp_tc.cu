// Split-BF16 MTTKRP on the tcgen05 tensor cores (sm_103a).
//
// Same row view and schedule as the plain kernel (internal.h): per fiber
// group (tile of 128 rows, outer index o) the inner contraction
//   T[row, r] = sum_k X[row, k] U[k, r]
// runs on the tensor cores as split products with FP32 accumulation in TMEM,
// hi = bf16(x), lo = bf16(x - hi), X_hi / X_lo split on the fly into 128-row operand
// tiles and U_hi / U_lo the two halves (rows 0..R_pad-1, R_pad..2 R_pad-1) of the
// split factor tile:
//   single-instance kernel: X_hi [U_hi; U_lo] + X_lo [U_hi; U_lo] (N = 2 R_pad), so that
//     T[:, r] + T[:, R_pad + r] holds all four products;
//   batched kernel: X_hi U_hi + X_hi U_lo + X_lo U_hi into R_pad columns (the dropped
//     X_lo U_lo is below 2^-16 * 2^-16 of |x u| per term).
// The remaining Khatri-Rao
// factors are applied as per-row weights when a fiber group is folded into the
// row accumulator (fused KRP + TDOT, never materialising the Khatri-Rao rows in
// HBM -- schedule P2 of Sec. IV-E; Sec. II-A decomposition).
//
// Warp roles (one CTA per SM, persistent over units):
//   warps 0-7    converters: raw FP32 tile (smem) -> split -> 128B-swizzled K-major
//                A tiles; one thread also bulk-copies the split factor tile B.
//                With packed outer indices and rows that are not 16-byte aligned
//                they load X from global themselves.
//   warps 8-11   epilogue: TMEM -> registers, weight, accumulate, write partials.
//   warp 12      TMEM allocation and the single-thread MMA issue.
//   warp 13      TMA: tiled tensor loads of raw X tiles into a ring of RS stages
//                (rows not 16-byte aligned: four loads per chunk, one per row class).
// Rings: raw X (RS stages: raw_full / raw_empty), operand tiles (AS stages:
// a_full / bfull / a_empty), two TMEM accumulators (accf / acce).  Every wait
// is bounded (mbar_wait) and warp-uniform where a warp barrier follows.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

#include "internal.h"
#include "sm100.cuh"
#include "tc_common.cuh"

namespace deinsum {
namespace {

using namespace sm100;

constexpr int kFoldEvery = 64;  // fiber groups accumulated in registers before a flush

// THREE: three split products into one accumulator of RP columns (X_hi U_hi + X_hi U_lo +
// X_lo U_hi); otherwise two MMAs with N = 2 RP (X_hi and X_lo against [U_hi; U_lo]) into an
// accumulator whose column r holds the U_hi products and column RP + r the U_lo products,
// all four split products.  Three products halve the epilogue's TMEM reads, but one
// accumulator takes 12 dependent MMAs per 64-k chunk against 8, which measured slower
// wherever the MMAs keep pace with HBM (1024^3: 0.687 against 0.652 ms), so only the
// batched kernel, whose short fiber groups make the epilogue weigh more, uses them.
template <int RP, bool THREE = false> struct TcCfg {
    static constexpr int N = 2 * RP;                       // rows of the split factor tile: hi, then lo
    static constexpr int ACC = THREE ? RP : 2 * RP;        // MMA N and accumulator columns
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
    // TMEM accumulators in flight: two, or four for the batched kernel, whose short fiber
    // groups would otherwise hold the MMAs up behind the epilogue
    static constexpr int NACC = THREE ? 4 : 2;
    static constexpr int TMEM_COLS = NACC * ACC < 32 ? 32 : NACC * ACC;   // a power of two, >= 32
    static constexpr int NBARS = 2 * RS + 3 * AS + 2 * NACC + 1 + 2 * WSLOTS;
    static constexpr size_t SMEM = size_t(RS) * RAW_STAGE + size_t(AS) * ASTAGE_BYTES + WBUF_BYTES + 1024 + 512;
    static_assert(SMEM <= 232448, "dynamic shared memory above the 227 KB per-CTA limit");
    static_assert(RAW_BYTES <= RAW_STAGE, "a tensor-map box fits a raw stage");
    static_assert(NBARS * 8 + 8 <= 512, "barrier area");
};

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

__global__ void weight_tables_kernel(const __grid_constant__ MttkrpArgs a) {
    weight_tables_body(a, int64_t(blockIdx.x) * blockDim.x + threadIdx.x, int64_t(gridDim.x) * blockDim.x);
}

__global__ void batched_weight_tables_kernel(const MttkrpArgs *__restrict__ insts) {
    weight_tables_body(insts[blockIdx.y], int64_t(blockIdx.x) * blockDim.x + threadIdx.x,
                       int64_t(gridDim.x) * blockDim.x);
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

// OP: outer indices packed into the tile; MN: MN-major A operand (the last mode);
// PW: per-row weights (packed outer indices, or narrow tiles of several p with L rows).
// RC: X through the four row-class tensor maps (rows not 16-byte aligned); otherwise through
// the tensor map when a.use_tma, else per-thread loads.
// Registers: 128 per thread at most.  The launch check counts a block's warps rounded up
// to a multiple of four (14 -> 16), and 16 x 32 x 128 is the SM's 65,536; a 144-register
// build of this 448-thread kernel fails to launch.  The rank-64 instances with per-row
// weights (64 accumulators and a float4 weight row per thread in the epilogue) spill there.
template <int RP, bool OP, bool MN, bool PW, bool RC>
__global__ void __maxnreg__(128)
mttkrp_tc_kernel(const __grid_constant__ MttkrpArgs a) {
    static_assert(!OP || PW, "packed outer indices weight every row group");
    static_assert(!(OP && RC), "row classes are not used with packed outer indices");
    using C = TcCfg<RP>;
    constexpr int RS = C::RS, AS = C::AS;
    const MttkrpGeom &g = a.g;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *raw_base = smem;
    unsigned char *a_base = smem + RS * C::RAW_STAGE;
    float *wbuf = reinterpret_cast<float *>(a_base + AS * C::ASTAGE_BYTES);   // weight ring
    uint64_t *bars = reinterpret_cast<uint64_t *>(a_base + AS * C::ASTAGE_BYTES + C::WBUF_BYTES);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + C::NBARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
    const uint64_t wlim = a.wait_ns;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t raw_s = smem_u32(raw_base), a_s = smem_u32(a_base);
    auto raw_addr = [&](int s) { return raw_s + uint32_t(s) * C::RAW_STAGE; };
    auto a_hi = [&](int s) { return a_s + uint32_t(s) * C::ASTAGE_BYTES; };
    auto a_lo = [&](int s) { return a_s + uint32_t(s) * C::ASTAGE_BYTES + C::A_BYTES; };
    auto b_t = [&](int s) { return a_s + uint32_t(s) * C::ASTAGE_BYTES + 2 * C::A_BYTES; };
    auto raw_full = [&](int s) { return smem_u32(bars + s); };
    auto raw_empty = [&](int s) { return smem_u32(bars + RS + s); };
    auto a_full = [&](int s) { return smem_u32(bars + 2 * RS + s); };
    auto bfull = [&](int s) { return smem_u32(bars + 2 * RS + AS + s); };
    auto a_empty = [&](int s) { return smem_u32(bars + 2 * RS + 2 * AS + s); };
    constexpr int AB = 2 * RS + 3 * AS;   // accumulator barriers, then the drain, then the weight ring
    auto accf = [&](int b) { return smem_u32(bars + AB + b); };
    auto acce = [&](int b) { return smem_u32(bars + AB + C::NACC + b); };
    const uint32_t drain = smem_u32(bars + AB + 2 * C::NACC);
    auto wfull = [&](int s) { return smem_u32(bars + AB + 2 * C::NACC + 1 + s); };
    auto wempty = [&](int s) { return smem_u32(bars + AB + 2 * C::NACC + 1 + C::WSLOTS + s); };
    auto wslot_addr = [&](int s) { return smem_u32(wbuf) + uint32_t(s) * uint32_t(C::WSLOT_FLOATS) * 4u; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < RS; ++s) {
            mbar_init(raw_full(s), 1);
            mbar_init(raw_empty(s), CONV_WARPS);
        }
        for (int s = 0; s < AS; ++s) {
            mbar_init(a_full(s), CONV_WARPS);
            mbar_init(bfull(s), 1);
            mbar_init(a_empty(s), 1);
        }
        for (int b = 0; b < C::NACC; ++b) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), EPI_WARPS);
        }
        mbar_init(drain, 1);
        for (int s = 0; s < C::WSLOTS; ++s) {
            mbar_init(wfull(s), 1);
            mbar_init(wempty(s), EPI_WARPS);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == C::MMA_WARP) {
        tmem_alloc(smem_u32(tmem_holder), C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp < CONV_WARPS) {
        // ----------------------------------------------------------- converters
        const int pt = threadIdx.x;
        const bool issuer = (pt == 0);
        const char *bsrc = static_cast<const char *>(a.Bsplit);
        Iter it;
        it.init(a);
        const MnPos mp = mn_pos(a.raw_pitch > 0 ? a.raw_pitch : BM, OP ? int(g.G) : 1, pt);
        uint32_t bpar = 0, bused = 0;  // per operand stage: parity of the last B copy, copy issued
        for (int64_t chunk = 0; !it.done; ++chunk) {
            float4 v[8];
            const int rs = int(chunk % RS);
            if (RC || a.use_tma) {
                const uint32_t rj = uint32_t(chunk / RS);
                if (!__all_sync(0xffffffffu, mbar_wait(raw_full(rs), rj & 1u, abort_flag, a.status, wlim))) break;
                const float *raw = reinterpret_cast<const float *>(raw_base + size_t(rs) * C::RAW_STAGE);
                if (RC) {
                    if (MN) conv_read_rowcls_mn(g, a.X, it.col, it.o, it.kb, raw, pt, v);
                    else conv_read_rowcls(g, a.X, it.col, it.tile, it.o, it.kb, raw, rowcls_thread(pt), v);
                } else if (MN && !OP && a.raw_pitch == BM) conv_read_smem_mn128(raw, pt, v);
                else if (MN) conv_read_smem_mn(mp, a.raw_pitch, raw, pt, v);
                else if (!g.narrow || g.G * g.I == BM) conv_read_smem_wide(raw, pt, v);   // all 128 rows
                else conv_read_smem_t<OP>(a.g, a.raw_pitch, raw, pt, v);
                // hand the raw stage back to the TMA warp before the split, so that its next
                // load overlaps it: the proxy fence orders these generic reads before that
                // async-proxy write (an mbarrier release alone does not)
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(raw_empty(rs));
            } else if (MN) {
                conv_read_global_mn<OP>(a, it, pt, v);
            } else {
                conv_read_global<OP>(a, it, pt, v);
            }
            const int as = int(chunk % AS);
            const uint32_t aj = uint32_t(chunk / AS);
            if (!__all_sync(0xffffffffu, mbar_wait(a_empty(as), (aj & 1u) ^ 1u, abort_flag, a.status, wlim))) break;
            // with a single inner chunk (n_kb = 1) every chunk uses the same factor tile:
            // each operand stage copies it once and keeps it
            if (issuer && (g.n_kb != 1 || aj == 0)) {
                mbar_arrive_expect_tx(bfull(as), C::B_BYTES);
                bulk_g2s(b_t(as), bsrc + size_t(it.kb) * C::B_BYTES, C::B_BYTES, bfull(as));
                bpar = (bpar & ~(1u << as)) | ((aj & 1u) << as);
                bused |= 1u << as;
            }
            if (MN && RC) conv_store_mn_cls(pt, a_hi(as), a_lo(as), v);
            else if (MN) conv_store_mn(pt, a_hi(as), a_lo(as), v);
            else conv_store(g, RC ? rowcls_thread(pt) : pt, a_hi(as), a_lo(as), v);
            // the proxy fence orders this thread's A stores before the tensor-core reads
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(a_full(as));
            it.next(a);
        }
        if (issuer) {  // every bulk copy into this CTA's smem has landed before exit
            for (int s = 0; s < AS; ++s)
                if ((bused >> s) & 1u) mbar_drain(bfull(s), (bpar >> s) & 1u, a.status);
        }
    } else if (warp == C::TMA_WARP) {
        // ------------------------------------------------------------------ TMA
        // (also the weight ring: every fiber group's weight rows, whether or not X goes by TMA)
        if (lane == 0) {
            Iter it;
            it.init(a);
            // per raw stage / weight slot: a copy was issued into it, and that copy's parity
            uint32_t r_used = 0, r_par = 0, w_used = 0, w_par = 0;
            int64_t fgi = 0;
            for (int64_t chunk = 0; !it.done; ++chunk) {
                if (it.kb == it.kb_lo) {
                    const int ws = int(fgi % C::WSLOTS);
                    const uint32_t wj = uint32_t(fgi / C::WSLOTS);
                    if (!mbar_wait(wempty(ws), (wj & 1u) ^ 1u, abort_flag, a.status, wlim)) break;
                    load_fg_weights(a.g, a.Lw, a.Ow, it.tile, it.o, wslot_addr(ws), wfull(ws));
                    w_used |= 1u << ws;
                    w_par = (w_par & ~(1u << ws)) | ((wj & 1u) << ws);
                    ++fgi;
                }
                if (RC || a.use_tma) {
                    const int rs = int(chunk % RS);
                    const uint32_t rj = uint32_t(chunk / RS);
                    if (!mbar_wait(raw_empty(rs), (rj & 1u) ^ 1u, abort_flag, a.status, wlim)) break;
                    const int kc = it.kb * BK;
                    if (RC) {
                        rowcls_load(a.g, a.X, a.xrow, it.col, it.tile, it.o, it.kb, raw_addr(rs), raw_full(rs));
                    } else if (OP) {
                        mbar_arrive_expect_tx(raw_full(rs), a.box_bytes);
                        const int o0 = int(it.tile * g.G);
                        if (g.kcase == 0) tma_load_4d(raw_addr(rs), &a.xmap, kc, 0, o0, 0, raw_full(rs));
                        else tma_load_3d(raw_addr(rs), &a.xmap, 0, kc, o0, raw_full(rs));
                    } else if (g.kcase == 0) {
                        mbar_arrive_expect_tx(raw_full(rs), a.box_bytes);
                        const int c2 = g.narrow ? 0 : int(it.col * BM);
                        const int c3 = g.narrow ? int(it.tile * g.G) : int(it.tile);
                        tma_load_4d(raw_addr(rs), &a.xmap, kc, int(it.o), c2, c3, raw_full(rs));
                    } else {
                        mbar_arrive_expect_tx(raw_full(rs), a.box_bytes);
                        tma_load_3d(raw_addr(rs), &a.xmap, int(it.col * BM), kc, int(it.o), raw_full(rs));
                    }
                    r_used |= 1u << rs;
                    r_par = (r_par & ~(1u << rs)) | ((rj & 1u) << rs);
                }
                it.next(a);
            }
            // every copy issued into this CTA's shared memory has landed before exit, also
            // when a role gave up and left some of them unconsumed (a completed phase
            // returns at once)
            for (int s2 = 0; s2 < RS; ++s2)
                if ((r_used >> s2) & 1u) mbar_drain(raw_full(s2), (r_par >> s2) & 1u, a.status);
            for (int s2 = 0; s2 < C::WSLOTS; ++s2)
                if ((w_used >> s2) & 1u) mbar_drain(wfull(s2), (w_par >> s2) & 1u, a.status);
        }
        __syncwarp();
    } else if (warp == C::MMA_WARP) {
        // -------------------------------------------------------------- MMA issue
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16_f32(BM, C::ACC) | (MN ? kIdescAMnMajor : 0u);
            int64_t chunk = 0;
            Iter itm;   // this CTA's fiber groups, for their chunk counts
            itm.init(a);
            bool ok = true;
            for (int64_t fgi = 0; ok && !itm.done; ++fgi, itm.next_fg(a)) {
                const int nkb = itm.kb_hi - itm.kb_lo;
                const int b = int(fgi % C::NACC);
                const uint32_t jb = uint32_t(fgi / C::NACC);
                if (!mbar_wait(acce(b), (jb & 1u) ^ 1u, abort_flag, a.status, wlim)) { ok = false; break; }
                tc_fence_after();
                const uint32_t dcol = tmem + uint32_t(b * C::ACC);
                for (int kb = 0; kb < nkb; ++kb) {
                    const int s = int(chunk % AS);
                    const uint32_t j = uint32_t(chunk / AS);
                    if (!mbar_wait(a_full(s), j & 1u, abort_flag, a.status, wlim) ||
                        ((g.n_kb != 1 || j == 0) && !mbar_wait(bfull(s), j & 1u, abort_flag, a.status, wlim))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t dh = MN ? desc_mnmajor_sw128(a_hi(s), kMnAtomStride, kMnKGroupStride)
                                           : desc_kmajor_sw128(a_hi(s));
                    const uint64_t dl = MN ? desc_mnmajor_sw128(a_lo(s), kMnAtomStride, kMnKGroupStride)
                                           : desc_kmajor_sw128(a_lo(s));
                    const uint64_t db = desc_kmajor_sw128(b_t(s));   // [U_hi; U_lo]: N = 2 RP rows
                    #pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        // K = 16 per step: 32 bytes along a K-major row, two 8-k groups of an MN-major tile
                        const uint64_t adv = uint64_t(kk * 32) >> 4;
                        const uint64_t adv_a = MN ? uint64_t(kk * 2 * kMnKGroupStride) >> 4 : adv;
                        mma_bf16(dcol, dh + adv_a, db + adv, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                        mma_bf16(dcol, dl + adv_a, db + adv, idesc, 1u);
                    }
                    mma_commit(a_empty(s));
                    ++chunk;
                }
                if (!ok) break;
                mma_commit(accf(b));
            }
            // all issued MMAs have completed before TMEM is released
            mma_commit(drain);
            mbar_drain(drain, 0, a.status);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------- epilogue
        const int quad = warp & 3;                 // TMEM lanes 32*quad .. 32*quad+31
        const int l = quad * 32 + lane;            // tile row of this thread
        constexpr bool lane_weights = PW;          // per-row weights (the launcher's choice)
        const bool has_common = OP ? g.n_lmodes > 0 : g.n_outer > 0;   // a row common to the tile
        const int lg = g.narrow ? int(l / g.I) : 0;   // narrow: p offset of row l within its tile
        Iter it;
        it.init(a);
        int64_t fgi = 0;
        bool ok = true;
        while (ok && !it.done) {
            const int64_t u = it.u;
            const int64_t ucol = it.col;
            float *part = a.partial + (u * BM + l) * RP;   // this row's partial sums (thread-private)
            bool first_flush = true;
            float acc[RP];
            #pragma unroll
            for (int c = 0; c < RP; ++c) acc[c] = 0.f;
            // fold the register accumulator into the unit's partial row
            auto flush = [&]() {
                #pragma unroll
                for (int c = 0; c < RP; c += 4) {
                    float4 s = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
                    if (!first_flush) {
                        const float4 p = *reinterpret_cast<const float4 *>(part + c);
                        s.x += p.x; s.y += p.y; s.z += p.z; s.w += p.w;
                    }
                    *reinterpret_cast<float4 *>(part + c) = s;
                    acc[c] = acc[c + 1] = acc[c + 2] = acc[c + 3] = 0.f;
                }
                first_flush = false;
            };
            int64_t tile = -1;
            int folded = 0;
            bool rv = true;  // narrow tiles: this thread's row holds a valid (p, i_n)
            while (!it.done && it.u == u) {
                if (it.tile != tile) {
                    tile = it.tile;
                    if (lane_weights) rv = OP ? opack_row_valid(g, tile, l) : row_valid(g, ucol, tile_rowbase(g, ucol, tile), l);
                }
                // weights of this fiber group, from its ring slot (rows of R_pad floats, zero past R)
                const int ws = int(fgi % C::WSLOTS);
                const uint32_t wj = uint32_t(fgi / C::WSLOTS);
                if (!__all_sync(0xffffffffu, mbar_wait(wfull(ws), wj & 1u, abort_flag, a.status, wlim))) {
                    ok = false;
                    break;
                }
                const float *wsl = wbuf + ws * C::WSLOT_FLOATS;
                const float *lrow = wsl + RP * (1 + lg);   // narrow: L row of this thread's p
                const bool wl = !lane_weights && g.n_lmodes > 0;   // one L row for the whole tile
                const int b = int(fgi % C::NACC);
                const uint32_t jb = uint32_t(fgi / C::NACC);
                if (!__all_sync(0xffffffffu, mbar_wait(accf(b), jb & 1u, abort_flag, a.status, wlim))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem + (uint32_t(quad * 32) << 16) + uint32_t(b * C::ACC);
                #pragma unroll
                for (int c = 0; c < RP; c += 16) {
                    uint32_t t[16], tl[16];   // the U_hi and U_lo columns of rank columns c .. c + 15
                    tmem_ld16(taddr + uint32_t(c), t);
                    tmem_ld16(taddr + uint32_t(RP + c), tl);
                    tmem_wait_ld();
                    #pragma unroll
                    for (int q = 0; q < 16; ++q) t[q] = __float_as_uint(__uint_as_float(t[q]) + __uint_as_float(tl[q]));
                    #pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const int col = c + 4 * q4;
                        float4 w4;
                        if constexpr (PW) {
                            // per-row weights: this thread's row-group row (zero for an invalid
                            // row) times the row common to the tile
                            w4 = rv ? *reinterpret_cast<const float4 *>(lrow + col) : make_float4(0.f, 0.f, 0.f, 0.f);
                            if (has_common) {
                                const float4 cw = *reinterpret_cast<const float4 *>(wsl + col);
                                w4.x *= cw.x; w4.y *= cw.y; w4.z *= cw.z; w4.w *= cw.w;
                            }
                        } else {
                            // the same row for every thread (a broadcast read): Ofac(o), times L(p)
                            w4 = has_common ? *reinterpret_cast<const float4 *>(wsl + col) : make_float4(1.f, 1.f, 1.f, 1.f);
                            if (wl) {
                                const float4 lw = *reinterpret_cast<const float4 *>(wsl + RP + col);
                                w4.x *= lw.x; w4.y *= lw.y; w4.z *= lw.z; w4.w *= lw.w;
                            }
                        }
                        const int q = 4 * q4;
                        acc[col] = fmaf(w4.x, __uint_as_float(t[q]), acc[col]);
                        acc[col + 1] = fmaf(w4.y, __uint_as_float(t[q + 1]), acc[col + 1]);
                        acc[col + 2] = fmaf(w4.z, __uint_as_float(t[q + 2]), acc[col + 2]);
                        acc[col + 3] = fmaf(w4.w, __uint_as_float(t[q + 3]), acc[col + 3]);
                    }
                }
                tc_fence_before();
                fence_proxy_async_smem();   // the slot's reads before its next bulk-copy write
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(wempty(ws));
                    mbar_arrive(acce(b));
                }
                ++fgi;
                if (++folded == kFoldEvery) {
                    folded = 0;
                    flush();
                }
                it.next_fg(a);   // to the next fiber group
            }
            if (!ok) break;
            flush();
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == C::MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

// Inner factor -> split BF16 tiles: tile kb holds rows n < RP = hi(U[64 kb + k, n]),
// rows RP + n = lo(...), zero beyond R and beyond K_in, in the 128B-swizzled K-major layout.
// With Ub (a merged inner mode) the factor row k is the Khatri-Rao row
// U[k / Ib, n] * Ub[k % Ib, n], formed in FP32.
__global__ void split_inner_factor_kernel(const float *__restrict__ U, const float *__restrict__ Ub, int64_t Ib,
                                          unsigned char *__restrict__ out, int64_t K_in, int R, int RP, int n_kb) {
    const int64_t total = int64_t(n_kb) * 2 * RP * BK;
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int k = int(idx % BK);
        const int n = int((idx / BK) % (2 * RP));
        const int64_t kb = idx / (int64_t(BK) * 2 * RP);
        const int r = n % RP;
        const int64_t kr = kb * BK + k;
        float v = 0.f;
        if (r < R && kr < K_in) v = Ub ? U[(kr / Ib) * R + r] * Ub[(kr % Ib) * R + r] : U[kr * R + r];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 e = n < RP ? h : __float2bfloat16_rn(v - __bfloat162float(h));
        *reinterpret_cast<__nv_bfloat16 *>(out + size_t(kb) * (2 * RP * BK * 2) + sw128_offset(uint32_t(n), uint32_t(k))) = e;
    }
}

template <int RP, bool OP, bool MN, bool PW, bool RC = false>
int launch_tc_rp_op(const MttkrpArgs &a, int n_sm, void *stream) {
    using C = TcCfg<RP>;
    cudaError_t e = cudaFuncSetAttribute(mttkrp_tc_kernel<RP, OP, MN, PW, RC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM));
    if (e != cudaSuccess) return int(e);
    int64_t grid = a.n_units < n_sm ? a.n_units : n_sm;
    if (grid < 1) grid = 1;
    MttkrpArgs ka = a;
    ka.wait_ns = wait_limit_ns();
    mttkrp_tc_kernel<RP, OP, MN, PW, RC><<<unsigned(grid), C::THREADS, C::SMEM, static_cast<cudaStream_t>(stream)>>>(ka);
    count_launch();
    return int(cudaGetLastError());
}

// case 1 (rows contiguous in memory) takes the MN-major A operand; tiles whose row
// groups carry their own weights (packed outer indices, or several p with L rows)
// the per-row-weight epilogue
template <int RP>
int launch_tc_rp(const MttkrpArgs &a, int n_sm, void *stream) {
    const MttkrpGeom &g = a.g;
    if (a.row_classes && !a.use_tma && !g.opack) {   // rows not 16-byte aligned
        if (g.kcase == 1) return launch_tc_rp_op<RP, false, true, false, true>(a, n_sm, stream);
        if (g.narrow && g.n_lmodes > 0) return launch_tc_rp_op<RP, false, false, true, true>(a, n_sm, stream);
        return launch_tc_rp_op<RP, false, false, false, true>(a, n_sm, stream);
    }
    if (g.kcase == 1)
        return g.opack ? launch_tc_rp_op<RP, true, true, true>(a, n_sm, stream)
                       : launch_tc_rp_op<RP, false, true, false>(a, n_sm, stream);
    if (g.opack) return launch_tc_rp_op<RP, true, false, true>(a, n_sm, stream);
    if (g.narrow && g.n_lmodes > 0) return launch_tc_rp_op<RP, false, false, true>(a, n_sm, stream);
    return launch_tc_rp_op<RP, false, false, false>(a, n_sm, stream);
}

// ---------------------------------------------------------------------------
// Batched form: one persistent launch over the work units of every instance.
// Each CTA walks the unit list the host assigned to it (largest first over the
// CTAs, then grouped by how the unit's instance loads X); every unit names its
// instance, whose arguments sit in device memory.  Each role reads a unit's
// fields once and runs its chunks in code specialised for the instance's loads
// (tensor map or row classes, K-major or MN-major operand) and, in the epilogue,
// for its padded rank, so that all kinds of instance share one launch and one
// tail.  The MMAs take the three split products into one accumulator of R_pad
// columns (N = R_pad, a runtime field of the instruction descriptor).
// ---------------------------------------------------------------------------
constexpr int RPB = 64;  // the batched kernel is shaped for the largest padded rank

// How a unit's instance reaches the converters (from its arguments; uniform per unit).
enum BatchKind : int { BK_TMA_K = 0, BK_TMA_MN = 1, BK_RC_K = 2, BK_RC_MN = 3, BK_GL_K = 4, BK_GL_MN = 5 };
__device__ __forceinline__ int batch_kind(const MttkrpArgs &a) {
    const int mn = a.g.kcase == 1 ? 1 : 0;
    return a.row_classes ? BK_RC_K + mn : (a.use_tma ? BK_TMA_K + mn : BK_GL_K + mn);
}
template <int K> using KindTag = std::integral_constant<int, K>;

// The geometry fields the per-chunk code reads, copied once per unit from device memory
// (the other fields of the local copy are never read).  K-major kinds fix kcase = 0 at
// compile time, so the case-1 branches of the shared helpers drop out.
template <bool MN>
__device__ __forceinline__ void batch_geometry(MttkrpGeom &l, const MttkrpGeom &g) {
    l.kcase = MN ? 1 : 0;
    l.narrow = g.narrow;
    l.opack = 0;
    l.R = g.R;
    l.R_pad = g.R_pad;
    l.n_kb = g.n_kb;
    l.n_lmodes = g.n_lmodes;
    l.n_outer = g.n_outer;
    l.P = g.P;
    l.I = g.I;
    l.Q = g.Q;
    l.K_in = g.K_in;
    l.O = g.O;
    l.G = g.G;
    l.O_iter = g.O_iter;
}

__global__ void __maxnreg__(128)   // the launch limit of 448 threads: see mttkrp_tc_kernel
mttkrp_tc_batched_kernel(const __grid_constant__ BatchArgs bargs) {
    using C = TcCfg<RPB, true>;
    constexpr int RS = C::RS, AS = C::AS;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *raw_base = smem;
    unsigned char *a_base = smem + RS * C::RAW_STAGE;
    float *wbuf = reinterpret_cast<float *>(a_base + AS * C::ASTAGE_BYTES);   // weight ring
    uint64_t *bars = reinterpret_cast<uint64_t *>(a_base + AS * C::ASTAGE_BYTES + C::WBUF_BYTES);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + C::NBARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
    int *status = bargs.status;
    const uint64_t wlim = bargs.wait_ns;
    const int64_t ubeg = bargs.cta_begin[blockIdx.x], uend = bargs.cta_begin[blockIdx.x + 1];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t raw_s = smem_u32(raw_base), a_s = smem_u32(a_base);
    auto raw_addr = [&](int s) { return raw_s + uint32_t(s) * C::RAW_STAGE; };
    auto a_hi = [&](int s) { return a_s + uint32_t(s) * C::ASTAGE_BYTES; };
    auto a_lo = [&](int s) { return a_s + uint32_t(s) * C::ASTAGE_BYTES + C::A_BYTES; };
    auto b_t = [&](int s) { return a_s + uint32_t(s) * C::ASTAGE_BYTES + 2 * C::A_BYTES; };
    auto raw_full = [&](int s) { return smem_u32(bars + s); };
    auto raw_empty = [&](int s) { return smem_u32(bars + RS + s); };
    auto a_full = [&](int s) { return smem_u32(bars + 2 * RS + s); };
    auto bfull = [&](int s) { return smem_u32(bars + 2 * RS + AS + s); };
    auto a_empty = [&](int s) { return smem_u32(bars + 2 * RS + 2 * AS + s); };
    constexpr int AB = 2 * RS + 3 * AS;   // accumulator barriers, then the drain, then the weight ring
    auto accf = [&](int b) { return smem_u32(bars + AB + b); };
    auto acce = [&](int b) { return smem_u32(bars + AB + C::NACC + b); };
    const uint32_t drain = smem_u32(bars + AB + 2 * C::NACC);
    auto wfull = [&](int s) { return smem_u32(bars + AB + 2 * C::NACC + 1 + s); };
    auto wempty = [&](int s) { return smem_u32(bars + AB + 2 * C::NACC + 1 + C::WSLOTS + s); };
    auto wslot_addr = [&](int s) { return smem_u32(wbuf) + uint32_t(s) * uint32_t(C::WSLOT_FLOATS) * 4u; };
    // unit u: its instance's arguments and (column, first fiber group, end, partial offset)
    auto unit_args = [&](int64_t u) -> const MttkrpArgs & { return bargs.insts[bargs.units[5 * u]]; };
    auto unit_field = [&](int64_t u, int f) { return bargs.units[5 * u + f]; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < RS; ++s) {
            mbar_init(raw_full(s), 1);
            mbar_init(raw_empty(s), CONV_WARPS);
        }
        for (int s = 0; s < AS; ++s) {
            mbar_init(a_full(s), CONV_WARPS);
            mbar_init(bfull(s), 1);
            mbar_init(a_empty(s), 1);
        }
        for (int b = 0; b < C::NACC; ++b) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), EPI_WARPS);
        }
        mbar_init(drain, 1);
        for (int s = 0; s < C::WSLOTS; ++s) {
            mbar_init(wfull(s), 1);
            mbar_init(wempty(s), EPI_WARPS);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == C::MMA_WARP) {
        tmem_alloc(smem_u32(tmem_holder), C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp < CONV_WARPS) {
        // ----------------------------------------------------------- converters
        const int pt = threadIdx.x;
        const bool issuer = (pt == 0);
        uint32_t bpar = 0, bused = 0;      // per operand stage: parity of the last B copy, copy issued
        int64_t chunk = 0, tchunk = 0;     // operand-ring and raw-ring sequence numbers
        auto run = [&](auto kt, const MttkrpArgs &a, int64_t col, int64_t f0, int64_t f1) -> bool {
            constexpr int K = decltype(kt)::value;
            constexpr bool MN = (K & 1) != 0;
            constexpr bool RING = K < BK_GL_K;   // X through the raw ring (tensor map or row classes)
            MttkrpGeom g;
            batch_geometry<MN>(g, a.g);
            const void *X = a.X;
            const char *bsrc = static_cast<const char *>(a.Bsplit);
            const uint32_t bbytes = uint32_t(2 * g.R_pad * BK * 2);
            const int pitch = a.raw_pitch;
            const bool wide = !g.narrow || g.G * g.I == BM;
            MnPos mp;
            if constexpr (K == BK_TMA_MN) mp = mn_pos(pitch > 0 ? pitch : BM, 1, pt);
            for (int64_t fg = f0; fg < f1; ++fg) {
                const int64_t tile = fg / g.O_iter, o = fg - tile * g.O_iter;
                for (int kb = 0; kb < g.n_kb; ++kb, ++chunk) {
                    float4 v[8];
                    if constexpr (RING) {
                        const int rs = int(tchunk % RS);
                        const uint32_t rj = uint32_t(tchunk / RS);
                        ++tchunk;
                        if (!__all_sync(0xffffffffu, mbar_wait(raw_full(rs), rj & 1u, abort_flag, status, wlim)))
                            return false;
                        const float *raw = reinterpret_cast<const float *>(raw_base + size_t(rs) * C::RAW_STAGE);
                        if constexpr (K == BK_RC_MN) {
                            conv_read_rowcls_mn(g, X, col, o, kb, raw, pt, v);
                        } else if constexpr (K == BK_RC_K) {
                            conv_read_rowcls(g, X, col, tile, o, kb, raw, rowcls_thread(pt), v);
                        } else if constexpr (K == BK_TMA_MN) {
                            if (pitch == BM) conv_read_smem_mn128(raw, pt, v);
                            else conv_read_smem_mn(mp, pitch, raw, pt, v);
                        } else {
                            if (wide) conv_read_smem_wide(raw, pt, v);
                            else conv_read_smem_t<false>(g, pitch, raw, pt, v);
                        }
                        fence_proxy_async_smem();   // these generic reads before the stage's next TMA write
                        __syncwarp();
                        if (lane == 0) mbar_arrive(raw_empty(rs));
                    } else {
                        Iter it;
                        it.col = col;
                        it.tile = tile;
                        it.o = o;
                        it.kb = kb;
                        if constexpr (MN) conv_read_global_mn<false>(a, it, pt, v);
                        else conv_read_global<false>(a, it, pt, v);
                    }
                    const int as = int(chunk % AS);
                    const uint32_t aj = uint32_t(chunk / AS);
                    if (!__all_sync(0xffffffffu, mbar_wait(a_empty(as), (aj & 1u) ^ 1u, abort_flag, status, wlim)))
                        return false;
                    if (issuer) {
                        mbar_arrive_expect_tx(bfull(as), bbytes);
                        bulk_g2s(b_t(as), bsrc + size_t(kb) * bbytes, bbytes, bfull(as));
                        bpar = (bpar & ~(1u << as)) | ((aj & 1u) << as);
                        bused |= 1u << as;
                    }
                    if constexpr (K == BK_RC_MN) conv_store_mn_cls(pt, a_hi(as), a_lo(as), v);
                    else if constexpr (MN) conv_store_mn(pt, a_hi(as), a_lo(as), v);
                    else conv_store(g, K == BK_RC_K ? rowcls_thread(pt) : pt, a_hi(as), a_lo(as), v);
                    fence_proxy_async_smem();   // the A stores before the tensor-core reads
                    __syncwarp();
                    if (lane == 0) mbar_arrive(a_full(as));
                }
            }
            return true;
        };
        bool ok = true;
        for (int64_t u = ubeg; ok && u < uend; ++u) {
            const MttkrpArgs &a = unit_args(u);
            const int64_t col = unit_field(u, 1), f0 = unit_field(u, 2), f1 = unit_field(u, 3);
            switch (batch_kind(a)) {
                case BK_TMA_K: ok = run(KindTag<BK_TMA_K>{}, a, col, f0, f1); break;
                case BK_TMA_MN: ok = run(KindTag<BK_TMA_MN>{}, a, col, f0, f1); break;
                case BK_RC_K: ok = run(KindTag<BK_RC_K>{}, a, col, f0, f1); break;
                case BK_RC_MN: ok = run(KindTag<BK_RC_MN>{}, a, col, f0, f1); break;
                case BK_GL_K: ok = run(KindTag<BK_GL_K>{}, a, col, f0, f1); break;
                default: ok = run(KindTag<BK_GL_MN>{}, a, col, f0, f1); break;
            }
        }
        if (issuer) {  // every bulk copy into this CTA's smem has landed before exit
            for (int s = 0; s < AS; ++s)
                if ((bused >> s) & 1u) mbar_drain(bfull(s), (bpar >> s) & 1u, status);
        }
    } else if (warp == C::TMA_WARP) {
        // ------------------------------------------------------------------ TMA
        // (also the weight ring: every fiber group's weight rows, whether or not X goes by TMA)
        if (lane == 0) {
            uint32_t r_used = 0, r_par = 0, w_used = 0, w_par = 0;   // as in the single-instance kernel
            int64_t tchunk = 0, fgi = 0;
            const MttkrpArgs *fenced = nullptr;
            auto run = [&](auto kt, const MttkrpArgs &a, int64_t col, int64_t f0, int64_t f1) -> bool {
                constexpr int K = decltype(kt)::value;
                constexpr bool MN = (K & 1) != 0;
                constexpr bool RING = K < BK_GL_K;
                MttkrpGeom g;
                batch_geometry<MN>(g, a.g);
                const float *Lw = a.Lw, *Ow = a.Ow;
                const void *X = a.X;
                const uint32_t box_bytes = a.box_bytes;
                if (RING && fenced != &a) {   // the descriptors were written since the last launch
                    if constexpr (K == BK_RC_K || K == BK_RC_MN)
                        for (int c = 0; c < 4; ++c) fence_tensormap_acquire(&a.xrow[c]);
                    else
                        fence_tensormap_acquire(&a.xmap);
                    fenced = &a;
                }
                for (int64_t fg = f0; fg < f1; ++fg) {
                    const int64_t tile = fg / g.O_iter, o = fg - tile * g.O_iter;
                    const int ws = int(fgi % C::WSLOTS);
                    const uint32_t wj = uint32_t(fgi / C::WSLOTS);
                    if (!mbar_wait(wempty(ws), (wj & 1u) ^ 1u, abort_flag, status, wlim)) return false;
                    load_fg_weights(g, Lw, Ow, tile, o, wslot_addr(ws), wfull(ws));
                    w_used |= 1u << ws;
                    w_par = (w_par & ~(1u << ws)) | ((wj & 1u) << ws);
                    ++fgi;
                    if constexpr (RING) {
                        for (int kb = 0; kb < g.n_kb; ++kb) {
                            const int rs = int(tchunk % RS);
                            const uint32_t rj = uint32_t(tchunk / RS);
                            ++tchunk;
                            if (!mbar_wait(raw_empty(rs), (rj & 1u) ^ 1u, abort_flag, status, wlim)) return false;
                            const int kc = kb * BK;
                            if constexpr (K == BK_RC_K || K == BK_RC_MN) {
                                rowcls_load(g, X, a.xrow, col, tile, o, kb, raw_addr(rs), raw_full(rs));
                            } else if constexpr (K == BK_TMA_K) {
                                mbar_arrive_expect_tx(raw_full(rs), box_bytes);
                                const int c2 = g.narrow ? 0 : int(col * BM);
                                const int c3 = g.narrow ? int(tile * g.G) : int(tile);
                                tma_load_4d(raw_addr(rs), &a.xmap, kc, int(o), c2, c3, raw_full(rs));
                            } else {
                                mbar_arrive_expect_tx(raw_full(rs), box_bytes);
                                tma_load_3d(raw_addr(rs), &a.xmap, int(col * BM), kc, int(o), raw_full(rs));
                            }
                            r_used |= 1u << rs;
                            r_par = (r_par & ~(1u << rs)) | ((rj & 1u) << rs);
                        }
                    }
                }
                return true;
            };
            bool ok = true;
            for (int64_t u = ubeg; ok && u < uend; ++u) {
                const MttkrpArgs &a = unit_args(u);
                const int64_t col = unit_field(u, 1), f0 = unit_field(u, 2), f1 = unit_field(u, 3);
                switch (batch_kind(a)) {
                    case BK_TMA_K: ok = run(KindTag<BK_TMA_K>{}, a, col, f0, f1); break;
                    case BK_TMA_MN: ok = run(KindTag<BK_TMA_MN>{}, a, col, f0, f1); break;
                    case BK_RC_K: ok = run(KindTag<BK_RC_K>{}, a, col, f0, f1); break;
                    case BK_RC_MN: ok = run(KindTag<BK_RC_MN>{}, a, col, f0, f1); break;
                    case BK_GL_K: ok = run(KindTag<BK_GL_K>{}, a, col, f0, f1); break;
                    default: ok = run(KindTag<BK_GL_MN>{}, a, col, f0, f1); break;
                }
            }
            // every copy issued into this CTA's shared memory has landed before exit
            for (int s2 = 0; s2 < RS; ++s2)
                if ((r_used >> s2) & 1u) mbar_drain(raw_full(s2), (r_par >> s2) & 1u, status);
            for (int s2 = 0; s2 < C::WSLOTS; ++s2)
                if ((w_used >> s2) & 1u) mbar_drain(wfull(s2), (w_par >> s2) & 1u, status);
        }
        __syncwarp();
    } else if (warp == C::MMA_WARP) {
        // -------------------------------------------------------------- MMA issue
        if (lane == 0) {
            int64_t chunk = 0, fgi = 0;
            auto run = [&](auto mt, const MttkrpArgs &a, int64_t f0, int64_t f1) -> bool {
                constexpr bool MN = decltype(mt)::value != 0;   // the last mode: MN-major A
                const int n_kb = a.g.n_kb;
                const int rp = a.g.R_pad;
                const uint32_t idesc = idesc_bf16_f32(BM, rp) | (MN ? kIdescAMnMajor : 0u);
                const uint32_t blo = uint32_t(rp * 128);   // U_lo rows of the split factor tile
                for (int64_t fg = f0; fg < f1; ++fg, ++fgi) {
                    const int b = int(fgi % C::NACC);
                    const uint32_t jb = uint32_t(fgi / C::NACC);
                    if (!mbar_wait(acce(b), (jb & 1u) ^ 1u, abort_flag, status, wlim)) return false;
                    tc_fence_after();
                    const uint32_t dcol = tmem + uint32_t(b * C::ACC);
                    for (int kb = 0; kb < n_kb; ++kb, ++chunk) {
                        const int s = int(chunk % AS);
                        const uint32_t j = uint32_t(chunk / AS);
                        if (!mbar_wait(a_full(s), j & 1u, abort_flag, status, wlim) ||
                            !mbar_wait(bfull(s), j & 1u, abort_flag, status, wlim))
                            return false;
                        tc_fence_after();
                        const uint64_t dh = MN ? desc_mnmajor_sw128(a_hi(s), kMnAtomStride, kMnKGroupStride)
                                               : desc_kmajor_sw128(a_hi(s));
                        const uint64_t dl = MN ? desc_mnmajor_sw128(a_lo(s), kMnAtomStride, kMnKGroupStride)
                                               : desc_kmajor_sw128(a_lo(s));
                        const uint64_t db = desc_kmajor_sw128(b_t(s));
                        const uint64_t dbl = desc_kmajor_sw128(b_t(s) + blo);
                        #pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            const uint64_t adv = uint64_t(kk * 32) >> 4;
                            const uint64_t adv_a = MN ? uint64_t(kk * 2 * kMnKGroupStride) >> 4 : adv;
                            mma_bf16(dcol, dh + adv_a, db + adv, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                            mma_bf16(dcol, dh + adv_a, dbl + adv, idesc, 1u);
                            mma_bf16(dcol, dl + adv_a, db + adv, idesc, 1u);
                        }
                        mma_commit(a_empty(s));
                    }
                    mma_commit(accf(b));
                }
                return true;
            };
            bool ok = true;
            for (int64_t u = ubeg; ok && u < uend; ++u) {
                const MttkrpArgs &a = unit_args(u);
                const int64_t f0 = unit_field(u, 2), f1 = unit_field(u, 3);
                ok = a.g.kcase == 1 ? run(KindTag<1>{}, a, f0, f1) : run(KindTag<0>{}, a, f0, f1);
            }
            // all issued MMAs have completed before TMEM is released
            mma_commit(drain);
            mbar_drain(drain, 0, status);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------- epilogue
        const int quad = warp & 3;
        const int l = quad * 32 + lane;
        int64_t fgi = 0;
        auto run = [&](auto rt, const MttkrpArgs &a, int64_t col, int64_t f0, int64_t f1, int64_t part_off) -> bool {
            constexpr int RP = decltype(rt)::value;
            MttkrpGeom g;
            batch_geometry<false>(g, a.g);
            g.kcase = a.g.kcase;
            // per-row weights: narrow case-0 tiles of several p with L rows
            const bool lane_weights = g.kcase == 0 && g.narrow && g.n_lmodes > 0;
            const bool has_common = g.n_outer > 0;                 // a row common to the tile
            const bool wl = !lane_weights && g.n_lmodes > 0;       // one L row for the whole tile
            float *part = bargs.partial + part_off + int64_t(l) * RP;
            bool first_flush = true;
            float acc[RP];
            #pragma unroll
            for (int c = 0; c < RP; ++c) acc[c] = 0.f;
            auto flush = [&]() {
                #pragma unroll
                for (int c = 0; c < RP; c += 4) {
                    float4 sv = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
                    if (!first_flush) {
                        const float4 pv = *reinterpret_cast<const float4 *>(part + c);
                        sv.x += pv.x; sv.y += pv.y; sv.z += pv.z; sv.w += pv.w;
                    }
                    *reinterpret_cast<float4 *>(part + c) = sv;
                    acc[c] = acc[c + 1] = acc[c + 2] = acc[c + 3] = 0.f;
                }
                first_flush = false;
            };
            int64_t tile = -1;
            int folded = 0;
            bool rv = true;  // narrow tiles: this thread's row holds a valid (p, i_n)
            const int lg = g.narrow ? int(l / g.I) : 0;
            for (int64_t fg = f0; fg < f1; ++fg, ++fgi) {
                const int64_t t = fg / g.O_iter;
                if (t != tile) {
                    tile = t;
                    if (lane_weights) rv = row_valid(g, col, tile_rowbase(g, col, tile), l);
                }
                const int ws = int(fgi % C::WSLOTS);
                const uint32_t wj = uint32_t(fgi / C::WSLOTS);
                if (!__all_sync(0xffffffffu, mbar_wait(wfull(ws), wj & 1u, abort_flag, status, wlim))) return false;
                const float *wsl = wbuf + ws * C::WSLOT_FLOATS;
                const float *lrow = wsl + RP * (1 + lg);
                const int b = int(fgi % C::NACC);
                const uint32_t jb = uint32_t(fgi / C::NACC);
                if (!__all_sync(0xffffffffu, mbar_wait(accf(b), jb & 1u, abort_flag, status, wlim))) return false;
                tc_fence_after();
                const uint32_t taddr = tmem + (uint32_t(quad * 32) << 16) + uint32_t(b * C::ACC);
                #pragma unroll
                for (int c = 0; c < RP; c += 16) {
                    uint32_t tv[16];
                    tmem_ld16(taddr + uint32_t(c), tv);
                    tmem_wait_ld();
                    #pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const int cc = c + 4 * q4;
                        // weight rows are zero past R: no column mask
                        float4 w4 = has_common ? *reinterpret_cast<const float4 *>(wsl + cc)
                                               : make_float4(1.f, 1.f, 1.f, 1.f);
                        if (lane_weights || wl) {
                            const float4 lw = lane_weights
                                ? (rv ? *reinterpret_cast<const float4 *>(lrow + cc) : make_float4(0.f, 0.f, 0.f, 0.f))
                                : *reinterpret_cast<const float4 *>(wsl + RP + cc);
                            w4.x *= lw.x; w4.y *= lw.y; w4.z *= lw.z; w4.w *= lw.w;
                        }
                        const int q = 4 * q4;
                        acc[cc] = fmaf(w4.x, __uint_as_float(tv[q]), acc[cc]);
                        acc[cc + 1] = fmaf(w4.y, __uint_as_float(tv[q + 1]), acc[cc + 1]);
                        acc[cc + 2] = fmaf(w4.z, __uint_as_float(tv[q + 2]), acc[cc + 2]);
                        acc[cc + 3] = fmaf(w4.w, __uint_as_float(tv[q + 3]), acc[cc + 3]);
                    }
                }
                tc_fence_before();
                fence_proxy_async_smem();   // the slot's reads before its next bulk-copy write
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(wempty(ws));
                    mbar_arrive(acce(b));
                }
                if (++folded == kFoldEvery) {
                    folded = 0;
                    flush();
                }
            }
            flush();
            return true;
        };
        bool ok = true;
        for (int64_t u = ubeg; ok && u < uend; ++u) {
            const MttkrpArgs &a = unit_args(u);
            const int64_t col = unit_field(u, 1), f0 = unit_field(u, 2), f1 = unit_field(u, 3);
            const int64_t off = unit_field(u, 4);
            const int rp = a.g.R_pad;
            ok = rp == 16 ? run(KindTag<16>{}, a, col, f0, f1, off)
               : rp == 32 ? run(KindTag<32>{}, a, col, f0, f1, off)
                          : run(KindTag<64>{}, a, col, f0, f1, off);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == C::MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

}  // namespace

size_t mttkrp_tc_batched_smem_bytes() { return TcCfg<RPB, true>::SMEM; }

int launch_mttkrp_tc_batched(const BatchArgs &b, int grid, void *stream) {
    using C = TcCfg<RPB, true>;
    cudaError_t e = cudaFuncSetAttribute(mttkrp_tc_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(C::SMEM));
    if (e != cudaSuccess) return int(e);
    BatchArgs kb = b;
    kb.wait_ns = wait_limit_ns();
    mttkrp_tc_batched_kernel<<<unsigned(grid), C::THREADS, C::SMEM, static_cast<cudaStream_t>(stream)>>>(kb);
    count_launch();
    return int(cudaGetLastError());
}

size_t mttkrp_tc_smem_bytes(int R_pad) {
    switch (R_pad) {
        case 16: return TcCfg<16>::SMEM;
        case 32: return TcCfg<32>::SMEM;
        case 64: return TcCfg<64>::SMEM;
    }
    return 0;
}

int launch_split_inner_factor(const MttkrpArgs &a, void *bsplit, void *stream) {
    const MttkrpGeom &g = a.g;
    const int inner = g.kcase == 0 ? g.order - 1 : g.order - 2;
    const int64_t total = int64_t(g.n_kb) * 2 * g.R_pad * BK;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    split_inner_factor_kernel<<<unsigned(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const float *>(a.U[inner]), static_cast<const float *>(a.Uk2), a.K_minor > 0 ? a.K_minor : 1,
        static_cast<unsigned char *>(bsplit), g.K_in, g.R, g.R_pad, g.n_kb);
    count_launch();
    return int(cudaGetLastError());
}

int launch_weight_tables(const MttkrpArgs &a, void *stream) {
    const int64_t total = int64_t(weight_table_floats_l(a.g) + weight_table_floats_o(a.g));
    if (total == 0) return 0;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    weight_tables_kernel<<<unsigned(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(a);
    count_launch();
    return int(cudaGetLastError());
}

int launch_weight_tables_batched(const MttkrpArgs *insts, int n, int64_t max_floats, void *stream) {
    if (max_floats == 0) return 0;
    int64_t bx = (max_floats + 255) / 256;
    if (bx > 64) bx = 64;
    batched_weight_tables_kernel<<<dim3(unsigned(bx), unsigned(n)), 256, 0, static_cast<cudaStream_t>(stream)>>>(insts);
    count_launch();
    return int(cudaGetLastError());
}

int launch_mttkrp_tc(const MttkrpArgs &a, int n_sm, void *stream) {
    switch (a.g.R_pad) {
        case 16: return launch_tc_rp<16>(a, n_sm, stream);
        case 32: return launch_tc_rp<32>(a, n_sm, stream);
        case 64: return launch_tc_rp<64>(a, n_sm, stream);
    }
    return int(cudaErrorInvalidValue);
}

}  // namespace deinsum
