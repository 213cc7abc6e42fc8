// Split-BF16 MTTKRP on the tcgen05 tensor cores (sm_103a).
//
// Same row view and schedule as the plain kernel (internal.h): per fiber
// group (tile of 128 rows, outer index o) the inner contraction
//   T[row, n] = sum_k A[row, k] * B[n, k]
// runs on the tensor cores with
//   A = [X_hi | X_lo]   (128 rows, split on the fly: hi = bf16(x), lo = bf16(x - hi))
//   B = [U_hi ; U_lo]   (2 R_pad rows: the inner factor's hi and lo parts)
// so that T[:, r] + T[:, R_pad + r] = (X_hi + X_lo)(U_hi + U_lo)[:, r]: the four
// split products with FP32 accumulation in TMEM.  The remaining Khatri-Rao
// factors are applied as per-row weights when a fiber group is folded into the
// row accumulator (fused KRP + TDOT, never materialising the Khatri-Rao rows in
// HBM -- schedule P2 of Sec. IV-E; Sec. II-A decomposition).
//
// Warp roles (one CTA per SM, persistent over units):
//   warps 0-7    producers: 128-bit streaming loads of X -> split -> 128B-swizzled
//                K-major smem tiles; one thread also bulk-copies the B tile.
//   warps 8..    epilogue: TMEM -> registers, weight, accumulate, write partials.
//   last warp    TMEM allocation and the single-thread MMA issue.
// Pipelines: STAGES smem stages (full/empty mbarriers) and two TMEM accumulators
// (acc-full/acc-empty mbarriers).  Every wait is bounded (mbar_wait).
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
constexpr int PRODUCER_WARPS = 8;
constexpr int EPI_WARPS = 4;
constexpr int kFoldEvery = 64;  // fiber groups accumulated in registers before a flush to smem
constexpr int kPrefetchAhead = 4;  // chunks of X bulk-prefetched into L2 ahead of the loads

template <int RP> struct TcCfg {
    static constexpr int N = 2 * RP;                       // MMA N: hi and lo columns of the factor
    static constexpr int STAGES = RP <= 32 ? 4 : 3;
    static constexpr int WARPS = PRODUCER_WARPS + EPI_WARPS + 1;
    static constexpr int THREADS = WARPS * 32;
    static constexpr int A_BYTES = BM * BK * 2;            // one of hi / lo
    static constexpr int B_BYTES = N * BK * 2;
    static constexpr int STAGE_BYTES = 2 * A_BYTES + B_BYTES;
    static constexpr int TMEM_COLS = 2 * N;                // two accumulators
    static constexpr int PRIV_BYTES = 2 * BM * RP * 4;     // per-row weights + flushed sums
    static constexpr size_t SMEM = size_t(STAGES) * STAGE_BYTES + PRIV_BYTES + 1024 + 256;
};

struct Iter {
    int64_t u, col, fg, fg1, tile, o;
    int kb;
    bool done;
    __device__ __forceinline__ void load_unit(const MttkrpArgs &a) {
        while (u < a.n_units) {
            col = a.units[3 * u];
            fg = a.units[3 * u + 1];
            fg1 = a.units[3 * u + 2];
            if (fg < fg1) {
                kb = 0;
                tile = fg / a.g.O;
                o = fg - tile * a.g.O;
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
    // advance by one chunk
    __device__ __forceinline__ void next(const MttkrpArgs &a) {
        if (++kb < a.g.n_kb) return;
        kb = 0;
        if (++fg < fg1) {
            if (++o == a.g.O) { o = 0; ++tile; }
            return;
        }
        u += gridDim.x;
        load_unit(a);
    }
};

// Case 0 rows of a tile: row l of tile t is the (p, i_n) pair with flat index
// rowbase + l in the P x I_n row space, where rowbase = t*G*I_n (narrow: the
// tile holds G consecutive p with all I_n rows) or t*I_n + col*128 (wide).
__device__ __forceinline__ int64_t tile_rowbase(const MttkrpGeom &g, int64_t col, int64_t t) {
    return g.narrow ? t * g.G * g.I : t * g.I + col * BM;
}
__device__ __forceinline__ bool row_valid(const MttkrpGeom &g, int64_t col, int64_t rowbase, int l) {
    if (g.kcase == 1) return col * BM + l < g.I;
    if (g.narrow) return l < g.G * g.I && rowbase + l < g.P * g.I;
    return col * BM + l < g.I;
}

// Load the 32 X values one producer thread owns in the chunk `it`.
//   case 0: rows rsub + 16 j (j < 8), elements k = 4 k4 .. 4 k4 + 3
//   case 1: row pt % 128, elements k = 32 (pt / 128) .. + 31
__device__ __forceinline__ void producer_load(const MttkrpArgs &a, const Iter &it, int pt, float4 (&v)[8]) {
    const MttkrpGeom &g = a.g;
    const float *X = static_cast<const float *>(a.X);
    const int64_t k0 = int64_t(it.kb) * BK;
    if (g.kcase == 0) {
        const int k4 = pt & 15, rsub = pt >> 4;
        const int64_t rowbase = tile_rowbase(g, it.col, it.tile);
        const int64_t kpos = k0 + 4 * k4;
        const float *p0 = X + (rowbase + rsub) * g.Q + it.o * g.K_in + kpos;
        const int64_t rstride = 16 * g.Q;
        if (g.vec_ok) {
            #pragma unroll
            for (int j = 0; j < 8; ++j)
                v[j] = (kpos < g.K_in && row_valid(g, it.col, rowbase, rsub + 16 * j))
                           ? ldg_stream4(p0 + j * rstride) : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            #pragma unroll
            for (int j = 0; j < 8; ++j) {
                float e[4] = {0.f, 0.f, 0.f, 0.f};
                if (row_valid(g, it.col, rowbase, rsub + 16 * j))
                    #pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (kpos + q < g.K_in) e[q] = __ldg(p0 + j * rstride + q);
                v[j] = make_float4(e[0], e[1], e[2], e[3]);
            }
        }
    } else {
        // one row per lane: a warp reads 32 consecutive rows (128 contiguous bytes) of one k
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
                e[q] = (rv && kbase + kk < g.K_in) ? ldg_stream1(base + int64_t(kk) * g.I) : 0.f;
            }
            v[j] = make_float4(e[0], e[1], e[2], e[3]);
        }
    }
}

// Bulk-prefetch into L2 the data kPrefetchAhead chunks after chunk `it` on the
// same rows.  A case-0 row is contiguous over all q = (o, k), and case-1 rows
// are contiguous over all p = (o, k), so that data sits a fixed distance
// further along: thread pt < 128 prefetches 64 elements of row pt (case 0);
// thread pt < 64 prefetches one 128-row slice (case 1).  Only with 16-byte
// aligned rows (vec_ok); a hint, bounded to the rows' extent.
__device__ __forceinline__ void producer_prefetch(const MttkrpArgs &a, const Iter &it, int pt) {
    const MttkrpGeom &g = a.g;
    if (!g.vec_ok) return;
    const float *X = static_cast<const float *>(a.X);
    const int64_t ahead = int64_t(kPrefetchAhead) * BK;
    if (g.kcase == 0) {
        if (pt >= BM) return;
        const int64_t rowbase = tile_rowbase(g, it.col, it.tile);
        const int64_t q = it.o * g.K_in + int64_t(it.kb) * BK + ahead;
        if (q >= g.Q || !row_valid(g, it.col, rowbase, pt)) return;
        const int64_t n = g.Q - q < BK ? g.Q - q : BK;
        prefetch_l2(X + (rowbase + pt) * g.Q + q, uint32_t(n * 4));
    } else {
        if (pt >= BK) return;
        const int64_t p = it.o * g.K_in + int64_t(it.kb) * BK + pt + ahead;
        if (p >= g.O * g.K_in) return;
        const int64_t r0 = it.col * BM;
        const int64_t n = g.I - r0 < BM ? g.I - r0 : BM;
        prefetch_l2(X + p * g.I + r0, uint32_t(n * 4));
    }
}

// Split and store the thread's 32 values into the stage's A_hi / A_lo tiles.
__device__ __forceinline__ void producer_store(const MttkrpGeom &g, int pt, uint32_t a_hi, uint32_t a_lo,
                                               const float4 (&v)[8]) {
    if (g.kcase == 0) {
        const int k4 = pt & 15, rsub = pt >> 4;
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t row = uint32_t(rsub + 16 * j);
            const uint32_t off = sw128_offset(row, uint32_t(4 * k4));
            uint32_t h0, l0, h1, l1;
            split2(v[j].x, v[j].y, h0, l0);
            split2(v[j].z, v[j].w, h1, l1);
            sts64(a_hi + off, h0, h1);
            sts64(a_lo + off, l0, l1);
        }
    } else {
        // row `row`, k = 32 kh .. 32 kh + 31: four 8-element groups; eight consecutive
        // lanes hold eight consecutive rows, so their 16-byte stores hit distinct banks
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

template <int RP>
__global__ void __launch_bounds__(TcCfg<RP>::THREADS, 1)
mttkrp_tc_kernel(const __grid_constant__ MttkrpArgs a) {
    using C = TcCfg<RP>;
    constexpr int STAGES = C::STAGES;
    const MttkrpGeom &g = a.g;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float *priv = reinterpret_cast<float *>(smem + STAGES * C::STAGE_BYTES);   // [2][RP][BM] thread-private
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * C::STAGE_BYTES + C::PRIV_BYTES);
    // bars: full[S], bfull[S], empty[S], accf[2], acce[2], drain
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 3 * STAGES + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = smem_u32(smem);
    auto a_hi = [&](int s) { return sbase + uint32_t(s) * C::STAGE_BYTES; };
    auto a_lo = [&](int s) { return sbase + uint32_t(s) * C::STAGE_BYTES + C::A_BYTES; };
    auto b_t = [&](int s) { return sbase + uint32_t(s) * C::STAGE_BYTES + 2 * C::A_BYTES; };
    auto full = [&](int s) { return smem_u32(bars + s); };
    auto bfull = [&](int s) { return smem_u32(bars + STAGES + s); };
    auto empty = [&](int s) { return smem_u32(bars + 2 * STAGES + s); };
    auto accf = [&](int b) { return smem_u32(bars + 3 * STAGES + b); };
    auto acce = [&](int b) { return smem_u32(bars + 3 * STAGES + 2 + b); };
    const uint32_t drain = smem_u32(bars + 3 * STAGES + 4);

    const int mma_warp = C::WARPS - 1;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full(s), PRODUCER_WARPS);
            mbar_init(bfull(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), EPI_WARPS);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == mma_warp) {
        tmem_alloc(smem_u32(tmem_holder), C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp < PRODUCER_WARPS) {
        // ------------------------------------------------------------ producers
        const int pt = threadIdx.x;
        const bool issuer = (pt == 0);
        const char *bsrc = static_cast<const char *>(a.Bsplit);
        Iter it;
        it.init(a);
        float4 va[8], vb[8];
        uint32_t bpar_issued = 0;  // bit s: parity of the last copy issued on stage s
        uint32_t bused = 0;        // bit s: a copy was issued on stage s
        int64_t chunk = 0;
        bool ok = true;
        if (!it.done) producer_load(a, it, pt, va);
        auto body = [&](float4 (&cur)[8], float4 (&nxt)[8]) -> bool {
            Iter nx = it;
            nx.next(a);
            if (!nx.done) {
                producer_load(a, nx, pt, nxt);
                producer_prefetch(a, nx, pt);
            }
            const int s = int(chunk % STAGES);
            const uint32_t j = uint32_t(chunk / STAGES);
            // warp-uniform outcome, so that no lane is left behind at a warp barrier
            if (!__all_sync(0xffffffffu, mbar_wait(empty(s), (j & 1u) ^ 1u, abort_flag, a.status))) return false;
            if (issuer) {
                mbar_arrive_expect_tx(bfull(s), C::B_BYTES);
                bulk_g2s(b_t(s), bsrc + size_t(it.kb) * C::B_BYTES, C::B_BYTES, bfull(s));
                bpar_issued = (bpar_issued & ~(1u << s)) | ((j & 1u) << s);
                bused |= 1u << s;
            }
            producer_store(g, pt, a_hi(s), a_lo(s), cur);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(full(s));
            it = nx;
            ++chunk;
            return true;
        };
        while (ok && !it.done) {
            ok = body(va, vb);
            if (!ok || it.done) break;
            ok = body(vb, va);
        }
        if (issuer) {  // every bulk copy into this CTA's smem has landed before exit
            for (int s = 0; s < STAGES; ++s)
                if ((bused >> s) & 1u) mbar_wait(bfull(s), (bpar_issued >> s) & 1u, abort_flag, a.status);
        }
    } else if (warp == mma_warp) {
        // -------------------------------------------------------------- MMA issue
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16_f32(BM, C::N);
            int64_t chunk = 0, fgi = 0, nfg = 0;
            {   // count the fiber groups of this CTA
                Iter it;
                it.init(a);
                while (!it.done) {
                    nfg += it.fg1 - it.fg;
                    it.u += gridDim.x;
                    it.load_unit(a);
                }
            }
            bool ok = true;
            for (fgi = 0; ok && fgi < nfg; ++fgi) {
                const int b = int(fgi & 1);
                const uint32_t jb = uint32_t(fgi >> 1);
                if (!mbar_wait(acce(b), (jb & 1u) ^ 1u, abort_flag, a.status)) { ok = false; break; }
                tc_fence_after();
                const uint32_t dcol = tmem + uint32_t(b * C::N);
                for (int kb = 0; kb < g.n_kb; ++kb) {
                    const int s = int(chunk % STAGES);
                    const uint32_t j = uint32_t(chunk / STAGES);
                    if (!mbar_wait(full(s), j & 1u, abort_flag, a.status) ||
                        !mbar_wait(bfull(s), j & 1u, abort_flag, a.status)) { ok = false; break; }
                    tc_fence_after();
                    const uint64_t dh = desc_kmajor_sw128(a_hi(s));
                    const uint64_t dl = desc_kmajor_sw128(a_lo(s));
                    const uint64_t db = desc_kmajor_sw128(b_t(s));
                    #pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint64_t adv = uint64_t(kk * 32) >> 4;  // 32 bytes per K=16 step
                        mma_bf16(dcol, dh + adv, db + adv, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                        mma_bf16(dcol, dl + adv, db + adv, idesc, 1u);
                    }
                    mma_commit(empty(s));
                    ++chunk;
                }
                if (!ok) break;
                mma_commit(accf(b));
            }
            // all issued MMAs have completed before TMEM is released
            mma_commit(drain);
            mbar_wait(drain, 0, abort_flag, a.status);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------- epilogue
        const int quad = warp & 3;                 // TMEM lanes 32*quad .. 32*quad+31
        const int l = quad * 32 + lane;            // tile row of this thread
        float *Lrow = priv;                        // [RP][BM]: per-row weights (narrow tiles)
        float *Sout = priv + RP * BM;              // [RP][BM]: flushed sums
        const bool lane_weights = g.kcase == 0 && g.narrow && g.n_lmodes > 0;
        Iter it;
        it.init(a);
        int64_t fgi = 0;
        bool ok = true;
        while (ok && !it.done) {
            const int64_t u = it.u;
            const int64_t ucol = it.col;
            float acc[RP];
            #pragma unroll
            for (int c = 0; c < RP; ++c) { acc[c] = 0.f; Sout[c * BM + l] = 0.f; }
            int64_t tile = -1;
            int folded = 0;
            float lw_lane0 = 0.f, lw_lane1 = 0.f;  // lane-independent row weights (wide tiles), columns lane, lane+32
            while (!it.done && it.u == u) {
                const int64_t rowbase = g.kcase == 0 ? tile_rowbase(g, ucol, it.tile) : 0;
                if (it.tile != tile) {
                    tile = it.tile;
                    if (lane_weights) {
                        // narrow tile: row l belongs to p = tile*G + l / I_n
                        lw_lane0 = 1.f;
                        lw_lane1 = 1.f;
                        const bool v = row_valid(g, ucol, rowbase, l);
                        const int64_t p = tile * g.G + l / g.I;
                        #pragma unroll 4
                        for (int c = 0; c < RP; ++c)
                            Lrow[c * BM + l] = (v && c < g.R) ? row_weight(a, p, c) : 0.f;
                    } else if (g.kcase == 0 && g.n_lmodes > 0) {
                        lw_lane0 = lane < g.R ? row_weight(a, tile, lane) : 0.f;
                        if (RP > 32) lw_lane1 = lane + 32 < g.R ? row_weight(a, tile, lane + 32) : 0.f;
                    } else {
                        lw_lane0 = 1.f;
                        lw_lane1 = 1.f;
                    }
                }
                // weights of this fiber group: lane c holds column c (and c + 32)
                const float w0 = lane < g.R ? lw_lane0 * outer_weight(a, it.o, lane) : 0.f;
                const float w1 = (RP > 32 && lane + 32 < g.R) ? lw_lane1 * outer_weight(a, it.o, lane + 32) : 0.f;
                const int b = int(fgi & 1);
                const uint32_t jb = uint32_t(fgi >> 1);
                if (!__all_sync(0xffffffffu, mbar_wait(accf(b), jb & 1u, abort_flag, a.status))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem + (uint32_t(quad * 32) << 16) + uint32_t(b * C::N);
                #pragma unroll
                for (int c = 0; c < RP; c += 16) {
                    uint32_t hi[16], lo[16];
                    tmem_ld16(taddr + uint32_t(c), hi);
                    tmem_ld16(taddr + uint32_t(RP + c), lo);
                    tmem_wait_ld();
                    #pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int col = c + q;
                        float w = __shfl_sync(0xffffffffu, col < 32 ? w0 : w1, col & 31);
                        if (lane_weights) w *= Lrow[col * BM + l];
                        acc[col] = fmaf(w, __uint_as_float(hi[q]) + __uint_as_float(lo[q]), acc[col]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce(b));
                ++fgi;
                if (++folded == kFoldEvery) {
                    folded = 0;
                    #pragma unroll
                    for (int c = 0; c < RP; ++c) { Sout[c * BM + l] += acc[c]; acc[c] = 0.f; }
                }
                for (int kb = 0; kb < g.n_kb; ++kb) it.next(a);  // to the next fiber group
            }
            if (!ok) break;
            float *part = a.partial + (u * BM + l) * RP;
            #pragma unroll
            for (int c = 0; c < RP; c += 4)
                *reinterpret_cast<float4 *>(part + c) =
                    make_float4(Sout[c * BM + l] + acc[c], Sout[(c + 1) * BM + l] + acc[c + 1],
                                Sout[(c + 2) * BM + l] + acc[c + 2], Sout[(c + 3) * BM + l] + acc[c + 3]);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == mma_warp) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

// Inner factor -> split BF16 tiles: tile kb holds rows n < RP = hi(U[64 kb + k, n]),
// rows RP + n = lo(...), zero beyond R and beyond K_in, in the 128B-swizzled K-major layout.
__global__ void split_inner_factor_kernel(const float *__restrict__ U, unsigned char *__restrict__ out,
                                          int64_t K_in, int R, int RP, int n_kb) {
    const int64_t total = int64_t(n_kb) * 2 * RP * BK;
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int k = int(idx % BK);
        const int n = int((idx / BK) % (2 * RP));
        const int64_t kb = idx / (int64_t(BK) * 2 * RP);
        const int r = n % RP;
        const int64_t kr = kb * BK + k;
        const float v = (r < R && kr < K_in) ? U[kr * R + r] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 e = n < RP ? h : __float2bfloat16_rn(v - __bfloat162float(h));
        *reinterpret_cast<__nv_bfloat16 *>(out + size_t(kb) * (2 * RP * BK * 2) + sw128_offset(uint32_t(n), uint32_t(k))) = e;
    }
}

template <int RP>
int launch_tc_rp(const MttkrpArgs &a, int n_sm, void *stream) {
    using C = TcCfg<RP>;
    cudaError_t e = cudaFuncSetAttribute(mttkrp_tc_kernel<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(C::SMEM));
    if (e != cudaSuccess) return int(e);
    int64_t grid = a.n_units < n_sm ? a.n_units : n_sm;
    if (grid < 1) grid = 1;
    mttkrp_tc_kernel<RP><<<unsigned(grid), C::THREADS, C::SMEM, static_cast<cudaStream_t>(stream)>>>(a);
    count_launch();
    return int(cudaGetLastError());
}

}  // namespace

size_t mttkrp_tc_smem_bytes(int R_pad) {  // NOLINT
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
        static_cast<const float *>(a.U[inner]), static_cast<unsigned char *>(bsplit), g.K_in, g.R, g.R_pad, g.n_kb);
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
