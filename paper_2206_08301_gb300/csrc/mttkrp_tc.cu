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
//   batched kernel (mttkrp_tc_batched.cu): X_hi U_hi + X_hi U_lo + X_lo U_hi into R_pad
//     columns (the dropped X_lo U_lo is below 2^-16 * 2^-16 of |x u| per term).
// The remaining Khatri-Rao factors are applied as per-row weights when a fiber group is folded into the
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
// a_full / bfull / a_empty), TMEM accumulators (accf / acce; TcCfg in mttkrp_tc.cuh).  Every wait
// is bounded (mbar_wait) and warp-uniform where a warp barrier follows.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"
#include "sm100.cuh"
#include "tc_common.cuh"
#include "mttkrp_tc.cuh"

namespace deinsum {
namespace {

using namespace sm100;

__global__ void weight_tables_kernel(const __grid_constant__ MttkrpArgs a) {
    weight_tables_body(a, int64_t(blockIdx.x) * blockDim.x + threadIdx.x, int64_t(gridDim.x) * blockDim.x);
}

// OP: outer indices packed into the tile; MN: MN-major A operand (the last mode);
// PW: per-row weights (packed outer indices, or narrow tiles of several p with L rows).
// RC: X through the four row-class tensor maps (rows not 16-byte aligned); otherwise through
// the tensor map when a.use_tma, else per-thread loads.
// Registers: 128 per thread at most.  The launch check counts a block's warps rounded up
// to a multiple of four (14 -> 16), and 16 x 32 x 128 is the SM's 65,536; a 144-register
// build of this 448-thread kernel fails to launch.  The rank-64 instances with per-row
// weights (64 accumulators and a float4 weight row per thread in the epilogue) spill there.
// TTM: one TTM of a chain (launch_ttm_tc): no weights; every fiber group's result is an
// output tile of its own, written to a.ttm_out.
template <int RP, bool OP, bool MN, bool PW, bool RC, bool TTM = false>
__global__ void __maxnreg__(128)
mttkrp_tc_kernel(const __grid_constant__ MttkrpArgs a) {
    static_assert(!TTM || (MN && !OP && !PW && !RC), "the TTM form takes the last-mode view through a tensor map");
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
                    else conv_read_rowcls_half(g, a.X, it.col, it.tile, it.o, it.kb, raw, pt, v);
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
            else if (RC) conv_store_rowcls_half(pt, a_hi(as), a_lo(as), v);
            else conv_store(g, pt, a_hi(as), a_lo(as), v);
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
                if (!TTM && it.kb == it.kb_lo) {
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
    } else if constexpr (TTM) {
        // ------------------------------------------------------- TTM write-out
        // every fiber group (a column of 128 rows b, outer index o = a) is one output tile:
        // Y[o, r, b] = T[b, r], the U_hi and U_lo columns added; rows past I_n are not written.
        // With I_n a multiple of 4 (and Y 16-byte aligned) each warp turns its 32 rows into
        // 16-byte words along b through 4 KB of scratch in the (unused) weight ring: PWC
        // columns r at a time, 8 lanes to a column; otherwise each lane stores its own row.
        const int quad = warp & 3;
        const int l = quad * 32 + lane;
        float *Y = a.ttm_out;
        constexpr int PWC = (C::WBUF_BYTES / 512) >= 16 ? 16 : 8;   // columns per scratch pass
        static_assert(C::WBUF_BYTES >= 4 * 32 * PWC * 4, "TTM write-out scratch");
        float *sc = wbuf + quad * 32 * PWC;
        const bool vec = (g.I & 3) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
        const int q4 = lane & 7, rr = lane >> 3;   // the 16-byte word this lane stores: b 4 q4, column rr + 4 i
        Iter it;
        it.init(a);
        int64_t fgi = 0;
        while (!it.done) {
            const int b = int(fgi % C::NACC);
            const uint32_t jb = uint32_t(fgi / C::NACC);
            if (!__all_sync(0xffffffffu, mbar_wait(accf(b), jb & 1u, abort_flag, a.status, wlim))) break;
            tc_fence_after();
            const uint32_t taddr = tmem + (uint32_t(quad * 32) << 16) + uint32_t(b * C::ACC);
            const int64_t row = it.col * BM + l;
            const bool rv = row < g.I;
            float *yr = Y + it.o * int64_t(g.R) * g.I + row;
            const int64_t b0 = it.col * BM + quad * 32;           // the warp's first row
            float *yw = Y + it.o * int64_t(g.R) * g.I + b0 + 4 * q4;
            const bool wv = b0 + 4 * q4 < g.I;                     // (all four rows, I_n % 4 == 0)
            #pragma unroll
            for (int c = 0; c < RP; c += 16) {
                uint32_t t[16], tl[16];
                tmem_ld16(taddr + uint32_t(c), t);
                tmem_ld16(taddr + uint32_t(RP + c), tl);
                tmem_wait_ld();
                if (vec) {
                    #pragma unroll
                    for (int h = 0; h < 16; h += PWC) {
                        if (c + h >= g.R) break;
                        #pragma unroll
                        for (int q = 0; q < PWC; ++q)
                            sc[q * 32 + lane] = __uint_as_float(t[h + q]) + __uint_as_float(tl[h + q]);
                        __syncwarp();
                        #pragma unroll
                        for (int i = 0; i < PWC / 4; ++i) {
                            const int r = c + h + rr + 4 * i;
                            if (wv && r < g.R)
                                *reinterpret_cast<float4 *>(yw + int64_t(r) * g.I) =
                                    *reinterpret_cast<const float4 *>(sc + (rr + 4 * i) * 32 + 4 * q4);
                        }
                        __syncwarp();   // read before the next pass overwrites the scratch
                    }
                } else {
                    #pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (rv && c + q < g.R) yr[int64_t(c + q) * g.I] = __uint_as_float(t[q]) + __uint_as_float(tl[q]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce(b));
            ++fgi;
            it.next_fg(a);
        }
    } else {
        // ------------------------------------------------------------- epilogue
        const int quad = warp & 3;                 // TMEM lanes 32*quad .. 32*quad+31
        // tile row of this thread's TMEM lane (row-class K-major tiles are stored class-major)
        const int l = (RC && !MN) ? rowcls_tile_row(quad * 32 + lane) : quad * 32 + lane;
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

template <int RP, bool OP, bool MN, bool PW, bool RC = false, bool TTM = false>
int launch_tc_rp_op(const MttkrpArgs &a, int n_sm, void *stream) {
    using C = TcCfg<RP>;
    cudaError_t e = cudaFuncSetAttribute(mttkrp_tc_kernel<RP, OP, MN, PW, RC, TTM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM));
    if (e != cudaSuccess) return int(e);
    int64_t grid = a.n_units < n_sm ? a.n_units : n_sm;
    if (grid < 1) grid = 1;
    MttkrpArgs ka = a;
    ka.wait_ns = wait_limit_ns();
    mttkrp_tc_kernel<RP, OP, MN, PW, RC, TTM><<<unsigned(grid), C::THREADS, C::SMEM, static_cast<cudaStream_t>(stream)>>>(ka);
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

}  // namespace


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

int launch_ttm_tc(const MttkrpArgs &a, int n_sm, void *stream) {
    if (!a.ttm_out || !a.use_tma || a.g.kcase != 1 || a.g.opack || a.g.kseg != 1) return int(cudaErrorInvalidValue);
    switch (a.g.R_pad) {
        case 16: return launch_tc_rp_op<16, false, true, false, false, true>(a, n_sm, stream);
        case 32: return launch_tc_rp_op<32, false, true, false, false, true>(a, n_sm, stream);
        case 64: return launch_tc_rp_op<64, false, true, false, false, true>(a, n_sm, stream);
    }
    return int(cudaErrorInvalidValue);
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
