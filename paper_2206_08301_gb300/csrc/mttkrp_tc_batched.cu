// Batched split-BF16 MTTKRP on the tcgen05 tensor cores (sm_103a): one persistent
// launch over the work units of many instances, with the launches around it (the factor
// split and weight tables before, the fixed-order reduction after); csrc/batched.cu is the
// host side (instance tables, the unit list, graph capture, autotuning).  The pipeline is the one of
// the single-instance kernel (mttkrp_tc.cu): TMA ring of raw FP32 chunks, converter warps
// splitting them into BF16 hi / lo operand tiles, one thread issuing tcgen05.mma, FP32
// accumulators in TMEM, epilogue warps folding fiber groups with their Khatri-Rao weights.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

#include "internal.h"
#include "sm100.cuh"
#include "tc_common.cuh"
#include "mttkrp_tc.cuh"

namespace deinsum {
namespace {

using namespace sm100;

// ---------------------------------------------------------------------------
// Batched form: one persistent launch over the work units of every instance.
// The CTAs take units in order from one list (grouped by how the unit's instance
// loads X, largest first within a group) through a device ticket counter: the TMA
// thread takes each ticket and hands it to the CTA's other roles through a small
// shared-memory ring, so a CTA takes its next unit only when its pipeline is ready
// for one and all CTAs finish together.  Every unit names its instance, whose
// arguments sit in device memory.  Each role reads a unit's
// fields once and runs its chunks in code specialised for the instance's loads
// (tensor map or row classes, K-major or MN-major operand) and, in the epilogue,
// for its padded rank, so that all kinds of instance share one launch and one
// tail.  The MMAs take all four split products as in the single-instance kernel
// (N = 2 R_pad, a runtime field of the instruction descriptor; the accumulator's
// column r holds the U_hi products and column R_pad + r the U_lo products).
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
    int64_t *uring = reinterpret_cast<int64_t *>(tmem_holder + 2);   // NQ unit tickets

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
    constexpr int QB = AB + 2 * C::NACC + 1 + 2 * C::WSLOTS;   // the ticket ring's barriers
    auto qfull = [&](int s) { return smem_u32(bars + QB + s); };
    auto qempty = [&](int s) { return smem_u32(bars + QB + C::NQ + s); };
    // readers of each ticket: the eight converter warps, the MMA thread, the four epilogue warps
    constexpr uint32_t kQReaders = CONV_WARPS + 1 + EPI_WARPS;
    auto wslot_addr = [&](int s) { return smem_u32(wbuf) + uint32_t(s) * uint32_t(C::WSLOT_FLOATS) * 4u; };
    // unit u: its instance's arguments and (column, first fiber group, end, partial offset)
    auto unit_args = [&](int64_t u) -> const MttkrpArgs & { return bargs.insts[bargs.units[5 * u]]; };
    auto unit_field = [&](int64_t u, int f) { return bargs.units[5 * u + f]; };
    // The q-th ticket of this CTA (q = 0, 1, ...): the TMA thread takes the next unit index
    // from the device counter (-1 once the list is exhausted) and publishes it in ring slot
    // q mod NQ; every other role reads it from there (a warp reads it with all its lanes,
    // lane 0 releases the slot).  Every role walks the same tickets in the same order.
    auto give_ticket = [&](int64_t q, int64_t &u) -> bool {
        const int slot = int(q % C::NQ);
        if (!mbar_wait(qempty(slot), uint32_t((q / C::NQ) & 1) ^ 1u, abort_flag, status, wlim)) return false;
        const int64_t t = int64_t(atomicAdd(bargs.ticket, 1ull));
        u = t < bargs.n_units ? t : -1;
        uring[slot] = u;
        mbar_arrive(qfull(slot));   // release: the slot's value is seen by whoever observes the phase
        return true;
    };
    auto take_ticket_warp = [&](int64_t q, int64_t &u) -> bool {
        const int slot = int(q % C::NQ);
        if (!__all_sync(0xffffffffu, mbar_wait(qfull(slot), uint32_t((q / C::NQ) & 1), abort_flag, status, wlim)))
            return false;
        u = uring[slot];
        __syncwarp();
        if (lane == 0) mbar_arrive(qempty(slot));
        return true;
    };
    auto take_ticket_thread = [&](int64_t q, int64_t &u) -> bool {
        const int slot = int(q % C::NQ);
        if (!mbar_wait(qfull(slot), uint32_t((q / C::NQ) & 1), abort_flag, status, wlim)) return false;
        u = uring[slot];
        mbar_arrive(qempty(slot));
        return true;
    };

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
        for (int s = 0; s < C::NQ; ++s) {
            mbar_init(qfull(s), 1);
            mbar_init(qempty(s), kQReaders);
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
                            conv_read_rowcls_half(g, X, col, tile, o, kb, raw, pt, v);
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
                    else if constexpr (K == BK_RC_K) conv_store_rowcls_half(pt, a_hi(as), a_lo(as), v);
                    else conv_store(g, pt, a_hi(as), a_lo(as), v);
                    fence_proxy_async_smem();   // the A stores before the tensor-core reads
                    __syncwarp();
                    if (lane == 0) mbar_arrive(a_full(as));
                }
            }
            return true;
        };
        bool ok = true;
        int64_t u = 0;
        for (int64_t q = 0; ok; ++q) {
            if (!take_ticket_warp(q, u) || u < 0) break;
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
            int64_t u = 0;
            for (int64_t q = 0; ok; ++q) {
                if (!give_ticket(q, u) || u < 0) break;
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
                const uint32_t idesc = idesc_bf16_f32(BM, 2 * rp) | (MN ? kIdescAMnMajor : 0u);
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
                        const uint64_t db = desc_kmajor_sw128(b_t(s));   // [U_hi; U_lo]: N = 2 R_pad rows
                        #pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            const uint64_t adv = uint64_t(kk * 32) >> 4;
                            const uint64_t adv_a = MN ? uint64_t(kk * 2 * kMnKGroupStride) >> 4 : adv;
                            mma_bf16(dcol, dh + adv_a, db + adv, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                            mma_bf16(dcol, dl + adv_a, db + adv, idesc, 1u);
                        }
                        mma_commit(a_empty(s));
                    }
                    mma_commit(accf(b));
                }
                return true;
            };
            bool ok = true;
            int64_t u = 0;
            for (int64_t q = 0; ok; ++q) {
                if (!take_ticket_thread(q, u) || u < 0) break;
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
        const int lane_row = quad * 32 + lane;   // this thread's TMEM lane (accumulator row)
        int64_t fgi = 0;
        auto run = [&](auto rt, const MttkrpArgs &a, int64_t col, int64_t f0, int64_t f1, int64_t part_off) -> bool {
            constexpr int RP = decltype(rt)::value;
            MttkrpGeom g;
            batch_geometry<false>(g, a.g);
            g.kcase = a.g.kcase;
            // the tile row of this lane: K-major row-class tiles are stored class-major
            const int l = batch_kind(a) == BK_RC_K ? rowcls_tile_row(lane_row) : lane_row;
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
                    uint32_t tv[16], tl[16];   // the U_hi and U_lo products of columns c .. c + 15
                    tmem_ld16(taddr + uint32_t(c), tv);
                    tmem_ld16(taddr + uint32_t(RP + c), tl);
                    tmem_wait_ld();
                    #pragma unroll
                    for (int q = 0; q < 16; ++q) tv[q] = __float_as_uint(__uint_as_float(tv[q]) + __uint_as_float(tl[q]));
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
        int64_t u = 0;
        for (int64_t q = 0; ok; ++q) {
            if (!take_ticket_warp(q, u) || u < 0) break;
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

// ---------------------------------------------------------------------------
// The launches around the tensor-core kernel.  Their grids are dealt out per instance
// (instance i owns blocks [start[i], start[i+1])): block_instance finds a block's instance
// by a binary search over start, done once per block.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int block_instance(const int *__restrict__ start, int n) {
    __shared__ int inst;
    if (threadIdx.x == 0) {
        const int b = int(blockIdx.x);
        int lo = 0, hi = n - 1;   // the last i with start[i] <= b
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (start[mid] <= b) lo = mid;
            else hi = mid - 1;
        }
        inst = lo;
    }
    __syncthreads();
    return inst;
}

// Split factor tiles and weight tables of every instance, before the tensor-core kernel.
__global__ void __launch_bounds__(256) batched_prep_kernel(const MttkrpArgs *__restrict__ insts,
                                                           const SplitInst *__restrict__ si,
                                                           const int *__restrict__ start, int n) {
    const int i = block_instance(start, n);
    const int64_t t0 = int64_t(int(blockIdx.x) - start[i]) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(start[i + 1] - start[i]) * blockDim.x;
    const SplitInst s = si[i];
    const int64_t total = int64_t(s.n_kb) * 2 * s.RP * BK;
    for (int64_t idx = t0; idx < total; idx += stride) {
        const int k = int(idx % BK);
        const int nn = int((idx / BK) % (2 * s.RP));
        const int64_t kb = idx / (int64_t(BK) * 2 * s.RP);
        const int r = nn % s.RP;
        const int64_t kr = kb * BK + k;
        const float v = (r < s.R && kr < s.K_in) ? s.U[kr * s.R + r] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 e = nn < s.RP ? h : __float2bfloat16_rn(v - __bfloat162float(h));
        *reinterpret_cast<__nv_bfloat16 *>(s.out + size_t(kb) * (2 * s.RP * BK * 2) +
                                           sw128_offset(uint32_t(nn), uint32_t(k))) = e;
    }
    weight_tables_body(insts[i], t0, stride);
}

// Each instance's output from its unit partials, in unit order (deterministic).
__global__ void __launch_bounds__(256) batched_reduce_kernel(const RedInst *__restrict__ ri,
                                                             const int *__restrict__ start, int n,
                                                             const int64_t *__restrict__ red_col,
                                                             const int64_t *__restrict__ red_off,
                                                             const float *__restrict__ partial) {
    const int i = block_instance(start, n);
    const RedInst r = ri[i];
    const int64_t stride = int64_t(start[i + 1] - start[i]) * blockDim.x;
    const int64_t total = r.I * r.R;
    for (int64_t e = int64_t(int(blockIdx.x) - start[i]) * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t row = e / r.R;
        const int c = int(e - row * r.R);
        const int64_t col = row / r.rows_per_col;
        const int64_t ii = row - col * r.rows_per_col;
        const int64_t k0 = red_col[r.col_table + col], k1 = red_col[r.col_table + col + 1];
        float acc = 0.f;
        if (r.narrow) {
            for (int64_t k = k0; k < k1; ++k) {
                const float *p = partial + red_off[k] + ii * r.RP + c;
                for (int64_t g = 0; g < r.G; ++g) acc += p[g * r.I * r.RP];
            }
        } else {
            #pragma unroll 4
            for (int64_t k = k0; k < k1; ++k) acc += partial[red_off[k] + ii * r.RP + c];
        }
        r.out[e] = acc;
    }
}

}  // namespace

int launch_batched_prep(const MttkrpArgs *insts, const SplitInst *splits, const int *start, int n, int n_blocks,
                        void *stream) {
    batched_prep_kernel<<<unsigned(n_blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(insts, splits, start, n);
    count_launch();
    return int(cudaGetLastError());
}

int launch_batched_reduce(const RedInst *red, const int *start, int n, int n_blocks, const int64_t *red_col,
                          const int64_t *red_off, const float *partial, void *stream) {
    batched_reduce_kernel<<<unsigned(n_blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(red, start, n, red_col,
                                                                                           red_off, partial);
    count_launch();
    return int(cudaGetLastError());
}

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

}  // namespace deinsum
