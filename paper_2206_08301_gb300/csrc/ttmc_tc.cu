// Fused TTMc stage on the tcgen05 tensor cores (sm_103a).
//
// A TTMc keeping mode n (Sec. III-B, Table IV: Y = X x_m U_m over every
// m != n) contracts every other mode of X with its factor.  When n < N-2 the
// last two modes are contracted here in a single pass over X:
//   T2[s, c, d] = sum_{k, l} X[s, k, l] U_{N-2}[k, c] U_{N-1}[l, d],
// s a slab (flat index over modes 0..N-3).  Per slab and 128-row k tile:
//   stage 1 (tensor cores): T1[k, d] = sum_l X[s, k, l] U_{N-1}[l, d] with the
//     MTTKRP pipeline -- TMA ring of raw FP32 chunks (128 k x 64 l), converter
//     warps splitting them into BF16 hi / lo operand tiles, one thread issuing
//     tcgen05.mma against the split factor tiles, FP32 accumulation in TMEM;
//   stage 2 (tensor cores, I_{N-2} <= 256): the epilogue warps split each T1
//     tile into BF16 hi / lo and write it to shared memory as an MN-major operand
//     (row k, n = (part, d)); a warp of its own issues
//       D2[c, (p, d)] += sum_k U_{N-2}[k, c] T1_p[k, d]
//     for both parts of U_{N-2} (resident split tiles, K-major) into a per-slab
//     TMEM accumulator (rows c on TMEM lanes 96 + c), and another warp reads D2 once
//     the slab is complete and writes T2.  Slabs with I_{N-2} <= 64 (<= 32) share a tile two
//     (four) at a time, 128 / SG rows apart, each contracted over its own rows, so
//     that short slabs still fill the tensor-core tile; there the operands swap (T1 the
//     MN-major A operand with rows (slab, d), U_{N-2} the B operand), so that 8 (4) MMAs
//     of M = 64 (128) serve the whole tile, and four warps of their own write T2 out.
//     The stage-2 issue never blocks the stage-1 issue: separate threads, separate commits.
//   stage 2 (CUDA cores, FP32, I_{N-2} > 256): each epilogue warp moves the 32 T1
//     rows of its TMEM lane quadrant to shared memory and adds U_{N-2}^T T1 over
//     them into its own partial block of T2; at the end of a slab the four
//     partials are added in warp order.  The factor rows of a k tile sit in one
//     of two shared-memory slots, copied one tile ahead by the epilogue itself.
// T1 never reaches HBM; T2 (R_{N-2} R_{N-1} / (I_{N-2} I_{N-1}) of X) is written
// once, and the remaining modes are contracted by the TTM chain.  Each
// CTA owns a contiguous range of slabs, so every T2 block is produced by one
// CTA in a fixed order (deterministic, no reduction pass).
//
// Warp roles: 0-7 converters, 8-11 epilogue (stage 2), 12 TMEM + stage-1 MMA
// issue, 13 TMA; with the tensor-core stage 2 also 14 (stage-2 MMA issue) and 15
// (T2 write-out from TMEM lanes 96-127); with packed slabs 12-15 write T2 out (one TMEM
// lane quadrant each) and 16, 17, 18 take the MMA, TMA and stage-2 issue roles.  Every wait is bounded (mbar_wait); the epilogue warps meet only
// through mbarriers (tensor-core stage 2: b2full / b2free for the T1 operand,
// d2full / d2free for the TMEM accumulators; CUDA-core stage 2: ufree for the U
// slots, t1full / t1free for the partial blocks), so a time-out anywhere ends
// every role.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"
#include "sm100.cuh"
#include "tc_common.cuh"

namespace deinsum {
namespace {

// RC: rows of X not 16-byte aligned, loaded through the four row-class tensor maps (four
// class boxes per chunk, 34 KB a stage: two raw stages instead of three).
// TC2: stage 2 on the tensor cores, with two more warps: 14 issues the stage-2 MMAs and 15
// reads the finished slabs' T2 out of TMEM (a 448-thread block is checked as 16 warps for
// its registers anyway, so they cost no registers).
// PACK (packed slabs, SG > 1): warps 12-15 write T2 out, one TMEM lane quadrant each, and
// the MMA, TMA and stage-2 issue roles move to warps 16-18 (608 threads, at most 104
// registers a thread).
template <bool RC = false, bool TC2 = false, bool PACK = false> struct TtmcCfg {
    static constexpr int RP = 32;                          // padded R_{N-1} and R_{N-2}
    static constexpr int N = 2 * RP;                       // rows of the split factor tile (hi, then lo)
    static constexpr int RS = RC ? 2 : 3;                  // raw X stages
    static constexpr int AS = 2;                           // operand stages
    static constexpr int OUT_WARP = CONV_WARPS + EPI_WARPS;  // PACK: first of the four T2 writers
    static constexpr int MMA_WARP = CONV_WARPS + EPI_WARPS + (PACK ? 4 : 0);
    static constexpr int TMA_WARP = MMA_WARP + 1;
    static constexpr int S2_WARP = TMA_WARP + 1;            // TC2: stage-2 issue (lane 0)
    static constexpr int T2_WARP = TMA_WARP + 2;            // TC2 without PACK: T2 writer (TMEM lanes 96-127)
    static constexpr int WARPS = PACK ? S2_WARP + 1 : (TC2 ? TMA_WARP + 3 : TMA_WARP + 1);
    static constexpr int THREADS = WARPS * 32;
    static constexpr int RAW_BYTES = BM * BK * 4;           // one box of the tensor map
    static constexpr int RAW_STAGE = RC ? kRcRawBytes : RAW_BYTES;
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = N * BK * 2;
    static constexpr int ASTAGE_BYTES = 2 * A_BYTES + B_BYTES;
    static constexpr int T1_BYTES = BM * RP * 4;           // one T1 tile, FP32, 16-byte slots swizzled by row
    static constexpr int USLOTS = 2;
    static constexpr int USLOT_BYTES = BM * RP * 4;        // 128 rows of U_{N-2}, 32 columns
    static constexpr int NACC = 2;                         // TMEM accumulators of N columns (tiles in flight)
    static constexpr int TMEM_COLS = NACC * N;
    // tensor-core stage 2: the region after the operand stages holds the split U_{N-2}
    // tiles (up to two k tiles, 16 KB each) and the split T1 tile B2 (128 k x 64 n, MN-major)
    static constexpr int U2S_BYTES = kTtmcTc2MaxKt * 16384;
    static constexpr int B2_BYTES = BM * 2 * RP * 2;
    static_assert(U2S_BYTES + B2_BYTES == T1_BYTES + USLOTS * USLOT_BYTES, "the two stage-2 layouts share one region");
    static constexpr int D2_SLOTS = 4;                     // TMEM accumulators of slabs' T2 (2 RP columns each)
    static constexpr int TMEM_COLS_TC2 = 512;              // NACC * N + D2_SLOTS * 2 RP = 384, as a power of two
    static_assert(NACC * N + D2_SLOTS * 2 * RP <= TMEM_COLS_TC2, "TMEM columns");
    static constexpr int ACC_BAR = 2 * RS + 3 * AS;        // accf[NACC], acce[NACC], drain follow the rings
    static constexpr int TC2_BAR = ACC_BAR + 2 * NACC + 1 + USLOTS + 3;   // u2full, b2full[2], b2free[2], d2full[], d2free[]
    static constexpr int NBARS = TC2_BAR + 5 + 2 * D2_SLOTS + 1;   // + the stage-2 issuer's drain
    static constexpr size_t SMEM = size_t(RS) * RAW_STAGE + size_t(AS) * ASTAGE_BYTES + T1_BYTES +
                                   size_t(USLOTS) * USLOT_BYTES + 1024 + 512;
    static_assert(SMEM <= 232448, "dynamic shared memory above the 227 KB per-CTA limit");
    static_assert(NBARS * 8 + 8 <= 512, "barrier area");
};

// Chunks of one CTA: slab groups [s, s1) (one slab each unless slabs share a
// tile), then k tiles, then l chunks.
struct TIter {
    int64_t s, s1;
    int kt, kb;
    bool done;
    __device__ __forceinline__ void init(int64_t S) {
        s = S * blockIdx.x / gridDim.x;
        s1 = S * (blockIdx.x + 1) / gridDim.x;
        kt = 0;
        kb = 0;
        done = s >= s1;
    }
    __device__ __forceinline__ void next(int n_kb, int n_kt) {
        if (++kb < n_kb) return;
        kb = 0;
        if (++kt < n_kt) return;
        kt = 0;
        if (++s >= s1) done = true;
    }
};

// T1 tile in shared memory: row r holds 32 floats as eight 16-byte slots,
// logical slot x stored at slot x ^ (r & 7) (conflict-free row writes and
// column-block reads).
__device__ __forceinline__ float4 *t1_slot(float *t1s, int r, int x) {
    return reinterpret_cast<float4 *>(t1s + r * TtmcCfg<>::RP) + (x ^ (r & 7));
}

// Row classes with SG > 1 packed slabs (I_{N-2} <= 128 / SG): slab g of the group fills tile
// rows g KP .. g KP + KP - 1 (KP = 128 / SG), rows past I_{N-2} in it being the next slab's
// rows (finite values against the zero rows of U_{N-2}) or zero past X.  The class boxes hold
// KP / 4 rows each (the maps are encoded so): for class c, slab g's box goes to rows
// g KP / 4 .. of the class's 32-row region, so tile row l of any slab sits at region row
// l / 4, as with one slab per tile, and only the class and word offset change per slab.
template <int SG>
__device__ __forceinline__ void rc_load_packed(const TtmcArgs &a, int64_t grp, int kb, uint32_t dst, uint32_t bar) {
    constexpr int KP = BM / SG;
    mbar_arrive_expect_tx(bar, kRcRawBytes);   // 4 classes x SG boxes of KP / 4 rows
    const uint64_t xw = word_index(a.X);
    const int64_t x0 = int64_t(kb) * BK;
    #pragma unroll
    for (int g = 0; g < SG; ++g) {
        const int64_t rowbase = (grp * SG + g) * a.g.I;
        #pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t rc = rowbase + ((c - rowbase) & 3);          // slab's first row of class c
            const int64_t x = int64_t((xw + uint64_t(c) * uint64_t(a.g.Q)) & 3u) + x0;
            tma_load_2d(dst + uint32_t((c * kRcRows0 + g * (KP / 4)) * kRcPitch0 * 4), &a.xrow[c],
                        int(x & ~int64_t(3)), int((rc - c) >> 2), bar);
        }
    }
}
// JN rows of one class run (4 words each, box rows 4 apart) starting at word d of address r.
template <int JN>
__device__ __forceinline__ void rc_read_run(uint32_t r, int d, float4 *v) {
    constexpr uint32_t JS = 4u * kRcPitch0 * 4u;
    switch (d) {
        case 0:
            #pragma unroll
            for (int j = 0; j < JN; ++j) v[j] = lds128(r + JS * j);
            break;
        case 1:
            #pragma unroll
            for (int j = 0; j < JN; ++j) v[j] = lds_words(r + JS * j, 1);
            break;
        case 2:
            #pragma unroll
            for (int j = 0; j < JN; ++j) v[j] = lds_words(r + JS * j, 2);
            break;
        default:
            #pragma unroll
            for (int j = 0; j < JN; ++j) v[j] = lds_words(r + JS * j, 3);
            break;
    }
}
// The converter's rows rsub + 16 j (rowcls_thread layout) of a packed group: j in
// [g 8 / SG, (g + 1) 8 / SG) belongs to slab g, of class (slab start + rsub) mod 4.
template <int SG>
__device__ __forceinline__ void rc_read_packed(const TtmcArgs &a, int64_t grp, int kb, const float *raw, int pt,
                                               float4 (&v)[8]) {
    constexpr int JG = 8 / SG;
    const int k4 = pt & 15, rsub = pt >> 4;
    const uint64_t xw = word_index(a.X);
    const uint64_t x0 = uint64_t(kb) * BK;
    #pragma unroll
    for (int g = 0; g < SG; ++g) {
        const uint64_t row = uint64_t((grp * SG + g) * a.g.I + rsub);
        const int d = int((xw + row * uint64_t(a.g.Q) + x0) & 3u);
        const int c = int(row & 3u);
        const uint32_t r = smem_u32(raw) +
                           uint32_t(((c * kRcRows0 + (rsub >> 2) + 4 * g * JG) * kRcPitch0 + 4 * k4) * 4);
        rc_read_run<JG>(r, d, v + g * JG);
    }
}

// STORE: the epilogue writes the T1 tiles to HBM (a.T2 as S x I_{N-2} x R_{N-1}:
// the TTM over the last mode alone) instead of running stage 2.  SG: slabs per
// tile (a.sg).  TC2: stage 2 on the tensor cores (a.tc2), else on CUDA cores.
// RC: X through the row-class maps a.xrow (rows of I_{N-1} words not 16-byte aligned; with
// SG = 1 the tile's rows s I_{N-2} + 128 kt + l as in the MTTKRP case-0 view, with SG > 1
// the packed slabs of rc_load_packed).
template <bool STORE, int SG, bool TC2, bool RC>
__global__ void __launch_bounds__(TtmcCfg<RC, TC2, (SG > 1)>::THREADS, 1)
ttmc_fused_kernel(const __grid_constant__ TtmcArgs a) {
    using C = TtmcCfg<RC, TC2, (SG > 1)>;
    constexpr int RS = C::RS, AS = C::AS, RP = C::RP;
    static_assert(!STORE || (SG == 1 && !TC2), "the last-mode TTM keeps one slab per tile");
    static_assert(TC2 || SG == 1, "packed slabs take the tensor-core stage 2");
    // Stage 1 takes two MMAs of N = 2 RP per 16 k (X_hi [U_hi U_lo], X_lo [U_hi U_lo]: four
    // split products, hi and lo columns added by the feed).  A three-product form for packed
    // slabs (12 MMAs of N = RP a chunk, half the feed's TMEM reads) measured no faster once
    // their T2 writes left the feed warps (60^5: 0.688 against 0.684 ms).
    constexpr uint32_t kTmemCols = TC2 ? C::TMEM_COLS_TC2 : C::TMEM_COLS;
    const int64_t ngroups = (a.S + SG - 1) / SG;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *raw_base = smem;
    unsigned char *a_base = smem + RS * C::RAW_STAGE;
    unsigned char *region = a_base + AS * C::ASTAGE_BYTES;   // CUDA-core: t1s, U slots; TC2: U2 tiles, B2
    float *t1s = reinterpret_cast<float *>(region);
    float *ubuf = t1s + C::T1_BYTES / 4;
    // TC2: the split U_{N-2} tiles (n_kt x 16 KB), then the B2 tiles: two when n_kt = 1, else one
    const uint32_t u2s_addr = smem_u32(region);
    const int nb2 = a.n_kt == 1 ? 2 : 1;
    auto b2_addr = [&](int i) { return u2s_addr + uint32_t(a.n_kt + i) * 16384u; };
    uint64_t *bars = reinterpret_cast<uint64_t *>(region + C::T1_BYTES + C::USLOTS * C::USLOT_BYTES);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + C::NBARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
    int *status = a.status;
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
    constexpr int UB = C::ACC_BAR + 2 * C::NACC + 1;   // first barrier after the accumulators and drain
    auto accf = [&](int b) { return smem_u32(bars + C::ACC_BAR + b); };
    auto acce = [&](int b) { return smem_u32(bars + C::ACC_BAR + C::NACC + b); };
    const uint32_t drain = smem_u32(bars + C::ACC_BAR + 2 * C::NACC);
    auto ufull = [&](int s) { return smem_u32(bars + UB + s); };
    const uint32_t ufree = smem_u32(bars + UB + C::USLOTS);
    const uint32_t t1full = smem_u32(bars + UB + C::USLOTS + 1);
    const uint32_t t1free = smem_u32(bars + UB + C::USLOTS + 2);
    const uint32_t u2full = smem_u32(bars + C::TC2_BAR);
    auto b2full = [&](int i) { return smem_u32(bars + C::TC2_BAR + 1 + i); };
    auto b2free = [&](int i) { return smem_u32(bars + C::TC2_BAR + 3 + i); };
    auto d2full = [&](int j) { return smem_u32(bars + C::TC2_BAR + 5 + j); };
    auto d2free = [&](int j) { return smem_u32(bars + C::TC2_BAR + 5 + C::D2_SLOTS + j); };
    const uint32_t drain2 = smem_u32(bars + C::TC2_BAR + 5 + 2 * C::D2_SLOTS);
    auto uslot_addr = [&](int s) { return smem_u32(ubuf) + uint32_t(s) * C::USLOT_BYTES; };

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
        for (int s = 0; s < C::USLOTS; ++s) mbar_init(ufull(s), 1);
        mbar_init(ufree, EPI_WARPS);
        mbar_init(t1full, EPI_WARPS);
        mbar_init(t1free, EPI_WARPS);
        mbar_init(u2full, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(b2full(i), EPI_WARPS);
            mbar_init(b2free(i), 1);
        }
        for (int j = 0; j < C::D2_SLOTS; ++j) {
            mbar_init(d2full(j), 1);
            mbar_init(d2free(j), SG > 1 ? 4 : 1);   // packed slabs: the four T2 writers
        }
        mbar_init(drain2, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == C::MMA_WARP) {
        tmem_alloc(smem_u32(tmem_holder), kTmemCols);
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
        TIter it;
        it.init(ngroups);
        uint32_t bpar = 0, bused = 0;
        for (int64_t chunk = 0; !it.done; ++chunk) {
            float4 v[8];
            const int rs = int(chunk % RS);
            const uint32_t rj = uint32_t(chunk / RS);
            if (!__all_sync(0xffffffffu, mbar_wait(raw_full(rs), rj & 1u, abort_flag, status, wlim))) break;
            const float *raw = reinterpret_cast<const float *>(raw_base + size_t(rs) * C::RAW_STAGE);
            if constexpr (RC && SG > 1) rc_read_packed<SG>(a, it.s, it.kb, raw, rowcls_thread(pt), v);
            else if constexpr (RC) conv_read_rowcls(a.g, a.X, it.kt, it.s, 0, it.kb, raw, rowcls_thread(pt), v);
            else if (!a.g.narrow) conv_read_smem_wide(raw, pt, v);
            else conv_read_smem_t<false>(a.g, BM, raw, pt, v);
            // hand the raw stage back to the TMA warp before the split, so that its next
            // load overlaps it: the proxy fence orders these generic reads before that
            // async-proxy write (an mbarrier release alone does not)
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(raw_empty(rs));
            const int as = int(chunk % AS);
            const uint32_t aj = uint32_t(chunk / AS);
            if (!__all_sync(0xffffffffu, mbar_wait(a_empty(as), (aj & 1u) ^ 1u, abort_flag, status, wlim))) break;
            // a single l chunk (n_kb = 1): every chunk uses the same factor tile, which each
            // operand stage copies once and keeps
            if (issuer && (a.n_kb != 1 || aj == 0)) {
                mbar_arrive_expect_tx(bfull(as), C::B_BYTES);
                bulk_g2s(b_t(as), bsrc + size_t(it.kb) * C::B_BYTES, C::B_BYTES, bfull(as));
                bpar = (bpar & ~(1u << as)) | ((aj & 1u) << as);
                bused |= 1u << as;
            }
            conv_store(a.g, RC ? rowcls_thread(pt) : pt, a_hi(as), a_lo(as), v);
            fence_proxy_async_smem();   // the A stores before the tensor-core reads
            __syncwarp();
            if (lane == 0) mbar_arrive(a_full(as));
            it.next(a.n_kb, a.n_kt);
        }
        if (issuer) {  // every bulk copy into this CTA's smem has landed before exit
            for (int s = 0; s < AS; ++s)
                if ((bused >> s) & 1u) mbar_drain(bfull(s), (bpar >> s) & 1u, status);
        }
    } else if (warp == C::TMA_WARP) {
        // ------------------------------------------------------------------ TMA
        // raw X chunks
        if (lane == 0) {
            TIter it;
            it.init(ngroups);
            uint32_t r_used = 0, r_par = 0;   // per raw stage: a copy was issued, its parity
            for (int64_t chunk = 0; !it.done; ++chunk) {
                const int rs = int(chunk % RS);
                const uint32_t rj = uint32_t(chunk / RS);
                if (!mbar_wait(raw_empty(rs), (rj & 1u) ^ 1u, abort_flag, status, wlim)) break;
                if constexpr (RC && SG > 1) {
                    rc_load_packed<SG>(a, it.s, it.kb, raw_addr(rs), raw_full(rs));
                } else if constexpr (RC) {
                    rowcls_load(a.g, a.X, a.xrow, it.kt, it.s, 0, it.kb, raw_addr(rs), raw_full(rs));
                } else {
                    mbar_arrive_expect_tx(raw_full(rs), a.box_bytes);
                    tma_load_3d(raw_addr(rs), &a.xmap, it.kb * BK, it.kt * BM, int(it.s * SG), raw_full(rs));
                }
                r_used |= 1u << rs;
                r_par = (r_par & ~(1u << rs)) | ((rj & 1u) << rs);
                it.next(a.n_kb, a.n_kt);
            }
            // every copy issued into this CTA's shared memory has landed before exit, also
            // when a role gave up and left some of them unconsumed
            for (int s2 = 0; s2 < RS; ++s2)
                if ((r_used >> s2) & 1u) mbar_drain(raw_full(s2), (r_par >> s2) & 1u, status);
        }
        __syncwarp();
    } else if (warp == C::MMA_WARP) {
        // -------------------------------------------------------------- MMA issue
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16_f32(BM, C::N);
            TIter it;
            it.init(ngroups);
            const int64_t nfg = (it.s1 - it.s) * a.n_kt;
            int64_t chunk = 0;
            bool ok = true;
            for (int64_t fgi = 0; ok && fgi < nfg; ++fgi) {
                const int b = int(fgi % C::NACC);
                const uint32_t jb = uint32_t(fgi / C::NACC);
                if (!mbar_wait(acce(b), (jb & 1u) ^ 1u, abort_flag, status, wlim)) { ok = false; break; }
                tc_fence_after();
                const uint32_t dcol = tmem + uint32_t(b * C::N);
                for (int kb = 0; kb < a.n_kb; ++kb) {
                    const int s = int(chunk % AS);
                    const uint32_t j = uint32_t(chunk / AS);
                    if (!mbar_wait(a_full(s), j & 1u, abort_flag, status, wlim) ||
                        ((a.n_kb != 1 || j == 0) && !mbar_wait(bfull(s), j & 1u, abort_flag, status, wlim))) {
                        ok = false;
                        break;
                    }
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
                    mma_commit(a_empty(s));
                    ++chunk;
                }
                if (!ok) break;
                mma_commit(accf(b));
            }
            // all issued MMAs have completed before TMEM is released
            mma_commit(drain);
            mbar_drain(drain, 0, status);
        }
        __syncwarp();
    } else if constexpr (STORE) {
        // ------------------------------------------- epilogue: T1 tiles to HBM
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        TIter it;
        it.init(ngroups);
        const int64_t nfg = (it.s1 - it.s) * a.n_kt;
        int64_t s = it.s;
        int kt = 0;
        const bool vec = (a.R3 & 3) == 0;
        for (int64_t fgi = 0; fgi < nfg; ++fgi) {
            const int b = int(fgi % C::NACC);
            const uint32_t jb = uint32_t(fgi / C::NACC);
            if (!__all_sync(0xffffffffu, mbar_wait(accf(b), jb & 1u, abort_flag, status, wlim))) break;
            tc_fence_after();
            const int64_t k = int64_t(kt) * BM + row;
            const bool valid = k < a.g.I;
            float *dst = a.T2 + (s * a.g.I + k) * a.R3;
            const uint32_t taddr = tmem + (uint32_t(quad * 32) << 16) + uint32_t(b * C::N);
            #pragma unroll
            for (int c0 = 0; c0 < RP; c0 += 16) {
                uint32_t hi[16], lo[16];
                tmem_ld16(taddr + uint32_t(c0), hi);
                tmem_ld16(taddr + uint32_t(RP + c0), lo);
                tmem_wait_ld();
                if (valid) {
                    #pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        const int d = c0 + 4 * x;
                        const float4 v4 = make_float4(__uint_as_float(hi[4 * x]) + __uint_as_float(lo[4 * x]),
                                                      __uint_as_float(hi[4 * x + 1]) + __uint_as_float(lo[4 * x + 1]),
                                                      __uint_as_float(hi[4 * x + 2]) + __uint_as_float(lo[4 * x + 2]),
                                                      __uint_as_float(hi[4 * x + 3]) + __uint_as_float(lo[4 * x + 3]));
                        if (vec) {
                            if (d < a.R3) *reinterpret_cast<float4 *>(dst + d) = v4;
                        } else {
                            if (d < a.R3) dst[d] = v4.x;
                            if (d + 1 < a.R3) dst[d + 1] = v4.y;
                            if (d + 2 < a.R3) dst[d + 2] = v4.z;
                            if (d + 3 < a.R3) dst[d + 3] = v4.w;
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce(b));
            if (++kt == a.n_kt) {
                kt = 0;
                ++s;
            }
        }
    } else if constexpr (TC2) {
        // ------------------------------ tensor-core stage 2: feed, issue, write-out
        // Epilogue warps 8-11 (feed): per tile, each thread takes its T1 row (TMEM lane =
        // tile row = k) from the stage-1 accumulator, splits it into BF16 hi / lo and writes
        // it as row k of an MN-major B2 tile (n = d for hi, 32 + d for lo).
        // Warp 14, lane 0 (issue): per tile, for each slab g of the tile and both parts q of
        // U_{N-2} = U_hi + U_lo,  D2[slot][c, (p, d)] += sum_k U_q[k, c] T1_p[k, d], with
        // A = the split U_{N-2} block of part q (K-major) placed so that its rows c land on
        // the MMA's rows 96 + c (the window starts 96 rows before the block; the rows before
        // it only feed D rows that nobody reads), B = the split T1 tile (MN-major,
        // n = (p, d)), k over the slab's rows of the tile.  Its commits track only its own MMAs.
        // Warp 15 (write-out): TMEM lanes 96-127 = c of each finished slab's D2 slot -> T2.
        // The three meet only through mbarriers (b2full / b2free, d2full / d2free).
        // Packed slabs (SG > 1) swap the operands, so that one group of MMAs serves the whole
        // tile: the feed writes T1 as an MN-major A tile with rows m = (g, d) (32 g + d) and
        // k index kk = (p, k) (KP p + k, k the row within slab g); B is the split U_{N-2}
        // block, K-major, rows (q, c) (32 q + c), the same 64 k for both p; so
        //   D2[tile][(g, d), (q, c)] = sum_{p, k} T1_p[g KP + k, d] U_q[k, c],
        // and T2[g, c, d] = D2[(g, d), c] + D2[(g, d), 32 + c].  SG = 4: M = 128 (row m on
        // TMEM lane m), K = 64, 4 MMAs; SG = 2: M = 64 (rows 16 i .. 16 i + 15 on lanes
        // 32 i .. 32 i + 15), K = 128, 8 MMAs -- against 16 MMAs of M = 128 with A = the
        // U_{N-2} window, of whose 128 rows R_{N-2} <= 32 are used.  Warps 12-15 write T2 out, each from its own
        // TMEM lane quadrant, up to four tiles (the D2 slots) behind the feed: stores issued
        // by the feed warps themselves held the feed back (0.69 against 0.90 ms at 60^5).
        TIter it;
        it.init(ngroups);
        const int64_t nfg = (it.s1 - it.s) * a.n_kt;
        const bool vec = (a.R3 & 3) == 0;
        constexpr uint32_t kD2Lanes = 96u << 16;   // TMEM lane offset of the D2 rows c
        constexpr int KP = BM / SG;                // tile rows of one slab
        constexpr int M2 = SG == 2 ? 64 : BM;      // packed slabs: rows (g, d) of the A tile
        // packed slabs: the U_{N-2} region's second half (unused with one k tile) holds 2 KB of
        // scratch per T2 writer, through which it turns its values into rows of d for 16-byte
        // stores
        constexpr int kScratchBytes = 2048;
        float *scratch = reinterpret_cast<float *>(region + 8192);
        auto issue_packed = [&](int64_t t, int bi) -> bool {
            constexpr uint32_t idesc2 = idesc_bf16_f32(M2, 2 * RP) | kIdescAMnMajor;
            const int slot = int(t % C::D2_SLOTS);
            if (!mbar_wait(b2full(bi), uint32_t((t / nb2) & 1), abort_flag, status, wlim)) return false;
            if (t == 0 && !mbar_wait(u2full, 0u, abort_flag, status, wlim)) return false;
            // the tile that last used the slot has been written out
            if (!mbar_wait(d2free(slot), uint32_t((t / C::D2_SLOTS) & 1) ^ 1u, abort_flag, status, wlim)) return false;
            tc_fence_after();
            const uint32_t dcol = tmem + uint32_t(C::NACC * C::N + slot * 2 * RP);
            const uint64_t bdesc = desc_kmajor_sw128(u2s_addr);   // U_{N-2} block: rows (q, c), 64 k
            #pragma unroll
            for (int ks = 0; ks < 2 * KP / 16; ++ks) {
                const uint64_t adesc =
                    SG == 2 ? desc_mnmajor_sw128(b2_addr(bi) + uint32_t(ks * 2048), 1024u, 1024u)
                            : desc_mnmajor_sw128(b2_addr(bi) + uint32_t(ks * 2 * kMnKGroupStride), kMnAtomStride,
                                                 kMnKGroupStride);
                const uint64_t adv = uint64_t((ks % (KP / 16)) * 32) >> 4;   // k = 16 ks mod KP
                mma_bf16(dcol, adesc, bdesc + adv, idesc2, ks > 0 ? 1u : 0u);
            }
            mma_commit(d2full(slot));
            mma_commit(b2free(bi));
            return true;
        };
        // Packed slabs: the T2 writer of TMEM quadrant qd writes tile t's T2 rows (g, d) held
        // in its lanes (SG = 4: g = qd, d = lane; SG = 2: g = qd / 2, d = 16 (qd mod 2) + lane
        // for lanes below 16), every c.  With R_{N-1} a multiple of 4 (and T2 16-byte aligned)
        // the lanes put their values in the warp's scratch as rows c of W d values (SG = 2:
        // W = 16, all 32 rows at once; SG = 4: W = 32, 16 rows at a time) and read them back
        // as 16-byte words, W / 4 lanes to a row; otherwise each lane stores its own values
        // (4-byte words, rows c R_{N-1} floats apart).
        auto write_packed = [&](int64_t t, int qd) -> bool {
            const int slot = int(t % C::D2_SLOTS);
            if (!__all_sync(0xffffffffu, mbar_wait(d2full(slot), uint32_t((t / C::D2_SLOTS) & 1), abort_flag, status,
                                                   wlim)))
                return false;
            tc_fence_after();
            const uint32_t d2 = tmem + (uint32_t(qd * 32) << 16) + uint32_t(C::NACC * C::N + slot * 2 * RP);
            uint32_t vh[2][16], vl[2][16];   // columns (hi part, c) and (lo part, c)
            tmem_ld16(d2, vh[0]);
            tmem_ld16(d2 + 16, vh[1]);
            tmem_ld16(d2 + RP, vl[0]);
            tmem_ld16(d2 + RP + 16, vl[1]);
            tmem_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(d2free(slot));
            constexpr int W = SG == 2 ? 16 : 32;           // d values per warp
            const int g = SG == 4 ? qd : (qd >> 1);
            const int d0 = SG == 4 ? 0 : 16 * (qd & 1);    // the warp's first d
            const int64_t sl = (it.s + t) * SG + g;
            if (sl >= a.S || d0 >= a.R3) return true;       // (warp-uniform)
            float *blk = a.T2 + sl * a.R2 * a.R3;
            if ((a.R3 & 3) == 0 && (reinterpret_cast<uintptr_t>(a.T2) & 15) == 0) {
                float *sc = scratch + qd * (kScratchBytes / 4);
                constexpr int RPASS = kScratchBytes / 4 / W;   // rows c per pass (32 or 16)
                constexpr int LPR = W / 4;                     // lanes per row
                constexpr int RPI = 32 / LPR;                  // rows per 16-byte read
                const int q = lane % LPR, rr = lane / LPR;
                const bool qok = d0 + 4 * q < a.R3;
                #pragma unroll
                for (int c0 = 0; c0 < RP; c0 += RPASS) {
                    if (c0 >= a.R2) break;
                    if (lane < W) {
                        #pragma unroll
                        for (int c = 0; c < RPASS; ++c)
                            sc[c * W + lane] = __uint_as_float(vh[(c0 + c) >> 4][(c0 + c) & 15]) +
                                               __uint_as_float(vl[(c0 + c) >> 4][(c0 + c) & 15]);
                    }
                    __syncwarp();
                    #pragma unroll
                    for (int r0 = 0; r0 < RPASS; r0 += RPI) {
                        const int c = c0 + r0 + rr;
                        if (c < a.R2 && qok) {
                            const float4 v4 = *reinterpret_cast<const float4 *>(sc + (r0 + rr) * W + 4 * q);
                            *reinterpret_cast<float4 *>(blk + int64_t(c) * a.R3 + d0 + 4 * q) = v4;
                        }
                    }
                    __syncwarp();   // the rows are read before the next pass overwrites them
                }
            } else {
                const int d = d0 + lane;
                if (lane < W && d < a.R3) {
                    #pragma unroll
                    for (int c = 0; c < RP; ++c)
                        if (c < a.R2)
                            blk[int64_t(c) * a.R3 + d] =
                                __uint_as_float(vh[c >> 4][c & 15]) + __uint_as_float(vl[c >> 4][c & 15]);
                }
            }
            return true;
        };
        auto issue_stage2 = [&](int64_t t, int bi) -> bool {
            if constexpr (SG > 1) return issue_packed(t, bi);   // (the rest: one slab per tile)
            constexpr uint32_t idesc2 = idesc_bf16_f32(BM, 2 * RP) | kIdescBMnMajor;
            const int tk = int(t % a.n_kt);
            const int64_t tg = t / a.n_kt;         // slab group within the CTA
            if (!mbar_wait(b2full(bi), uint32_t((t / nb2) & 1), abort_flag, status, wlim)) return false;
            if (t == 0 && !mbar_wait(u2full, 0u, abort_flag, status, wlim)) return false;
            tc_fence_after();
            for (int g = 0; g < SG; ++g) {
                const int64_t j = tg * SG + g;     // slab index within the CTA
                const int slot = int(j % C::D2_SLOTS);
                // the slab that last used the slot has been written out
                if (tk == 0 && !mbar_wait(d2free(slot), uint32_t((j / C::D2_SLOTS) & 1) ^ 1u, abort_flag, status, wlim))
                    return false;
                tc_fence_after();
                const uint32_t dcol = tmem + uint32_t(C::NACC * C::N + slot * 2 * RP);
                #pragma unroll
                for (int ks = 0; ks < KP / 16; ++ks) {
                    const int ku = 16 * ks;                       // k within the tile's k range
                    const int h = ku >> 6, st = (ku & 63) >> 4;   // 64-k half, 16-k step in it
                    const uint32_t ahi = u2s_addr + uint32_t(((tk * 2 + h) * 2 + 0) * 4096) - 12288u;
                    const uint32_t alo = u2s_addr + uint32_t(((tk * 2 + h) * 2 + 1) * 4096) - 12288u;
                    const uint64_t adv = uint64_t(st * 32) >> 4;
                    const uint64_t db =
                        desc_mnmajor_sw128(b2_addr(bi) + uint32_t(((g * KP + ku) >> 3) * 1024), 1024u, 1024u);
                    mma_bf16(dcol, desc_kmajor_sw128(ahi) + adv, db, idesc2, (tk > 0 || ks > 0) ? 1u : 0u);
                    mma_bf16(dcol, desc_kmajor_sw128(alo) + adv, db, idesc2, 1u);
                }
                if (tk == a.n_kt - 1) mma_commit(d2full(slot));
            }
            mma_commit(b2free(bi));
            return true;
        };
        auto write_t2 = [&](int64_t pg) -> bool {
            for (int g = 0; g < SG; ++g) {
                const int64_t j = (pg - it.s) * SG + g;   // slab index within the CTA
                const int slot = int(j % C::D2_SLOTS);
                if (!__all_sync(0xffffffffu,
                                mbar_wait(d2full(slot), uint32_t((j / C::D2_SLOTS) & 1), abort_flag, status, wlim)))
                    return false;
                tc_fence_after();
                const uint32_t d2 = tmem + kD2Lanes + uint32_t(C::NACC * C::N + slot * 2 * RP);   // lanes 96-127
                uint32_t vh[2][16], vl[2][16];   // columns (hi part, d) and (lo part, d)
                tmem_ld16(d2, vh[0]);
                tmem_ld16(d2 + 16, vh[1]);
                tmem_ld16(d2 + RP, vl[0]);
                tmem_ld16(d2 + RP + 16, vl[1]);
                tmem_wait_ld();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(d2free(slot));
                const int64_t sl = pg * SG + g;
                const int c = lane;
                if (sl < a.S && c < a.R2) {
                    float *dst = a.T2 + (sl * a.R2 + c) * a.R3;
                    #pragma unroll
                    for (int d = 0; d < RP; d += 4) {
                        const uint32_t *h4 = &vh[d >> 4][d & 15], *l4 = &vl[d >> 4][d & 15];
                        const float4 t4 = make_float4(__uint_as_float(h4[0]) + __uint_as_float(l4[0]),
                                                      __uint_as_float(h4[1]) + __uint_as_float(l4[1]),
                                                      __uint_as_float(h4[2]) + __uint_as_float(l4[2]),
                                                      __uint_as_float(h4[3]) + __uint_as_float(l4[3]));
                        if (vec) {
                            if (d < a.R3) *reinterpret_cast<float4 *>(dst + d) = t4;
                        } else {
                            if (d < a.R3) dst[d] = t4.x;
                            if (d + 1 < a.R3) dst[d + 1] = t4.y;
                            if (d + 2 < a.R3) dst[d + 2] = t4.z;
                            if (d + 3 < a.R3) dst[d + 3] = t4.w;
                        }
                    }
                }
            }
            return true;
        };
        if (warp == C::S2_WARP) {
            if (lane == 0 && nfg > 0) {
                // the split U_{N-2} tiles stay for the whole kernel
                // (packed slabs: only the first 8 KB, rows (q, c) for k < 64; the rest of the
                // region is the feed warps' T2 scratch)
                const uint32_t u2bytes = SG > 1 ? 8192u : uint32_t(a.n_kt) * 16384u;
                mbar_arrive_expect_tx(u2full, u2bytes);
                bulk_g2s(u2s_addr, a.U2split, u2bytes, u2full);
                for (int64_t fgi = 0; fgi < nfg; ++fgi)
                    if (!issue_stage2(fgi, int(fgi % nb2))) break;
                // the U_{N-2} copy has landed and every stage-2 MMA has completed before exit
                // (and before TMEM is released), also when the loop ended early
                mbar_drain(u2full, 0u, status);
                mma_commit(drain2);
                mbar_drain(drain2, 0u, status);
            }
            __syncwarp();
        } else if (warp == C::T2_WARP) {
            if constexpr (SG == 1) {
                for (int64_t pg = it.s; pg < it.s1; ++pg)
                    if (!write_t2(pg)) break;
            }
        } else if (SG > 1 && warp >= C::OUT_WARP && warp < C::OUT_WARP + 4) {
            // packed slabs: the T2 writers, one TMEM lane quadrant each (warp mod 4), as far
            // as four tiles behind the feed (the D2 slots)
            for (int64_t t = 0; t < nfg; ++t)
                if (!write_packed(t, warp & 3)) break;
        } else {
            const int quad = warp & 3;
            const int row = quad * 32 + lane;
            for (int64_t fgi = 0; fgi < nfg; ++fgi) {
                const int b = int(fgi % C::NACC);
                const uint32_t jb = uint32_t(fgi / C::NACC);
                const int bi = int(fgi % nb2);
                if (!__all_sync(0xffffffffu, mbar_wait(accf(b), jb & 1u, abort_flag, status, wlim))) break;
                // the stage-2 MMAs of the tile that last used this B2 buffer have read it
                if (fgi >= nb2 && !__all_sync(0xffffffffu, mbar_wait(b2free(bi), uint32_t(((fgi / nb2) & 1) ^ 1),
                                                                     abort_flag, status, wlim)))
                    break;
                tc_fence_after();
                const uint32_t taddr = tmem + (uint32_t(quad * 32) << 16) + uint32_t(b * C::N);
                uint32_t ph[RP / 2], pl[RP / 2];   // T1 row: packed BF16 pairs, hi and lo parts
                #pragma unroll
                for (int c0 = 0; c0 < RP; c0 += 16) {
                    uint32_t hi[16], lo[16];
                    tmem_ld16(taddr + uint32_t(c0), hi);
                    tmem_ld16(taddr + uint32_t(RP + c0), lo);
                    tmem_wait_ld();
                    #pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float x0 = __uint_as_float(hi[2 * q]) + __uint_as_float(lo[2 * q]);
                        const float x1 = __uint_as_float(hi[2 * q + 1]) + __uint_as_float(lo[2 * q + 1]);
                        split2(x0, x1, ph[c0 / 2 + q], pl[c0 / 2 + q]);
                    }
                }
                tc_fence_before();
                const uint32_t b2 = b2_addr(bi);
                if constexpr (SG > 1) {
                    // A tile element (m, kk) = (32 g + d, KP p + k) for tile row g KP + k
                    const uint32_t m0 = uint32_t(row / KP) * 32u, k = uint32_t(row % KP);
                    #pragma unroll
                    for (int ch = 0; ch < 4; ++ch) {
                        const uint32_t m = m0 + uint32_t(8 * ch);
                        const uint32_t oh = SG == 2 ? sw128_mn64_offset(m, k) : sw128_mn_offset(m, k);
                        const uint32_t ol = SG == 2 ? sw128_mn64_offset(m, KP + k) : sw128_mn_offset(m, KP + k);
                        sts128(b2 + oh, ph[4 * ch], ph[4 * ch + 1], ph[4 * ch + 2], ph[4 * ch + 3]);
                        sts128(b2 + ol, pl[4 * ch], pl[4 * ch + 1], pl[4 * ch + 2], pl[4 * ch + 3]);
                    }
                } else {
                    #pragma unroll
                    for (int ch = 0; ch < 4; ++ch) {
                        sts128(b2 + sw128_mn64_offset(uint32_t(8 * ch), uint32_t(row)), ph[4 * ch], ph[4 * ch + 1],
                               ph[4 * ch + 2], ph[4 * ch + 3]);
                        sts128(b2 + sw128_mn64_offset(uint32_t(RP + 8 * ch), uint32_t(row)), pl[4 * ch],
                               pl[4 * ch + 1], pl[4 * ch + 2], pl[4 * ch + 3]);
                    }
                }
                fence_proxy_async_smem();   // the B2 stores before the tensor-core reads
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(acce(b));
                    mbar_arrive(b2full(bi));
                }
            }
        }
    } else {
        // ------------------------------------ epilogue (stage 2), one slab per tile
        // Each warp adds U_{N-2}^T T1 over its own 32 rows into a partial block of the
        // slab's T2 (4 x 8 outputs per thread); at the end of the slab the four partials
        // are added in warp order (t1full: partials written, t1free: partials read).
        const int quad = warp & 3;                 // TMEM lanes (= tile rows) 32*quad .. 32*quad+31
        const int row = quad * 32 + lane;          // the T1 row this thread moves to smem
        const int cb = lane >> 2, dg = lane & 3;   // stage 2: T2[4 cb .. 4 cb + 3, 8 dg .. 8 dg + 7]
        const int et = threadIdx.x - CONV_WARPS * 32;
        float acc[4][8];
        #pragma unroll
        for (int i = 0; i < 4; ++i)
            #pragma unroll
            for (int q = 0; q < 8; ++q) acc[i][q] = 0.f;
        TIter it;
        it.init(ngroups);
        const int64_t nfg = (it.s1 - it.s) * a.n_kt;
        int64_t s = it.s;
        int kt = 0;
        uint32_t slab = 0;                         // slabs finished by this CTA
        // U_{N-2} rows of k tile kt.  With at most two tiles (I_{N-2} <= 256) every tile
        // is copied once into slot kt and stays; otherwise the rows of fiber group f go
        // to slot f % 2, copied by one thread one group ahead (groups 0 and 1 now, group
        // f + 1 once every warp is done with group f - 1).
        const bool uissuer = (et == 0);
        const bool uresident = a.n_kt <= C::USLOTS;
        uint32_t u_loads[C::USLOTS] = {0u, 0u};   // copies issued into each slot (the issuer's count)
        auto load_u = [&](int us, int ktile) {
            mbar_arrive_expect_tx(ufull(us), C::USLOT_BYTES);
            bulk_g2s(uslot_addr(us), a.U2pad + size_t(ktile) * BM * RP, C::USLOT_BYTES, ufull(us));
            ++u_loads[us];
        };
        if (uissuer && nfg > 0) {
            if (uresident) {
                for (int t = 0; t < a.n_kt; ++t) load_u(t, t);
            } else {
                load_u(0, 0);
                if (nfg > 1) load_u(1, 1 % a.n_kt);
            }
        }
        for (int64_t fgi = 0; fgi < nfg; ++fgi) {
            const int b = int(fgi % C::NACC);
            const uint32_t jb = uint32_t(fgi / C::NACC);
            if (!__all_sync(0xffffffffu, mbar_wait(accf(b), jb & 1u, abort_flag, status, wlim))) break;
            tc_fence_after();
            // the block of t1s this warp writes held the previous slab's partials:
            // every warp has finished reading them
            if (kt == 0 && !__all_sync(0xffffffffu, mbar_wait(t1free, (slab & 1u) ^ 1u, abort_flag, status, wlim))) break;
            const uint32_t taddr = tmem + (uint32_t(quad * 32) << 16) + uint32_t(b * C::N);
            #pragma unroll
            for (int c0 = 0; c0 < RP; c0 += 16) {
                uint32_t hi[16], lo[16];
                tmem_ld16(taddr + uint32_t(c0), hi);
                tmem_ld16(taddr + uint32_t(RP + c0), lo);
                tmem_wait_ld();
                #pragma unroll
                for (int x = 0; x < 4; ++x) {
                    const int q = 4 * x;
                    *t1_slot(t1s, row, c0 / 4 + x) =
                        make_float4(__uint_as_float(hi[q]) + __uint_as_float(lo[q]),
                                    __uint_as_float(hi[q + 1]) + __uint_as_float(lo[q + 1]),
                                    __uint_as_float(hi[q + 2]) + __uint_as_float(lo[q + 2]),
                                    __uint_as_float(hi[q + 3]) + __uint_as_float(lo[q + 3]));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce(b));
            {
                // every warp has finished group fgi - 1, whose slot the next group uses
                bool ok = true;
                if (uissuer && !uresident && fgi >= 1 && fgi + 1 < nfg) {
                    ok = mbar_wait(ufree, uint32_t((fgi - 1) & 1), abort_flag, status, wlim);
                    if (ok) load_u(int((fgi + 1) % C::USLOTS), (kt + 1) % a.n_kt);
                }
                if (!__all_sync(0xffffffffu, ok)) break;
            }
            const int us = uresident ? kt : int(fgi % C::USLOTS);
            const uint32_t uj = uresident ? 0u : uint32_t(fgi / C::USLOTS);
            if (!__all_sync(0xffffffffu, mbar_wait(ufull(us), uj & 1u, abort_flag, status, wlim))) break;
            // stage 2 over this warp's rows that lie inside I_{N-2}, in groups of four
            // (the rows past it are zero in both operands: TMA zero fill and the
            // padded factor, so a partial group is harmless)
            const float *u = ubuf + us * (C::USLOT_BYTES / 4) + 4 * cb;
            const int64_t left = a.g.I - int64_t(kt) * BM - quad * 32;
            const int nrows = left <= 0 ? 0 : (left >= 32 ? 32 : int((left + 3) & ~int64_t(3)));
            #pragma unroll 1
            for (int r0 = quad * 32; r0 < quad * 32 + nrows; r0 += 4) {
                float4 w[4], x0[4], x1[4];
                #pragma unroll
                for (int i = 0; i < 4; ++i) {
                    w[i] = *reinterpret_cast<const float4 *>(u + (r0 + i) * RP);
                    x0[i] = *t1_slot(t1s, r0 + i, 2 * dg);
                    x1[i] = *t1_slot(t1s, r0 + i, 2 * dg + 1);
                }
                #pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float wc[4] = {w[i].x, w[i].y, w[i].z, w[i].w};
                    const float xd[8] = {x0[i].x, x0[i].y, x0[i].z, x0[i].w, x1[i].x, x1[i].y, x1[i].z, x1[i].w};
                    #pragma unroll
                    for (int cc = 0; cc < 4; ++cc)
                        #pragma unroll
                        for (int q = 0; q < 8; ++q) acc[cc][q] = fmaf(wc[cc], xd[q], acc[cc][q]);
                }
            }
            fence_proxy_async_smem();   // the slot's reads before its next bulk-copy write
            __syncwarp();
            if (lane == 0) mbar_arrive(ufree);
            if (++kt == a.n_kt) {
                // slab done: the warp's partial block goes to its own 32 rows of t1s
                // (32 x 32 floats, c-major), then the four partials are added in warp order
                float *pw = t1s + quad * 32 * RP;
                #pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    float4 *dst = reinterpret_cast<float4 *>(pw + (4 * cb + cc) * RP + 8 * dg);
                    dst[0] = make_float4(acc[cc][0], acc[cc][1], acc[cc][2], acc[cc][3]);
                    dst[1] = make_float4(acc[cc][4], acc[cc][5], acc[cc][6], acc[cc][7]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(t1full);
                if (!__all_sync(0xffffffffu, mbar_wait(t1full, slab & 1u, abort_flag, status, wlim))) break;
                // this warp reduces rows c = 8 quad .. 8 quad + 7 of the block
                const int c = 8 * quad + (lane >> 2), d0 = 8 * (lane & 3);
                float sum[8];
                #pragma unroll
                for (int q = 0; q < 8; ++q) sum[q] = 0.f;
                #pragma unroll
                for (int wq = 0; wq < 4; ++wq) {
                    const float4 *src = reinterpret_cast<const float4 *>(t1s + wq * 32 * RP + c * RP + d0);
                    const float4 p0 = src[0], p1 = src[1];
                    sum[0] += p0.x; sum[1] += p0.y; sum[2] += p0.z; sum[3] += p0.w;
                    sum[4] += p1.x; sum[5] += p1.y; sum[6] += p1.z; sum[7] += p1.w;
                }
                if (c < a.R2) {
                    float *dst = a.T2 + (s * a.R2 + c) * a.R3;
                    #pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (d0 + q < a.R3) dst[d0 + q] = sum[q];
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(t1free);
                #pragma unroll
                for (int i = 0; i < 4; ++i)
                    #pragma unroll
                    for (int q = 0; q < 8; ++q) acc[i][q] = 0.f;
                kt = 0;
                ++s;
                ++slab;
            }
        }
        // the U copies have landed before exit, also when the loop ended early
        if (uissuer)
            for (int us = 0; us < C::USLOTS; ++us)
                if (u_loads[us]) mbar_drain(ufull(us), (u_loads[us] - 1u) & 1u, status);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == C::MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// U (rows x R, row-major) -> out (n_kt*128 rows x 32), zero beyond rows x R.
__global__ void pad_factor_kernel(const float *__restrict__ U, int64_t rows, int R, float *__restrict__ out,
                                  int64_t total) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = i / TtmcCfg<>::RP;
        const int c = int(i - r * TtmcCfg<>::RP);
        out[i] = (r < rows && c < R) ? U[r * R + c] : 0.f;
    }
}

}  // namespace

namespace {
template <bool STORE, int SG, bool TC2, bool RC = false>
int launch_ttmc_variant(const TtmcArgs &a, int n_sm, void *stream) {
    using C = TtmcCfg<RC, TC2, (SG > 1)>;
    cudaError_t e = cudaFuncSetAttribute(ttmc_fused_kernel<STORE, SG, TC2, RC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM));
    if (e != cudaSuccess) return int(e);
    const int64_t groups = (a.S + SG - 1) / SG;
    int64_t grid = groups < n_sm ? groups : n_sm;
    if (grid < 1) grid = 1;
    TtmcArgs ka = a;
    ka.wait_ns = wait_limit_ns();
    ttmc_fused_kernel<STORE, SG, TC2, RC><<<unsigned(grid), C::THREADS, C::SMEM, static_cast<cudaStream_t>(stream)>>>(ka);
    count_launch();
    return int(cudaGetLastError());
}
}  // namespace

int launch_ttmc_fused(const TtmcArgs &a, int n_sm, void *stream) {
    if (a.row_classes) {
        if (a.sg != 1 && (!a.tc2 || a.sg != ttmc_slab_group(a.g.I))) return int(cudaErrorInvalidValue);
        if (a.tc2) {
            if (a.n_kt > kTtmcTc2MaxKt) return int(cudaErrorInvalidValue);
            if (a.sg == 4) return launch_ttmc_variant<false, 4, true, true>(a, n_sm, stream);
            if (a.sg == 2) return launch_ttmc_variant<false, 2, true, true>(a, n_sm, stream);
            return launch_ttmc_variant<false, 1, true, true>(a, n_sm, stream);
        }
        return launch_ttmc_variant<false, 1, false, true>(a, n_sm, stream);
    }
    if (a.tc2) {
        if (a.n_kt > kTtmcTc2MaxKt) return int(cudaErrorInvalidValue);
        if (a.sg == 4) return launch_ttmc_variant<false, 4, true>(a, n_sm, stream);
        if (a.sg == 2) return launch_ttmc_variant<false, 2, true>(a, n_sm, stream);
        if (a.sg == 1) return launch_ttmc_variant<false, 1, true>(a, n_sm, stream);
        return int(cudaErrorInvalidValue);
    }
    if (a.sg != 1) return int(cudaErrorInvalidValue);
    return launch_ttmc_variant<false, 1, false>(a, n_sm, stream);
}
int launch_ttm_last_tc(const TtmcArgs &a, int n_sm, void *stream) {
    if (a.sg != 1 || a.tc2 || a.row_classes) return int(cudaErrorInvalidValue);
    return launch_ttmc_variant<true, 1, false>(a, n_sm, stream);
}

namespace {
// U (rows x R) -> split BF16 blocks ((kt * 2 + h) * 2 + p) * 4096: 32 rows c x 64 k,
// K-major 128-byte swizzle; hi = bf16(u), lo = bf16(u - hi); zero beyond rows x R.
__global__ void u2_split_kernel(const float *__restrict__ U, int64_t rows, int R, unsigned char *__restrict__ out,
                                int64_t total) {
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int kq = int(idx & 63);
        const int c = int((idx >> 6) & 31);
        const int h = int((idx >> 11) & 1);
        const int p = int((idx >> 12) & 1);
        const int64_t kt = idx >> 13;
        const int64_t k = kt * BM + h * 64 + kq;
        const float v = (c < R && k < rows) ? U[k * R + c] : 0.f;
        const __nv_bfloat16 hb = __float2bfloat16_rn(v);
        const __nv_bfloat16 e = p == 0 ? hb : __float2bfloat16_rn(v - __bfloat162float(hb));
        *reinterpret_cast<__nv_bfloat16 *>(out + size_t(((kt * 2 + h) * 2 + p) * 4096) +
                                           sw128_offset(uint32_t(c), uint32_t(kq))) = e;
    }
}
}  // namespace

int launch_ttmc_pad_factor(const float *U, int64_t rows, int R, float *out, int n_kt, void *stream) {
    const int64_t total = int64_t(n_kt) * BM * TtmcCfg<>::RP;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    pad_factor_kernel<<<unsigned(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(U, rows, R, out, total);
    count_launch();
    return int(cudaGetLastError());
}

int launch_ttmc_u2_split(const float *U, int64_t rows, int R, void *out, int n_kt, void *stream) {
    if (n_kt < 1 || n_kt > kTtmcTc2MaxKt || R > TtmcCfg<>::RP) return int(cudaErrorInvalidValue);
    const int64_t total = int64_t(n_kt) * 2 * 2 * 32 * 64;
    u2_split_kernel<<<unsigned((total + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        U, rows, R, static_cast<unsigned char *>(out), total);
    count_launch();
    return int(cudaGetLastError());
}

}  // namespace deinsum
