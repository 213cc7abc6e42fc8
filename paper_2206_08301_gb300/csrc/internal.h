// Internal declarations shared by the library's translation units.
//
// The MTTKRP kernels see X through one "row view" (see MttkrpGeom).  For
// mode n of an order-N tensor, with P = prod_{m<n} I_m and Q = prod_{m>n} I_m:
//
//   case 0 (n < N-1, "K-contiguous"): a row is a (p, i_n) pair; its elements
//     run over q = (o, k), where k indexes the last mode I_{N-1} (the "inner"
//     mode contracted on the tensor cores, stride 1 in memory) and o the modes
//     n+1..N-2 ("outer" modes).  Rows are grouped 128 to a tile: one p and 128
//     consecutive i_n when I_n >= 128 ("wide"), else G = min(floor(128/I_n), 32)
//     consecutive p with all I_n rows each ("narrow").  On the tensor-core path,
//     when there is no p to pack (P = 1) and I_n <= 64, the G groups run over
//     consecutive outer indices o instead ("opack"; also in case 1 with I_n <= 64).
//   case 1 (n = N-1, "M-contiguous"): a row is one i_n; its elements run over
//     p = (o, k) with k indexing mode N-2 (inner) and o modes 0..N-3 (outer);
//     consecutive rows are adjacent in memory.
//
// The inner contraction over k runs in chunks of 64 (BK).  For a fixed tile
// and outer index o (and, on the tensor-core path, a segment of at most 16
// chunks of k: a "fiber group"), the chunks are accumulated into
// T[row, r] = sum_k X[row, (o, k)] U_inner[k, r]; the fiber group is then
// folded into the row's accumulator with the weight
//   w[row, r] = L(p(row))[r] * Ofac(o)[r],
//   L(p) = prod_{m<n} U^m[i_m(p), r]   (case 0 only),  Ofac(o) = prod_{outer m} U^m[i_m(o), r].
// This is the MTTKRP sum regrouped by distributivity (Sec. III-B einsum).
//
// Work is split into units = (column of 128 output rows, range of fiber
// groups); every unit writes its own 128 x R_pad block of partial sums and a
// reduction kernel adds the blocks of each column in unit order, so results do
// not depend on which CTA ran which unit.
#pragma once

#include <cstdint>
#include <cstddef>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/deinsum.h"

#define DEINSUM_MAX_ORDER 8
#define DEINSUM_BM 128
#define DEINSUM_BK 64
#define DEINSUM_GMAX 16  // most p values in one narrow tile (bounds the weight-ring slots)

namespace deinsum {

struct MttkrpGeom {
    int order;
    int mode;
    int kcase;            // 0: K-contiguous rows, 1: M-contiguous rows (mode == order-1)
    int narrow;           // case 0 with I < 128
    int R;                // rank
    int R_pad;            // rank padded for the kernels (16, 32 or 64)
    int n_kb;             // ceil(K_in / 64)
    int n_outer;          // number of outer modes
    int n_lmodes;         // case 0: modes 0..mode-1 (weights L); case 1: 0
    int vec_ok;           // rows allow 16-byte vector loads (checked with the X pointer)
    int64_t dims[DEINSUM_MAX_ORDER];
    int64_t P, I, Q;
    int64_t K_in;         // extent of the inner mode
    int64_t O;            // product of outer extents (1 if none)
    int outer_mode[DEINSUM_MAX_ORDER];
    int64_t outer_dim[DEINSUM_MAX_ORDER];
    int64_t G;            // narrow: p values (o values with opack) per tile, else 1
    int64_t n_cols;       // columns of 128 output rows (narrow: 1)
    int64_t tiles_per_col;
    int64_t fg_per_col;   // tiles_per_col * O_iter
    int64_t rows_per_col; // min(I, 128)
    int opack;            // tensor-core path, I <= 64 and no p to pack (case 0 with P = 1, or
                          // case 1): tile rows are (o_local, i_n), G >= 2 consecutive outer indices
    int64_t O_iter;       // outer indices iterated per tile: O, or 1 with opack (folded into the tile)
    int kseg;             // tensor-core path: segments of the inner range per (tile, o) -- each a fiber
    int n_kb_seg;         //   group of at most n_kb_seg chunks, so that TMEM accumulates <= 1024 k
};

struct MttkrpArgs {
    // TMA descriptor of X for the tensor-core kernel (valid when use_tma != 0):
    //   case 0: 4-D {K_in, O, I, P}, box {64, 1, min(I,128), G}  (opack: {K_in, I, O, P}, box {64, I, G, 1})
    //   case 1: 3-D {I, K_in, O},    box {min(I,128), 64, 1}     (opack: box {I, 64, G})
    CUtensorMap xmap;     // (the type carries its own 128-byte alignment)
    int use_tma;
    uint32_t box_bytes;   // bytes one box load writes (out-of-bounds parts are zero-filled)
    // Rows not 16-byte aligned (no xmap), no packed outer indices: four 2-D tensor maps, one per
    // class c of rows (case 0: rows r = p I + i of Q words) or k lines (case 1: lines o K_in + k
    // of I words) congruent to c mod 4.  Members of a class start at the same word offset d_c
    // within their 16-byte granule and lie 4 Q (4 I) words apart, a multiple of 16 bytes, so
    // map c has base = its first member's start rounded down to 16 bytes, inner extent
    // Q + d_c (I + d_c), row stride 4 Q (4 I); see encode_x_rowclass_maps.
    CUtensorMap xrow[4];
    int row_classes;
    int raw_pitch;        // elements per row of the raw tile in shared memory
    MttkrpGeom g;
    const void *X;
    const void *U[DEINSUM_MAX_ORDER];  // factor of each mode (U[mode] unused)
    const void *Uk2;                   // merged inner mode: the inner factor is the Khatri-Rao
    int64_t K_minor;                   //   product, row k = U[inner][k / K_minor] * Uk2[k % K_minor]
    const void *Bsplit;                // split-BF16 tiles of the inner factor (TC path)
    float *Lw;                         // TC path, n_lmodes > 0: P x R_pad row weights (weight_tables)
    float *Ow;                         // TC path, n_outer > 0:  O x R_pad fiber weights
    const int64_t *units;              // n_units x 3: column, first fiber group, end
    int64_t n_units;
    float *partial;                    // n_units x 128 x R_pad (F32 paths)
    double *partial64;                 // n_units x 128 x R_pad (F64 path)
    int *status;                       // device status word
    uint64_t wait_ns;                  // limit of a pipeline wait (set by the launcher)
    float *ttm_out;                    // launch_ttm_tc only: Y (see there)
};

// Many MTTKRP instances in one persistent launch of the tensor-core kernel: per-instance
// arguments (geometry, TMA descriptors of X, factor pointers, split factor tiles) live in
// device memory; the units, each = (instance, column, first fiber group, end, offset of
// its 128 x R_pad partial block in `partial`), form one list that the CTAs take in order
// from the ticket counter (zero at launch).  The kernel reads how an instance loads X
// (tensor map or row classes, the operand layout of its mode) from its arguments, once
// per unit.
struct BatchArgs {
    const MttkrpArgs *insts;
    const int64_t *units;       // 5 per unit
    int64_t n_units;
    unsigned long long *ticket; // next unit to hand out
    float *partial;
    int *status;
    uint64_t wait_ns;           // limit of a pipeline wait (set by the launcher)
};
int launch_mttkrp_tc_batched(const BatchArgs &b, int grid, void *stream);
size_t mttkrp_tc_batched_smem_bytes();

// The batched launches around the tensor-core kernel (mttkrp_tc_batched.cu).  Both run on a
// 1-D grid whose blocks are dealt out per instance: instance i owns blocks
// [start[i], start[i+1]) (start has n + 1 entries, every range non-empty), so that each
// instance gets blocks in proportion to its work and no block idles.
//   preparation: instance i's inner factor U (K_in x R) into n_kb split-BF16 tiles at `out`
//     (128-byte-swizzled K-major, rows U_hi then U_lo, zero past R and K_in), and its weight
//     tables (MttkrpArgs::Lw / Ow, as weight_tables_kernel);
//   reduction: out[col * rows_per_col + r, c] = the column's unit partials added in unit order
//     (narrow tiles: and over their G row groups).
struct SplitInst {
    const float *U;
    unsigned char *out;
    int64_t K_in;
    int R, RP, n_kb;
};
struct RedInst {
    float *out;
    int64_t I;
    int R, RP;
    int64_t rows_per_col, G;
    int narrow;
    int64_t col_table;  // first entry of this instance's column table in red_col
};
int launch_batched_prep(const MttkrpArgs *insts, const SplitInst *splits, const int *start, int n, int n_blocks,
                        void *stream);
int launch_batched_reduce(const RedInst *red, const int *start, int n, int n_blocks, const int64_t *red_col,
                          const int64_t *red_off, const float *partial, void *stream);

// Fused last-two-mode stage of a TTMc keeping a mode n < N-2 (ttmc_tc.cu):
//   T2[s, c, d] = sum_{k, l} X[s, k, l] U_{N-2}[k, c] U_{N-1}[l, d]
// for every slab s (flat index over modes 0..N-3), k over I_{N-2}, l over
// I_{N-1}.  The contraction over l runs on the tensor cores (split BF16, 128 k
// at a time), the one over k on the tensor cores as well while I_{N-2} <= 256 (tc2),
// else on CUDA cores in FP32; T1 = X U_{N-1} stays on chip.
// Short slabs share a 128-row tile: sg = 2 (I_{N-2} <= 64) or 4 (<= 32) slabs at a
// row pitch of 128 / sg, the rows past I_{N-2} zero-filled by the TMA (the next slab's
// rows, or zero past X, with row classes).
struct TtmcArgs {
    CUtensorMap xmap;     // 3-D {I_{N-1}, I_{N-2}, S}, box {64, min(I_{N-2}, 128), 1}; sg > 1: {64, 128/sg, sg}
    // rows of X (I_{N-1} words) not 16-byte aligned: the four row-class maps of the case-0 view
    // g, X's address; sg = 1 (boxes of 32 rows), or sg = 2 / 4 with tc2 (boxes of 32 / sg rows)
    CUtensorMap xrow[4];
    const void *X;
    int row_classes;
    uint32_t box_bytes;
    MttkrpGeom g;         // converter view of a chunk: case 0, I = I_{N-2}, narrow = I < 128 and sg = 1, G = 1
    const void *Bsplit;   // split-BF16 tiles of U_{N-1} (R_pad 32, n_kb tiles)
    const float *U2pad;   // CUDA-core stage 2: U_{N-2} as n_kt*128 rows x 32 FP32, zero beyond I_{N-2} x R_{N-2}
    const void *U2split;  // tensor-core stage 2 (tc2): split BF16 tiles of U_{N-2} (launch_ttmc_u2_split)
    float *T2;            // S x R_{N-2} x R_{N-1}, row-major
    int64_t S;            // slabs
    int n_kt;             // tiles of 128 along k
    int n_kb;             // chunks of 64 along l
    int R2, R3;           // R_{N-2}, R_{N-1} (<= 32)
    int sg;               // slabs per tile (1, 2 or 4; n_kt = 1 when sg > 1)
    int tc2;              // stage 2 on the tensor cores (n_kt <= 2), else on CUDA cores (sg = 1)
    int *status;
    uint64_t wait_ns;     // limit of a pipeline wait (set by the launcher)
};
// Slabs per tile of the fused kernel for I_{N-2} = K.
inline int ttmc_slab_group(int64_t K) { return K <= 32 ? 4 : (K <= 64 ? 2 : 1); }
int launch_ttmc_fused(const TtmcArgs &a, int n_sm, void *stream);
// The same pipeline without stage 2: T[s, k, d] = sum_l X[s, k, l] U_{N-1}[l, d] written to
// a.T2 (S x I_{N-2} x R_{N-1}); a.U2pad and a.R2 are unused (the TTM over the last mode; sg = 1).
int launch_ttm_last_tc(const TtmcArgs &a, int n_sm, void *stream);
// 3-D tensor map of X for those kernels ({I_{N-1}, I_{N-2}, S}, box {64, min(I_{N-2}, 128), 1},
// or {64, 128/sg, sg} for sg > 1); false when X or its rows are not 16-byte aligned.
bool encode_ttm_last_map(const void *X, int64_t S, int64_t K, int64_t L, CUtensorMap *map, uint32_t *box_bytes,
                         int sg = 1);

// The four row-class tensor maps of an MTTKRP row view (MttkrpArgs::xrow) for X whose rows are
// not 16-byte aligned; false with packed outer indices, fewer than 4 rows (lines), extents
// beyond int32 coordinates or no encoder.
bool encode_x_rowclass_maps(const MttkrpGeom &g, const void *X, CUtensorMap *maps);
// Whether the geometry allows them (the conditions above other than X and the encoder).
bool rowclass_supported(const MttkrpGeom &g);
// Their converter view of a chunk (case 0, I = K, narrow when K < 128 and sg = 1 -- with sg > 1
// the box fills all 128 rows --, R_pad 32, ceil(L/64) chunks).
void ttm_last_geometry(int order, int64_t S, int64_t K, int64_t L, int R, MttkrpGeom *g, int sg = 1);
int launch_ttmc_pad_factor(const float *U, int64_t rows, int R, float *out, int n_kt, void *stream);
// U_{N-2} (rows x R, rows <= 256) -> the tensor-core stage-2 operand: for k tile kt < n_kt,
// part p (hi, lo) and half h of the tile, a 4 KB block at ((kt * 2 + p) * 2 + h) * 4096 holding
// 32 rows c x 64 k (K-major, 128-byte swizzle), zero beyond rows x R.  n_kt * 16 KB in all.
int launch_ttmc_u2_split(const float *U, int64_t rows, int R, void *out, int n_kt, void *stream);
constexpr int kTtmcTc2MaxKt = 2;   // k tiles the tensor-core stage 2 keeps resident

// Launch helpers implemented in the .cu files.  They return a CUDA error code
// (0 on success) and increment the library's launch counter.
int launch_mttkrp_plain_f32(const MttkrpArgs &a, int n_sm, void *stream);
int launch_mttkrp_plain_f64(const MttkrpArgs &a, int n_sm, void *stream);
int launch_mttkrp_tc(const MttkrpArgs &a, int n_sm, void *stream);
// One TTM of a chain on the tensor cores, Y[a, r, b] = sum_i X[a, i, b] U[i, r] (split BF16,
// FP32 accumulation), with X seen as the order-3 tensor (A, I, B) whose last mode b is the
// row of the MTTKRP view (geometry of mttkrp_prepare_oneoff(3, {A, I, B}, 2, R, X, a, false),
// X through its tensor map): every fiber group (128 rows b, one outer index a) is one output
// tile, written to a.ttm_out (A x R x B, FP32) instead of being folded with weights.  Needs
// a.U[1] = U, its split tiles in a.Bsplit (launch_split_inner_factor) and a unit table.
int launch_ttm_tc(const MttkrpArgs &a, int n_sm, void *stream);
int launch_split_inner_factor(const MttkrpArgs &a, void *bsplit, void *stream);
// Weight tables of the tensor-core kernel (a.Lw, a.Ow; sizes below).
int launch_weight_tables(const MttkrpArgs &a, void *stream);
// Floats of the two tables: P x R_pad (if n_lmodes > 0) and O x R_pad (if n_outer > 0).
inline size_t weight_table_floats_l(const MttkrpGeom &g) { return g.n_lmodes > 0 ? size_t(g.P) * size_t(g.R_pad) : 0; }
inline size_t weight_table_floats_o(const MttkrpGeom &g) { return g.n_outer > 0 ? size_t(g.O) * size_t(g.R_pad) : 0; }
// The final reduction of the unit partials into the I_n x R output; with C (R x L,
// device) it writes out = M C instead (I_n x L), the MTTKRP + MM epilogue.
int launch_mttkrp_reduce_f32(const MttkrpArgs &a, const int64_t *col_unit_begin, void *out, void *stream,
                             const void *C = nullptr, int64_t L = 0);
int launch_mttkrp_reduce_f64(const MttkrpArgs &a, const int64_t *col_unit_begin, void *out, void *stream,
                             const void *C = nullptr, int64_t L = 0);
size_t mttkrp_tc_smem_bytes(int R_pad);
int mttkrp_plain_ctas_per_sm(int f64, int R_pad);  // resident CTAs per SM of the plain kernel

// Plain TTM on a (A, Im, B) view: Y[a, r, b] = sum_i X[a, i, b] U[i, r].
int launch_ttm_plain_f32(const float *X, const float *U, float *Y, int64_t A, int64_t Im,
                         int64_t B, int64_t Rm, void *stream);
int launch_ttm_plain_f64(const double *X, const double *U, double *Y, int64_t A, int64_t Im,
                         int64_t B, int64_t Rm, void *stream);

void count_launch(int n = 1);

// Limit (ns) of every bounded pipeline wait of the tensor-core kernels launched from now on:
// 2 s unless deinsum_set_wait_limit_ns changed it.  Launchers copy it into the kernel arguments.
uint64_t wait_limit_ns();

// cudaMalloc / cudaMallocHost that count successful allocations (deinsum_alloc_count).
cudaError_t counted_malloc(void **p, size_t bytes);
cudaError_t counted_malloc_host(void **p, size_t bytes);

// Units per column of 128 output rows (each column's fiber groups cut into that many
// contiguous units) such that the busiest of `target` persistent CTAs, which take units
// round-robin, is as close as possible to the mean: it runs ceil(units / target) units
// of up to ceil(fg_per_col / per_col) fiber groups.  The smallest count within 1 % of
// the best is taken (fewer partial blocks to reduce); at most max_units units.
inline int64_t balanced_units_per_col(int64_t n_cols, int64_t fg_per_col, int64_t target, int64_t max_units) {
    if (n_cols < 1 || fg_per_col < 1 || target < 1) return 1;
    const double mean = double(n_cols) * double(fg_per_col) / double(target);
    auto eff = [&](int64_t p) {
        const int64_t units = n_cols * p;
        const int64_t waves = (units + target - 1) / target;
        const int64_t fg_unit = (fg_per_col + p - 1) / p;
        return mean / double(waves * fg_unit);
    };
    int64_t lo = target / n_cols;
    if (lo < 1) lo = 1;
    if (lo > fg_per_col) lo = fg_per_col;
    int64_t best = lo;
    double best_eff = eff(lo);
    for (int64_t p = lo + 1; p <= 8 * lo + 8 && p <= fg_per_col && n_cols * p <= max_units; ++p) {
        const double e = eff(p);
        if (e > best_eff + 0.01) {
            best = p;
            best_eff = e;
        }
    }
    return best;
}

int deinsum_internal_operand_mode(deinsum_plan_t pl, int k);

// Row view (and TMA descriptor of X when possible) of a one-off split-BF16
// MTTKRP, computed without heap or device allocation.  allow_opack = false keeps
// one outer index per tile (the batched kernel: its many small instances ran
// slower with packing, 16.1 vs 14.4 ms for the 512-instance batch).
bool mttkrp_prepare_oneoff(int order, const int64_t *dims, int mode, int R, const void *X, MttkrpArgs *a,
                           bool allow_opack = true);

}  // namespace deinsum
