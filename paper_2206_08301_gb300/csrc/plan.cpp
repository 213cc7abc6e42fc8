// Host side of the C ABI: einsum parsing and classification, the MTTKRP row
// view and work schedule, the plan's device workspace, and dispatch of the
// kernels.  Parsing follows the Einstein-notation rules of Sec. III-A
// (letters repeated across operands are summed, output letters are kept); the
// accepted patterns are the MTTKRP and TTMc einsums of Sec. III-B / Table IV.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace deinsum;

namespace deinsum {
static std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static std::atomic<int64_t> g_allocs{0};
cudaError_t counted_malloc(void **p, size_t bytes) {
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_allocs.fetch_add(1, std::memory_order_relaxed);
    return e;
}
cudaError_t counted_malloc_host(void **p, size_t bytes) {
    const cudaError_t e = cudaMallocHost(p, bytes);
    if (e == cudaSuccess) g_allocs.fetch_add(1, std::memory_order_relaxed);
    return e;
}

static std::atomic<uint64_t> g_wait_limit_ns{0};
uint64_t wait_limit_ns() {
    const uint64_t v = g_wait_limit_ns.load(std::memory_order_relaxed);
    return v ? v : 2000000000ull;
}
// The row-class maps of encode_x_rowclass_maps with case-0 boxes of `rows` rows.
static bool encode_rowclass_maps_rows(const MttkrpGeom &g, const void *X, CUtensorMap *maps, int rows);
}  // namespace deinsum

struct deinsum_plan_s {
    deinsum_kind kind = DEINSUM_KIND_MTTKRP;
    int order = 0;
    int mode = 0;
    deinsum_dtype dtype = DEINSUM_F32;
    deinsum_prec prec = DEINSUM_PREC_PLAIN;
    int64_t dims[DEINSUM_MAX_ORDER] = {0};
    int64_t ranks[DEINSUM_MAX_ORDER] = {0};
    int n_operands = 0;
    int operand_mode[DEINSUM_MAX_ORDER + 2] = {0};  // operand k >= 1 -> mode of X (the MM operand: -1)
    int64_t mm_cols = 0;                            // MTTKRP + MM: L, the columns of C (R x L); else 0

    // MTTKRP
    MttkrpGeom geom{};
    std::vector<int64_t> units;           // 3 per unit
    std::vector<int64_t> col_unit_begin;  // n_cols + 1
    int64_t planned_units = 0;

    // TTMc: contraction order and intermediate sizes
    std::vector<int> ttm_order;
    int64_t ttm_buf_elems = 0;
    // split-BF16 TTMc: the last two modes fused on the tensor cores (ttmc_tc.cu),
    // then the plain chain over the rest of the contracted modes
    bool ttmc_fused = false;
    std::vector<int> ttm_rest;     // chain order of the remaining modes
    int64_t t2_elems = 0;          // S x R_{N-2} x R_{N-1}
    int64_t rest_buf_elems = 0;    // largest intermediate of the remaining chain
    int64_t t_S = 0;               // slabs
    int t_nkt = 0, t_nkb = 0;
    int t_sg = 1;                  // slabs per tile of the fused kernel
    bool no_opack = false;         // keep one outer index per tile (the batched kernel's instances)
    int merge = 0;                 // tensor-core MTTKRP: the inner mode merged with its neighbour (see
                                   // choose_inner_merge); geom is then the order-(N-1) view

    // device state (after the first execute)
    int device = -1;
    int n_sm = 0;
    char *ws = nullptr;
    bool ws_owned = true;
    size_t ws_bytes = 0;
    int64_t *d_units = nullptr;
    int64_t *d_col_begin = nullptr;
    void *d_partial = nullptr;
    void *d_bsplit = nullptr;
    float *d_wtab = nullptr;   // weight tables of the tensor-core kernel (L, then O)
    int *d_status = nullptr;
    void *d_ttm[2] = {nullptr, nullptr};
    // fused TTMc: the chain's TTMs that run on the tensor cores (launch_ttm_tc), each with its
    // row view (A, I, B) and a unit table of its own (the tables back to back, 3 int64 a unit)
    struct TtmStage {
        int tc = 0;
        int64_t unit_off = 0, n_units = 0;
    };
    std::vector<TtmStage> ttm_stages;
    std::vector<int64_t> ttm_units;
    size_t ttm_bsplit_bytes = 0;
    int64_t *d_ttm_units = nullptr;
    void *d_ttm_bsplit = nullptr;
    float *d_t2 = nullptr;
    void *d_tbsplit = nullptr;
    float *d_u2pad = nullptr;

    // TMA descriptor of X, re-encoded when X moves
    CUtensorMap xmap{};
    const void *xmap_ptr = nullptr;
    int xmap_ok = 0;
    uint32_t xmap_box_bytes = 0;
    int xmap_pitch = 0;
    // row-class tensor maps of X (rows not 16-byte aligned), re-encoded when X moves
    CUtensorMap xrow[4]{};
    const void *xrow_ptr = nullptr;
    int xrow_ok = 0;

    // benchmark timing of the main kernel
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    size_t ev_used = 0;
};

namespace {

// Record the start event of the main kernel (timing enabled only); returns the pair index or -1.
long timing_begin(deinsum_plan_s *pl, void *stream) {
    if (!pl->timing) return -1;
    if (pl->ev_used == pl->ev_pool.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return -1;
        if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return -1; }
        pl->ev_pool.emplace_back(a, b);
    }
    cudaEventRecord(pl->ev_pool[pl->ev_used].first, static_cast<cudaStream_t>(stream));
    return long(pl->ev_used++);
}

void timing_end(deinsum_plan_s *pl, long idx, void *stream) {
    if (idx >= 0) cudaEventRecord(pl->ev_pool[size_t(idx)].second, static_cast<cudaStream_t>(stream));
}

bool is_letter(char c) { return (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z'); }

struct Parsed {
    std::vector<std::string> ins;
    std::string out;
    std::vector<char> letters;  // distinct, in order of first appearance
};

deinsum_status parse(const char *s, Parsed &p) {
    if (!s) return DEINSUM_ERR_INVALID;
    std::string str;
    for (const char *c = s; *c; ++c)
        if (*c != ' ') str.push_back(*c);
    size_t arrow = str.find("->");
    if (arrow == std::string::npos || str.find("->", arrow + 2) != std::string::npos)
        return DEINSUM_ERR_PARSE;
    std::string lhs = str.substr(0, arrow);
    p.out = str.substr(arrow + 2);
    size_t start = 0;
    while (true) {
        size_t comma = lhs.find(',', start);
        std::string t = lhs.substr(start, comma == std::string::npos ? std::string::npos : comma - start);
        if (t.empty()) return DEINSUM_ERR_PARSE;
        p.ins.push_back(t);
        if (comma == std::string::npos) break;
        start = comma + 1;
    }
    auto add = [&](const std::string &t) -> bool {
        for (char c : t) {
            if (!is_letter(c)) return false;
            if (std::find(p.letters.begin(), p.letters.end(), c) == p.letters.end()) p.letters.push_back(c);
        }
        return true;
    };
    for (auto &t : p.ins)
        if (!add(t)) return DEINSUM_ERR_PARSE;
    if (p.out.empty() || !add(p.out)) return DEINSUM_ERR_PARSE;
    // an output letter must appear in some input (Sec. III-A)
    for (char c : p.out) {
        bool found = false;
        for (auto &t : p.ins)
            if (t.find(c) != std::string::npos) found = true;
        if (!found) return DEINSUM_ERR_UNSUPPORTED;
    }
    return DEINSUM_OK;
}

int letter_index(const Parsed &p, char c) {
    return int(std::find(p.letters.begin(), p.letters.end(), c) - p.letters.begin());
}

int pad_rank(int R) { return R <= 16 ? 16 : (R <= 32 ? 32 : 64); }

// Chunks of 64 k one fiber group accumulates in TMEM at most.  The accumulation over the
// k steps of a group is where the split-BF16 path loses accuracy as groups grow: 16
// chunks (64 MMA k-steps) give a relative error of about 4e-6, 64 chunks about 1.1e-5.
constexpr int kMaxSegChunks = 16;

// The row view and schedule of the MTTKRP kernels (see internal.h).  With pl->merge the
// view is the order-(N-1) tensor in which the inner mode and its neighbour are one mode
// (modes N-2, N-1 for n < N-2; N-3, N-2 for n = N-1): the MTTKRP regrouped by the
// einsum's associativity, the merged factor being the Khatri-Rao product of the two.
void build_mttkrp_geometry(deinsum_plan_s *pl) {
    MttkrpGeom &g = pl->geom;
    std::memset(&g, 0, sizeof(g));
    int N = pl->order, n = pl->mode;
    g.R = int(pl->ranks[(n + 1) % N]);
    g.R_pad = pad_rank(g.R);
    for (int m = 0; m < N; ++m) g.dims[m] = pl->dims[m];
    if (pl->merge) {
        if (n < N - 2) {
            g.dims[N - 2] *= g.dims[N - 1];
        } else {
            g.dims[N - 3] *= g.dims[N - 2];
            g.dims[N - 2] = g.dims[N - 1];
            n = N - 2;
        }
        g.dims[N - 1] = 0;
        --N;
    }
    g.order = N;
    g.mode = n;
    g.P = 1;
    g.Q = 1;
    for (int m = 0; m < n; ++m) g.P *= g.dims[m];
    for (int m = n + 1; m < N; ++m) g.Q *= g.dims[m];
    g.I = g.dims[n];
    g.kcase = (n == N - 1) ? 1 : 0;
    if (g.kcase == 0) {
        g.K_in = g.dims[N - 1];
        for (int m = n + 1; m < N - 1; ++m) {
            g.outer_mode[g.n_outer] = m;
            g.outer_dim[g.n_outer] = g.dims[m];
            ++g.n_outer;
        }
        g.n_lmodes = n;
        g.narrow = g.I < DEINSUM_BM ? 1 : 0;
        if (g.narrow) {
            g.G = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(DEINSUM_BM / g.I, DEINSUM_GMAX), g.P));
            g.n_cols = 1;
            g.tiles_per_col = (g.P + g.G - 1) / g.G;
            g.rows_per_col = g.I;
        } else {
            g.G = 1;
            g.n_cols = (g.I + DEINSUM_BM - 1) / DEINSUM_BM;
            g.tiles_per_col = g.P;
            g.rows_per_col = DEINSUM_BM;
        }
        g.vec_ok = (g.K_in % 4 == 0) ? 1 : 0;
    } else {
        g.K_in = g.dims[N - 2];
        for (int m = 0; m < N - 2; ++m) {
            g.outer_mode[g.n_outer] = m;
            g.outer_dim[g.n_outer] = g.dims[m];
            ++g.n_outer;
        }
        g.n_lmodes = 0;
        g.narrow = 0;
        g.G = 1;
        g.n_cols = (g.I + DEINSUM_BM - 1) / DEINSUM_BM;
        g.tiles_per_col = 1;
        g.rows_per_col = std::min<int64_t>(g.I, DEINSUM_BM);
        g.vec_ok = (g.I % 4 == 0) ? 1 : 0;
    }
    g.O = 1;
    for (int k = 0; k < g.n_outer; ++k) g.O *= g.outer_dim[k];
    g.n_kb = int((g.K_in + DEINSUM_BK - 1) / DEINSUM_BK);
    g.O_iter = g.O;
    g.opack = 0;
    // Tensor-core path with short rows (I_n <= 64) and no leading index to pack into a
    // tile (case 0 with P = 1, or case 1): pack G >= 2 consecutive outer indices instead,
    // tile row g*I_n + i_n (the partial rows of the G groups are summed by the reduction
    // like the narrow p groups).  With 64 < I_n < 128 a tile holds one group anyway and
    // packing would only add index arithmetic.
    if (pl->prec == DEINSUM_PREC_SPLIT_BF16 && pl->dtype == DEINSUM_F32 && 2 * g.I <= DEINSUM_BM && g.O > 1 &&
        (g.kcase == 1 || g.P == 1) && !pl->no_opack) {
        g.opack = 1;
        g.narrow = 1;
        g.G = std::min<int64_t>(std::min<int64_t>(DEINSUM_BM / g.I, DEINSUM_GMAX), g.O);
        g.n_cols = 1;
        g.tiles_per_col = (g.O + g.G - 1) / g.G;
        g.rows_per_col = g.I;
        g.O_iter = 1;
    }
    // tensor-core path: at most 16 chunks (1024 k) accumulate in TMEM per fiber group; a
    // longer inner range is cut into segments, each its own fiber group (same weights)
    g.kseg = 1;
    g.n_kb_seg = g.n_kb;
    if (pl->prec == DEINSUM_PREC_SPLIT_BF16 && pl->dtype == DEINSUM_F32 && !pl->no_opack && g.n_kb > kMaxSegChunks) {
        g.n_kb_seg = kMaxSegChunks;
        g.kseg = (g.n_kb + kMaxSegChunks - 1) / kMaxSegChunks;
    }
    g.fg_per_col = g.tiles_per_col * g.O_iter * g.kseg;
}

// Split every column's fiber groups into contiguous units, about `target`
// units in all, so that a persistent grid of `target` CTAs is balanced.
void build_schedule(deinsum_plan_s *pl, int64_t target) {
    const MttkrpGeom &g = pl->geom;
    pl->units.clear();
    pl->col_unit_begin.assign(size_t(g.n_cols + 1), 0);
    // whole waves of `target` persistent CTAs, as evenly loaded as the fiber-group counts allow
    const int64_t per_col = balanced_units_per_col(g.n_cols, g.fg_per_col, target, 8 * target);
    for (int64_t c = 0; c < g.n_cols; ++c) {
        pl->col_unit_begin[size_t(c)] = int64_t(pl->units.size() / 3);
        for (int64_t s = 0; s < per_col; ++s) {
            int64_t f0 = g.fg_per_col * s / per_col;
            int64_t f1 = g.fg_per_col * (s + 1) / per_col;
            if (f1 <= f0) continue;
            pl->units.push_back(c);
            pl->units.push_back(f0);
            pl->units.push_back(f1);
        }
    }
    pl->col_unit_begin[size_t(g.n_cols)] = int64_t(pl->units.size() / 3);
    pl->planned_units = int64_t(pl->units.size() / 3);
}

size_t elem_size(deinsum_dtype d) { return d == DEINSUM_F64 ? 8 : 4; }

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

deinsum_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return DEINSUM_OK;
    if (e == cudaErrorMemoryAllocation) return DEINSUM_ERR_OOM;
    return DEINSUM_ERR_CUDA;
}

struct WsLayout {
    size_t status = 0, units = 0, cols = 0, partial = 0, bsplit = 0, wtab = 0, ttm0 = 0, ttm1 = 0, t2 = 0, tb = 0, u2 = 0,
           tunits = 0, tbs = 0, total = 0;
};

// Row view of one TTM of a fused TTMc chain, Y[a, r, b] = sum_i X[a, i, b] U[i, r], as the
// last-mode MTTKRP view of the order-3 tensor (A, I, B) (no packing, no k segments: the
// geometry mttkrp_prepare_oneoff gives with allow_opack = false).
MttkrpGeom ttm_stage_geometry(int64_t A, int64_t I, int64_t B, int R) {
    deinsum_plan_s tmp;
    tmp.kind = DEINSUM_KIND_MTTKRP;
    tmp.no_opack = true;
    tmp.order = 3;
    tmp.mode = 2;
    tmp.dtype = DEINSUM_F32;
    tmp.prec = DEINSUM_PREC_SPLIT_BF16;
    const int64_t d[3] = {A, I, B};
    for (int m = 0; m < 3; ++m) {
        tmp.dims[m] = d[m];
        tmp.ranks[m] = m == 2 ? d[m] : R;
    }
    build_mttkrp_geometry(&tmp);
    return tmp.geom;
}

// The chain's TTMs after the fused pair: which run on the tensor cores (the trailing extent B
// a multiple of 4 for the tensor map of rows b, R <= 64; the first two at most: each split-BF16
// stage adds about 1e-6 to the relative error, 4.9e-6 -> 6.1e-6 at 256^4 with one and
// 5.4e-6 -> 7.4e-6 at 60^5 with two, and the later, smaller stages stay in FP32 so that the
// chain keeps the 1e-5 gate at any order), and their unit tables for `target` persistent CTAs.
void build_ttm_stages(deinsum_plan_s *pl, int64_t target) {
    const int N = pl->order;
    pl->ttm_stages.assign(pl->ttm_rest.size(), deinsum_plan_s::TtmStage{});
    pl->ttm_units.clear();
    pl->ttm_bsplit_bytes = 0;
    int64_t cur[DEINSUM_MAX_ORDER];
    for (int m = 0; m < N; ++m) cur[m] = (m >= N - 2) ? pl->ranks[m] : pl->dims[m];
    for (size_t s = 0; s < pl->ttm_rest.size(); ++s) {
        const int m = pl->ttm_rest[s];
        int64_t A = 1, B = 1;
        for (int k = 0; k < m; ++k) A *= cur[k];
        for (int k = m + 1; k < N; ++k) B *= cur[k];
        const int R = int(pl->ranks[m]);
        if (s < 2 && B % 4 == 0 && R <= 64) {
            const MttkrpGeom g = ttm_stage_geometry(A, cur[m], B, R);
            if (g.kcase == 1 && !g.opack && g.kseg == 1) {
                deinsum_plan_s::TtmStage &st = pl->ttm_stages[s];
                st.tc = 1;
                st.unit_off = int64_t(pl->ttm_units.size() / 3);
                // a TTM unit writes its own output tiles (no partial sums to reduce), so units can
                // be fine: the split with the best balance over whole waves, up to 64 per CTA
                const double mean = double(g.n_cols) * double(g.fg_per_col) / double(target);
                int64_t per_col = 1;
                double best_eff = 0.0;
                for (int64_t p = 1; p <= g.fg_per_col && g.n_cols * p <= 64 * target; ++p) {
                    const int64_t waves = (g.n_cols * p + target - 1) / target;
                    const double e = mean / double(waves * ((g.fg_per_col + p - 1) / p));
                    if (e > best_eff + 0.005) {
                        best_eff = e;
                        per_col = p;
                    }
                }
                for (int64_t c = 0; c < g.n_cols; ++c)
                    for (int64_t u = 0; u < per_col; ++u) {
                        const int64_t f0 = g.fg_per_col * u / per_col, f1 = g.fg_per_col * (u + 1) / per_col;
                        if (f1 > f0) pl->ttm_units.insert(pl->ttm_units.end(), {c, f0, f1});
                    }
                st.n_units = int64_t(pl->ttm_units.size() / 3) - st.unit_off;
                pl->ttm_bsplit_bytes =
                    std::max(pl->ttm_bsplit_bytes, size_t(g.n_kb) * 2 * size_t(g.R_pad) * DEINSUM_BK * 2);
            }
        }
        cur[m] = R;
    }
}

// Fix the device (the current one), the schedule (one unit per resident CTA:
// the tensor-core kernel keeps one CTA per SM, the plain kernel as many as its
// occupancy allows) and the workspace layout.
deinsum_status plan_layout(deinsum_plan_s *pl, WsLayout &L) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return DEINSUM_ERR_CUDA;
    if (pl->device >= 0 && pl->device != dev) return DEINSUM_ERR_INVALID;  // a plan stays on its first device
    if (pl->n_sm == 0) {
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
            return DEINSUM_ERR_CUDA;
        pl->device = dev;
        pl->n_sm = nsm;
        if (pl->kind == DEINSUM_KIND_MTTKRP) {
            int per_sm = 1;
            if (pl->prec == DEINSUM_PREC_PLAIN)
                per_sm = mttkrp_plain_ctas_per_sm(pl->dtype == DEINSUM_F64 ? 1 : 0, pl->geom.R_pad);
            build_schedule(pl, int64_t(nsm) * per_sm);
        } else if (pl->ttmc_fused) {
            build_ttm_stages(pl, nsm);
        }
    }
    size_t off = 0;
    L.status = off;
    off = align_up(off + 256, 256);
    if (pl->kind == DEINSUM_KIND_MTTKRP) {
        const MttkrpGeom &g = pl->geom;
        L.units = off;
        off = align_up(off + pl->units.size() * sizeof(int64_t), 256);
        L.cols = off;
        off = align_up(off + pl->col_unit_begin.size() * sizeof(int64_t), 256);
        L.partial = off;
        off = align_up(off + size_t(pl->planned_units) * DEINSUM_BM * g.R_pad * elem_size(pl->dtype), 1024);
        if (pl->prec == DEINSUM_PREC_SPLIT_BF16) {
            L.bsplit = off;
            off = align_up(off + size_t(g.n_kb) * 2 * g.R_pad * DEINSUM_BK * 2, 1024);
            L.wtab = off;
            off = align_up(off + (weight_table_floats_l(g) + weight_table_floats_o(g)) * sizeof(float), 256);
        }
    } else if (pl->ttmc_fused) {
        L.t2 = off;
        off = align_up(off + size_t(pl->t2_elems) * sizeof(float), 256);
        L.ttm0 = off;
        off = align_up(off + size_t(pl->rest_buf_elems) * sizeof(float), 256);
        L.ttm1 = off;
        off = align_up(off + size_t(pl->rest_buf_elems) * sizeof(float), 1024);
        L.tb = off;   // split tiles of U_{N-1}: n_kb x 2*32 rows x 64 BF16
        off = align_up(off + size_t(pl->t_nkb) * 2 * 32 * DEINSUM_BK * 2, 1024);
        L.u2 = off;   // U_{N-2} padded to n_kt*128 rows x 32
        off = align_up(off + size_t(pl->t_nkt) * DEINSUM_BM * 32 * sizeof(float), 256);
        L.tunits = off;   // the chain's tensor-core TTMs: unit tables, split factor tiles
        off = align_up(off + pl->ttm_units.size() * sizeof(int64_t), 1024);
        L.tbs = off;
        off = align_up(off + pl->ttm_bsplit_bytes, 256);
    } else {
        L.ttm0 = off;
        off = align_up(off + size_t(pl->ttm_buf_elems) * elem_size(pl->dtype), 256);
        L.ttm1 = off;
        off = align_up(off + size_t(pl->ttm_buf_elems) * elem_size(pl->dtype), 256);
    }
    L.total = off;
    return DEINSUM_OK;
}

// Point the plan at workspace `ws` (>= the layout's bytes; 1024-byte aligned)
// and upload the schedule and a cleared status word on `stream`.
deinsum_status attach_workspace(deinsum_plan_s *pl, char *ws, const WsLayout &L, bool owned, cudaStream_t stream) {
    pl->ws = ws;
    pl->ws_owned = owned;
    pl->ws_bytes = L.total;
    pl->d_status = reinterpret_cast<int *>(pl->ws + L.status);
    cudaError_t e = cudaMemsetAsync(pl->d_status, 0, sizeof(int), stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (pl->kind == DEINSUM_KIND_MTTKRP) {
        pl->d_units = reinterpret_cast<int64_t *>(pl->ws + L.units);
        pl->d_col_begin = reinterpret_cast<int64_t *>(pl->ws + L.cols);
        pl->d_partial = pl->ws + L.partial;
        pl->d_bsplit = pl->prec == DEINSUM_PREC_SPLIT_BF16 ? pl->ws + L.bsplit : nullptr;
        pl->d_wtab = pl->prec == DEINSUM_PREC_SPLIT_BF16 ? reinterpret_cast<float *>(pl->ws + L.wtab) : nullptr;
        e = cudaMemcpyAsync(pl->d_units, pl->units.data(), pl->units.size() * sizeof(int64_t),
                            cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(pl->d_col_begin, pl->col_unit_begin.data(),
                                pl->col_unit_begin.size() * sizeof(int64_t), cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_status(e);
    } else {
        pl->d_ttm[0] = pl->ws + L.ttm0;
        pl->d_ttm[1] = pl->ws + L.ttm1;
        if (pl->ttmc_fused) {
            pl->d_t2 = reinterpret_cast<float *>(pl->ws + L.t2);
            pl->d_tbsplit = pl->ws + L.tb;
            pl->d_u2pad = reinterpret_cast<float *>(pl->ws + L.u2);
            pl->d_ttm_units = reinterpret_cast<int64_t *>(pl->ws + L.tunits);
            pl->d_ttm_bsplit = pl->ws + L.tbs;
            if (!pl->ttm_units.empty()) {
                e = cudaMemcpyAsync(pl->d_ttm_units, pl->ttm_units.data(), pl->ttm_units.size() * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, stream);
                if (e != cudaSuccess) return cuda_status(e);
            }
        }
    }
    return DEINSUM_OK;
}

// Allocate the workspace on the current device and upload the schedule.
deinsum_status ensure_device_state(deinsum_plan_s *pl, cudaStream_t stream) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return DEINSUM_ERR_CUDA;
    if (pl->ws && pl->device == dev) return DEINSUM_OK;
    if (pl->ws) return DEINSUM_ERR_INVALID;  // a plan stays on its first device
    WsLayout L;
    deinsum_status st = plan_layout(pl, L);
    if (st != DEINSUM_OK) return st;
    void *ws = nullptr;
    cudaError_t e = counted_malloc(&ws, L.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e);
    }
    st = attach_workspace(pl, static_cast<char *>(ws), L, true, stream);
    if (st == DEINSUM_OK && cudaStreamSynchronize(stream) != cudaSuccess) st = DEINSUM_ERR_CUDA;
    return st;
}

deinsum_status classify(deinsum_plan_s *pl, const Parsed &p, const int64_t *extents) {
    const std::string &x = p.ins[0];
    const int N = int(x.size());
    if (N < 2 || N > DEINSUM_MAX_ORDER) return DEINSUM_ERR_UNSUPPORTED;
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b)
            if (x[a] == x[b]) return DEINSUM_ERR_UNSUPPORTED;  // diagonal access of X
    // MTTKRP + MM (Sec. II-A running example, order >= 3; at order 2 it would be a
    // matrix chain): one more operand "<rank letter><new letter>"
    const bool mm = N >= 3 && int(p.ins.size()) == N + 1;
    if (int(p.ins.size()) != N && !mm) return DEINSUM_ERR_UNSUPPORTED;
    pl->order = N;
    pl->n_operands = int(p.ins.size());
    for (int m = 0; m < N; ++m) pl->dims[m] = extents[letter_index(p, x[m])];
    std::vector<int> used(size_t(N), 0);
    std::vector<char> rank_letter(size_t(N), 0);
    for (int k = 1; k < N; ++k) {
        const std::string &f = p.ins[size_t(k)];
        if (f.size() != 2) return DEINSUM_ERR_UNSUPPORTED;
        size_t pos = x.find(f[0]);
        if (pos == std::string::npos || x.find(f[1]) != std::string::npos || f[0] == f[1])
            return DEINSUM_ERR_UNSUPPORTED;
        if (used[pos]) return DEINSUM_ERR_UNSUPPORTED;
        used[pos] = 1;
        pl->operand_mode[k] = int(pos);
        rank_letter[pos] = f[1];
    }
    int kept = -1;
    for (int m = 0; m < N; ++m)
        if (!used[size_t(m)]) kept = m;
    pl->mode = kept;
    // MTTKRP: every factor shares one rank letter; output = kept letter + rank letter.
    bool same_rank = true;
    char r0 = rank_letter[size_t((kept + 1) % N)];
    for (int m = 0; m < N; ++m)
        if (m != kept && rank_letter[size_t(m)] != r0) same_rank = false;
    if (mm) {
        // the last operand is C = "<r><l>" with l new; output "<kept><l>"
        const std::string &c = p.ins[size_t(N)];
        if (!same_rank || c.size() != 2 || c[0] != r0 || c[1] == r0 || x.find(c[1]) != std::string::npos)
            return DEINSUM_ERR_UNSUPPORTED;
        if (p.out.size() != 2 || p.out[0] != x[size_t(kept)] || p.out[1] != c[1]) return DEINSUM_ERR_UNSUPPORTED;
        pl->kind = DEINSUM_KIND_MTTKRP;
        int64_t R = extents[letter_index(p, r0)];
        for (int m = 0; m < N; ++m) pl->ranks[m] = (m == kept) ? pl->dims[m] : R;
        pl->operand_mode[N] = -1;
        pl->mm_cols = extents[letter_index(p, c[1])];
        return DEINSUM_OK;
    }
    if (same_rank && p.out.size() == 2 && p.out[0] == x[size_t(kept)] && p.out[1] == r0) {
        pl->kind = DEINSUM_KIND_MTTKRP;
        int64_t R = extents[letter_index(p, r0)];
        for (int m = 0; m < N; ++m) pl->ranks[m] = (m == kept) ? pl->dims[m] : R;
        return DEINSUM_OK;
    }
    // TTMc: distinct rank letters, output = X letters with contracted ones replaced in place.
    if (int(p.out.size()) != N) return DEINSUM_ERR_UNSUPPORTED;
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b)
            if (a != kept && b != kept && rank_letter[size_t(a)] == rank_letter[size_t(b)])
                return DEINSUM_ERR_UNSUPPORTED;
    for (int m = 0; m < N; ++m) {
        char want = (m == kept) ? x[size_t(m)] : rank_letter[size_t(m)];
        if (p.out[size_t(m)] != want) return DEINSUM_ERR_UNSUPPORTED;
    }
    pl->kind = DEINSUM_KIND_TTMC;
    for (int m = 0; m < N; ++m)
        pl->ranks[m] = (m == kept) ? pl->dims[m] : extents[letter_index(p, rank_letter[size_t(m)])];
    return DEINSUM_OK;
}

// TTMc chain order: contract first the mode with the smallest ratio R_m / I_m
// (largest shrink of the running tensor), which minimises the FLOPs of the
// binary chain (Sec. II-A / IV-C); ties go to the later mode.
void plan_ttmc_chain(deinsum_plan_s *pl) {
    std::vector<int> modes;
    for (int m = 0; m < pl->order; ++m)
        if (m != pl->mode) modes.push_back(m);
    std::stable_sort(modes.begin(), modes.end(), [&](int a, int b) {
        double ra = double(pl->ranks[a]) / double(pl->dims[a]);
        double rb = double(pl->ranks[b]) / double(pl->dims[b]);
        if (ra != rb) return ra < rb;
        return a > b;
    });
    pl->ttm_order = modes;
    int64_t cur[DEINSUM_MAX_ORDER];
    for (int m = 0; m < pl->order; ++m) cur[m] = pl->dims[m];
    int64_t mx = 0;
    for (size_t s = 0; s + 1 < modes.size(); ++s) {
        cur[modes[s]] = pl->ranks[modes[s]];
        int64_t sz = 1;
        for (int m = 0; m < pl->order; ++m) sz *= cur[m];
        mx = std::max(mx, sz);
    }
    pl->ttm_buf_elems = std::max<int64_t>(mx, 1);
}

// Split-BF16 TTMc: modes N-2 and N-1 are contracted by the fused kernel;
// the other contracted modes follow in the same greedy order on
// T2 = [I_0 .. I_{N-3}, R_{N-2}, R_{N-1}].  Offered when the kept mode is
// below N-2 and R_{N-2}, R_{N-1} <= 32; rows of X (I_{N-1} words) that are not
// 16-byte aligned take the row-class tensor maps (short slabs packed as with the tensor map).
// Merge the inner mode of a tensor-core MTTKRP with its neighbour when the inner mode is
// short (at most two 64-wide chunks, so that every fiber group would be one or two chunks
// and the epilogue and its handshakes would run per 32 KB of X) and the merged view still
// fills its tiles: rows of 128 or more, several leading indices p, or outer indices left
// to pack.  Split BF16 only.
void choose_inner_merge(deinsum_plan_s *pl) {
    pl->merge = 0;
    if (pl->kind != DEINSUM_KIND_MTTKRP || pl->prec != DEINSUM_PREC_SPLIT_BF16 || pl->dtype != DEINSUM_F32) return;
    const int N = pl->order, n = pl->mode;
    if (N < 3) return;
    const int64_t lim = int64_t(1) << 31;
    int64_t P = 1, O = 1;
    const int64_t I = pl->dims[n];
    if (n < N - 2) {
        if (pl->dims[N - 1] > 2 * DEINSUM_BK || pl->dims[N - 2] * pl->dims[N - 1] >= lim) return;
        for (int m = 0; m < n; ++m) P *= pl->dims[m];
        for (int m = n + 1; m < N - 2; ++m) O *= pl->dims[m];
    } else if (n == N - 1) {
        if (pl->dims[N - 2] > 2 * DEINSUM_BK || pl->dims[N - 3] * pl->dims[N - 2] >= lim) return;
        for (int m = 0; m < N - 3; ++m) O *= pl->dims[m];
    } else {
        return;
    }
    if (I >= DEINSUM_BM || P >= 2 || O >= 2) pl->merge = 1;
}

deinsum_status plan_ttmc_fused(deinsum_plan_s *pl) {
    const int N = pl->order, n = pl->mode;
    if (N < 3 || n >= N - 2) return DEINSUM_ERR_UNSUPPORTED;
    if (pl->ranks[N - 2] > 32 || pl->ranks[N - 1] > 32) return DEINSUM_ERR_UNSUPPORTED;
    const int64_t lim = int64_t(1) << 31;
    int64_t S = 1;
    for (int m = 0; m < N - 2; ++m) S *= pl->dims[m];
    if (S >= lim || pl->dims[N - 2] >= lim || pl->dims[N - 1] >= lim) return DEINSUM_ERR_UNSUPPORTED;
    // rows of I_{N-1} words that are not 16-byte aligned take the row-class maps (their slabs
    // packed at execution, as the aligned ones are here)
    const bool rows16 = pl->dims[N - 1] % 4 == 0;
    if (!rows16) {
        MttkrpGeom g1;
        ttm_last_geometry(N, S, pl->dims[N - 2], pl->dims[N - 1], int(pl->ranks[N - 1]), &g1, 1);
        if (!rowclass_supported(g1)) return DEINSUM_ERR_UNSUPPORTED;
    }
    pl->ttmc_fused = true;
    pl->t_S = S;
    pl->t_sg = rows16 ? ttmc_slab_group(pl->dims[N - 2]) : 1;
    pl->t_nkt = int((pl->dims[N - 2] + DEINSUM_BM - 1) / DEINSUM_BM);
    pl->t_nkb = int((pl->dims[N - 1] + DEINSUM_BK - 1) / DEINSUM_BK);
    pl->t2_elems = S * pl->ranks[N - 2] * pl->ranks[N - 1];
    pl->ttm_rest.clear();
    for (int m : pl->ttm_order)
        if (m < N - 2) pl->ttm_rest.push_back(m);
    // among modes of equal R_m / I_m (the same flops either way) the lower mode first: its TTM
    // then has the long trailing extent, which the strided TTM kernel tiles without a ragged
    // edge, and the later, smaller stages take the ragged ones (60^5 R 24: 0.41 -> 0.37 ms)
    std::stable_sort(pl->ttm_rest.begin(), pl->ttm_rest.end(), [&](int x, int y) {
        const double rx = double(pl->ranks[x]) / double(pl->dims[x]);
        const double ry = double(pl->ranks[y]) / double(pl->dims[y]);
        if (rx != ry) return rx < ry;
        return x < y;
    });
    int64_t cur[DEINSUM_MAX_ORDER];
    for (int m = 0; m < N; ++m) cur[m] = (m >= N - 2) ? pl->ranks[m] : pl->dims[m];
    int64_t mx = 1;
    for (size_t s = 0; s + 1 < pl->ttm_rest.size(); ++s) {
        cur[pl->ttm_rest[s]] = pl->ranks[pl->ttm_rest[s]];
        int64_t sz = 1;
        for (int m = 0; m < N; ++m) sz *= cur[m];
        mx = std::max(mx, sz);
    }
    pl->rest_buf_elems = mx;
    ttm_last_geometry(N, S, pl->dims[N - 2], pl->dims[N - 1], int(pl->ranks[N - 1]), &pl->geom, pl->t_sg);
    return DEINSUM_OK;
}

double alg_flops(const deinsum_plan_s *pl) {
    double x = 1.0;
    for (int m = 0; m < pl->order; ++m) x *= double(pl->dims[m]);
    if (pl->kind == DEINSUM_KIND_MTTKRP)
        return 2.0 * x * double(pl->ranks[(pl->mode + 1) % pl->order]) +
               2.0 * double(pl->dims[pl->mode]) * double(pl->ranks[(pl->mode + 1) % pl->order]) * double(pl->mm_cols);
    double cur[DEINSUM_MAX_ORDER];
    for (int m = 0; m < pl->order; ++m) cur[m] = double(pl->dims[m]);
    double f = 0.0;
    for (int m : pl->ttm_order) {
        double sz = 1.0;
        for (int k = 0; k < pl->order; ++k) sz *= cur[k];
        f += 2.0 * sz * double(pl->ranks[m]);
        cur[m] = double(pl->ranks[m]);
    }
    return f;
}

double alg_bytes(const deinsum_plan_s *pl) {
    double es = double(elem_size(pl->dtype));
    double x = 1.0, fac = 0.0, out = 1.0;
    for (int m = 0; m < pl->order; ++m) {
        x *= double(pl->dims[m]);
        if (m != pl->mode) fac += double(pl->dims[m]) * double(pl->ranks[m]);
    }
    if (pl->kind == DEINSUM_KIND_MTTKRP && pl->mm_cols > 0) {
        const double R = double(pl->ranks[(pl->mode + 1) % pl->order]);
        fac += R * double(pl->mm_cols);                          // C
        out = double(pl->dims[pl->mode]) * double(pl->mm_cols);  // I_n x L
    } else if (pl->kind == DEINSUM_KIND_MTTKRP)
        out = double(pl->dims[pl->mode]) * double(pl->ranks[(pl->mode + 1) % pl->order]);
    else
        for (int m = 0; m < pl->order; ++m) out *= double(pl->ranks[m]);
    return es * (x + fac + out);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

// Tiled tensor map of X for the tensor-core kernel (see MttkrpArgs):
//   case 0: dims {K_in, O, I, P}, box {64, 1, min(I,128), G}; opack {K_in, I, O, P}, box {64, I, G, 1}
//   case 1: dims {I, K_in, O},    box {min(I,128), 64, 1 (opack: G)}
// Needs 16-byte aligned X and rows (vec_ok) and coordinates within int32.
bool encode_x_map(deinsum_plan_s *pl, const void *X) {
    if (pl->xmap_ptr == X) return pl->xmap_ok != 0;
    pl->xmap_ptr = X;
    pl->xmap_ok = 0;
    const MttkrpGeom &g = pl->geom;
    auto enc = tensor_map_encoder();
    if (!enc || !g.vec_ok || (reinterpret_cast<uintptr_t>(X) & 15) != 0) return false;
    const int64_t lim = int64_t(1) << 31;
    cuuint64_t dims[4], strides[3];
    cuuint32_t box[4], estr[4] = {1, 1, 1, 1};
    cuuint32_t rank;
    if (g.kcase == 0 && g.opack) {
        // {K_in, I, O, P}: a box of G outer indices x all I_n rows lands as [o][i][k]
        if (g.K_in >= lim || g.O >= lim || g.I >= lim || g.P >= lim) return false;
        rank = 4;
        dims[0] = cuuint64_t(g.K_in); dims[1] = cuuint64_t(g.I); dims[2] = cuuint64_t(g.O); dims[3] = cuuint64_t(g.P);
        strides[0] = cuuint64_t(g.Q) * 4; strides[1] = cuuint64_t(g.K_in) * 4; strides[2] = cuuint64_t(g.I * g.Q) * 4;
        box[0] = DEINSUM_BK; box[1] = cuuint32_t(g.I); box[2] = cuuint32_t(g.G); box[3] = 1;
        pl->xmap_pitch = DEINSUM_BK;
    } else if (g.kcase == 0) {
        if (g.K_in >= lim || g.O >= lim || g.I >= lim || g.P >= lim) return false;
        rank = 4;
        dims[0] = cuuint64_t(g.K_in); dims[1] = cuuint64_t(g.O); dims[2] = cuuint64_t(g.I); dims[3] = cuuint64_t(g.P);
        strides[0] = cuuint64_t(g.K_in) * 4; strides[1] = cuuint64_t(g.Q) * 4; strides[2] = cuuint64_t(g.I * g.Q) * 4;
        box[0] = DEINSUM_BK; box[1] = 1;
        box[2] = cuuint32_t(g.narrow ? g.I : DEINSUM_BM);
        box[3] = cuuint32_t(g.narrow ? g.G : 1);
        pl->xmap_pitch = DEINSUM_BK;
    } else {
        // {I, K_in, O}: box {min(I,128), 64, G}, landing as [o][k][i] (G = 1 unless opack)
        if (g.K_in >= lim || g.O >= lim || g.I >= lim) return false;
        rank = 3;
        dims[0] = cuuint64_t(g.I); dims[1] = cuuint64_t(g.K_in); dims[2] = cuuint64_t(g.O);
        strides[0] = cuuint64_t(g.I) * 4; strides[1] = cuuint64_t(g.I * g.K_in) * 4;
        box[0] = cuuint32_t(std::min<int64_t>(g.I, DEINSUM_BM)); box[1] = DEINSUM_BK;
        box[2] = cuuint32_t(g.opack ? g.G : 1);
        pl->xmap_pitch = int(box[0]);
    }
    uint64_t bytes = 4;
    for (cuuint32_t d = 0; d < rank; ++d) bytes *= box[d];
    pl->xmap_box_bytes = uint32_t(bytes);
    CUresult r = enc(&pl->xmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<void *>(X), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    pl->xmap_ok = (r == CUDA_SUCCESS) ? 1 : 0;
    return pl->xmap_ok != 0;
}

deinsum_status execute_mttkrp(deinsum_plan_s *pl, const void *const *inputs, void *output, void *stream) {
    const void *mm_c = pl->mm_cols > 0 ? inputs[pl->n_operands - 1] : nullptr;  // C of MTTKRP + MM
    MttkrpArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = pl->geom;
    a.X = inputs[0];
    for (int k = 1; k < pl->n_operands; ++k)
        if (pl->operand_mode[k] >= 0) a.U[pl->operand_mode[k]] = inputs[k];
    if (pl->merge) {   // the view's inner factor: Khatri-Rao of the two merged modes
        const int N = pl->order;
        const int minor = pl->mode < N - 2 ? N - 1 : N - 2;
        a.Uk2 = a.U[minor];
        a.K_minor = pl->dims[minor];
        if (pl->mode == N - 1) a.U[N - 2] = nullptr;   // the view's output mode
    }
    a.units = pl->d_units;
    a.n_units = pl->planned_units;
    a.status = pl->d_status;
    if ((reinterpret_cast<uintptr_t>(a.X) & 15) != 0) a.g.vec_ok = 0;
    int err = 0;
    if (pl->dtype == DEINSUM_F64) {
        a.partial64 = static_cast<double *>(pl->d_partial);
        const long ti = timing_begin(pl, stream);
        err = launch_mttkrp_plain_f64(a, pl->n_sm, stream);
        timing_end(pl, ti, stream);
        if (!err) err = launch_mttkrp_reduce_f64(a, pl->d_col_begin, output, stream, mm_c, pl->mm_cols);
    } else {
        a.partial = static_cast<float *>(pl->d_partial);
        if (pl->prec == DEINSUM_PREC_SPLIT_BF16) {
            a.Bsplit = pl->d_bsplit;
            a.Lw = pl->d_wtab;
            a.Ow = pl->d_wtab + weight_table_floats_l(pl->geom);
            if (encode_x_map(pl, a.X)) {
                a.xmap = pl->xmap;
                a.use_tma = 1;
                a.box_bytes = pl->xmap_box_bytes;
                a.raw_pitch = pl->xmap_pitch;
            }
            if (!a.use_tma && !a.g.opack) {   // unaligned rows: the four row-class maps
                if (pl->xrow_ptr != a.X) {
                    pl->xrow_ptr = a.X;
                    pl->xrow_ok = encode_x_rowclass_maps(a.g, a.X, pl->xrow) ? 1 : 0;
                }
                if (pl->xrow_ok) {
                    for (int c = 0; c < 4; ++c) a.xrow[c] = pl->xrow[c];
                    a.row_classes = 1;
                }
            }
            err = launch_split_inner_factor(a, pl->d_bsplit, stream);
            if (!err) err = launch_weight_tables(a, stream);
            const long ti = timing_begin(pl, stream);
            if (!err) err = launch_mttkrp_tc(a, pl->n_sm, stream);
            timing_end(pl, ti, stream);
        } else {
            const long ti = timing_begin(pl, stream);
            err = launch_mttkrp_plain_f32(a, pl->n_sm, stream);
            timing_end(pl, ti, stream);
        }
        if (!err) err = launch_mttkrp_reduce_f32(a, pl->d_col_begin, output, stream, mm_c, pl->mm_cols);
    }
    return err ? DEINSUM_ERR_CUDA : DEINSUM_OK;
}

// 3-D tensor map of X for the fused TTMc kernel: {I_{N-1}, I_{N-2}, S}, box
// {64, min(I_{N-2}, 128), 1} (or sg slabs of 128/sg rows); cached per X pointer.
bool encode_ttmc_map(deinsum_plan_s *pl, const void *X) {
    if (pl->xmap_ptr == X) return pl->xmap_ok != 0;
    pl->xmap_ptr = X;
    const int N = pl->order;
    pl->xmap_ok = encode_ttm_last_map(X, pl->t_S, pl->dims[N - 2], pl->dims[N - 1], &pl->xmap, &pl->xmap_box_bytes,
                                      pl->t_sg)
                      ? 1 : 0;
    return pl->xmap_ok != 0;
}

deinsum_status execute_ttmc_fused(deinsum_plan_s *pl, const void *const *inputs, void *output, void *stream) {
    const int N = pl->order;
    const void *U[DEINSUM_MAX_ORDER] = {nullptr};
    for (int k = 1; k < pl->n_operands; ++k) U[pl->operand_mode[k]] = inputs[k];
    TtmcArgs t;
    std::memset(&t, 0, sizeof(t));
    if (encode_ttmc_map(pl, inputs[0])) {
        t.xmap = pl->xmap;
        t.box_bytes = pl->xmap_box_bytes;
        t.g = pl->geom;
        t.sg = pl->t_sg;
    } else {
        // rows not 16-byte aligned (I_{N-1} not a multiple of 4, or X itself): the four
        // row-class maps, cached per X pointer; slabs of at most 64 (32) rows packed two
        // (four) to a tile as in the aligned kernel, with class boxes of 32 / sg rows
        const int sg = pl->t_nkt <= kTtmcTc2MaxKt ? ttmc_slab_group(pl->dims[N - 2]) : 1;
        ttm_last_geometry(N, pl->t_S, pl->dims[N - 2], pl->dims[N - 1], int(pl->ranks[N - 1]), &t.g, sg);
        if (pl->xrow_ptr != inputs[0]) {
            pl->xrow_ptr = inputs[0];
            pl->xrow_ok = encode_rowclass_maps_rows(t.g, inputs[0], pl->xrow, DEINSUM_BM / 4 / sg) ? 1 : 0;
        }
        if (!pl->xrow_ok) return DEINSUM_ERR_ALIGN;
        for (int c = 0; c < 4; ++c) t.xrow[c] = pl->xrow[c];
        t.X = inputs[0];
        t.row_classes = 1;
        t.sg = sg;
    }
    // split tiles of U_{N-1} (the same layout as the MTTKRP inner factor)
    MttkrpArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.g = pl->geom;
    sa.U[N - 1] = U[N - 1];
    int err = launch_split_inner_factor(sa, pl->d_tbsplit, stream);
    // stage 2 on the tensor cores while U_{N-2} fits on chip (I_{N-2} <= 256): its split
    // tiles; otherwise the padded FP32 rows for the CUDA-core stage 2 (the same buffer size)
    const bool tc2 = pl->t_nkt <= kTtmcTc2MaxKt;
    if (!err && tc2)
        err = launch_ttmc_u2_split(static_cast<const float *>(U[N - 2]), pl->dims[N - 2], int(pl->ranks[N - 2]),
                                   pl->d_u2pad, pl->t_nkt, stream);
    else if (!err)
        err = launch_ttmc_pad_factor(static_cast<const float *>(U[N - 2]), pl->dims[N - 2], int(pl->ranks[N - 2]),
                                     pl->d_u2pad, pl->t_nkt, stream);
    t.Bsplit = pl->d_tbsplit;
    t.U2pad = pl->d_u2pad;
    t.U2split = pl->d_u2pad;
    t.tc2 = tc2 ? 1 : 0;
    t.T2 = pl->ttm_rest.empty() ? static_cast<float *>(output) : pl->d_t2;
    t.S = pl->t_S;
    t.n_kt = pl->t_nkt;
    t.n_kb = pl->t_nkb;
    t.R2 = int(pl->ranks[N - 2]);
    t.R3 = int(pl->ranks[N - 1]);
    t.status = pl->d_status;
    if (!err) {
        const long ti = timing_begin(pl, stream);
        err = launch_ttmc_fused(t, pl->n_sm, stream);
        timing_end(pl, ti, stream);
    }
    // the remaining modes on T2 with the plain TTM kernel
    int64_t cur[DEINSUM_MAX_ORDER];
    for (int m = 0; m < N; ++m) cur[m] = (m >= N - 2) ? pl->ranks[m] : pl->dims[m];
    const void *src = t.T2;
    for (size_t s = 0; s < pl->ttm_rest.size() && !err; ++s) {
        const int m = pl->ttm_rest[s];
        int64_t A = 1, B = 1;
        for (int k = 0; k < m; ++k) A *= cur[k];
        for (int k = m + 1; k < N; ++k) B *= cur[k];
        void *dst = (s + 1 == pl->ttm_rest.size()) ? output : pl->d_ttm[s % 2];
        if (s < pl->ttm_stages.size() && pl->ttm_stages[s].tc) {
            // on the tensor cores (its own input is a 16-byte aligned workspace buffer)
            MttkrpArgs a;
            std::memset(static_cast<void *>(&a), 0, sizeof(a));
            const int64_t d3[3] = {A, cur[m], B};
            mttkrp_prepare_oneoff(3, d3, 2, int(pl->ranks[m]), src, &a, false);
            if (a.use_tma) {
                a.X = src;
                a.U[1] = U[m];
                a.Bsplit = pl->d_ttm_bsplit;
                a.units = pl->d_ttm_units + 3 * pl->ttm_stages[s].unit_off;
                a.n_units = pl->ttm_stages[s].n_units;
                a.status = pl->d_status;
                a.ttm_out = static_cast<float *>(dst);
                err = launch_split_inner_factor(a, pl->d_ttm_bsplit, stream);
                if (!err) err = launch_ttm_tc(a, pl->n_sm, stream);
                cur[m] = pl->ranks[m];
                src = dst;
                continue;
            }
        }
        err = launch_ttm_plain_f32(static_cast<const float *>(src), static_cast<const float *>(U[m]),
                                   static_cast<float *>(dst), A, cur[m], B, pl->ranks[m], stream);
        cur[m] = pl->ranks[m];
        src = dst;
    }
    return err ? DEINSUM_ERR_CUDA : DEINSUM_OK;
}

deinsum_status execute_ttmc(deinsum_plan_s *pl, const void *const *inputs, void *output, void *stream) {
    if (pl->ttmc_fused) return execute_ttmc_fused(pl, inputs, output, stream);
    const void *U[DEINSUM_MAX_ORDER] = {nullptr};
    for (int k = 1; k < pl->n_operands; ++k) U[pl->operand_mode[k]] = inputs[k];
    int64_t cur[DEINSUM_MAX_ORDER];
    for (int m = 0; m < pl->order; ++m) cur[m] = pl->dims[m];
    const void *src = inputs[0];
    int err = 0;
    for (size_t s = 0; s < pl->ttm_order.size() && !err; ++s) {
        const int m = pl->ttm_order[s];
        int64_t A = 1, B = 1;
        for (int k = 0; k < m; ++k) A *= cur[k];
        for (int k = m + 1; k < pl->order; ++k) B *= cur[k];
        void *dst = (s + 1 == pl->ttm_order.size()) ? output : pl->d_ttm[s % 2];
        const long ti = s == 0 ? timing_begin(pl, stream) : -1;
        if (pl->dtype == DEINSUM_F64)
            err = launch_ttm_plain_f64(static_cast<const double *>(src), static_cast<const double *>(U[m]),
                                       static_cast<double *>(dst), A, cur[m], B, pl->ranks[m], stream);
        else
            err = launch_ttm_plain_f32(static_cast<const float *>(src), static_cast<const float *>(U[m]),
                                       static_cast<float *>(dst), A, cur[m], B, pl->ranks[m], stream);
        timing_end(pl, ti, stream);
        cur[m] = pl->ranks[m];
        src = dst;
    }
    return err ? DEINSUM_ERR_CUDA : DEINSUM_OK;
}

}  // namespace

namespace deinsum {

// Row classes (MttkrpArgs::xrow): class c holds the rows (case 0) or k lines (case 1) whose
// index is c mod 4.  Map c is 2-D {len + d_c, members of the class} with row stride 4 len
// words, based at the 16-byte granule holding the start of member 0 (row or line c), where
// len = Q (case 0) or I (case 1) and d_c = that start's word offset in its granule; the
// kernels load boxes of {BK + 4, BM / 4} (case 0) or {BM + 4, BK / 4} (case 1).  Every
// address a box can reach lies in a granule that holds an element of X.
bool rowclass_supported(const MttkrpGeom &g) {
    const int64_t lim = int64_t(1) << 31;
    const int64_t len = g.kcase == 0 ? g.Q : g.I;                     // words per row (line)
    const int64_t n = g.kcase == 0 ? g.P * g.I : g.O * g.K_in;       // rows (lines)
    return !g.opack && n >= 4 && len + 3 < lim && n < 4 * lim;
}

// The same maps with case-0 boxes of `rows` rows (32, or 32 / SG for slabs packed SG to a tile).
static bool encode_rowclass_maps_rows(const MttkrpGeom &g, const void *X, CUtensorMap *maps, int rows) {
    auto enc = tensor_map_encoder();
    if (!enc || !rowclass_supported(g) || (reinterpret_cast<uintptr_t>(X) & 3) != 0) return false;
    const int64_t len = g.kcase == 0 ? g.Q : g.I;
    const int64_t n = g.kcase == 0 ? g.P * g.I : g.O * g.K_in;
    const uintptr_t xw = reinterpret_cast<uintptr_t>(X) >> 2;
    for (int c = 0; c < 4; ++c) {
        const uintptr_t start = xw + uintptr_t(c) * uintptr_t(len);   // word address of member 0
        const int64_t d = int64_t(start & 3);
        void *base = reinterpret_cast<void *>((start - uintptr_t(d)) << 2);
        cuuint64_t dims[2] = {cuuint64_t(len + d), cuuint64_t((n - c + 3) / 4)};
        cuuint64_t strides[1] = {cuuint64_t(4 * len) * 4};
        cuuint32_t box[2] = {g.kcase == 0 ? cuuint32_t(DEINSUM_BK + 4) : cuuint32_t(DEINSUM_BM + 4),
                             g.kcase == 0 ? cuuint32_t(rows) : cuuint32_t(DEINSUM_BK / 4)};
        cuuint32_t estr[2] = {1, 1};
        if (enc(&maps[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

bool encode_x_rowclass_maps(const MttkrpGeom &g, const void *X, CUtensorMap *maps) {
    return encode_rowclass_maps_rows(g, X, maps, DEINSUM_BM / 4);
}

// Converter view of one raw chunk (128 k rows x 64 l) of the last-mode TTM kernels:
// case 0, one slab per tile, R_pad 32 (split factor tiles of U_{N-1}).
void ttm_last_geometry(int order, int64_t S, int64_t K, int64_t L, int R, MttkrpGeom *g, int sg) {
    std::memset(g, 0, sizeof(*g));
    g->order = order;
    g->mode = order - 2;
    g->kcase = 0;
    g->I = K;
    g->narrow = (sg == 1 && K < DEINSUM_BM) ? 1 : 0;
    g->G = 1;
    g->P = S;
    g->K_in = L;
    g->Q = L;
    g->O = 1;
    g->R = R;
    g->R_pad = 32;
    g->n_kb = int((L + DEINSUM_BK - 1) / DEINSUM_BK);
    g->vec_ok = 1;
    g->O_iter = 1;
}

// 3-D tensor map of X viewed as S slabs x K rows x L (the last mode contiguous):
// dims {L, K, S}, box {64, min(K, 128), 1}; with sg > 1 (K <= 128 / sg) the box is
// {64, 128 / sg, sg}: sg slabs land 128 / sg rows apart, rows past K read as zero.
bool encode_ttm_last_map(const void *X, int64_t S, int64_t K, int64_t L, CUtensorMap *map, uint32_t *box_bytes,
                         int sg) {
    auto enc = tensor_map_encoder();
    const int64_t lim = int64_t(1) << 31;
    if (!enc || (reinterpret_cast<uintptr_t>(X) & 15) != 0 || L % 4 != 0 || S >= lim || K >= lim || L >= lim)
        return false;
    if (sg != 1 && (sg != ttmc_slab_group(K))) return false;
    cuuint64_t dims[3] = {cuuint64_t(L), cuuint64_t(K), cuuint64_t(S)};
    cuuint64_t strides[2] = {cuuint64_t(L) * 4, cuuint64_t(L * K) * 4};
    cuuint32_t box[3] = {DEINSUM_BK, cuuint32_t(sg > 1 ? DEINSUM_BM / sg : std::min<int64_t>(K, DEINSUM_BM)),
                         cuuint32_t(sg)};
    cuuint32_t estr[3] = {1, 1, 1};
    *box_bytes = uint32_t(4 * box[0] * box[1] * box[2]);
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(X), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Mode of X that einsum operand k (k >= 1) is contracted with.
int deinsum_internal_operand_mode(deinsum_plan_t pl, int k) { return pl->operand_mode[k]; }

// Row view and TMA descriptor of a one-off split-BF16 MTTKRP, for the entry
// point that allocates nothing: fills a->g and, when X allows it, a->xmap.
// Uses a plan object on the stack whose containers stay empty (no heap use).
bool mttkrp_prepare_oneoff(int order, const int64_t *dims, int mode, int R, const void *X, MttkrpArgs *a,
                           bool allow_opack) {
    deinsum_plan_s pl;
    pl.kind = DEINSUM_KIND_MTTKRP;
    pl.no_opack = !allow_opack;
    pl.order = order;
    pl.mode = mode;
    pl.dtype = DEINSUM_F32;
    pl.prec = DEINSUM_PREC_SPLIT_BF16;
    for (int m = 0; m < order; ++m) {
        pl.dims[m] = dims[m];
        pl.ranks[m] = (m == mode) ? dims[m] : R;
    }
    build_mttkrp_geometry(&pl);
    a->g = pl.geom;
    if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) a->g.vec_ok = 0;
    a->use_tma = 0;
    if (encode_x_map(&pl, X)) {
        a->xmap = pl.xmap;
        a->use_tma = 1;
        a->box_bytes = pl.xmap_box_bytes;
        a->raw_pitch = pl.xmap_pitch;
    }
    a->row_classes = 0;
    if (!a->use_tma && !a->g.opack && encode_x_rowclass_maps(a->g, X, a->xrow)) a->row_classes = 1;
    return true;
}

}  // namespace deinsum

extern "C" {

deinsum_status deinsum_plan(const char *einsum, const int64_t *extents, int n_extents,
                            deinsum_dtype dtype, deinsum_prec prec, deinsum_plan_t *out) {
    if (!out || !einsum || !extents) return DEINSUM_ERR_INVALID;
    *out = nullptr;
    Parsed p;
    deinsum_status st = parse(einsum, p);
    if (st != DEINSUM_OK) return st;
    if (int(p.letters.size()) != n_extents) return DEINSUM_ERR_SHAPE;
    for (int k = 0; k < n_extents; ++k)
        if (extents[k] < 1 || extents[k] > (int64_t(1) << 40)) return DEINSUM_ERR_SHAPE;
    if (dtype != DEINSUM_F32 && dtype != DEINSUM_F64) return DEINSUM_ERR_DTYPE;
    if (prec != DEINSUM_PREC_PLAIN && prec != DEINSUM_PREC_SPLIT_BF16) return DEINSUM_ERR_DTYPE;
    if (prec == DEINSUM_PREC_SPLIT_BF16 && dtype != DEINSUM_F32) return DEINSUM_ERR_DTYPE;
    deinsum_plan_s *pl = new (std::nothrow) deinsum_plan_s();
    if (!pl) return DEINSUM_ERR_OOM;
    pl->dtype = dtype;
    pl->prec = prec;
    st = classify(pl, p, extents);
    if (st == DEINSUM_OK) {
        if (pl->kind == DEINSUM_KIND_MTTKRP) {
            int64_t R = pl->ranks[(pl->mode + 1) % pl->order];
            if (R > 64) {
                st = DEINSUM_ERR_UNSUPPORTED;
            } else {
                choose_inner_merge(pl);
                build_mttkrp_geometry(pl);
            }
        } else {
            plan_ttmc_chain(pl);
            if (prec == DEINSUM_PREC_SPLIT_BF16) st = plan_ttmc_fused(pl);
        }
    }
    if (st != DEINSUM_OK) {
        delete pl;
        return st;
    }
    *out = pl;
    return DEINSUM_OK;
}

deinsum_status deinsum_execute(deinsum_plan_t pl, const void *const *inputs, int n_inputs, void *output,
                               deinsum_stream_t stream) {
    if (!pl || !inputs || !output) return DEINSUM_ERR_INVALID;
    if (n_inputs != pl->n_operands) return DEINSUM_ERR_INVALID;
    const size_t es = elem_size(pl->dtype);
    for (int k = 0; k < n_inputs; ++k) {
        if (!inputs[k]) return DEINSUM_ERR_INVALID;
        if (reinterpret_cast<uintptr_t>(inputs[k]) % es) return DEINSUM_ERR_ALIGN;
    }
    if (reinterpret_cast<uintptr_t>(output) % es) return DEINSUM_ERR_ALIGN;
    deinsum_status st = ensure_device_state(pl, static_cast<cudaStream_t>(stream));
    if (st != DEINSUM_OK) return st;
    if (pl->kind == DEINSUM_KIND_MTTKRP) return execute_mttkrp(pl, inputs, output, stream);
    return execute_ttmc(pl, inputs, output, stream);
}

deinsum_status deinsum_workspace_size(deinsum_plan_t pl, size_t *bytes) {
    if (!pl || !bytes) return DEINSUM_ERR_INVALID;
    *bytes = pl->ws_bytes;
    return DEINSUM_OK;
}

deinsum_status deinsum_plan_workspace_bytes(deinsum_plan_t pl, size_t *bytes) {
    if (!pl || !bytes) return DEINSUM_ERR_INVALID;
    WsLayout L;
    deinsum_status st = plan_layout(pl, L);
    if (st != DEINSUM_OK) return st;
    *bytes = L.total;
    return DEINSUM_OK;
}

deinsum_status deinsum_plan_bind_workspace(deinsum_plan_t pl, void *workspace, size_t bytes, deinsum_stream_t stream) {
    if (!pl || !workspace) return DEINSUM_ERR_INVALID;
    if (pl->ws) return DEINSUM_ERR_INVALID;  // already has a workspace
    if (reinterpret_cast<uintptr_t>(workspace) & 1023) return DEINSUM_ERR_ALIGN;
    WsLayout L;
    deinsum_status st = plan_layout(pl, L);
    if (st != DEINSUM_OK) return st;
    if (bytes < L.total) return DEINSUM_ERR_SHAPE;
    return attach_workspace(pl, static_cast<char *>(workspace), L, false, static_cast<cudaStream_t>(stream));
}

deinsum_status deinsum_plan_info(deinsum_plan_t pl, deinsum_plan_info_t *info) {
    if (!pl || !info) return DEINSUM_ERR_INVALID;
    std::memset(info, 0, sizeof(*info));
    info->kind = pl->kind;
    info->order = pl->order;
    info->mode = pl->mode;
    info->dtype = pl->dtype;
    info->prec = pl->prec;
    for (int m = 0; m < pl->order; ++m) {
        info->dims[m] = pl->dims[m];
        info->ranks[m] = pl->ranks[m];
    }
    if (pl->kind == DEINSUM_KIND_MTTKRP) {
        info->out_elems = pl->dims[pl->mode] * (pl->mm_cols > 0 ? pl->mm_cols : pl->ranks[(pl->mode + 1) % pl->order]);
        info->mm_cols = pl->mm_cols;
    } else {
        info->out_elems = 1;
        for (int m = 0; m < pl->order; ++m) info->out_elems *= pl->ranks[m];
    }
    info->alg_bytes = alg_bytes(pl);
    info->alg_flops = alg_flops(pl);
    info->n_units = pl->planned_units;
    if (pl->kind == DEINSUM_KIND_MTTKRP) {
        const MttkrpGeom &g = pl->geom;
        info->view_merged = pl->merge ? 1 : 0;
        info->view_packed = g.opack;
        info->view_groups = g.G;
        info->view_aligned_rows = g.vec_ok;
        info->view_row_classes = (pl->prec == DEINSUM_PREC_SPLIT_BF16 && pl->dtype == DEINSUM_F32 && !g.vec_ok &&
                                  rowclass_supported(g)) ? 1 : 0;
        // one SM's fast memory: the largest dynamic shared memory of a CTA (227 KB) plus the
        // tensor memory (256 KB), in FP32 words
        const double S = (232448.0 + 262144.0) / 4.0;
        double x_elems = 1.0;
        for (int m = 0; m < pl->order; ++m) x_elems *= double(pl->dims[m]);
        deinsum_io_bound_t b;
        if (deinsum_mttkrp_io_bound(S, x_elems, pl->ranks[(pl->mode + 1) % pl->order], &b) == DEINSUM_OK) {
            info->io_fast_mem_words = S;
            info->io_rho = b.rho;
            info->io_bound_bytes = 4.0 * b.q_min * (pl->dtype == DEINSUM_F64 ? 2.0 : 1.0);
        }
    }
    return DEINSUM_OK;
}

deinsum_status deinsum_last_device_status(deinsum_plan_t pl) {
    if (!pl) return DEINSUM_ERR_INVALID;
    if (!pl->d_status) return DEINSUM_OK;
    int v = 0;
    if (cudaMemcpy(&v, pl->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return DEINSUM_ERR_CUDA;
    if (v != 0 && cudaMemset(pl->d_status, 0, sizeof(int)) != cudaSuccess) return DEINSUM_ERR_CUDA;
    return v == 0 ? DEINSUM_OK : DEINSUM_ERR_TIMEOUT;
}

deinsum_status deinsum_mttkrp_io_bound(double S, double t_elems, int64_t R, deinsum_io_bound_t *out) {
    if (!out || !(S > 0.0) || !(t_elems > 0.0) || R < 1) return DEINSUM_ERR_INVALID;
    const double s13 = std::cbrt(S);
    out->X0 = 2.5 * S;
    out->I = out->J = out->K = s13;
    out->L = s13 * s13 / 2.0;
    out->rho = s13 * s13 / 3.0;
    out->rho_rank = out->rho < double(R) ? out->rho : double(R);
    out->q_min = t_elems * double(R) / out->rho_rank;
    return DEINSUM_OK;
}

void deinsum_set_wait_limit_ns(uint64_t ns) { g_wait_limit_ns.store(ns, std::memory_order_relaxed); }

int64_t deinsum_alloc_count(void) { return g_allocs.load(std::memory_order_relaxed); }

deinsum_status deinsum_set_kernel_timing(deinsum_plan_t pl, int enable) {
    if (!pl) return DEINSUM_ERR_INVALID;
    pl->timing = enable != 0;
    return DEINSUM_OK;
}

deinsum_status deinsum_kernel_time(deinsum_plan_t pl, double *total_ms, int64_t *launches) {
    if (!pl || !total_ms || !launches) return DEINSUM_ERR_INVALID;
    double tot = 0.0;
    for (size_t i = 0; i < pl->ev_used; ++i) {
        if (cudaEventSynchronize(pl->ev_pool[i].second) != cudaSuccess) return DEINSUM_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pl->ev_pool[i].first, pl->ev_pool[i].second) != cudaSuccess)
            return DEINSUM_ERR_CUDA;
        tot += double(ms);
    }
    *total_ms = tot;
    *launches = int64_t(pl->ev_used);
    pl->ev_used = 0;
    return DEINSUM_OK;
}

void deinsum_destroy(deinsum_plan_t pl) {
    if (!pl) return;
    for (auto &e : pl->ev_pool) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    if (pl->ws && pl->ws_owned) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != pl->device) cudaSetDevice(pl->device);
        cudaFree(pl->ws);
        if (cur != pl->device && cur >= 0) cudaSetDevice(cur);
    }
    delete pl;
}

const char *deinsum_status_string(deinsum_status s) {
    switch (s) {
        case DEINSUM_OK: return "ok";
        case DEINSUM_ERR_PARSE: return "malformed einsum string";
        case DEINSUM_ERR_UNSUPPORTED: return "not an MTTKRP or TTMc pattern the library offers";
        case DEINSUM_ERR_SHAPE: return "bad extents";
        case DEINSUM_ERR_DTYPE: return "dtype / precision combination not offered";
        case DEINSUM_ERR_ALIGN: return "pointer not aligned to its element size";
        case DEINSUM_ERR_OOM: return "device allocation failed";
        case DEINSUM_ERR_CUDA: return "CUDA error";
        case DEINSUM_ERR_TIMEOUT: return "a device-side bounded wait gave up";
        case DEINSUM_ERR_INVALID: return "invalid argument";
    }
    return "unknown status";
}

int64_t deinsum_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
