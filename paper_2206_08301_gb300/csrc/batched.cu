// Batched MTTKRP: many instances of uneven extents and ranks in one persistent
// tensor-core launch, replayed from a captured CUDA graph.  Instances whose rows
// are 16-byte aligned load X through a tensor map, the others through four
// row-class tensor maps; the kernel runs each unit in code specialised for its
// instance's loads and operand layout, read once per unit.
//
// Host side: every instance is classified by a regular plan (Sec. III-B MTTKRP
// einsum); its row view is cut into work units (column of 128 output rows x a
// range of fiber groups) of about `unit_bytes` of X each; the units form one list,
// grouped by kind of instance and largest first within a kind (by a cost that counts
// a unit's chunks and fiber-group epilogues), which the persistent CTAs take in order
// from a device ticket counter: each CTA takes its next unit when it is ready for one,
// so that they finish together whatever the cost model misjudges, and a CTA stays
// within one kind's specialised loop for long stretches.  The granularity is picked by
// an autotuner that times candidate schedules on the device and remembers the winner
// per batch signature.
// Device side (mttkrp_tc_batched.cu): one launch that splits every instance's inner factor
// and fills its weight tables, the batched tensor-core kernel, and a fixed-order reduction
// of the unit partials into each instance's output; the two around the kernel deal their
// blocks out per instance in proportion to its work.  With plain precision the
// batch runs as separate launches of the plain kernel (the baseline).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <queue>
#include <string>
#include <vector>

#include "internal.h"

namespace deinsum {
namespace {

constexpr int BM = DEINSUM_BM;
constexpr int BK = DEINSUM_BK;

size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Inst {
    int order = 0, mode = 0, R = 0, n_ops = 0;
    int64_t dims[DEINSUM_MAX_ORDER] = {0};
    int opmode[DEINSUM_MAX_ORDER + 1] = {0};
    MttkrpGeom g{};
    double xbytes = 0.0;
    int kind = 0;   // 0: tensor map (or per-thread loads); 1 / 2: row classes, case 0 / case 1
};

// Kinds of instance the schedule tunes separately: 2 * load kind (tensor map, row classes case 0,
// row classes case 1) + operand layout (K-major, MN-major).
constexpr int kKinds = 6;
struct TuneEntry {
    int div = 4;              // units of about total / (grid * div) bytes ...
    int shift[kKinds] = {};   // ... times 2^shift[k] more of them for the instances of kind k
};

std::mutex g_tune_mutex;
std::map<std::string, TuneEntry> g_tune_cache;  // batch signature -> unit sizes
bool g_tune_loaded = false;

void load_tune_cache() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("DEINSUM_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char key[256];
    TuneEntry e;
    while (std::fscanf(f, "%255s %d %d %d %d %d %d %d", key, &e.div, &e.shift[0], &e.shift[1], &e.shift[2],
                       &e.shift[3], &e.shift[4], &e.shift[5]) == 8)
        g_tune_cache[key] = e;
    std::fclose(f);
}

void store_tune_cache(const std::string &key, const TuneEntry &e) {
    g_tune_cache[key] = e;
    const char *path = std::getenv("DEINSUM_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d %d %d %d %d\n", key.c_str(), e.div, e.shift[0], e.shift[1], e.shift[2], e.shift[3],
                 e.shift[4], e.shift[5]);
    std::fclose(f);
}

}  // namespace
}  // namespace deinsum

using namespace deinsum;

struct deinsum_batch_s {
    int n = 0;
    deinsum_prec prec = DEINSUM_PREC_SPLIT_BF16;
    std::vector<deinsum_plan_t> plans;
    std::vector<Inst> inst;
    double total_bytes = 0.0;
    std::string signature;
    int unit_div = 4;   // units of about total / (grid * unit_div) bytes ...
    int kind_shift[kKinds] = {};   // ... times 2^kind_shift[k] more for instances of kind k (kind_key)
    int n_sm = 0, grid = 0;          // CTAs of the launch (one per SM, at most one per unit)
    // schedule (host)
    std::vector<int64_t> units;      // 5 per unit, in the order the CTAs take them
    std::vector<int64_t> red_off;    // partial offsets, per instance, column, split
    std::vector<int64_t> red_col;    // per instance: n_cols + 1 starts into red_off
    std::vector<int64_t> red_col_base;
    std::vector<size_t> bsplit_off;
    std::vector<size_t> wtab_off;    // per instance: its weight tables (L, then O)
    size_t partial_floats = 0, bsplit_bytes = 0, wtab_bytes = 0;
    std::vector<int> prep_start;     // per instance: its blocks of the preparation launch (n + 1)
    std::vector<int> red_start;      // per instance: its blocks of the reduction launch (n + 1)
    // device
    char *ws = nullptr;
    size_t ws_bytes = 0;
    size_t o_status = 0, o_insts = 0, o_split = 0, o_red = 0, o_units = 0, o_ticket = 0, o_redoff = 0, o_redcol = 0,
           o_pstart = 0, o_rstart = 0, o_bsplit = 0, o_wtab = 0, o_partial = 0, o_end = 0;
    char *staging = nullptr;  // pinned: insts + split table + reduce table
    size_t staging_bytes = 0;
    bool tables_uploaded = false;
    std::vector<const void *> ptrs;  // cached pointers of the last execute
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap = nullptr;  // capture stream
};

namespace {

void destroy_graph(deinsum_batch_s *b) {
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
}

// Relative time of a unit of `fgs` fiber groups: its 64-wide chunks (the converters' and
// the TMA's work, a quarter more through the row-class maps, whose reads realign the
// rows) plus one epilogue per fiber group (TMEM columns read, the instance's padded rank).
double unit_cost(const Inst &in, int64_t fgs) {
    const double chunk = in.kind ? 1.25 : 1.0;
    return double(fgs) * (double(in.g.n_kb) * chunk + double(in.g.R_pad) / 128.0);
}

int kind_key(const Inst &in) { return 2 * in.kind + in.g.kcase; }

// Units of about total / (grid * unit_div * 2^kind_shift) bytes of X, in the order the CTAs
// take them.
void build_batch_schedule(deinsum_batch_s *b) {
    const double target_units = double(b->n_sm) * double(b->unit_div);
    struct U {
        int64_t inst, col, f0, f1, off;
        double cost;
    };
    std::vector<U> all;
    b->red_off.clear();
    b->red_col.clear();
    b->red_col_base.assign(size_t(b->n), 0);
    b->bsplit_off.assign(size_t(b->n), 0);
    b->wtab_off.assign(size_t(b->n), 0);
    b->partial_floats = 0;
    b->bsplit_bytes = 0;
    b->wtab_bytes = 0;
    b->prep_start.assign(1, 0);
    b->red_start.assign(1, 0);
    // blocks of the launches around the tensor-core kernel, in proportion to each instance's
    // work: about 8 split or weight entries and 2 output entries per thread
    auto blocks = [](int64_t work, int64_t per_block) {
        return int(std::min<int64_t>(256, std::max<int64_t>(1, (work + per_block - 1) / per_block)));
    };
    for (int i = 0; i < b->n; ++i) {
        const MttkrpGeom &g = b->inst[size_t(i)].g;
        const int64_t max_units = g.n_cols * g.fg_per_col;
        const double scale = std::ldexp(1.0, b->kind_shift[kind_key(b->inst[size_t(i)])]);
        const double unit_bytes = std::max(1.0, b->total_bytes / (target_units * scale));
        int64_t want = int64_t(std::ceil(b->inst[size_t(i)].xbytes / unit_bytes));
        want = std::max<int64_t>(1, std::min(want, max_units));
        const int64_t per_col = std::min<int64_t>(g.fg_per_col, std::max<int64_t>(1, (want + g.n_cols - 1) / g.n_cols));
        b->red_col_base[size_t(i)] = int64_t(b->red_col.size());
        for (int64_t c = 0; c < g.n_cols; ++c) {
            b->red_col.push_back(int64_t(b->red_off.size()));
            for (int64_t s = 0; s < per_col; ++s) {
                const int64_t f0 = g.fg_per_col * s / per_col, f1 = g.fg_per_col * (s + 1) / per_col;
                if (f1 <= f0) continue;
                const int64_t off = int64_t(b->partial_floats);
                b->partial_floats += size_t(BM) * size_t(g.R_pad);
                b->red_off.push_back(off);
                all.push_back({i, c, f0, f1, off, unit_cost(b->inst[size_t(i)], f1 - f0)});
            }
        }
        b->red_col.push_back(int64_t(b->red_off.size()));
        b->bsplit_off[size_t(i)] = b->bsplit_bytes;
        b->bsplit_bytes += up(size_t(g.n_kb) * 2 * size_t(g.R_pad) * BK * 2, 1024);
        const size_t wf = weight_table_floats_l(g) + weight_table_floats_o(g);
        b->wtab_off[size_t(i)] = b->wtab_bytes;
        b->wtab_bytes += up(wf * 4, 256);
        const int64_t split_elems = int64_t(g.n_kb) * 2 * g.R_pad * BK;
        b->prep_start.push_back(b->prep_start.back() + blocks(split_elems + int64_t(wf), 256 * 8));
        b->red_start.push_back(b->red_start.back() + blocks(g.I * int64_t(g.R), 256 * 2));
    }
    // one global list of units that the launch's CTAs take in order from a device ticket
    // counter: grouped by kind of instance (the kernel's specialised loops; a CTA then stays in
    // one kind for long stretches), largest first within a kind, so that the last units taken
    // are the smallest
    b->units.clear();
    std::vector<size_t> order(all.size());
    for (size_t k = 0; k < all.size(); ++k) order[k] = k;
    auto key = [&](size_t k) { return kind_key(b->inst[size_t(all[k].inst)]); };   // load, then layout
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        if (key(x) != key(y)) return key(x) < key(y);
        return all[x].cost > all[y].cost;
    });
    for (size_t k : order) {
        const U &u = all[k];
        b->units.insert(b->units.end(), {u.inst, u.col, u.f0, u.f1, u.off});
    }
    b->grid = int(std::max<int64_t>(1, std::min<int64_t>(b->n_sm, int64_t(all.size()))));
}

deinsum_status layout_and_upload(deinsum_batch_s *b, cudaStream_t s) {
    size_t off = 0;
    auto take = [&](size_t bytes, size_t align) {
        off = up(off, align);
        const size_t r = off;
        off += bytes;
        return r;
    };
    b->o_status = take(256, 256);
    b->o_insts = take(sizeof(MttkrpArgs) * size_t(b->n), 128);
    b->o_split = take(sizeof(SplitInst) * size_t(b->n), 64);
    b->o_red = take(sizeof(RedInst) * size_t(b->n), 64);
    b->o_units = take(b->units.size() * 8, 256);
    b->o_ticket = take(8, 256);
    b->o_redoff = take(b->red_off.size() * 8, 256);
    b->o_redcol = take(b->red_col.size() * 8, 256);
    b->o_pstart = take(b->prep_start.size() * 4, 256);
    b->o_rstart = take(b->red_start.size() * 4, 256);
    b->o_bsplit = take(b->bsplit_bytes, 1024);
    b->o_wtab = take(b->wtab_bytes, 256);
    b->o_partial = take(b->partial_floats * 4, 1024);
    b->o_end = up(off, 1024);
    if (b->o_end > b->ws_bytes) {
        if (b->ws) cudaFree(b->ws);
        b->ws = nullptr;
        b->ws_bytes = 0;
        void *p = nullptr;
        cudaError_t e = counted_malloc(&p, b->o_end);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? DEINSUM_ERR_OOM : DEINSUM_ERR_CUDA;
        }
        b->ws = static_cast<char *>(p);
        b->ws_bytes = b->o_end;
    }
    const size_t stage = up(sizeof(MttkrpArgs) * size_t(b->n), 128) + up(sizeof(SplitInst) * size_t(b->n), 64) +
                         up(sizeof(RedInst) * size_t(b->n), 64);
    if (stage > b->staging_bytes) {
        if (b->staging) cudaFreeHost(b->staging);
        b->staging = nullptr;
        if (counted_malloc_host(reinterpret_cast<void **>(&b->staging), stage) != cudaSuccess) return DEINSUM_ERR_OOM;
        b->staging_bytes = stage;
    }
    cudaMemsetAsync(b->ws + b->o_status, 0, 256, s);
    cudaMemcpyAsync(b->ws + b->o_units, b->units.data(), b->units.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->ws + b->o_redoff, b->red_off.data(), b->red_off.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->ws + b->o_redcol, b->red_col.data(), b->red_col.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->ws + b->o_pstart, b->prep_start.data(), b->prep_start.size() * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->ws + b->o_rstart, b->red_start.data(), b->red_start.size() * 4, cudaMemcpyHostToDevice, s);
    b->tables_uploaded = true;
    b->ptrs.clear();  // instance tables must be rebuilt for the new layout
    destroy_graph(b);
    return cudaGetLastError() == cudaSuccess ? DEINSUM_OK : DEINSUM_ERR_CUDA;
}

// Instance arguments (pointers, TMA descriptors), split and reduce tables.
deinsum_status upload_instances(deinsum_batch_s *b, const void *const *const *inputs, void *const *outputs,
                                cudaStream_t s) {
    cudaStreamSynchronize(s);  // the staging buffer may still feed an earlier copy
    MttkrpArgs *A = reinterpret_cast<MttkrpArgs *>(b->staging);
    SplitInst *S = reinterpret_cast<SplitInst *>(b->staging + up(sizeof(MttkrpArgs) * size_t(b->n), 128));
    RedInst *Rd = reinterpret_cast<RedInst *>(reinterpret_cast<char *>(S) + up(sizeof(SplitInst) * size_t(b->n), 64));
    for (int i = 0; i < b->n; ++i) {
        const Inst &in = b->inst[size_t(i)];
        MttkrpArgs &a = A[i];
        std::memset(static_cast<void *>(&a), 0, sizeof(a));
        mttkrp_prepare_oneoff(in.order, in.dims, in.mode, in.R, inputs[i][0], &a, false);
        if (in.kind && !a.row_classes) return DEINSUM_ERR_CUDA;   // the maps of a planned row-class instance
        if (!in.kind) a.row_classes = 0;
        a.X = inputs[i][0];
        for (int k = 1; k < in.n_ops; ++k) a.U[in.opmode[k]] = inputs[i][k];
        a.Bsplit = b->ws + b->o_bsplit + b->bsplit_off[size_t(i)];
        a.Lw = reinterpret_cast<float *>(b->ws + b->o_wtab + b->wtab_off[size_t(i)]);
        a.Ow = a.Lw + weight_table_floats_l(a.g);
        a.status = reinterpret_cast<int *>(b->ws + b->o_status);
        const int inner = a.g.kcase == 0 ? a.g.order - 1 : a.g.order - 2;
        S[i] = {static_cast<const float *>(a.U[inner]), static_cast<unsigned char *>(const_cast<void *>(a.Bsplit)),
                a.g.K_in, a.g.R, a.g.R_pad, a.g.n_kb};
        Rd[i] = {static_cast<float *>(outputs[i]), a.g.I, a.g.R, a.g.R_pad, a.g.rows_per_col, a.g.G, a.g.narrow,
                 b->red_col_base[size_t(i)]};
    }
    const size_t bytes = up(sizeof(MttkrpArgs) * size_t(b->n), 128) + up(sizeof(SplitInst) * size_t(b->n), 64) +
                         up(sizeof(RedInst) * size_t(b->n), 64);
    // the three tables are laid out back to back in the workspace as in the staging buffer
    cudaMemcpyAsync(b->ws + b->o_insts, b->staging, bytes, cudaMemcpyHostToDevice, s);
    return cudaGetLastError() == cudaSuccess ? DEINSUM_OK : DEINSUM_ERR_CUDA;
}

deinsum_status launch_batch(deinsum_batch_s *b, cudaStream_t s) {
    if (launch_batched_prep(reinterpret_cast<const MttkrpArgs *>(b->ws + b->o_insts),
                            reinterpret_cast<const SplitInst *>(b->ws + b->o_split),
                            reinterpret_cast<const int *>(b->ws + b->o_pstart), b->n, b->prep_start.back(), s))
        return DEINSUM_ERR_CUDA;
    BatchArgs ba;
    ba.insts = reinterpret_cast<const MttkrpArgs *>(b->ws + b->o_insts);
    ba.units = reinterpret_cast<const int64_t *>(b->ws + b->o_units);
    ba.partial = reinterpret_cast<float *>(b->ws + b->o_partial);
    ba.status = reinterpret_cast<int *>(b->ws + b->o_status);
    ba.n_units = int64_t(b->units.size() / 5);
    ba.ticket = reinterpret_cast<unsigned long long *>(b->ws + b->o_ticket);
    if (cudaMemsetAsync(ba.ticket, 0, sizeof(unsigned long long), s) != cudaSuccess) return DEINSUM_ERR_CUDA;
    if (launch_mttkrp_tc_batched(ba, b->grid, s)) return DEINSUM_ERR_CUDA;
    if (launch_batched_reduce(reinterpret_cast<const RedInst *>(b->ws + b->o_red),
                              reinterpret_cast<const int *>(b->ws + b->o_rstart), b->n, b->red_start.back(),
                              reinterpret_cast<const int64_t *>(b->ws + b->o_redcol),
                              reinterpret_cast<const int64_t *>(b->ws + b->o_redoff),
                              reinterpret_cast<const float *>(b->ws + b->o_partial), s))
        return DEINSUM_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? DEINSUM_OK : DEINSUM_ERR_CUDA;
}

deinsum_status ensure_ready(deinsum_batch_s *b, const void *const *const *inputs, void *const *outputs,
                            cudaStream_t s) {
    if (b->n_sm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return DEINSUM_ERR_CUDA;
        if (cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DEINSUM_ERR_CUDA;
    }
    if (!b->tables_uploaded) {
        build_batch_schedule(b);
        deinsum_status st = layout_and_upload(b, s);
        if (st != DEINSUM_OK) return st;
    }
    std::vector<const void *> p;
    for (int i = 0; i < b->n; ++i) {
        for (int k = 0; k < b->inst[size_t(i)].n_ops; ++k) p.push_back(inputs[i][k]);
        p.push_back(outputs[i]);
    }
    if (p != b->ptrs) {
        destroy_graph(b);
        deinsum_status st = upload_instances(b, inputs, outputs, s);
        if (st != DEINSUM_OK) return st;
        b->ptrs = p;
    }
    return DEINSUM_OK;
}

}  // namespace

extern "C" {

deinsum_status deinsum_plan_batched(int n, const char *const *einsums, const int64_t *const *extents,
                                    const int *n_extents, deinsum_dtype dtype, deinsum_prec prec,
                                    deinsum_batch_t *out) {
    if (!out || n < 1 || !einsums || !extents || !n_extents) return DEINSUM_ERR_INVALID;
    *out = nullptr;
    if (dtype != DEINSUM_F32) return DEINSUM_ERR_DTYPE;
    deinsum_batch_s *b = new (std::nothrow) deinsum_batch_s();
    if (!b) return DEINSUM_ERR_OOM;
    b->n = n;
    b->prec = prec;
    b->plans.assign(size_t(n), nullptr);
    b->inst.resize(size_t(n));
    char sig[64];
    std::snprintf(sig, sizeof(sig), "n%d", n);
    b->signature = sig;
    for (int i = 0; i < n; ++i) {
        deinsum_status st = deinsum_plan(einsums[i], extents[i], n_extents[i], dtype, prec, &b->plans[size_t(i)]);
        if (st != DEINSUM_OK) {
            deinsum_batched_destroy(b);
            return st;
        }
        deinsum_plan_info_t info;
        deinsum_plan_info(b->plans[size_t(i)], &info);
        if (info.kind != DEINSUM_KIND_MTTKRP || info.mm_cols != 0) {   // plain MTTKRP instances only
            deinsum_batched_destroy(b);
            return DEINSUM_ERR_UNSUPPORTED;
        }
        Inst &in = b->inst[size_t(i)];
        in.order = info.order;
        in.mode = info.mode;
        in.n_ops = info.order;
        in.R = int(info.ranks[(info.mode + 1) % info.order]);
        for (int m = 0; m < in.order; ++m) in.dims[m] = info.dims[m];
        for (int k = 1; k < in.n_ops; ++k) in.opmode[k] = deinsum_internal_operand_mode(b->plans[size_t(i)], k);
        MttkrpArgs tmp;
        std::memset(static_cast<void *>(&tmp), 0, sizeof(tmp));
        mttkrp_prepare_oneoff(in.order, in.dims, in.mode, in.R, nullptr, &tmp, false);
        in.g = tmp.g;
        // rows not 16-byte aligned: row classes (X itself 4-byte aligned suffices), one launch per case
        in.kind = (!tmp.g.vec_ok && rowclass_supported(tmp.g)) ? (tmp.g.kcase == 1 ? 2 : 1) : 0;
        in.xbytes = 4.0;
        for (int m = 0; m < in.order; ++m) in.xbytes *= double(in.dims[m]);
        b->total_bytes += in.xbytes;
    }
    // signature for the autotune cache: count, total size and rank mix, rounded
    int rhist[4] = {0, 0, 0, 0};
    for (auto &in : b->inst) rhist[in.R <= 8 ? 0 : in.R <= 16 ? 1 : in.R <= 32 ? 2 : 3]++;
    std::snprintf(sig, sizeof(sig), "n%d_gb%.1f_r%d.%d.%d.%d", n, b->total_bytes / 1e9, rhist[0], rhist[1], rhist[2],
                  rhist[3]);
    b->signature = sig;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        load_tune_cache();
        auto it = g_tune_cache.find(b->signature);
        if (it != g_tune_cache.end()) {
            b->unit_div = it->second.div;
            for (int k = 0; k < kKinds; ++k) b->kind_shift[k] = it->second.shift[k];
        }
    }
    *out = b;
    return DEINSUM_OK;
}

deinsum_status deinsum_execute_batched(deinsum_batch_t b, const void *const *const *inputs, void *const *outputs,
                                       deinsum_stream_t stream) {
    if (!b || !inputs || !outputs) return DEINSUM_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (b->prec == DEINSUM_PREC_PLAIN) {
        for (int i = 0; i < b->n; ++i) {
            deinsum_status st = deinsum_execute(b->plans[size_t(i)], inputs[i], b->inst[size_t(i)].n_ops, outputs[i], stream);
            if (st != DEINSUM_OK) return st;
        }
        return DEINSUM_OK;
    }
    for (int i = 0; i < b->n; ++i)
        for (int k = 0; k < b->inst[size_t(i)].n_ops; ++k)
            if (!inputs[i] || !inputs[i][k] || (reinterpret_cast<uintptr_t>(inputs[i][k]) & 3)) return DEINSUM_ERR_INVALID;
    deinsum_status st = ensure_ready(b, inputs, outputs, s);
    if (st != DEINSUM_OK) return st;
    if (!b->gexec) {
        // first run with these pointers: launch directly (sets kernel attributes), then capture
        st = launch_batch(b, s);
        if (st != DEINSUM_OK) return st;
        // capture on the plan's own stream (the caller's may be the legacy default
        // stream, which cannot be captured); the graph is launched on the caller's
        if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return DEINSUM_ERR_CUDA;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return DEINSUM_ERR_CUDA;
        st = launch_batch(b, b->cap);
        cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
        if (st != DEINSUM_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return DEINSUM_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->gexec = nullptr;
            cudaGetLastError();
            return DEINSUM_ERR_CUDA;
        }
        return DEINSUM_OK;
    }
    if (cudaGraphLaunch(b->gexec, s) != cudaSuccess) return DEINSUM_ERR_CUDA;
    count_launch(3);   // the graph's kernels: preparation, tensor-core kernel, reduction
    return DEINSUM_OK;
}

deinsum_status deinsum_batched_autotune(deinsum_batch_t b, const void *const *const *inputs, void *const *outputs,
                                        deinsum_stream_t stream, double *best_ms) {
    if (!b || !inputs || !outputs) return DEINSUM_ERR_INVALID;
    if (b->prec != DEINSUM_PREC_SPLIT_BF16) return DEINSUM_ERR_DTYPE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // ms per execute of the current schedule (two untimed, three timed; < 0 on an error)
    auto time_it = [&]() -> double {
        b->tables_uploaded = false;
        if (ensure_ready(b, inputs, outputs, s) != DEINSUM_OK) return -1.0;
        for (int r = 0; r < 2; ++r) launch_batch(b, s);
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) launch_batch(b, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / 3.0;
    };
    auto fail = [&]() {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return DEINSUM_ERR_CUDA;
    };
    // the unit size of the whole batch, then one pass over the kinds of instance present,
    // halving or doubling each kind's unit count while that is faster
    for (int k = 0; k < kKinds; ++k) b->kind_shift[k] = 0;
    const int cand[] = {1, 2, 4, 8, 16, 32, 64};
    int best = b->unit_div;
    double best_t = 1e30;
    for (int div : cand) {
        b->unit_div = div;
        const double t = time_it();
        if (t < 0) return fail();
        if (t < best_t) {
            best_t = t;
            best = div;
        }
    }
    b->unit_div = best;
    bool present[kKinds] = {};
    for (const Inst &in : b->inst) present[kind_key(in)] = true;
    for (int k = 0; k < kKinds; ++k) {
        if (!present[k]) continue;
        for (int step : {1, -1}) {
            while (std::abs(b->kind_shift[k] + step) <= 3) {
                b->kind_shift[k] += step;
                const double t = time_it();
                if (t < 0) return fail();
                if (t < best_t) {
                    best_t = t;
                } else {
                    b->kind_shift[k] -= step;
                    break;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tables_uploaded = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        TuneEntry e;
        e.div = b->unit_div;
        for (int k = 0; k < kKinds; ++k) e.shift[k] = b->kind_shift[k];
        store_tune_cache(b->signature, e);
    }
    if (best_ms) *best_ms = best_t;
    return ensure_ready(b, inputs, outputs, s);
}

deinsum_status deinsum_batched_info(deinsum_batch_t b, int64_t *n_units, int *grid, int *unit_div, double *alg_bytes) {
    if (!b) return DEINSUM_ERR_INVALID;
    if (n_units) *n_units = int64_t(b->units.size() / 5);
    if (grid) *grid = b->grid;
    if (unit_div) *unit_div = b->unit_div;
    if (alg_bytes) {
        double t = 0.0;
        for (int i = 0; i < b->n; ++i) {
            deinsum_plan_info_t info;
            deinsum_plan_info(b->plans[size_t(i)], &info);
            t += info.alg_bytes;
        }
        *alg_bytes = t;
    }
    return DEINSUM_OK;
}

deinsum_status deinsum_batched_status(deinsum_batch_t b) {
    if (!b) return DEINSUM_ERR_INVALID;
    if (!b->ws) return DEINSUM_OK;
    int v = 0;
    if (cudaMemcpy(&v, b->ws + b->o_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return DEINSUM_ERR_CUDA;
    if (v != 0 && cudaMemset(b->ws + b->o_status, 0, sizeof(int)) != cudaSuccess) return DEINSUM_ERR_CUDA;
    return v == 0 ? DEINSUM_OK : DEINSUM_ERR_TIMEOUT;
}

void deinsum_batched_destroy(deinsum_batch_t b) {
    if (!b) return;
    destroy_graph(b);
    for (auto p : b->plans)
        if (p) deinsum_destroy(p);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ws) cudaFree(b->ws);
    if (b->staging) cudaFreeHost(b->staging);
    delete b;
}

}  // extern "C"
