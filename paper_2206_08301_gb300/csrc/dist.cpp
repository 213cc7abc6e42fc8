// Block distribution of iteration spaces over Cartesian process grids and the
// redistribution of a tensor between two such distributions (paper Sec. II-C/D
// and Sec. V: the block distribution i = p*B + o of Eqs. (12)-(13) with one block
// per process, replication over the Cartesian sub-grids that drop the dimensions
// a tensor does not use, and the per-dimension partitioning and message
// matching of Eqs. (20)-(25)).  Host-only: no CUDA call.  A multi-GPU (or
// multi-node) sharding of the contractions would use these plans; on this
// build's single GPU they are exercised by CPU ranks.
#include <algorithm>
#include <cstdint>
#include <cstring>

#include "internal.h"

namespace {

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

bool grid_ok(const deinsum_grid_t *g) {
    if (!g || g->ndim < 1 || g->ndim > 8) return false;
    for (int j = 0; j < g->ndim; ++j)
        if (g->extent[j] < 1 || g->procs[j] < 1) return false;
    return true;
}

int64_t grid_size(const deinsum_grid_t *g) {
    int64_t P = 1;
    for (int j = 0; j < g->ndim; ++j) P *= g->procs[j];
    return P;
}

void coords_of(const deinsum_grid_t *g, int64_t rank, int *c) {
    for (int j = g->ndim - 1; j >= 0; --j) {
        c[j] = int(rank % g->procs[j]);
        rank /= g->procs[j];
    }
}

int64_t rank_of(const deinsum_grid_t *g, const int *c) {
    int64_t r = 0;
    for (int j = 0; j < g->ndim; ++j) r = r * g->procs[j] + c[j];
    return r;
}

// block of process coordinate p along dimension j: [p B, min((p + 1) B, N))
void block_range(const deinsum_grid_t *g, int j, int p, int64_t *lo, int64_t *hi) {
    const int64_t B = ceil_div(g->extent[j], g->procs[j]);
    *lo = std::min<int64_t>(int64_t(p) * B, g->extent[j]);
    *hi = std::min<int64_t>(int64_t(p + 1) * B, g->extent[j]);
}

// the tensor's modes on a grid: mode t is grid dimension dims[t]; check distinct and in range
bool tensor_dims_ok(const deinsum_grid_t *g, const int *dims, int order) {
    if (!dims || order < 1 || order > g->ndim) return false;
    for (int t = 0; t < order; ++t) {
        if (dims[t] < 0 || dims[t] >= g->ndim) return false;
        for (int u = 0; u < t; ++u)
            if (dims[u] == dims[t]) return false;
    }
    return true;
}

bool uses(const int *dims, int order, int j) {
    for (int t = 0; t < order; ++t)
        if (dims[t] == j) return true;
    return false;
}

}  // namespace

extern "C" {

int64_t deinsum_grid_block(const deinsum_grid_t *g, int j) {
    if (!grid_ok(g) || j < 0 || j >= g->ndim) return 0;
    return ceil_div(g->extent[j], g->procs[j]);
}

deinsum_status deinsum_grid_coords(const deinsum_grid_t *g, int64_t rank, int *coords) {
    if (!grid_ok(g) || !coords || rank < 0 || rank >= grid_size(g)) return DEINSUM_ERR_INVALID;
    coords_of(g, rank, coords);
    return DEINSUM_OK;
}

int64_t deinsum_grid_rank(const deinsum_grid_t *g, const int *coords) {
    if (!grid_ok(g) || !coords) return -1;
    for (int j = 0; j < g->ndim; ++j)
        if (coords[j] < 0 || coords[j] >= g->procs[j]) return -1;
    return rank_of(g, coords);
}

deinsum_status deinsum_grid_block_range(const deinsum_grid_t *g, int64_t rank, int64_t *lo, int64_t *hi) {
    if (!grid_ok(g) || !lo || !hi || rank < 0 || rank >= grid_size(g)) return DEINSUM_ERR_INVALID;
    int c[8];
    coords_of(g, rank, c);
    for (int j = 0; j < g->ndim; ++j) block_range(g, j, c[j], lo + j, hi + j);
    return DEINSUM_OK;
}

deinsum_status deinsum_grid_sub(const deinsum_grid_t *g, const int *remain, int64_t rank, int64_t *color,
                                int64_t *key) {
    if (!grid_ok(g) || !remain || !color || !key || rank < 0 || rank >= grid_size(g)) return DEINSUM_ERR_INVALID;
    int c[8];
    coords_of(g, rank, c);
    int64_t col = 0, k = 0;
    for (int j = 0; j < g->ndim; ++j) {
        if (remain[j]) k = k * g->procs[j] + c[j];
        else col = col * g->procs[j] + c[j];
    }
    *color = col;
    *key = k;
    return DEINSUM_OK;
}

int deinsum_redist_dim_partitions(int64_t Bx, int64_t By, int64_t py, deinsum_dim_part_t *parts, int max_parts) {
    if (Bx < 1 || By < 1 || py < 0 || !parts) return -1;
    // p^(y) B^(y) = xi B^(x) + lambda (Eqs. 20-21); the k runs of o^(y) map to x-process xi + m
    const int64_t xi = (py * By) / Bx;
    const int64_t lambda = (py * By) % Bx;
    const int64_t k = ceil_div(By + lambda, Bx);  // Eq. (24)
    if (k > max_parts) return -1;
    for (int64_t m = 0; m < k; ++m) {
        deinsum_dim_part_t &p = parts[m];
        p.px = xi + m;
        p.oy_lo = std::max<int64_t>(0, m * Bx - lambda);
        p.oy_hi = std::min<int64_t>(By, (m + 1) * Bx - lambda);
        p.ox_lo = (m == 0) ? lambda : 0;          // Eq. (23)
        p.ox_hi = p.ox_lo + (p.oy_hi - p.oy_lo);
    }
    return int(k);
}

void deinsum_redist_match(int64_t Bx, int64_t By, int64_t px, int64_t *py_lo, int64_t *py_hi) {
    // Eq. (25): the y-processes whose block meets x-block px, as a half-open range
    *py_lo = ceil_div(px * Bx + 1, By) - 1;
    *py_hi = ceil_div((px + 1) * Bx, By);
}

int deinsum_redist_plan(const deinsum_grid_t *gx, const int *xdims, const deinsum_grid_t *gy, const int *ydims,
                        int order, int64_t rank, int sending, deinsum_msg_t *msgs, int max_msgs) {
    if (!grid_ok(gx) || !grid_ok(gy) || !tensor_dims_ok(gx, xdims, order) || !tensor_dims_ok(gy, ydims, order))
        return -1;
    for (int t = 0; t < order; ++t)
        if (gx->extent[xdims[t]] != gy->extent[ydims[t]]) return -1;
    const deinsum_grid_t *gs = sending ? gx : gy;   // this rank's grid
    const deinsum_grid_t *go = sending ? gy : gx;   // the peers' grid
    const int *ds = sending ? xdims : ydims;
    const int *dp = sending ? ydims : xdims;
    if (rank < 0 || rank >= grid_size(gs)) return -1;
    int c[8];
    coords_of(gs, rank, c);
    // a block replicated over the x-grid dimensions the tensor does not use is sent
    // once, by its replica with zero coordinates there; every y-replica receives it
    if (sending)
        for (int j = 0; j < gx->ndim; ++j)
            if (!uses(xdims, order, j) && c[j] != 0) return 0;
    // per tensor mode, the peer coordinates whose blocks meet this rank's block
    int64_t plo[8], phi[8];
    for (int t = 0; t < order; ++t) {
        const int64_t Bs = ceil_div(gs->extent[ds[t]], gs->procs[ds[t]]);
        const int64_t Bo = ceil_div(go->extent[dp[t]], go->procs[dp[t]]);
        if (sending) {
            deinsum_redist_match(Bs, Bo, c[ds[t]], plo + t, phi + t);
        } else {
            // the x-processes of this y-block: xi .. xi + k - 1 (Eqs. 20-24)
            const int64_t py = c[ds[t]];
            plo[t] = (py * Bs) / Bo;
            phi[t] = plo[t] + ceil_div(Bs + (py * Bs) % Bo, Bo);
        }
        plo[t] = std::max<int64_t>(plo[t], 0);
        phi[t] = std::min<int64_t>(phi[t], go->procs[dp[t]]);
    }
    // enumerate peer coordinates: tensor dims over [plo, phi); other peer dims over
    // every coordinate when receiving replicas (sending), else 0 (the sending replica)
    int pc[8] = {0};
    int lo_c[8], hi_c[8];
    for (int j = 0; j < go->ndim; ++j) {
        lo_c[j] = 0;
        hi_c[j] = sending ? go->procs[j] : 1;
    }
    for (int t = 0; t < order; ++t) {
        lo_c[dp[t]] = int(plo[t]);
        hi_c[dp[t]] = int(phi[t]);
    }
    for (int j = 0; j < go->ndim; ++j) {
        if (lo_c[j] >= hi_c[j]) return 0;
        pc[j] = lo_c[j];
    }
    int n = 0;
    while (true) {
        // the intersection of the two blocks, in global tensor coordinates
        deinsum_msg_t m;
        std::memset(&m, 0, sizeof(m));
        bool empty = false;
        for (int t = 0; t < order; ++t) {
            int64_t slo, shi, olo, ohi;
            block_range(gs, ds[t], c[ds[t]], &slo, &shi);
            block_range(go, dp[t], pc[dp[t]], &olo, &ohi);
            m.lo[t] = std::max(slo, olo);
            m.hi[t] = std::min(shi, ohi);
            if (m.lo[t] >= m.hi[t]) empty = true;
        }
        if (!empty) {
            m.peer = rank_of(go, pc);
            if (msgs) {
                if (n >= max_msgs) return -1;
                msgs[n] = m;
            }
            ++n;
        }
        int j = go->ndim - 1;
        while (j >= 0) {
            if (++pc[j] < hi_c[j]) break;
            pc[j] = lo_c[j];
            --j;
        }
        if (j < 0) break;
    }
    return n;
}

}  // extern "C"
