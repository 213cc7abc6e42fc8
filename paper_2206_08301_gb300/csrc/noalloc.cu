// Allocation-free split-BF16 MTTKRP entry point.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// another allocator (a framework's caching allocator that has reserved the
// HBM budget), or latency-critical loops where the implicit device
// synchronisation of cudaMalloc / cudaFree is not acceptable.  This entry
// point runs the same kernels as deinsum_execute for a split-BF16 MTTKRP, but
// its scratch (schedule table, per-unit partial sums, split factor tiles,
// weight tables and status word) lives in one fixed file-scope device array, so no call
// allocates device memory.  The array is created with the library's module
// on every GPU that loads it and is held until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace deinsum {
namespace {

// Limits of the fixed scratch (see include/deinsum.h).
constexpr int64_t kMaxUnits = 256;                          // work units of one call
constexpr int64_t kMaxCols = 256;                           // columns of 128 output rows
constexpr size_t kOffStatus = 0;
constexpr size_t kOffUnits = 256;                           // kMaxUnits x 3 int64
constexpr size_t kOffCols = kOffUnits + size_t(kMaxUnits) * 3 * 8;  // kMaxCols + 1 int64
constexpr size_t kOffBsplit = 16384;                        // split factor tiles: offset a multiple of
                                                            // 1024, address only 256-aligned (the array's
                                                            // alignment); bulk copies need 16 bytes
constexpr size_t kBsplitBytes = size_t(1) << 20;            // 64 tiles at rank 64
constexpr size_t kOffPartial = kOffBsplit + kBsplitBytes;
constexpr size_t kPartialBytes = size_t(kMaxUnits) * DEINSUM_BM * 64 * 4;  // 8 MiB
constexpr size_t kOffWtab = kOffPartial + kPartialBytes;
constexpr size_t kWtabBytes = size_t(1) << 22;              // weight tables, 1 Mi floats
constexpr size_t kScratchBytes = kOffWtab + kWtabBytes;
static_assert(kOffCols + size_t(kMaxCols + 1) * 8 <= kOffBsplit, "scratch layout overlap");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host-side cache of each device's scratch address (the symbol's device
// address differs from its host-side name) and SM count.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_dev[kMaxDevices] = {nullptr};
int g_sms[kMaxDevices] = {0};

// Fill the unit table and the column table of the schedule (the same split as
// the planned path: per_col contiguous ranges of fiber groups per column) and
// clear the status word.
__global__ void noalloc_schedule_kernel(int64_t *units, int64_t *cols, int *status, int64_t n_cols,
                                        int64_t per_col, int64_t fg_per_col) {
    const int64_t n_units = n_cols * per_col;
    const int64_t n = n_units > n_cols + 1 ? n_units : n_cols + 1;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        if (i < n_units) {
            const int64_t c = i / per_col, s = i - c * per_col;
            units[3 * i] = c;
            units[3 * i + 1] = fg_per_col * s / per_col;
            units[3 * i + 2] = fg_per_col * (s + 1) / per_col;
        }
        if (i <= n_cols) cols[i] = i * per_col;
        if (i == 0) *status = 0;
    }
}

}  // namespace
}  // namespace deinsum

using namespace deinsum;

extern "C" deinsum_status deinsum_mttkrp_noalloc(int order, const int64_t *dims, int mode, int rank,
                                                 const float *X, const float *const *factors, float *out,
                                                 deinsum_stream_t stream) {
    if (order < 2 || order > DEINSUM_MAX_ORDER || mode < 0 || mode >= order || !dims || !X || !factors || !out)
        return DEINSUM_ERR_INVALID;
    if (rank < 1 || rank > 64) return DEINSUM_ERR_SHAPE;
    for (int m = 0; m < order; ++m) {
        if (dims[m] < 1) return DEINSUM_ERR_SHAPE;
        if (m != mode && !factors[m]) return DEINSUM_ERR_INVALID;
        if (m != mode && (reinterpret_cast<uintptr_t>(factors[m]) & 3)) return DEINSUM_ERR_ALIGN;
    }
    if ((reinterpret_cast<uintptr_t>(X) & 3) || (reinterpret_cast<uintptr_t>(out) & 3)) return DEINSUM_ERR_ALIGN;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DEINSUM_ERR_CUDA;
    unsigned char *scratch = nullptr;
    int n_sm = 0;
    {
        // once per device, with that device current: the scratch array's device address
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_dev[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return DEINSUM_ERR_CUDA;
            }
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
                return DEINSUM_ERR_CUDA;
            g_scratch_dev[dev] = static_cast<unsigned char *>(p);
            g_sms[dev] = sms;
        }
        scratch = g_scratch_dev[dev];
        n_sm = g_sms[dev];
    }

    MttkrpArgs a;
    std::memset(&a, 0, sizeof(a));
    mttkrp_prepare_oneoff(order, dims, mode, rank, X, &a);
    const MttkrpGeom &g = a.g;
    const int64_t max_units_here = std::min<int64_t>(
        kMaxUnits, int64_t(kPartialBytes / (size_t(DEINSUM_BM) * size_t(g.R_pad) * 4)));
    const int64_t per_col = balanced_units_per_col(g.n_cols, g.fg_per_col, n_sm, max_units_here);
    const int64_t n_units = g.n_cols * per_col;
    const size_t bsplit_bytes = size_t(g.n_kb) * 2 * size_t(g.R_pad) * DEINSUM_BK * 2;
    const size_t wtab_floats_l = weight_table_floats_l(g);
    if (g.n_cols > kMaxCols || n_units > kMaxUnits || bsplit_bytes > kBsplitBytes ||
        size_t(n_units) * DEINSUM_BM * size_t(g.R_pad) * 4 > kPartialBytes ||
        (wtab_floats_l + weight_table_floats_o(g)) * 4 > kWtabBytes)
        return DEINSUM_ERR_SHAPE;

    for (int m = 0; m < order; ++m) a.U[m] = (m == mode) ? nullptr : factors[m];
    a.X = X;
    a.units = reinterpret_cast<const int64_t *>(scratch + kOffUnits);
    a.n_units = n_units;
    a.partial = reinterpret_cast<float *>(scratch + kOffPartial);
    a.status = reinterpret_cast<int *>(scratch + kOffStatus);
    a.Bsplit = scratch + kOffBsplit;
    a.Lw = reinterpret_cast<float *>(scratch + kOffWtab);
    a.Ow = a.Lw + wtab_floats_l;
    int64_t *cols = reinterpret_cast<int64_t *>(scratch + kOffCols);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    noalloc_schedule_kernel<<<2, 256, 0, s>>>(reinterpret_cast<int64_t *>(scratch + kOffUnits), cols,
                                              reinterpret_cast<int *>(scratch + kOffStatus), g.n_cols, per_col,
                                              g.fg_per_col);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return DEINSUM_ERR_CUDA;
    int err = launch_split_inner_factor(a, scratch + kOffBsplit, stream);
    if (!err) err = launch_weight_tables(a, stream);
    if (!err) err = launch_mttkrp_tc(a, n_sm, stream);
    if (!err) err = launch_mttkrp_reduce_f32(a, cols, out, stream);
    return err ? DEINSUM_ERR_CUDA : DEINSUM_OK;
}

// The status word sits at the start of the array: read it on the current device with a
// symbol copy (no allocation).  Each call of deinsum_mttkrp_noalloc clears it first, so it
// describes the latest call on this device.
extern "C" deinsum_status deinsum_mttkrp_noalloc_status(void) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_scratch, sizeof(int), kOffStatus, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return DEINSUM_ERR_CUDA;
    }
    return v == 0 ? DEINSUM_OK : DEINSUM_ERR_TIMEOUT;
}
