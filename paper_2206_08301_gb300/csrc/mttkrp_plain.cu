// Plain CUDA-core MTTKRP (FP32 or FP64 FMA), and the fixed-order reduction of
// unit partial sums shared by every MTTKRP path.
//
// Computes the mode-n MTTKRP of Sec. III-B through the row view described in
// internal.h: per fiber group (tile of 128 rows, outer index o) the inner
// contraction T[row, r] = sum_k X[row, (o, k)] U_inner[k, r] runs as a
// register-tiled product on CUDA cores, chunk by chunk of 64 k staged in
// shared memory; the fiber group is then folded into the row accumulator with
// the weight L(p(row))[r] * Ofac(o)[r] (the remaining Khatri-Rao factors,
// formed on the fly and never stored in HBM -- the fused schedule P2 of
// Sec. IV-E).
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace deinsum {
namespace {

constexpr int kThreads = 256;
constexpr int BM = DEINSUM_BM;
constexpr int BK = DEINSUM_BK;
constexpr int kFlushEvery = 64;  // fiber groups folded into the inner accumulator before it is flushed

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
struct PlainSmem {
    static constexpr int VW = Vec<T>::n;
    static constexpr int XP = BK + VW;       // case 0 row pitch (elements), keeps vector alignment
    static constexpr int XTP = BM + VW;      // case 1 row pitch
    static constexpr int XS = (BM * XP > BK * XTP) ? BM * XP : BK * XTP;
};

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// Product of the factor rows of modes `modes[0..n)` at the multi-index of `lin`
// (decomposed row-major over `dims`), column r.
template <typename T>
__device__ __forceinline__ T factor_product(const MttkrpArgs &a, int n, const int *modes, const int64_t *dims,
                                            int64_t lin, int r) {
    T v = T(1);
    for (int k = n - 1; k >= 0; --k) {
        const int64_t d = dims[k];
        const int64_t i = lin % d;
        lin /= d;
        v = v * ldg(static_cast<const T *>(a.U[modes[k]]) + i * a.g.R + r);
    }
    return v;
}

template <typename T, int RP>
__global__ void __launch_bounds__(kThreads)
mttkrp_plain_kernel(const MttkrpArgs a) {
    constexpr int VW = Vec<T>::n;
    using VT = typename Vec<T>::type;
    constexpr int TN = RP / 8;
    const MttkrpGeom &g = a.g;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);                               // tile of X
    T *Us = Xs + PlainSmem<T>::XS;                                        // BK x RP inner factor chunk
    T *Ls = Us + BK * RP;                                                 // BM x RP row weights L
    T *Ofs = Ls + BM * RP;                                                // RP outer weights
    int64_t *rowoff = reinterpret_cast<int64_t *>(Ofs + RP);              // BM row offsets (case 0)
    int *rowvalid = reinterpret_cast<int *>(rowoff + BM);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int rq = lane >> 3, rc = lane & 7;
    int myrow[4];
    for (int i = 0; i < 4; ++i)
        myrow[i] = g.kcase == 0 ? warp * 16 + rq + 4 * i : warp * 16 + 4 * rq + i;

    int lmodes[DEINSUM_MAX_ORDER];
    int64_t ldims[DEINSUM_MAX_ORDER];
    for (int m = 0; m < g.n_lmodes; ++m) { lmodes[m] = m; ldims[m] = g.dims[m]; }

    for (int64_t u = blockIdx.x; u < a.n_units; u += gridDim.x) {
        const int64_t col = a.units[3 * u + 0];
        const int64_t fg0 = a.units[3 * u + 1];
        const int64_t fg1 = a.units[3 * u + 2];
        T acc_out[4][TN], acc_in[4][TN];
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < TN; ++j) { acc_out[i][j] = T(0); acc_in[i][j] = T(0); }
        int64_t cur_tile = -1;
        int folded = 0;

        for (int64_t fg = fg0; fg < fg1; ++fg) {
            const int64_t t = fg / g.O;
            const int64_t o = fg - t * g.O;
            __syncthreads();  // previous users of rowoff / Ls / Ofs are done
            if (t != cur_tile) {
                for (int l = tid; l < BM; l += kThreads) {
                    int64_t p = 0, in = 0;
                    int valid = 0;
                    if (g.kcase == 0) {
                        if (g.narrow) {
                            const int64_t gi = l / g.I;
                            in = l - gi * g.I;
                            p = t * g.G + gi;
                            valid = (gi < g.G) && (p < g.P);
                        } else {
                            in = col * BM + l;
                            p = t;
                            valid = in < g.I;
                        }
                        rowoff[l] = valid ? (p * g.I + in) * g.Q : 0;
                    } else {
                        in = col * BM + l;
                        valid = in < g.I;
                        rowoff[l] = in;
                    }
                    rowvalid[l] = valid;
                    for (int r = 0; r < RP; ++r) {
                        T w = T(0);
                        if (valid && r < g.R)
                            w = g.n_lmodes ? factor_product<T>(a, g.n_lmodes, lmodes, ldims, p, r) : T(1);
                        Ls[l * RP + r] = w;
                    }
                }
                cur_tile = t;
            }
            for (int r = tid; r < RP; r += kThreads)
                Ofs[r] = r < g.R ? factor_product<T>(a, g.n_outer, g.outer_mode, g.outer_dim, o, r) : T(0);

            T tacc[4][TN];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < TN; ++j) tacc[i][j] = T(0);

            const T *X = static_cast<const T *>(a.X);
            const T *Uin = static_cast<const T *>(a.U[g.kcase == 0 ? g.order - 1 : g.order - 2]);
            for (int kb = 0; kb < g.n_kb; ++kb) {
                const int64_t k0 = int64_t(kb) * BK;
                __syncthreads();  // Xs / Us free, rowoff visible
                // ---- stage the X tile
                if (g.kcase == 0) {
                    const int64_t base = o * g.K_in + k0;
                    if (g.vec_ok && VW == 4) {
                        for (int idx = tid; idx < BM * (BK / VW); idx += kThreads) {
                            const int l = idx / (BK / VW), kv = idx % (BK / VW);
                            VT v;
                            if (rowvalid[l] && k0 + kv * VW < g.K_in)
                                v = __ldg(reinterpret_cast<const VT *>(X + rowoff[l] + base + kv * VW));
                            else
                                v = VT{};
                            *reinterpret_cast<VT *>(Xs + l * PlainSmem<T>::XP + kv * VW) = v;
                        }
                    } else {
                        for (int idx = tid; idx < BM * BK; idx += kThreads) {
                            const int l = idx / BK, k = idx % BK;
                            T v = T(0);
                            if (rowvalid[l] && k0 + k < g.K_in) v = ldg(X + rowoff[l] + base + k);
                            Xs[l * PlainSmem<T>::XP + k] = v;
                        }
                    }
                } else {
                    const int64_t cb = col * BM;
                    if (g.vec_ok && VW == 4) {
                        for (int idx = tid; idx < BK * (BM / VW); idx += kThreads) {
                            const int k = idx / (BM / VW), lv = idx % (BM / VW);
                            VT v;
                            if (k0 + k < g.K_in && cb + lv * VW < g.I)
                                v = __ldg(reinterpret_cast<const VT *>(
                                    X + (o * g.K_in + k0 + k) * g.I + cb + lv * VW));
                            else
                                v = VT{};
                            *reinterpret_cast<VT *>(Xs + k * PlainSmem<T>::XTP + lv * VW) = v;
                        }
                    } else {
                        for (int idx = tid; idx < BK * BM; idx += kThreads) {
                            const int k = idx / BM, l = idx % BM;
                            T v = T(0);
                            if (k0 + k < g.K_in && cb + l < g.I) v = ldg(X + (o * g.K_in + k0 + k) * g.I + cb + l);
                            Xs[k * PlainSmem<T>::XTP + l] = v;
                        }
                    }
                }
                // ---- stage the inner factor chunk
                for (int idx = tid; idx < BK * RP; idx += kThreads) {
                    const int k = idx / RP, r = idx % RP;
                    T v = T(0);
                    if (r < g.R && k0 + k < g.K_in) v = ldg(Uin + (k0 + k) * g.R + r);
                    Us[idx] = v;
                }
                __syncthreads();
                // ---- register-tiled product
                if (g.kcase == 0) {
                    #pragma unroll 2
                    for (int k = 0; k < BK; k += VW) {
                        VT xv[4];
                        #pragma unroll
                        for (int i = 0; i < 4; ++i)
                            xv[i] = *reinterpret_cast<const VT *>(Xs + myrow[i] * PlainSmem<T>::XP + k);
                        #pragma unroll
                        for (int kk = 0; kk < VW; ++kk) {
                            T uv[TN];
                            #pragma unroll
                            for (int j = 0; j < TN; ++j) uv[j] = Us[(k + kk) * RP + rc * TN + j];
                            #pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const T x = reinterpret_cast<const T *>(&xv[i])[kk];
                                #pragma unroll
                                for (int j = 0; j < TN; ++j) tacc[i][j] = fma(x, uv[j], tacc[i][j]);
                            }
                        }
                    }
                } else {
                    #pragma unroll 4
                    for (int k = 0; k < BK; ++k) {
                        T xr[4];
                        #pragma unroll
                        for (int i = 0; i < 4; i += VW) {
                            VT v = *reinterpret_cast<const VT *>(Xs + k * PlainSmem<T>::XTP + warp * 16 + 4 * rq + i);
                            #pragma unroll
                            for (int e = 0; e < VW; ++e) xr[i + e] = reinterpret_cast<const T *>(&v)[e];
                        }
                        T uv[TN];
                        #pragma unroll
                        for (int j = 0; j < TN; ++j) uv[j] = Us[k * RP + rc * TN + j];
                        #pragma unroll
                        for (int i = 0; i < 4; ++i)
                            #pragma unroll
                            for (int j = 0; j < TN; ++j) tacc[i][j] = fma(xr[i], uv[j], tacc[i][j]);
                    }
                }
            }
            // ---- fold the fiber group with its Khatri-Rao weight
            #pragma unroll
            for (int i = 0; i < 4; ++i)
                #pragma unroll
                for (int j = 0; j < TN; ++j) {
                    const int r = rc * TN + j;
                    const T w = Ls[myrow[i] * RP + r] * Ofs[r];
                    acc_in[i][j] = fma(w, tacc[i][j], acc_in[i][j]);
                }
            if (++folded == kFlushEvery) {
                folded = 0;
                for (int i = 0; i < 4; ++i)
                    for (int j = 0; j < TN; ++j) { acc_out[i][j] += acc_in[i][j]; acc_in[i][j] = T(0); }
            }
        }
        // ---- unit partial: one 128 x RP block per unit
        T *part = (sizeof(T) == 8) ? reinterpret_cast<T *>(a.partial64) : reinterpret_cast<T *>(a.partial);
        part += u * BM * RP;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < TN; ++j)
                part[myrow[i] * RP + rc * TN + j] = acc_out[i][j] + acc_in[i][j];
    }
}

template <typename T>
size_t plain_smem_bytes(int RP) {
    return sizeof(T) * (size_t(PlainSmem<T>::XS) + size_t(BK) * RP + size_t(BM) * RP + RP) +
           sizeof(int64_t) * BM + sizeof(int) * BM;
}

template <typename T, int RP>
int launch_plain_rp(const MttkrpArgs &a, int n_sm, void *stream) {
    const size_t smem = plain_smem_bytes<T>(RP);
    cudaError_t e = cudaFuncSetAttribute(mttkrp_plain_kernel<T, RP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return int(e);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mttkrp_plain_kernel<T, RP>, kThreads, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = int64_t(n_sm) * per_sm;
    if (grid > a.n_units) grid = a.n_units;
    if (grid < 1) grid = 1;
    mttkrp_plain_kernel<T, RP><<<unsigned(grid), kThreads, smem, static_cast<cudaStream_t>(stream)>>>(a);
    count_launch();
    return int(cudaGetLastError());
}

template <typename T>
int launch_plain(const MttkrpArgs &a, int n_sm, void *stream) {
    switch (a.g.R_pad) {
        case 16: return launch_plain_rp<T, 16>(a, n_sm, stream);
        case 32: return launch_plain_rp<T, 32>(a, n_sm, stream);
        case 64: return launch_plain_rp<T, 64>(a, n_sm, stream);
    }
    return int(cudaErrorInvalidValue);
}

// M[col*128 + i, r] = sum over the column's units (in order) and, for narrow
// rows, over the G row groups of the tile, of the unit partials.
template <typename T>
__global__ void mttkrp_reduce_kernel(const T *__restrict__ partial, const int64_t *__restrict__ col_begin,
                                     T *__restrict__ out, int64_t I, int R, int RP, int64_t rows_per_col,
                                     int64_t G, int narrow) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= I * R) return;
    const int64_t row = idx / R;
    const int r = int(idx - row * R);
    const int64_t col = row / rows_per_col;
    const int64_t i = row - col * rows_per_col;
    T s = T(0);
    for (int64_t u = col_begin[col]; u < col_begin[col + 1]; ++u) {
        const T *p = partial + u * BM * RP;
        if (narrow) {
            for (int64_t gi = 0; gi < G; ++gi) s += p[(gi * I + i) * RP + r];
        } else {
            s += p[i * RP + r];
        }
    }
    out[idx] = s;
}

// The same sum for columns with many partial blocks (few output rows, long contracted
// modes: e.g. mode 0 of an order-5 tensor, hundreds of units in one column): each block
// takes 32 consecutive output elements; its eight warps each add one contiguous eighth of
// the column's (unit, row group) terms in order, and thread 0 of each element's slot adds
// the eight segment sums in order.  The order is fixed by the schedule alone, so results
// stay bit-reproducible.
template <typename T>
__global__ void mttkrp_reduce_seg_kernel(const T *__restrict__ partial, const int64_t *__restrict__ col_begin,
                                         T *__restrict__ out, int64_t I, int R, int RP, int64_t rows_per_col,
                                         int64_t G, int narrow) {
    __shared__ T seg[8][32];
    const int e = threadIdx.x & 31, sg = threadIdx.x >> 5;
    const int64_t idx = int64_t(blockIdx.x) * 32 + e;
    T s = T(0);
    if (idx < I * R) {
        const int64_t row = idx / R;
        const int r = int(idx - row * R);
        const int64_t col = row / rows_per_col;
        const int64_t i = row - col * rows_per_col;
        const int64_t g = narrow ? G : 1;
        const int64_t u0 = col_begin[col], nterm = (col_begin[col + 1] - u0) * g;
        const int64_t t0 = nterm * sg / 8, t1 = nterm * (sg + 1) / 8;
        for (int64_t t = t0; t < t1; ++t) {
            const int64_t u = u0 + t / g, gi = t - (t / g) * g;
            s += partial[(u * BM + (narrow ? gi * I + i : i)) * RP + r];
        }
    }
    seg[sg][e] = s;
    __syncthreads();
    if (sg == 0 && idx < I * R) {
        T tot = T(0);
        #pragma unroll
        for (int k = 0; k < 8; ++k) tot += seg[k][e];
        out[idx] = tot;
    }
}

// MTTKRP followed by a matrix product (Sec. II-A running example): per output
// row, M[row, :] is summed from the unit partials in the same fixed order as
// above into shared memory, then out[row, l] = sum_r M[row, r] C[r, l] (r in
// order).  M never reaches HBM.
template <typename T>
__global__ void mttkrp_reduce_mm_kernel(const T *__restrict__ partial, const int64_t *__restrict__ col_begin,
                                        const T *__restrict__ C, T *__restrict__ out, int64_t I, int R, int RP,
                                        int64_t rows_per_col, int64_t G, int narrow, int64_t L) {
    __shared__ T m[64];
    for (int64_t row = blockIdx.x; row < I; row += gridDim.x) {
        const int64_t col = row / rows_per_col;
        const int64_t i = row - col * rows_per_col;
        for (int r = threadIdx.x; r < R; r += blockDim.x) {
            T s = T(0);
            for (int64_t u = col_begin[col]; u < col_begin[col + 1]; ++u) {
                const T *p = partial + u * BM * RP;
                if (narrow) {
                    for (int64_t gi = 0; gi < G; ++gi) s += p[(gi * I + i) * RP + r];
                } else {
                    s += p[i * RP + r];
                }
            }
            m[r] = s;
        }
        __syncthreads();
        for (int64_t l = threadIdx.x; l < L; l += blockDim.x) {
            T acc = T(0);
            for (int r = 0; r < R; ++r) acc += m[r] * C[int64_t(r) * L + l];
            out[row * L + l] = acc;
        }
        __syncthreads();
    }
}

template <typename T>
int launch_reduce(const MttkrpArgs &a, const T *partial, const int64_t *col_begin, void *out, void *stream,
                  const void *C, int64_t L) {
    if (C) {
        const int64_t blocks = a.g.I < 8192 ? a.g.I : 8192;
        mttkrp_reduce_mm_kernel<T><<<unsigned(blocks), 128, 0, static_cast<cudaStream_t>(stream)>>>(
            partial, col_begin, static_cast<const T *>(C), static_cast<T *>(out), a.g.I, a.g.R, a.g.R_pad,
            a.g.rows_per_col, a.g.G, a.g.narrow, L);
        count_launch();
        return int(cudaGetLastError());
    }
    const int64_t n = a.g.I * a.g.R;
    // terms per output element: the units of a column times the row groups of a narrow tile
    const int64_t cols = a.g.n_cols > 0 ? a.g.n_cols : 1;
    const int64_t terms = (a.n_units + cols - 1) / cols * (a.g.narrow ? a.g.G : 1);
    if (terms > 64) {
        mttkrp_reduce_seg_kernel<T><<<unsigned((n + 31) / 32), 256, 0, static_cast<cudaStream_t>(stream)>>>(
            partial, col_begin, static_cast<T *>(out), a.g.I, a.g.R, a.g.R_pad, a.g.rows_per_col, a.g.G, a.g.narrow);
    } else {
        const int threads = 256;
        const int64_t blocks = (n + threads - 1) / threads;
        mttkrp_reduce_kernel<T><<<unsigned(blocks), threads, 0, static_cast<cudaStream_t>(stream)>>>(
            partial, col_begin, static_cast<T *>(out), a.g.I, a.g.R, a.g.R_pad, a.g.rows_per_col, a.g.G, a.g.narrow);
    }
    count_launch();
    return int(cudaGetLastError());
}

}  // namespace

template <typename T>
int plain_ctas_per_sm(int RP) {
    int per_sm = 1;
    switch (RP) {
        case 16:
            cudaFuncSetAttribute(mttkrp_plain_kernel<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(plain_smem_bytes<T>(16)));
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mttkrp_plain_kernel<T, 16>, kThreads, plain_smem_bytes<T>(16));
            break;
        case 32:
            cudaFuncSetAttribute(mttkrp_plain_kernel<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(plain_smem_bytes<T>(32)));
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mttkrp_plain_kernel<T, 32>, kThreads, plain_smem_bytes<T>(32));
            break;
        default:
            cudaFuncSetAttribute(mttkrp_plain_kernel<T, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(plain_smem_bytes<T>(64)));
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mttkrp_plain_kernel<T, 64>, kThreads, plain_smem_bytes<T>(64));
            break;
    }
    cudaGetLastError();
    return per_sm < 1 ? 1 : per_sm;
}

int mttkrp_plain_ctas_per_sm(int f64, int R_pad) { return f64 ? plain_ctas_per_sm<double>(R_pad) : plain_ctas_per_sm<float>(R_pad); }

int launch_mttkrp_plain_f32(const MttkrpArgs &a, int n_sm, void *stream) { return launch_plain<float>(a, n_sm, stream); }
int launch_mttkrp_plain_f64(const MttkrpArgs &a, int n_sm, void *stream) { return launch_plain<double>(a, n_sm, stream); }
int launch_mttkrp_reduce_f32(const MttkrpArgs &a, const int64_t *col_begin, void *out, void *stream,
                             const void *C, int64_t L) {
    return launch_reduce<float>(a, a.partial, col_begin, out, stream, C, L);
}
int launch_mttkrp_reduce_f64(const MttkrpArgs &a, const int64_t *col_begin, void *out, void *stream,
                             const void *C, int64_t L) {
    return launch_reduce<double>(a, a.partial64, col_begin, out, stream, C, L);
}

}  // namespace deinsum
