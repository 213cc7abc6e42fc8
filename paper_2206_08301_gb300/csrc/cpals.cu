// CP-ALS on the device: the decomposition whose bottleneck the paper's MTTKRP
// serves (Sec. I).  The ALS steps follow Kolda & Bader, "Tensor Decompositions
// and Applications", SIAM Review 2009, Sec. 3.4: for each mode n in turn
// (Gauss-Seidel),
//   M   = MTTKRP_n(X, U)                         (split-BF16 tensor-core kernel)
//   V   = Hadamard_{m != n} G_m,  G_m = U_m^T U_m    (FP64, R x R)
//   U_n = M V^{-1}                               (Cholesky of V, FP64 solves per row)
//   lambda_r = ||U_n[:, r]||_2,  U_n[:, r] /= lambda_r   (FP64 norms)
//   G_n = U_n^T U_n
// and after the sweep fit = 1 - sqrt(max(0, ||X||^2 + ||Xhat||^2 - 2 <X, Xhat>)) / ||X||
// with ||Xhat||^2 = lambda^T (Hadamard_m G_m) lambda and
// <X, Xhat> = sum_r lambda_r sum_i M_last[i, r] U_last[i, r].
// Only the MTTKRP runs in (split) FP32; every R x R quantity, the solves, the
// norms and the fit are FP64.  Everything stays on the device; the host only
// enqueues kernels.
//
// Dimension tree (order 3, split-BF16, R <= 32, I_2 a multiple of 4): modes 0
// and 1 share the partial contraction T = X x_2 U_2 (T[i, j, r] = sum_k X[i, j, k]
// U_2[k, r], an I_0 x I_1 x R tensor written once by the tensor-core TTM kernel):
//   M_0[i, r] = sum_j T[i, j, r] U_1[j, r],   M_1[j, r] = sum_i T[i, j, r] U_0[i, r],
// the latter with U_0 already updated -- T depends only on U_2, which the sweep
// updates last.  X is then streamed twice per sweep instead of three times.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace deinsum {
namespace {

constexpr int kMaxR = 64;

// Dimension tree: M_0[i, r] = sum_j T[i, j, r] U_1[j, r].  One block per i; thread
// (r, jg) sums j = jg, jg + 4, ...; the four partial sums are added in order.
__global__ void __launch_bounds__(128) tree_m0_kernel(const float *__restrict__ T, const float *__restrict__ U1,
                                                      float *__restrict__ M, int64_t J, int R) {
    const int64_t i = blockIdx.x;
    const int r = threadIdx.x & 31, jg = threadIdx.x >> 5;
    __shared__ float red[4][32];
    float acc = 0.f;
    if (r < R)
        for (int64_t j = jg; j < J; j += 4) acc = fmaf(T[(i * J + j) * R + r], U1[j * R + r], acc);
    red[jg][r] = acc;
    __syncthreads();
    if (threadIdx.x < R) M[i * R + threadIdx.x] = ((red[0][r] + red[1][r]) + red[2][r]) + red[3][r];
}

// The same for R a multiple of 4 (the common case), with 16-byte loads: thread (c, jg) of a
// block of 256 holds rank columns 4 c .. 4 c + 3 (c < R / 4) and sums j = jg, jg + 32, ...
// in two independent chains (j 32 apart); the 32 j groups are added in a fixed order.
__global__ void __launch_bounds__(256) tree_m0_vec_kernel(const float *__restrict__ T, const float *__restrict__ U1,
                                                          float *__restrict__ M, int64_t J, int R) {
    const int64_t i = blockIdx.x;
    const int c = threadIdx.x & 7, jg = threadIdx.x >> 3;
    const int R4 = R >> 2;
    __shared__ float4 red[32][8];
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
    if (c < R4) {
        const float4 *Ti = reinterpret_cast<const float4 *>(T + i * J * R);
        const float4 *U4 = reinterpret_cast<const float4 *>(U1);
        int64_t j = jg;
        for (; j + 32 < J; j += 64) {
            const float4 t0 = Ti[j * R4 + c], u0 = U4[j * R4 + c];
            const float4 t1 = Ti[(j + 32) * R4 + c], u1 = U4[(j + 32) * R4 + c];
            a0.x = fmaf(t0.x, u0.x, a0.x); a0.y = fmaf(t0.y, u0.y, a0.y);
            a0.z = fmaf(t0.z, u0.z, a0.z); a0.w = fmaf(t0.w, u0.w, a0.w);
            a1.x = fmaf(t1.x, u1.x, a1.x); a1.y = fmaf(t1.y, u1.y, a1.y);
            a1.z = fmaf(t1.z, u1.z, a1.z); a1.w = fmaf(t1.w, u1.w, a1.w);
        }
        for (; j < J; j += 32) {
            const float4 t0 = Ti[j * R4 + c], u0 = U4[j * R4 + c];
            a0.x = fmaf(t0.x, u0.x, a0.x); a0.y = fmaf(t0.y, u0.y, a0.y);
            a0.z = fmaf(t0.z, u0.z, a0.z); a0.w = fmaf(t0.w, u0.w, a0.w);
        }
    }
    red[jg][c] = make_float4(a0.x + a1.x, a0.y + a1.y, a0.z + a1.z, a0.w + a1.w);
    __syncthreads();
    if (threadIdx.x < R) {
        const int cc = threadIdx.x >> 2, q = threadIdx.x & 3;
        float t = 0.f;
        for (int k = 0; k < 32; ++k) {
            const float4 v = red[k][cc];
            t += q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
        }
        M[i * R + threadIdx.x] = t;
    }
}

// Dimension tree: M_1[j, r] = sum_i T[i, j, r] U_0[i, r].  Block (jb, is): four j, the
// i of slice is (kTreeSplit slices); thread (j, r) runs over them in order into
// part[is][j][r]; tree_m1_sum adds the slices in order.
constexpr int kTreeSplit = 8;
__global__ void __launch_bounds__(128) tree_m1_kernel(const float *__restrict__ T, const float *__restrict__ U0,
                                                      float *__restrict__ part, int64_t I, int64_t J, int R) {
    const int r = threadIdx.x & 31;
    const int64_t j = int64_t(blockIdx.x) * 4 + (threadIdx.x >> 5);
    if (r >= R || j >= J) return;
    const int64_t i0 = I * blockIdx.y / kTreeSplit, i1 = I * (blockIdx.y + 1) / kTreeSplit;
    float acc = 0.f;
    #pragma unroll 4
    for (int64_t i = i0; i < i1; ++i) acc = fmaf(T[(i * J + j) * R + r], U0[i * R + r], acc);
    part[(int64_t(blockIdx.y) * J + j) * R + r] = acc;
}

__global__ void tree_m1_sum(const float *__restrict__ part, float *__restrict__ M, int64_t n) {
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        float v = 0.f;
        for (int q = 0; q < kTreeSplit; ++q) v += part[q * n + e];
        M[e] = v;
    }
}

bool tree_eligible(int order, const int64_t *dims, int R, deinsum_prec prec) {
    return order == 3 && prec == DEINSUM_PREC_SPLIT_BF16 && R <= 32 && dims[2] % 4 == 0 &&
           dims[0] < (int64_t(1) << 31) && dims[1] < (int64_t(1) << 31) && dims[2] < (int64_t(1) << 31);
}

// G = U^T U in FP64 (U: I x R float, row-major).  One block per row r1 of G, 1024 threads:
// thread (r2, slice) sums rows slice, slice + 16, ... of U[i, r1] U[i, r2] in four
// independent FP32 chains (rows 16 apart), folded into an FP64 accumulator every 8 products
// per chain (the FP64 pipe is narrow); the 16 slices are added in a fixed order.
constexpr int kGramSlices = 16;
__global__ void __launch_bounds__(1024) gram_kernel(const float *__restrict__ U, int64_t I, int R,
                                                    double *__restrict__ G) {
    const int r1 = blockIdx.x;
    const int r2 = threadIdx.x & 63, sl = threadIdx.x >> 6;
    __shared__ double red[kGramSlices][64];
    double acc = 0.0;
    if (r2 < R) {
        constexpr int64_t step = 4 * kGramSlices;
        int64_t i = sl;
        float p[4] = {0.f, 0.f, 0.f, 0.f};
        int cnt = 0;
        for (; i + 3 * kGramSlices < I; i += step) {
            #pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t row = (i + q * kGramSlices) * R;
                p[q] = fmaf(U[row + r1], U[row + r2], p[q]);
            }
            if (++cnt == 8) {
                acc += (double(p[0]) + double(p[1])) + (double(p[2]) + double(p[3]));
                p[0] = p[1] = p[2] = p[3] = 0.f;
                cnt = 0;
            }
        }
        for (; i < I; i += kGramSlices) p[0] = fmaf(U[i * R + r1], U[i * R + r2], p[0]);
        acc += (double(p[0]) + double(p[1])) + (double(p[2]) + double(p[3]));
    }
    red[sl][r2] = acc;
    __syncthreads();
    if (sl == 0 && r2 < R) {
        double t = 0.0;
        #pragma unroll
        for (int k = 0; k < kGramSlices; ++k) t += red[k][r2];
        G[r1 * R + r2] = t;
    }
}

// One block: V = Hadamard of the Grams of every mode except `mode`, its
// Cholesky factor L (V = L L^T), then W = V^{-1} = L^{-T} L^{-1}, written to
// global memory for apply_kernel.  A pivot that is not positive (V singular
// to FP64 precision) is replaced by a tiny positive value and the status word
// records it.
__global__ void __launch_bounds__(256) inverse_kernel(const double *__restrict__ grams, int order, int mode, int R,
                                                      double *__restrict__ W, int *status) {
    extern __shared__ double inv_smem[];   // L and L^{-1}, kMaxR x (kMaxR + 1) each
    double(*L)[kMaxR + 1] = reinterpret_cast<double(*)[kMaxR + 1]>(inv_smem);
    double(*Li)[kMaxR + 1] = reinterpret_cast<double(*)[kMaxR + 1]>(inv_smem + kMaxR * (kMaxR + 1));
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        const int a = e / R, b = e % R;
        double v = 1.0;
        for (int m = 0; m < order; ++m)
            if (m != mode) v *= grams[(size_t(m) * R + a) * R + b];
        L[a][b] = v;
    }
    __syncthreads();
    // in-place Cholesky of the lower triangle, right-looking: per column k the
    // pivot, the scaled column, then the rank-1 update of the trailing block
    __shared__ double floor_pivot;
    if (threadIdx.x == 0) {
        double dmax = 0.0;
        for (int k = 0; k < R; ++k) dmax = fmax(dmax, fabs(L[k][k]));
        floor_pivot = dmax > 0.0 ? dmax * 1e-300 : 1e-300;
    }
    __syncthreads();
    __shared__ double rinv[kMaxR];   // 1 / L[k][k]: one FP64 division per column
    for (int k = 0; k < R; ++k) {
        if (threadIdx.x == 0) {
            double d = L[k][k];
            if (!(d > 0.0)) {
                d = floor_pivot;
                atomicOr(status, 2);
            }
            const double sd = sqrt(d);
            L[k][k] = sd;
            rinv[k] = 1.0 / sd;
        }
        __syncthreads();
        for (int i = k + 1 + int(threadIdx.x); i < R; i += blockDim.x) L[i][k] *= rinv[k];
        __syncthreads();
        const int rem = R - k - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            const int i = k + 1 + e / rem, j = k + 1 + e % rem;
            if (j <= i) L[i][j] -= L[i][k] * L[j][k];
        }
        __syncthreads();
    }
    // L^{-1} by elimination on [L | I], all threads per step: row k of the
    // right-hand side is divided by L[k][k], then removed from the rows below
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) Li[e / R][e % R] = (e / R == e % R) ? 1.0 : 0.0;
    for (int k = 0; k < R; ++k) {
        __syncthreads();
        for (int j = threadIdx.x; j <= k; j += blockDim.x) Li[k][j] *= rinv[k];
        __syncthreads();
        const int rows_below = R - k - 1;
        for (int e = threadIdx.x; e < rows_below * (k + 1); e += blockDim.x) {
            const int i = k + 1 + e / (k + 1), j = e % (k + 1);
            Li[i][j] -= L[i][k] * Li[k][j];
        }
    }
    __syncthreads();
    // W = L^{-T} L^{-1}: W[a][b] = sum_{p >= max(a, b)} Li[p][a] Li[p][b]
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        const int a = e / R, b = e % R;
        double s = 0.0;
        for (int p = a > b ? a : b; p < R; ++p) s += Li[p][a] * Li[p][b];
        W[e] = s;
    }
}

// U_n[i, b] = sum_a M[i, a] W[a, b]  (FP64 products of the FP32 MTTKRP rows, rounded once to FP32).
__global__ void __launch_bounds__(256) apply_kernel(const float *__restrict__ M, const double *__restrict__ W,
                                                    float *__restrict__ Un, int64_t I, int R) {
    __shared__ double Ws[kMaxR * kMaxR];
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) Ws[e] = W[e];
    __syncthreads();
    const int64_t n = I * R;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = e / R;
        const int b = int(e - i * R);
        const float *m = M + i * R;
        double s = 0.0;
        for (int a = 0; a < R; ++a) s += double(m[a]) * Ws[a * R + b];
        Un[e] = float(s);
    }
}

// lambda_r = ||U[:, r]||_2 in FP64, then U[:, r] /= lambda_r (a zero column keeps lambda = 0).
__global__ void normalize_kernel(float *__restrict__ U, int64_t I, int R, double *__restrict__ lambda) {
    const int r = blockIdx.x;
    __shared__ double red[32];
    double s = 0.0;
    {
        float part = 0.f;
        int cnt = 0;
        for (int64_t i = threadIdx.x; i < I; i += blockDim.x) {
            const float v = U[i * R + r];
            part = fmaf(v, v, part);
            if (++cnt == 16) {
                s += double(part);
                part = 0.f;
                cnt = 0;
            }
        }
        s += double(part);
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    __shared__ double nrm;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
        nrm = sqrt(t);
        lambda[r] = nrm;
    }
    __syncthreads();
    if (nrm > 0.0) {
        const double inv = 1.0 / nrm;
        for (int64_t i = threadIdx.x; i < I; i += blockDim.x) U[i * R + r] = float(double(U[i * R + r]) * inv);
    }
}

// ||X||^2 in FP64: per-block partial sums, then a single-block finish.
// ||X||^2 partial sums: each thread takes four float4 loads per step (independent,
// so they are in flight together), accumulates up to a few thousand squares in four
// FP32 partials, and the block adds the threads' sums in FP64.  (||X||^2 only
// enters the fit; FP32 partials of <= 2^13 squares keep it to ~1e-6 relative.)
__global__ void __launch_bounds__(256) sumsq_partial_kernel(const float *__restrict__ X, int64_t n,
                                                            double *__restrict__ partial) {
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nth = int64_t(gridDim.x) * blockDim.x;
    const bool vec = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    const int64_t n4 = vec ? n / 4 : 0;
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    double s = 0.0;
    float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
    int steps = 0;
    int64_t i = tid;
    for (; i + 3 * nth < n4; i += 4 * nth) {
        const float4 a = X4[i], b = X4[i + nth], c = X4[i + 2 * nth], d = X4[i + 3 * nth];
        p0 = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, p0))));
        p1 = fmaf(b.x, b.x, fmaf(b.y, b.y, fmaf(b.z, b.z, fmaf(b.w, b.w, p1))));
        p2 = fmaf(c.x, c.x, fmaf(c.y, c.y, fmaf(c.z, c.z, fmaf(c.w, c.w, p2))));
        p3 = fmaf(d.x, d.x, fmaf(d.y, d.y, fmaf(d.z, d.z, fmaf(d.w, d.w, p3))));
        if (++steps == 512) {   // 2^13 squares per partial
            s += (double(p0) + double(p1)) + (double(p2) + double(p3));
            p0 = p1 = p2 = p3 = 0.f;
            steps = 0;
        }
    }
    for (; i < n4; i += nth) {
        const float4 a = X4[i];
        p0 = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, p0))));
    }
    s += (double(p0) + double(p1)) + (double(p2) + double(p3));
    for (int64_t e = 4 * n4 + tid; e < n; e += nth) s += double(X[e]) * double(X[e]);
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void sum_kernel(const double *__restrict__ partial, int n, double *__restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

// fit after a sweep (one block): inner = sum_r lambda_r sum_i M[i, r] U[i, r]
// over the last mode; normXhat^2 = lambda^T (Hadamard_m G_m) lambda.
// The final fit takes the direct residual only when the expansion can cancel: its
// error in res^2 is about twice the MTTKRP's relative error times ||X||^2 (~1e-5 ||X||^2
// on the split path), i.e. below 5e-5 in the fit while res^2 >= 1e-2 ||X||^2.
constexpr double kDirectResidualBelow = 1e-2;

__global__ void fit_kernel(const float *__restrict__ M, const float *__restrict__ U, int64_t I, int R,
                           const double *__restrict__ lambda, const double *__restrict__ grams, int order,
                           const double *__restrict__ normx2, double *__restrict__ fit_out,
                           int *__restrict__ need_direct) {
    // blockDim = 256: thread (r = tid % 64, slice = tid / 64) sums rows slice,
    // slice + 4, ... of M[i, r] U[i, r] (FP32 partials of 8, FP64 accumulation);
    // every thread also takes a share of the R x R terms of ||Xhat||^2
    __shared__ double red[4][64];
    __shared__ double xr[256];
    const int r = threadIdx.x & 63, sl = threadIdx.x >> 6;
    double acc = 0.0;
    if (r < R) {
        float part = 0.f;
        int cnt = 0;
        for (int64_t i = sl; i < I; i += 4) {
            part = fmaf(M[i * R + r], U[i * R + r], part);
            if (++cnt == 8) {
                acc += double(part);
                part = 0.f;
                cnt = 0;
            }
        }
        acc += double(part);
        acc *= lambda[r];
    }
    red[sl][r] = acc;
    double xh = 0.0;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        const int a = e / R, b = e % R;
        double h = lambda[a] * lambda[b];
        for (int m = 0; m < order; ++m) h *= grams[(size_t(m) * R + a) * R + b];
        xh += h;
    }
    xr[threadIdx.x] = xh;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (int(threadIdx.x) < w) xr[threadIdx.x] += xr[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 64) red[0][threadIdx.x] = (red[0][threadIdx.x] + red[1][threadIdx.x]) +
                                                 (red[2][threadIdx.x] + red[3][threadIdx.x]);
    __syncthreads();
    if (threadIdx.x == 0) {
        double inner = 0.0;
        for (int q = 0; q < R; ++q) inner += red[0][q];
        const double res2 = fmax(0.0, *normx2 + xr[0] - 2.0 * inner);
        *fit_out = 1.0 - sqrt(res2) / sqrt(*normx2);
        if (need_direct) *need_direct = res2 < kDirectResidualBelow * *normx2 ? 1 : 0;
    }
}

// Direct residual ||X - Xhat||^2 with Xhat = [[lambda; U]]: X is viewed as
// rows (all modes but the last) x K (the last mode).  A block takes 64-row tiles and
// sweeps their k in chunks of 64: W[row, r] = lambda_r prod_{m < N-1} U_m[i_m(row), r]
// (once per row tile) and the last factor's chunk are staged in shared memory
// (r-major), each thread forms 4 x 4 reconstructed entries in FP32 (R
// multiply-adds each), squares the residuals, sums them in FP32 over its chunk
// and adds that sum to an FP64 per-block partial.  Accurate where the expansion
// of the fit cancels.
struct ResidualArgs {
    const float *X;
    const float *U[DEINSUM_MAX_ORDER];
    int64_t dims[DEINSUM_MAX_ORDER];
    int order, R;
    const double *lambda;
    double *partial;  // gridDim.x
    const int *need;  // 0: the expansion's fit stands, nothing to compute
};

__global__ void __launch_bounds__(256) residual_kernel(const ResidualArgs a) {
    __shared__ float Ws[kMaxR][64 + 4];
    __shared__ float Cs[kMaxR][64 + 4];
    __shared__ double red[8];
    if (a.need && *a.need == 0) {   // the same value for every thread
        if (threadIdx.x == 0) a.partial[blockIdx.x] = 0.0;
        return;
    }
    const int R = a.R;
    const int64_t K = a.dims[a.order - 1];
    int64_t rows = 1;
    for (int m = 0; m < a.order - 1; ++m) rows *= a.dims[m];
    const int64_t rtiles = (rows + 63) / 64, ktiles = (K + 63) / 64;
    const int t = threadIdx.x, tr = t >> 4, tk = t & 15;
    const float *C = a.U[a.order - 1];
    double block_sum = 0.0;
    // a row tile's weights W[row, r] = lambda_r prod_{m < N-1} U_m[i_m(row), r] are built
    // once (FP64 products, stored in FP32) and reused for every k tile of the row
    for (int64_t rt = blockIdx.x; rt < rtiles; rt += gridDim.x) {
        const int64_t r0 = rt * 64;
        __syncthreads();
        for (int e = t; e < 64 * R; e += 256) {
            const int rl = e / R, r = e % R;
            const int64_t row = r0 + rl;
            float w = 0.f;
            if (row < rows) {
                double v = a.lambda[r];
                int64_t rem = row;
                for (int m = a.order - 2; m >= 0; --m) {
                    const int64_t i = rem % a.dims[m];
                    rem /= a.dims[m];
                    v *= double(a.U[m][i * R + r]);
                }
                w = float(v);
            }
            Ws[r][rl] = w;
        }
        for (int64_t kt = 0; kt < ktiles; ++kt) {
        const int64_t k0 = kt * 64;
        __syncthreads();
        for (int e = t; e < 64 * R; e += 256) {
            const int kl = e / R, r = e % R;
            Cs[r][kl] = (k0 + kl < K) ? C[(k0 + kl) * R + r] : 0.f;
        }
        __syncthreads();
        float xh[4][4] = {};
        for (int r = 0; r < R; ++r) {
            const float4 w4 = *reinterpret_cast<const float4 *>(&Ws[r][4 * tr]);
            const float4 c4 = *reinterpret_cast<const float4 *>(&Cs[r][4 * tk]);
            const float wv[4] = {w4.x, w4.y, w4.z, w4.w}, cv[4] = {c4.x, c4.y, c4.z, c4.w};
            #pragma unroll
            for (int i = 0; i < 4; ++i)
                #pragma unroll
                for (int j = 0; j < 4; ++j) xh[i][j] = fmaf(wv[i], cv[j], xh[i][j]);
        }
        float s = 0.f;
        #pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t row = r0 + 4 * tr + i;
            if (row >= rows) continue;
            #pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t k = k0 + 4 * tk + j;
                if (k < K) {
                    const float d = a.X[row * K + k] - xh[i][j];
                    s = fmaf(d, d, s);
                }
            }
        }
        block_sum += double(s);
        }
    }
    for (int off = 16; off > 0; off >>= 1) block_sum += __shfl_down_sync(0xffffffffu, block_sum, off);
    if ((t & 31) == 0) red[t >> 5] = block_sum;
    __syncthreads();
    if (t == 0) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[w];
        a.partial[blockIdx.x] = v;
    }
}

// fit = 1 - sqrt(residual^2) / ||X|| from the summed residual partials (one block),
// when the direct residual was needed (*need != 0); else the expansion's fit stays.
__global__ void fit_from_residual_kernel(const double *__restrict__ partial, int n, const double *__restrict__ normx2,
                                         double *__restrict__ fit_out, const int *__restrict__ need) {
    if (need && *need == 0) return;
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
        *fit_out = 1.0 - sqrt(t) / sqrt(*normx2);
    }
}

}  // namespace
}  // namespace deinsum

using namespace deinsum;

struct deinsum_cpals_s {
    int order = 0;
    int R = 0;
    int64_t dims[DEINSUM_MAX_ORDER] = {0};
    deinsum_prec prec = DEINSUM_PREC_SPLIT_BF16;
    deinsum_plan_t plans[DEINSUM_MAX_ORDER] = {nullptr};
    int device = -1;
    char *ws = nullptr;
    bool ws_owned = true;
    float *M = nullptr;          // max_n I_n x R
    double *grams = nullptr;     // order x R x R
    double *normx2 = nullptr;    // 1
    double *partial = nullptr;   // kSumBlocks
    double *W = nullptr;         // R x R inverse of the Gram-Hadamard matrix
    int *status = nullptr;       // 1
    // dimension tree (see the top of the file)
    bool tree_ok = false;        // the shape allows it
    bool tree_on = true;         // enabled (deinsum_cpals_set_dimension_tree)
    float *T = nullptr;          // I_0 x I_1 x R
    unsigned char *tb = nullptr; // split-BF16 tiles of U_2
    CUtensorMap tmap{};
    const void *tmap_ptr = nullptr;
    bool tmap_ok = false;
    uint32_t tmap_box = 0;
};

namespace {
constexpr int kSumBlocks = 1024;
constexpr size_t kInvSmem = size_t(2) * kMaxR * (kMaxR + 1) * sizeof(double);

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// The handle's own workspace: M (max_n I_n x R float), the Grams (N x R x R
// double), ||X||^2, the status word, the FP64 partial sums.
size_t tree_T_bytes(const deinsum_cpals_s *h) {
    return h->tree_ok ? round_up(size_t(h->dims[0]) * size_t(h->dims[1]) * size_t(h->R) * 4, 1024) : 0;
}
size_t tree_tb_bytes(const deinsum_cpals_s *h) {
    // split tiles of U_2, then the kTreeSplit partial blocks of M_1
    return h->tree_ok ? round_up(size_t((h->dims[2] + 63) / 64) * 2 * 32 * 64 * 2, 1024) +
                            round_up(size_t(kTreeSplit) * size_t(h->dims[1]) * size_t(h->R) * 4, 1024)
                      : 0;
}

size_t cpals_own_bytes(const deinsum_cpals_s *h) {
    int64_t imax = 0;
    for (int m = 0; m < h->order; ++m) imax = h->dims[m] > imax ? h->dims[m] : imax;
    const size_t bM = round_up(size_t(imax) * h->R * 4, 256);
    const size_t bG = round_up(size_t(h->order) * h->R * h->R * 8, 256);
    return round_up(bM + bG + 256 + size_t(kSumBlocks) * 8 + size_t(h->R) * h->R * 8, 1024) + tree_T_bytes(h) +
           tree_tb_bytes(h);
}

void cpals_attach_own(deinsum_cpals_s *h, char *p, bool owned, int dev) {
    int64_t imax = 0;
    for (int m = 0; m < h->order; ++m) imax = h->dims[m] > imax ? h->dims[m] : imax;
    const size_t bM = round_up(size_t(imax) * h->R * 4, 256);
    const size_t bG = round_up(size_t(h->order) * h->R * h->R * 8, 256);
    h->ws = p;
    h->ws_owned = owned;
    h->device = dev;
    h->M = reinterpret_cast<float *>(h->ws);
    h->grams = reinterpret_cast<double *>(h->ws + bM);
    h->normx2 = reinterpret_cast<double *>(h->ws + bM + bG);
    h->status = reinterpret_cast<int *>(h->ws + bM + bG + 8);
    h->partial = reinterpret_cast<double *>(h->ws + bM + bG + 256);
    h->W = h->partial + kSumBlocks;
    const size_t base = round_up(bM + bG + 256 + size_t(kSumBlocks) * 8 + size_t(h->R) * h->R * 8, 1024);
    h->T = h->tree_ok ? reinterpret_cast<float *>(h->ws + base) : nullptr;
    h->tb = h->tree_ok ? reinterpret_cast<unsigned char *>(h->ws + base + tree_T_bytes(h)) : nullptr;
}

std::string mttkrp_spec(int order, int mode) {
    const char *x = "abcdefgh";
    std::string s(x, size_t(order));
    for (int m = 0; m < order; ++m)
        if (m != mode) {
            s += ',';
            s += x[m];
            s += 'r';
        }
    s += "->";
    s += x[mode];
    s += 'r';
    return s;
}
}  // namespace

extern "C" {

deinsum_status deinsum_cpals_create(int order, const int64_t *dims, int rank, deinsum_prec prec,
                                    deinsum_cpals_t *out) {
    if (!out || !dims || order < 2 || order > DEINSUM_MAX_ORDER) return DEINSUM_ERR_INVALID;
    *out = nullptr;
    if (rank < 1 || rank > kMaxR) return DEINSUM_ERR_SHAPE;
    if (prec != DEINSUM_PREC_PLAIN && prec != DEINSUM_PREC_SPLIT_BF16) return DEINSUM_ERR_DTYPE;
    deinsum_cpals_s *h = new (std::nothrow) deinsum_cpals_s();
    if (!h) return DEINSUM_ERR_OOM;
    h->order = order;
    h->R = rank;
    h->prec = prec;
    for (int m = 0; m < order; ++m) {
        if (dims[m] < 1) { delete h; return DEINSUM_ERR_SHAPE; }
        h->dims[m] = dims[m];
    }
    h->tree_ok = tree_eligible(order, dims, rank, prec);
    for (int n = 0; n < order; ++n) {
        std::vector<int64_t> ext(dims, dims + order);
        ext.push_back(rank);
        deinsum_status st = deinsum_plan(mttkrp_spec(order, n).c_str(), ext.data(), order + 1, DEINSUM_F32, prec,
                                         &h->plans[n]);
        if (st != DEINSUM_OK) {
            deinsum_cpals_destroy(h);
            return st;
        }
    }
    *out = h;
    return DEINSUM_OK;
}

deinsum_status deinsum_cpals_run(deinsum_cpals_t h, const float *X, float *const *factors, double *lambda,
                                 int sweeps, double *fits, deinsum_stream_t stream) {
    if (!h || !X || !factors || !lambda || !fits || sweeps < 1) return DEINSUM_ERR_INVALID;
    for (int m = 0; m < h->order; ++m)
        if (!factors[m]) return DEINSUM_ERR_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return DEINSUM_ERR_CUDA;
    const int R = h->R;
    if (!h->ws) {
        void *p = nullptr;
        cudaError_t e = counted_malloc(&p, cpals_own_bytes(h));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? DEINSUM_ERR_OOM : DEINSUM_ERR_CUDA;
        }
        cpals_attach_own(h, static_cast<char *>(p), true, dev);
    } else if (dev != h->device) {
        return DEINSUM_ERR_INVALID;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaFuncSetAttribute(inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kInvSmem)) !=
        cudaSuccess)
        return DEINSUM_ERR_CUDA;
    int64_t nx = 1;
    for (int m = 0; m < h->order; ++m) nx *= h->dims[m];
    // ||X||^2 and the Grams of the initial factors
    cudaMemsetAsync(h->status, 0, sizeof(int), s);
    sumsq_partial_kernel<<<kSumBlocks, 256, 0, s>>>(X, nx, h->partial);
    sum_kernel<<<1, 256, 0, s>>>(h->partial, kSumBlocks, h->normx2);
    count_launch(2);
    for (int m = 0; m < h->order; ++m) {
        gram_kernel<<<R, 1024, 0, s>>>(factors[m], h->dims[m], R, h->grams + size_t(m) * R * R);
        count_launch();
    }
    if (cudaGetLastError() != cudaSuccess) return DEINSUM_ERR_CUDA;
    std::vector<const void *> ins(size_t(h->order));
    // dimension tree for this X (its tensor map needs 16-byte aligned rows)
    bool tree = h->tree_ok && h->tree_on;
    if (tree && h->tmap_ptr != X) {
        h->tmap_ptr = X;
        h->tmap_ok = encode_ttm_last_map(X, h->dims[0], h->dims[1], h->dims[2], &h->tmap, &h->tmap_box);
    }
    tree = tree && h->tmap_ok;
    TtmcArgs ta;
    MttkrpArgs sa;
    if (tree) {
        std::memset(&ta, 0, sizeof(ta));
        ta.xmap = h->tmap;
        ta.box_bytes = h->tmap_box;
        ttm_last_geometry(3, h->dims[0], h->dims[1], h->dims[2], R, &ta.g);
        ta.Bsplit = h->tb;
        ta.T2 = h->T;
        ta.S = h->dims[0];
        ta.n_kt = int((h->dims[1] + 127) / 128);
        ta.n_kb = ta.g.n_kb;
        ta.R3 = R;
        ta.sg = 1;
        ta.status = h->status;
        std::memset(&sa, 0, sizeof(sa));
        sa.g = ta.g;
    }
    int nsm = 0;
    if (tree && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DEINSUM_ERR_CUDA;
    for (int sw = 0; sw < sweeps; ++sw) {
        for (int n = 0; n < h->order; ++n) {
            if (tree && n == 0) {
                // T = X x_2 U_2 (one stream of X), then M_0 from T
                sa.U[2] = factors[2];
                if (launch_split_inner_factor(sa, h->tb, stream) || launch_ttm_last_tc(ta, nsm, stream))
                    return DEINSUM_ERR_CUDA;
                if (R % 4 == 0 && (reinterpret_cast<uintptr_t>(factors[1]) & 15) == 0)
                    tree_m0_vec_kernel<<<unsigned(h->dims[0]), 256, 0, s>>>(h->T, factors[1], h->M, h->dims[1], R);
                else
                    tree_m0_kernel<<<unsigned(h->dims[0]), 128, 0, s>>>(h->T, factors[1], h->M, h->dims[1], R);
                count_launch();
            } else if (tree && n == 1) {
                float *part = reinterpret_cast<float *>(h->tb + round_up(size_t((h->dims[2] + 63) / 64) * 8192, 1024));
                tree_m1_kernel<<<dim3(unsigned((h->dims[1] + 3) / 4), kTreeSplit), 128, 0, s>>>(
                    h->T, factors[0], part, h->dims[0], h->dims[1], R);
                const int64_t nm = h->dims[1] * R;
                tree_m1_sum<<<unsigned(std::min<int64_t>(1024, (nm + 255) / 256)), 256, 0, s>>>(part, h->M, nm);
                count_launch(2);
            } else {
                ins[0] = X;
                int k = 1;
                for (int m = 0; m < h->order; ++m)
                    if (m != n) ins[size_t(k++)] = factors[m];
                deinsum_status st = deinsum_execute(h->plans[n], ins.data(), h->order, h->M, stream);
                if (st != DEINSUM_OK) return st;
            }
            const int64_t I = h->dims[n];
            inverse_kernel<<<1, 256, kInvSmem, s>>>(h->grams, h->order, n, R, h->W, h->status);
            int blocks = int((I * R + 255) / 256);
            if (blocks > 1024) blocks = 1024;
            apply_kernel<<<blocks, 256, 0, s>>>(h->M, h->W, factors[n], I, R);
            normalize_kernel<<<R, 256, 0, s>>>(factors[n], I, R, lambda);
            gram_kernel<<<R, 1024, 0, s>>>(factors[n], I, R, h->grams + size_t(n) * R * R);
            count_launch(4);
        }
        const int last = h->order - 1;
        // expansion of the residual from quantities the sweep already has; after the last
        // sweep it also decides whether the direct residual is needed (it cancels when small)
        int *need_direct = reinterpret_cast<int *>(h->normx2 + 1);
        fit_kernel<<<1, 256, 0, s>>>(h->M, factors[last], h->dims[last], R, lambda, h->grams, h->order, h->normx2,
                                     fits + sw, sw + 1 < sweeps ? nullptr : need_direct);
        count_launch();
        if (sw + 1 == sweeps) {
            // final fit from the residual itself when the expansion may have cancelled (the
            // flag fit_kernel just set; otherwise both kernels return at once)
            ResidualArgs ra;
            std::memset(&ra, 0, sizeof(ra));
            ra.X = X;
            for (int m = 0; m < h->order; ++m) {
                ra.U[m] = factors[m];
                ra.dims[m] = h->dims[m];
            }
            ra.order = h->order;
            ra.R = R;
            ra.lambda = lambda;
            ra.partial = h->partial;
            ra.need = need_direct;
            residual_kernel<<<kSumBlocks, 256, 0, s>>>(ra);
            fit_from_residual_kernel<<<1, 256, 0, s>>>(h->partial, kSumBlocks, h->normx2, fits + sw, need_direct);
            count_launch(2);
        }
        if (cudaGetLastError() != cudaSuccess) return DEINSUM_ERR_CUDA;
    }
    return DEINSUM_OK;
}

deinsum_status deinsum_cpals_workspace_bytes(deinsum_cpals_t h, size_t *bytes) {
    if (!h || !bytes) return DEINSUM_ERR_INVALID;
    size_t total = cpals_own_bytes(h);
    for (int n = 0; n < h->order; ++n) {
        size_t b = 0;
        deinsum_status st = deinsum_plan_workspace_bytes(h->plans[n], &b);
        if (st != DEINSUM_OK) return st;
        total += round_up(b, 1024);
    }
    *bytes = total;
    return DEINSUM_OK;
}

deinsum_status deinsum_cpals_bind_workspace(deinsum_cpals_t h, void *workspace, size_t bytes,
                                            deinsum_stream_t stream) {
    if (!h || !workspace || h->ws) return DEINSUM_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(workspace) & 1023) return DEINSUM_ERR_ALIGN;
    size_t need = 0;
    deinsum_status st = deinsum_cpals_workspace_bytes(h, &need);
    if (st != DEINSUM_OK) return st;
    if (bytes < need) return DEINSUM_ERR_SHAPE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return DEINSUM_ERR_CUDA;
    char *p = static_cast<char *>(workspace);
    cpals_attach_own(h, p, false, dev);
    size_t off = cpals_own_bytes(h);
    for (int n = 0; n < h->order; ++n) {
        size_t b = 0;
        deinsum_plan_workspace_bytes(h->plans[n], &b);
        st = deinsum_plan_bind_workspace(h->plans[n], p + off, b, stream);
        if (st != DEINSUM_OK) return st;
        off += round_up(b, 1024);
    }
    return DEINSUM_OK;
}

deinsum_status deinsum_cpals_set_dimension_tree(deinsum_cpals_t h, int enable) {
    if (!h) return DEINSUM_ERR_INVALID;
    h->tree_on = enable != 0;
    return DEINSUM_OK;
}

int deinsum_cpals_uses_dimension_tree(deinsum_cpals_t h) { return h && h->tree_ok && h->tree_on ? 1 : 0; }

deinsum_status deinsum_cpals_status(deinsum_cpals_t h) {
    if (!h) return DEINSUM_ERR_INVALID;
    if (!h->status) return DEINSUM_OK;
    int v = 0;
    if (cudaMemcpy(&v, h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DEINSUM_ERR_CUDA;
    deinsum_status plans_st = DEINSUM_OK;
    for (int n = 0; n < h->order; ++n) {
        const deinsum_status st = deinsum_last_device_status(h->plans[n]);
        if (st != DEINSUM_OK && plans_st == DEINSUM_OK) plans_st = st;
    }
    if (plans_st != DEINSUM_OK) return plans_st;
    // bit 0: a bounded wait of the dimension-tree kernel gave up; bit 1: a floored pivot
    if (v & 1) return DEINSUM_ERR_TIMEOUT;
    return v == 0 ? DEINSUM_OK : DEINSUM_ERR_INVALID;
}

void deinsum_cpals_destroy(deinsum_cpals_t h) {
    if (!h) return;
    for (int n = 0; n < DEINSUM_MAX_ORDER; ++n)
        if (h->plans[n]) deinsum_destroy(h->plans[n]);
    if (h->ws && h->ws_owned) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != h->device) cudaSetDevice(h->device);
        cudaFree(h->ws);
        if (cur != h->device && cur >= 0) cudaSetDevice(cur);
    }
    delete h;
}

}  // extern "C"
