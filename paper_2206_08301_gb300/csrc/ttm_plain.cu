// Plain CUDA-core TTM, the mode-m tensor product of Sec. III-B
//   Y[a, r, b] = sum_i X[a, i, b] U[i, r]      (X viewed as A x I_m x B)
// used one mode at a time for the TTMc chain (the binary decomposition of
// Sec. II-A).  Each TTM runs as a strided product C[m, n] = sum_k A(m,k) B(k,n)
// with m the long dimension (a when B == 1, else b within one a), n = r, on a
// 128 x 32 register-tiled CUDA-core kernel (FP32 or FP64 FMA); FP32 TTMs over a
// middle mode with a trailing extent B >= 64, a multiple of 4, take the
// 256 x 32 kernel with 16-byte loads below.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "internal.h"

namespace deinsum {
namespace {

constexpr int TBM = 128, TBN = 32, TBK = 16, TTHREADS = 256;

struct Strides {
    int64_t M, N, K, batch;
    int64_t sAm, sAk, sAb;
    int64_t sBk, sBn;
    int64_t sCm, sCn, sCb;
};

template <typename T>
__global__ void __launch_bounds__(TTHREADS)
ttm_kernel(const T *__restrict__ A, const T *__restrict__ B, T *__restrict__ C, const Strides s) {
    __shared__ T As[TBK][TBM + 4];
    __shared__ T Bs[TBK][TBN + 4];
    const int64_t mtiles = (s.M + TBM - 1) / TBM;
    const int64_t ntiles = (s.N + TBN - 1) / TBN;
    const int64_t bid = blockIdx.x;
    const int64_t nt = bid % ntiles;
    const int64_t mt = (bid / ntiles) % mtiles;
    const int64_t bt = bid / (ntiles * mtiles);
    const int64_t m0 = mt * TBM, n0 = nt * TBN;
    const T *Ab = A + bt * s.sAb;
    T *Cb = C + bt * s.sCb;
    const int t = threadIdx.x;
    const int tm = t >> 3, tn = t & 7;  // rows tm*4.., cols tn*4..
    T acc[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int64_t k0 = 0; k0 < s.K; k0 += TBK) {
        // A tile: TBM x TBK
        for (int idx = t; idx < TBM * TBK; idx += TTHREADS) {
            int mm, kk;
            if (s.sAk == 1) { kk = idx % TBK; mm = idx / TBK; }
            else { mm = idx % TBM; kk = idx / TBM; }
            const int64_t gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < s.M && gk < s.K) ? Ab[gm * s.sAm + gk * s.sAk] : T(0);
        }
        for (int idx = t; idx < TBK * TBN; idx += TTHREADS) {
            const int nn = idx % TBN, kk = idx / TBN;
            const int64_t gn = n0 + nn, gk = k0 + kk;
            Bs[kk][nn] = (gn < s.N && gk < s.K) ? B[gk * s.sBk + gn * s.sBn] : T(0);
        }
        __syncthreads();
        #pragma unroll
        for (int kk = 0; kk < TBK; ++kk) {
            T a[4], b[4];
            #pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tm * 4 + i];
            #pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tn * 4 + j];
            #pragma unroll
            for (int i = 0; i < 4; ++i)
                #pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            const int64_t gm = m0 + tm * 4 + i, gn = n0 + tn * 4 + j;
            if (gm < s.M && gn < s.N) Cb[gm * s.sCm + gn * s.sCn] = acc[i][j];
        }
}

// FP32 TTM over a middle mode with a contiguous trailing extent B (a multiple of 4, X and Y
// 16-byte aligned): Y[a, r, b] = sum_i X[a, i, b] U[i, r].  A CTA takes one a, 256 b and up to
// 32 r; thread (bg = lane, rg = warp) accumulates b = b0 + 4 bg .. + 3 and b0 + 128 + 4 bg .. + 3
// for RPW ranks r = r0 + RPW rg .. + RPW - 1, RPW = ceil(min(R, 32) / 8) (8 RPW FMA per k and
// thread; the U values are warp broadcasts), so that R = 8, 16 or 24 costs no FMA on
// padding.  Chunks of 16 i are read with 16-byte loads into registers one chunk ahead and
// stored into the other of two shared-memory buffers.
constexpr int SB = 256, SR = 32, SK = 16, STHREADS = 256;

template <int RPW>
__global__ void __launch_bounds__(STHREADS)
ttm_strided_f32_kernel(const float *__restrict__ X, const float *__restrict__ U, float *__restrict__ Y,
                       int64_t I, int64_t B, int64_t R) {
    __shared__ float4 xs[2][SK][SB / 4];
    __shared__ float4 us[2][SK][SR / 4];
    const int64_t nbt = (B + SB - 1) / SB, nrt = (R + SR - 1) / SR;
    const int64_t bid = blockIdx.x;
    const int64_t rt = bid % nrt;
    const int64_t bt = (bid / nrt) % nbt;
    const int64_t a = bid / (nrt * nbt);
    const int64_t b0 = bt * SB, r0 = rt * SR;
    const int t = threadIdx.x, bg = t & 31, rg = t >> 5;
    const float *Xa = X + a * I * B;
    // this thread's loads of a chunk: X rows k = (t >> 6) + 4 q (q < 4), float4 column t & 63;
    // U row k = t >> 3 (t < 128), columns r0 + 4 (t & 7) .. + 3
    const int xc = t & 63, xk = t >> 6;
    const bool xcol_ok = b0 + 4 * xc < B;
    const int uk = t >> 3, uc = t & 7;
    float4 px[4], pu;
    auto fetch = [&](int64_t i0) {
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t i = i0 + xk + 4 * q;
            px[q] = (xcol_ok && i < I) ? *reinterpret_cast<const float4 *>(Xa + i * B + b0 + 4 * xc)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (t < 128) {
            const int64_t i = i0 + uk;
            float e[4];
            #pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t r = r0 + 4 * uc + q;
                e[q] = (i < I && r < R) ? U[i * R + r] : 0.f;
            }
            pu = make_float4(e[0], e[1], e[2], e[3]);
        }
    };
    auto stash = [&](int buf) {
        #pragma unroll
        for (int q = 0; q < 4; ++q) xs[buf][xk + 4 * q][xc] = px[q];
        if (t < 128) us[buf][uk][uc] = pu;
    };
    float acc[RPW][8];
    #pragma unroll
    for (int j = 0; j < RPW; ++j)
        #pragma unroll
        for (int q = 0; q < 8; ++q) acc[j][q] = 0.f;
    fetch(0);
    stash(0);
    __syncthreads();
    int buf = 0;
    for (int64_t i0 = 0; i0 < I; i0 += SK) {
        const bool more = i0 + SK < I;
        if (more) fetch(i0 + SK);
        #pragma unroll
        for (int k = 0; k < SK; ++k) {
            const float4 x0 = xs[buf][k][bg], x1 = xs[buf][k][32 + bg];
            const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            float uv[RPW];
            if constexpr (RPW == 4) {
                const float4 u = us[buf][k][rg];
                uv[0] = u.x; uv[1] = u.y; uv[2] = u.z; uv[3] = u.w;
            } else {
                const float *uk = reinterpret_cast<const float *>(us[buf][k]) + RPW * rg;
                #pragma unroll
                for (int j = 0; j < RPW; ++j) uv[j] = uk[j];
            }
            #pragma unroll
            for (int j = 0; j < RPW; ++j)
                #pragma unroll
                for (int q = 0; q < 8; ++q) acc[j][q] = fmaf(uv[j], xv[q], acc[j][q]);
        }
        if (more) {
            stash(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
    #pragma unroll
    for (int j = 0; j < RPW; ++j) {
        const int64_t r = r0 + RPW * rg + j;
        if (r >= R) continue;
        float *yr = Y + (a * R + r) * B + b0;
        if (b0 + 4 * bg < B)
            *reinterpret_cast<float4 *>(yr + 4 * bg) = make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
        if (b0 + 128 + 4 * bg < B)
            *reinterpret_cast<float4 *>(yr + 128 + 4 * bg) = make_float4(acc[j][4], acc[j][5], acc[j][6], acc[j][7]);
    }
}

// FP32 TTM with R <= 32 over a contiguous trailing extent B (a multiple of 4, X and Y 16-byte
// aligned): each thread owns two consecutive b of one a and all RT >= R ranks (2 RT
// accumulators) and reads its pair X[a, i, b .. b + 1] straight from global memory (a warp
// reads 256 contiguous bytes), RPF rows ahead through a ring of registers; the rows of U come
// from shared memory, 64 at a time, as warp-uniform 16-byte reads (broadcasts).  Every X value
// feeds RT FMAs from registers; four CTAs per SM (at most 128 registers a thread).
constexpr int RTHREADS = 128, RPF = 4, RUROWS = 64;

template <int RT>
__global__ void __launch_bounds__(RTHREADS, 4)
ttm_rows_f32_kernel(const float *__restrict__ X, const float *__restrict__ U, float *__restrict__ Y, int64_t A,
                    int64_t I, int64_t B, int R) {
    __shared__ float4 us[RUROWS][RT / 4];
    const int64_t B2 = B / 2;
    const int64_t gid = int64_t(blockIdx.x) * RTHREADS + threadIdx.x;
    const bool live = gid < A * B2;   // threads past the end still help stage U
    const int64_t a = live ? gid / B2 : 0, b = live ? 2 * (gid - a * B2) : 0;
    const float *xp = X + a * I * B + b;
    auto ldx = [&](int64_t i) {
        return (live && i < I) ? __ldg(reinterpret_cast<const float2 *>(xp + i * B)) : make_float2(0.f, 0.f);
    };
    float acc[RT][2];
    #pragma unroll
    for (int r = 0; r < RT; ++r) acc[r][0] = acc[r][1] = 0.f;
    float2 xq[RPF];
    #pragma unroll
    for (int j = 0; j < RPF; ++j) xq[j] = ldx(j);
    for (int64_t c0 = 0; c0 < I; c0 += RUROWS) {
        __syncthreads();   // the previous chunk of U is no longer read
        for (int e = threadIdx.x; e < RUROWS * RT; e += RTHREADS) {
            const int k = e / RT, r = e - k * RT;
            const int64_t i = c0 + k;
            reinterpret_cast<float *>(us[k])[r] = (i < I && r < R) ? U[i * R + r] : 0.f;
        }
        __syncthreads();
        const int64_t c1 = I - c0 < RUROWS ? I : c0 + RUROWS;
        for (int64_t i0 = c0; i0 < c1; i0 += RPF) {   // RUROWS is a multiple of RPF
            #pragma unroll
            for (int j = 0; j < RPF; ++j) {
                const int64_t i = i0 + j;
                const float2 x = xq[j];
                xq[j] = ldx(i + RPF);
                const float4 *ur = us[i - c0];
                #pragma unroll
                for (int q = 0; q < RT / 4; ++q) {
                    const float4 u = ur[q];
                    acc[4 * q][0] = fmaf(u.x, x.x, acc[4 * q][0]);
                    acc[4 * q][1] = fmaf(u.x, x.y, acc[4 * q][1]);
                    acc[4 * q + 1][0] = fmaf(u.y, x.x, acc[4 * q + 1][0]);
                    acc[4 * q + 1][1] = fmaf(u.y, x.y, acc[4 * q + 1][1]);
                    acc[4 * q + 2][0] = fmaf(u.z, x.x, acc[4 * q + 2][0]);
                    acc[4 * q + 2][1] = fmaf(u.z, x.y, acc[4 * q + 2][1]);
                    acc[4 * q + 3][0] = fmaf(u.w, x.x, acc[4 * q + 3][0]);
                    acc[4 * q + 3][1] = fmaf(u.w, x.y, acc[4 * q + 3][1]);
                }
            }
        }
    }
    if (!live) return;
    float *yp = Y + a * int64_t(R) * B + b;
    #pragma unroll
    for (int r = 0; r < RT; ++r)
        if (r < R) *reinterpret_cast<float2 *>(yp + int64_t(r) * B) = make_float2(acc[r][0], acc[r][1]);
}

template <typename T>
int launch_ttm(const T *X, const T *U, T *Y, int64_t Aext, int64_t Im, int64_t Bext, int64_t Rm, void *stream) {
    if constexpr (sizeof(T) == 4) {
        if (Bext >= 64 && Bext % 4 == 0 && Rm <= 32 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
            (reinterpret_cast<uintptr_t>(Y) & 15) == 0) {
            const int64_t threads = Aext * (Bext / 2);
            const int64_t blocks = (threads + RTHREADS - 1) / RTHREADS;
            if (blocks < 1 || blocks > 0x7FFFFFFFll) return int(cudaErrorInvalidValue);
            const int rt = int((Rm + 7) / 8) * 8;
            auto kern = rt == 8 ? ttm_rows_f32_kernel<8>
                      : rt == 16 ? ttm_rows_f32_kernel<16>
                      : rt == 24 ? ttm_rows_f32_kernel<24> : ttm_rows_f32_kernel<32>;
            kern<<<unsigned(blocks), RTHREADS, 0, static_cast<cudaStream_t>(stream)>>>(
                reinterpret_cast<const float *>(X), reinterpret_cast<const float *>(U), reinterpret_cast<float *>(Y),
                Aext, Im, Bext, int(Rm));
            count_launch();
            return int(cudaGetLastError());
        }
        if (Bext >= 64 && Bext % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
            (reinterpret_cast<uintptr_t>(Y) & 15) == 0) {
            const int64_t blocks = Aext * ((Bext + SB - 1) / SB) * ((Rm + SR - 1) / SR);
            if (blocks < 1 || blocks > 0x7FFFFFFFll) return int(cudaErrorInvalidValue);
            const int64_t rw = ((Rm < SR ? Rm : SR) + 7) / 8;   // ranks per warp
            auto kern = rw == 1 ? ttm_strided_f32_kernel<1>
                      : rw == 2 ? ttm_strided_f32_kernel<2>
                      : rw == 3 ? ttm_strided_f32_kernel<3> : ttm_strided_f32_kernel<4>;
            kern<<<unsigned(blocks), STHREADS, 0, static_cast<cudaStream_t>(stream)>>>(
                reinterpret_cast<const float *>(X), reinterpret_cast<const float *>(U), reinterpret_cast<float *>(Y),
                Im, Bext, Rm);
            count_launch();
            return int(cudaGetLastError());
        }
    }
    Strides s{};
    if (Bext == 1) {
        s.M = Aext; s.N = Rm; s.K = Im; s.batch = 1;
        s.sAm = Im; s.sAk = 1; s.sAb = 0;
        s.sBk = Rm; s.sBn = 1;
        s.sCm = Rm; s.sCn = 1; s.sCb = 0;
    } else {
        // per a: C'[b, r] = sum_i X[a, i, b] U[i, r], written to Y[a, r, b]
        s.M = Bext; s.N = Rm; s.K = Im; s.batch = Aext;
        s.sAm = 1; s.sAk = Bext; s.sAb = Im * Bext;
        s.sBk = Rm; s.sBn = 1;
        s.sCm = 1; s.sCn = Bext; s.sCb = Rm * Bext;
    }
    const int64_t blocks = s.batch * ((s.M + TBM - 1) / TBM) * ((s.N + TBN - 1) / TBN);
    if (blocks < 1 || blocks > 0x7FFFFFFFll) return int(cudaErrorInvalidValue);
    ttm_kernel<T><<<unsigned(blocks), TTHREADS, 0, static_cast<cudaStream_t>(stream)>>>(X, U, Y, s);
    count_launch();
    return int(cudaGetLastError());
}

}  // namespace

int launch_ttm_plain_f32(const float *X, const float *U, float *Y, int64_t A, int64_t Im, int64_t B, int64_t Rm,
                         void *stream) {
    return launch_ttm<float>(X, U, Y, A, Im, B, Rm, stream);
}
int launch_ttm_plain_f64(const double *X, const double *U, double *Y, int64_t A, int64_t Im, int64_t B,
                         int64_t Rm, void *stream) {
    return launch_ttm<double>(X, U, Y, A, Im, B, Rm, stream);
}

}  // namespace deinsum
