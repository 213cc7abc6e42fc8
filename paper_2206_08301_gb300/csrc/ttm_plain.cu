// Plain CUDA-core TTM, the mode-m tensor product of Sec. III-B
//   Y[a, r, b] = sum_i X[a, i, b] U[i, r]      (X viewed as A x I_m x B)
// used one mode at a time for the TTMc chain (the binary decomposition of
// Sec. II-A).  Each TTM runs as a strided product C[m, n] = sum_k A(m,k) B(k,n)
// with m the long dimension (a when B == 1, else b within one a), n = r, on a
// 128 x 32 register-tiled CUDA-core kernel (FP32 or FP64 FMA).
#include <cuda_runtime.h>

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

template <typename T>
int launch_ttm(const T *X, const T *U, T *Y, int64_t Aext, int64_t Im, int64_t Bext, int64_t Rm, void *stream) {
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
