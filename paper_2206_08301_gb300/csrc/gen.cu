// Seeded synthetic inputs on the device.  Bit-for-bit the counter-based
// definitions of the project's input module: SplitMix64 (S. Vigna's public
// generator; state advances by the golden-ratio increment, each output is the
// 64-bit finaliser of the state) addressed by element index.  No contraction
// arithmetic lives here.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace deinsum {
namespace {

constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ull;
// sqrt(3) * 2^-16, the scale of the four-lane Irwin-Hall noise draw (the same
// float64 value as the input module's NOISE_SCALE)
__device__ constexpr double kNoiseScale = 1.7320508075688772 * 0x1p-16;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t state0(uint64_t seed, uint64_t stream) {
    return mix64(seed + stream * GAMMA);
}

__device__ __forceinline__ uint64_t raw(uint64_t s0, uint64_t i) { return mix64(s0 + (i + 1) * GAMMA); }

__global__ void gen_uniform_f32_kernel(uint64_t s0, int64_t n, float *out) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t u = uint32_t(raw(s0, uint64_t(i)) >> 40);
        out[i] = float(double(u) * 0x1p-23 - 1.0);
    }
}

__global__ void gen_uniform_f64_kernel(uint64_t s0, int64_t n, double *out) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint64_t u = raw(s0, uint64_t(i)) >> 11;
        out[i] = double(u) * 0x1p-52 - 1.0;
    }
}

struct CpArgs {
    int order, rank;
    int64_t dims[DEINSUM_MAX_ORDER];
    const float *A[DEINSUM_MAX_ORDER];
    float sigma;
    uint64_t noise_s0;
};

// X[idx] = sum_s prod_m A_m[i_m, s] + sigma * f32(z(idx)), each float
// operation explicitly rounded (no contraction into FMA), in the order the
// input module states.
// Each thread owns 4 consecutive entries of one row (all modes but the last
// fixed): the row's partial products w[s] = A_0[i_0, s] * ... * A_{N-2}[i_{N-2}, s]
// are formed once (the same left-to-right products the definition forms),
// then every entry multiplies them by the last factor's row and sums over s.
constexpr int kGenMaxRank = 64;

// Tiles of 16 rows x 64 entries of the last mode: blockIdx.x picks the
// 64-wide chunk k, whose last-factor rows are staged once (As[s][k]); the
// block then walks row tiles, forms the rows' partial products into
// ws[s][row], and thread (row group, k) produces 4 rows x 1 entry.
constexpr int kGenRows = 16, kGenK = 64;

__global__ void __launch_bounds__(256) gen_cp_f32_kernel(const __grid_constant__ CpArgs a, int64_t n, float *out) {
    extern __shared__ float gsm[];
    const int N = a.order, R = a.rank;
    float *As = gsm;                       // [R][kGenK]
    float *ws = gsm + R * kGenK;           // [R][kGenRows]
    const int64_t K = a.dims[N - 1];
    const int64_t rows = n / K;
    const int64_t k0 = int64_t(blockIdx.x) * kGenK;
    const float *Alast = a.A[N - 1];
    for (int e = threadIdx.x; e < R * kGenK; e += blockDim.x) {
        const int s = e / kGenK, kk = e % kGenK;
        As[e] = (k0 + kk < K) ? Alast[(k0 + kk) * R + s] : 0.f;
    }
    const int kk = threadIdx.x & (kGenK - 1), rg = threadIdx.x >> 6;   // rows 4 rg .. 4 rg + 3
    const int64_t k = k0 + kk;
    const int64_t rtiles = (rows + kGenRows - 1) / kGenRows;
    for (int64_t rt = blockIdx.y; rt < rtiles; rt += gridDim.y) {
        const int64_t r0 = rt * kGenRows;
        __syncthreads();
        for (int e = threadIdx.x; e < R * kGenRows; e += blockDim.x) {
            const int s = e / kGenRows, rl = e % kGenRows;
            const int64_t row = r0 + rl;
            float t = 1.f;
            if (row < rows && N > 1) {
                int64_t idx[DEINSUM_MAX_ORDER];
                int64_t rem = row;
                for (int m = N - 2; m >= 0; --m) {
                    idx[m] = rem % a.dims[m];
                    rem /= a.dims[m];
                }
                t = a.A[0][idx[0] * R + s];
                for (int m = 1; m < N - 1; ++m) t = __fmul_rn(t, a.A[m][idx[m] * R + s]);
            }
            ws[e] = t;
        }
        __syncthreads();
        if (k >= K) continue;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int s = 0; s < R; ++s) {
            const float4 w4 = *reinterpret_cast<const float4 *>(ws + s * kGenRows + 4 * rg);
            const float av = As[s * kGenK + kk];
            const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
            #pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = __fadd_rn(acc[q], N > 1 ? __fmul_rn(wv[q], av) : av);
        }
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t row = r0 + 4 * rg + q;
            if (row >= rows) break;
            const int64_t i = row * K + k;
            float v = acc[q];
            if (a.sigma != 0.f) {
                const uint64_t r = raw(a.noise_s0, uint64_t(i));
                const uint64_t sum = (r & 0xFFFFull) + ((r >> 16) & 0xFFFFull) + ((r >> 32) & 0xFFFFull) + (r >> 48);
                const float z = __double2float_rn(__dmul_rn(double(int64_t(sum) - (int64_t(1) << 17)), kNoiseScale));
                v = __fadd_rn(v, __fmul_rn(a.sigma, z));
            }
            out[i] = v;
        }
    }
}

unsigned grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return unsigned(b);
}

}  // namespace
}  // namespace deinsum

using namespace deinsum;

extern "C" {

deinsum_status deinsum_gen_uniform_f32(uint64_t seed, uint64_t stream_id, int64_t n, float *out,
                                       deinsum_stream_t stream) {
    if (n < 0 || (n > 0 && !out)) return DEINSUM_ERR_INVALID;
    if (n == 0) return DEINSUM_OK;
    gen_uniform_f32_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(state0(seed, stream_id), n, out);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DEINSUM_OK : DEINSUM_ERR_CUDA;
}

deinsum_status deinsum_gen_uniform_f64(uint64_t seed, uint64_t stream_id, int64_t n, double *out,
                                       deinsum_stream_t stream) {
    if (n < 0 || (n > 0 && !out)) return DEINSUM_ERR_INVALID;
    if (n == 0) return DEINSUM_OK;
    gen_uniform_f64_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(state0(seed, stream_id), n, out);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DEINSUM_OK : DEINSUM_ERR_CUDA;
}

deinsum_status deinsum_gen_cp_f32(uint64_t seed, int order, const int64_t *dims, int rank,
                                  const float *const *factors, double sigma, float *out,
                                  deinsum_stream_t stream) {
    if (order < 1 || order > DEINSUM_MAX_ORDER || rank < 1 || !dims || !factors || !out)
        return DEINSUM_ERR_INVALID;
    if (rank > kGenMaxRank) return DEINSUM_ERR_SHAPE;
    CpArgs a{};
    a.order = order;
    a.rank = rank;
    int64_t n = 1;
    for (int m = 0; m < order; ++m) {
        if (dims[m] < 1 || !factors[m]) return DEINSUM_ERR_INVALID;
        a.dims[m] = dims[m];
        a.A[m] = factors[m];
        n *= dims[m];
    }
    a.sigma = float(sigma);  // rounded to nearest, as the input module does
    a.noise_s0 = state0(seed, 2);  // the noise stream of the input module
    const int64_t K = dims[order - 1];
    const int64_t ktiles = (K + kGenK - 1) / kGenK;
    const int64_t rtiles = (n / K + kGenRows - 1) / kGenRows;
    int64_t gy = (int64_t(152) * 8 + ktiles - 1) / ktiles;
    if (gy > rtiles) gy = rtiles;
    if (gy > 65535) gy = 65535;
    if (gy < 1) gy = 1;
    if (ktiles > 0x7FFFFFFF) return DEINSUM_ERR_SHAPE;
    const size_t smem = size_t(rank) * (kGenK + kGenRows) * sizeof(float);
    gen_cp_f32_kernel<<<dim3(unsigned(ktiles), unsigned(gy)), 256, smem, static_cast<cudaStream_t>(stream)>>>(a, n, out);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DEINSUM_OK : DEINSUM_ERR_CUDA;
}

}  // extern "C"
