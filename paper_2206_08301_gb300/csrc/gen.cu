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

__global__ void __launch_bounds__(256) gen_cp_f32_kernel(const __grid_constant__ CpArgs a, int64_t n, float *out) {
    const int N = a.order, R = a.rank;
    const int64_t K = a.dims[N - 1];
    const int64_t kq = (K + 3) / 4;
    const int64_t chunks = (n / K) * kq;
    const float *Alast = a.A[N - 1];
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < chunks; c += int64_t(gridDim.x) * blockDim.x) {
        const int64_t row = c / kq;
        const int64_t k0 = (c - row * kq) * 4;
        int64_t idx[DEINSUM_MAX_ORDER];
        int64_t rem = row;
        for (int m = N - 2; m >= 0; --m) {
            idx[m] = rem % a.dims[m];
            rem /= a.dims[m];
        }
        float w[kGenMaxRank];
        #pragma unroll
        for (int s = 0; s < kGenMaxRank; ++s) {
            if (s < R && N > 1) {
                float t = a.A[0][idx[0] * R + s];
                for (int m = 1; m < N - 1; ++m) t = __fmul_rn(t, a.A[m][idx[m] * R + s]);
                w[s] = t;
            }
        }
        for (int q = 0; q < 4; ++q) {
            const int64_t k = k0 + q;
            if (k >= K) break;
            const float *ar = Alast + k * R;
            float acc = 0.f;
            #pragma unroll
            for (int s = 0; s < kGenMaxRank; ++s)
                if (s < R) acc = __fadd_rn(acc, N > 1 ? __fmul_rn(w[s], __ldg(ar + s)) : __ldg(ar + s));
            const int64_t i = row * K + k;
            if (a.sigma != 0.f) {
                const uint64_t r = raw(a.noise_s0, uint64_t(i));
                const uint64_t sum = (r & 0xFFFFull) + ((r >> 16) & 0xFFFFull) + ((r >> 32) & 0xFFFFull) + (r >> 48);
                const float z = __double2float_rn(__dmul_rn(double(int64_t(sum) - (int64_t(1) << 17)), kNoiseScale));
                acc = __fadd_rn(acc, __fmul_rn(a.sigma, z));
            }
            out[i] = acc;
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
    gen_cp_f32_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(a, n, out);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DEINSUM_OK : DEINSUM_ERR_CUDA;
}

}  // extern "C"
