// Loading the sample into the device store (Sec. 2: amplitudes are computed
// once per event and kept; Sec. 5, Table 1: "Start-up" and "Lookup table
// creation").
//
//  pack:  event-major interleaved complex [n][N] (float or double pairs) ->
//         structure-of-arrays planes, plane 2a = Re A_a, plane 2a+1 = Im A_a,
//         events contiguous. Doubles are rounded to nearest float.
//  table: planes -> per-event Hermitian table of Sec. 2, coefficient-major
//         t[p][i]: p < N holds |A_a|^2, then for each pair a < b in
//         row-major order two planes Re(A_a conj A_b), Im(A_a conj A_b).
#include <cuda_bf16.h>

#include <algorithm>

#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int kPackEvents = 64;

template <typename T2>
__global__ void pack_kernel(const T2 *__restrict__ src, int64_t n, int N, float *__restrict__ planes,
                            int64_t pitch)
{
    extern __shared__ float sm[];  // [2N][kPackEvents + 1]
    constexpr int LD = kPackEvents + 1;
    const int64_t e0 = (int64_t)blockIdx.x * kPackEvents;
    const int cnt = (int)((n - e0) < kPackEvents ? (n - e0) : kPackEvents);
    const T2 *in = src + e0 * N;
    for (int idx = threadIdx.x; idx < cnt * N; idx += blockDim.x) {
        const int e = idx / N, w = idx - e * N;
        const T2 v = in[idx];
        sm[(2 * w) * LD + e] = (float)v.x;   // round-to-nearest for doubles
        sm[(2 * w + 1) * LD + e] = (float)v.y;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 2 * N * kPackEvents; idx += blockDim.x) {
        const int r = idx / kPackEvents, e = idx - r * kPackEvents;
        if (e < cnt)
            planes[r * pitch + e0 + e] = sm[r * LD + e];
    }
}

// Each entry is the float nearest to its exact value: the products of two
// floats are exact in double and each entry adds two of them, so the double
// result carries one rounding and the final rounding to float is the only
// one that matters. (One-time work; FP64 is acceptable here.)
__global__ void table_kernel(const float *__restrict__ planes, int64_t pitch, int64_t n, int N,
                             float *__restrict__ table, int64_t tpitch)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    for (int w = 0; w < N; ++w) {
        const double ar = planes[(2 * w) * pitch + i], ai = planes[(2 * w + 1) * pitch + i];
        table[w * tpitch + i] = __double2float_rn(ar * ar + ai * ai);
    }
    int p = N;
    for (int x = 0; x < N; ++x) {
        const double xr = planes[(2 * x) * pitch + i], xi = planes[(2 * x + 1) * pitch + i];
        for (int y = x + 1; y < N; ++y) {
            const double yr = planes[(2 * y) * pitch + i], yi = planes[(2 * y + 1) * pitch + i];
            // A_x conj(A_y) = (xr yr + xi yi) + i (xi yr - xr yi)
            table[(int64_t)p * tpitch + i] = __double2float_rn(xr * yr + xi * yi);
            table[(int64_t)(p + 1) * tpitch + i] = __double2float_rn(xi * yr - xr * yi);
            p += 2;
        }
    }
}

// Per-event table of an incoherent sum over L components (planes of L N
// waves, component l of wave a at plane 2 (l N + a)): products of floats are
// exact in double, summed over components in double and rounded once.
__global__ void table_incoh_kernel(const float *__restrict__ planes, int64_t pitch, int64_t n,
                                   int N, int L, float *__restrict__ table, int64_t tpitch)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    auto re = [&](int l, int w) { return (double)planes[(2 * (l * N + w)) * pitch + i]; };
    auto im = [&](int l, int w) { return (double)planes[(2 * (l * N + w) + 1) * pitch + i]; };
    for (int w = 0; w < N; ++w) {
        double d = 0.0;
        for (int l = 0; l < L; ++l)
            d += re(l, w) * re(l, w) + im(l, w) * im(l, w);
        table[w * tpitch + i] = __double2float_rn(d);
    }
    int p = N;
    for (int x = 0; x < N; ++x)
        for (int y = x + 1; y < N; ++y) {
            double tr = 0.0, ti = 0.0;
            for (int l = 0; l < L; ++l) {
                // A_x conj(A_y) = (xr yr + xi yi) + i (xi yr - xr yi)
                tr += re(l, x) * re(l, y) + im(l, x) * im(l, y);
                ti += im(l, x) * re(l, y) - re(l, x) * im(l, y);
            }
            table[(int64_t)p * tpitch + i] = __double2float_rn(tr);
            table[(int64_t)(p + 1) * tpitch + i] = __double2float_rn(ti);
            p += 2;
        }
}

__global__ void amp_max_kernel(const float *__restrict__ planes, int64_t pitch, int64_t n, int N,
                               float *__restrict__ amax)
{
    const int w = blockIdx.y;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(planes[(2 * w) * pitch + i]) + fabsf(planes[(2 * w + 1) * pitch + i]));
    for (int o = 16; o > 0; o >>= 1)
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)  // non-negative floats order like their bit patterns
        atomicMax(reinterpret_cast<int *>(amax + w), __float_as_int(m));
}

__global__ void plane_absmax_kernel(const float *__restrict__ planes, int64_t pitch, int64_t n,
                                    float *__restrict__ out)
{
    const int r = blockIdx.y;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(planes[(int64_t)r * pitch + i]));
    for (int o = 16; o > 0; o >>= 1)
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<int *>(out + r), __float_as_int(m));
}

__global__ void to_float_kernel(const double *__restrict__ src, int64_t n, float *__restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __double2float_rn(src[i]);
}

}  // namespace

cudaError_t launch_to_float(const double *src, int64_t n, float *dst, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    to_float_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(src, n, dst);
    return cudaGetLastError();
}

cudaError_t launch_plane_absmax(const float *planes, int64_t pitch, int64_t n, int rows, float *out,
                                cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)rows);
    plane_absmax_kernel<<<grid, 256, 0, s>>>(planes, pitch, n, out);
    return cudaGetLastError();
}

cudaError_t launch_amp_max(const Planes &amp, float *amax, cudaStream_t s)
{
    if (amp.n <= 0)
        return cudaSuccess;
    dim3 grid((unsigned)std::min<int64_t>((amp.n + 255) / 256, 256), (unsigned)amp.n_waves);
    amp_max_kernel<<<grid, 256, 0, s>>>(amp.ptr, amp.pitch, amp.n, amp.n_waves, amax);
    return cudaGetLastError();
}

cudaError_t launch_pack(const void *src, int dtype, int64_t n, int n_waves, float *planes,
                        int64_t pitch, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    const int64_t blocks = (n + kPackEvents - 1) / kPackEvents;
    const size_t smem = (size_t)2 * n_waves * (kPackEvents + 1) * sizeof(float);
    if (dtype == PWA_C64)
        pack_kernel<float2><<<(unsigned)blocks, 256, smem, s>>>(
            static_cast<const float2 *>(src), n, n_waves, planes, pitch);
    else
        pack_kernel<double2><<<(unsigned)blocks, 256, smem, s>>>(
            static_cast<const double2 *>(src), n, n_waves, planes, pitch);
    return cudaGetLastError();
}

cudaError_t launch_table_build(const Planes &amp, float *table, int64_t table_pitch, cudaStream_t s)
{
    if (amp.n <= 0)
        return cudaSuccess;
    const int64_t blocks = (amp.n + 127) / 128;
    table_kernel<<<(unsigned)blocks, 128, 0, s>>>(amp.ptr, amp.pitch, amp.n, amp.n_waves, table,
                                                   table_pitch);
    return cudaGetLastError();
}

cudaError_t launch_table_build_incoh(const Planes &amp, int n_lambda, float *table,
                                     int64_t table_pitch, cudaStream_t s)
{
    if (amp.n <= 0)
        return cudaSuccess;
    if (n_lambda < 1 || amp.n_waves % n_lambda)
        return cudaErrorInvalidValue;
    const int64_t blocks = (amp.n + 127) / 128;
    table_incoh_kernel<<<(unsigned)blocks, 128, 0, s>>>(amp.ptr, amp.pitch, amp.n,
                                                        amp.n_waves / n_lambda, n_lambda, table,
                                                        table_pitch);
    return cudaGetLastError();
}

}  // namespace pwa
