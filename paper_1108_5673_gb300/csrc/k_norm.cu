// MC normalisation matrix (the inner bracket of the second term of Eq. 3,
// built once per sample as Sec. 2 says it can be when masses and widths are
// fixed):
//
//   M[a][b] = (1/N_gen) sum_{j in accepted MC} conj(A_a(j)) A_b(j).
//
// Exactness: a product of two floats is exact in double, so every term is
// formed exactly and summed in FP64; the matrix carries ~1e-15 relative
// rounding, far below what the NLL needs (V^H M V ~ N_data).
//
// Layout: a grid of CTAs splits the events; each CTA stages tiles of 32
// events x 2N planes in shared memory and each thread owns a few entries
// (a <= b) of the upper triangle. CTA partials [grid][P][2] are summed in
// block order by a second kernel (deterministic), which also fills the lower
// triangle by Hermitian symmetry.
#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int kNormThreads = 256;
constexpr int kNormTile = 32;
constexpr int kMaxPairsPerThread = (kMaxWaves * (kMaxWaves + 1) / 2 + kNormThreads - 1) / kNormThreads;

__global__ void __launch_bounds__(kNormThreads)
    norm_partial_kernel(const float *__restrict__ planes, int64_t pitch, int64_t n, int N,
                        int64_t chunk, double *__restrict__ partials)
{
    __shared__ float tile[2 * kMaxWaves][kNormTile + 1];
    __shared__ short pa[kMaxWaves * (kMaxWaves + 1) / 2], pb[kMaxWaves * (kMaxWaves + 1) / 2];
    const int P = N * (N + 1) / 2;
    if (threadIdx.x == 0) {
        int p = 0;
        for (int x = 0; x < N; ++x)
            for (int y = x; y < N; ++y, ++p) {
                pa[p] = (short)x;
                pb[p] = (short)y;
            }
    }
    double acc_r[kMaxPairsPerThread], acc_i[kMaxPairsPerThread];
#pragma unroll
    for (int q = 0; q < kMaxPairsPerThread; ++q)
        acc_r[q] = acc_i[q] = 0.0;

    const int64_t begin = (int64_t)blockIdx.x * chunk;
    const int64_t end = (begin + chunk < n) ? begin + chunk : n;
    for (int64_t t0 = begin; t0 < end; t0 += kNormTile) {
        const int cnt = (int)((end - t0) < kNormTile ? (end - t0) : kNormTile);
        __syncthreads();
        for (int idx = threadIdx.x; idx < 2 * N * kNormTile; idx += kNormThreads) {
            const int r = idx / kNormTile, e = idx - r * kNormTile;
            tile[r][e] = (e < cnt) ? planes[r * pitch + t0 + e] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kMaxPairsPerThread; ++q) {
            const int p = threadIdx.x + q * kNormThreads;
            if (p < P) {
                const int x = pa[p], y = pb[p];
                double sr = 0.0, si = 0.0;
                for (int e = 0; e < cnt; ++e) {
                    const double xr = tile[2 * x][e], xi = tile[2 * x + 1][e];
                    const double yr = tile[2 * y][e], yi = tile[2 * y + 1][e];
                    // conj(A_x) A_y = (xr yr + xi yi) + i (xr yi - xi yr)
                    sr = fma(xr, yr, fma(xi, yi, sr));
                    si = fma(xr, yi, fma(-xi, yr, si));
                }
                acc_r[q] += sr;
                acc_i[q] += si;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kMaxPairsPerThread; ++q) {
        const int p = threadIdx.x + q * kNormThreads;
        if (p < P) {
            partials[((size_t)blockIdx.x * P + p) * 2] = acc_r[q];
            partials[((size_t)blockIdx.x * P + p) * 2 + 1] = acc_i[q];
        }
    }
}

__global__ void norm_reduce_kernel(const double *__restrict__ partials, int grid, int N,
                                   double n_gen, double *__restrict__ M)
{
    const int P = N * (N + 1) / 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * P)
        return;
    double s = 0.0;
    for (int b = 0; b < grid; ++b)
        s += partials[(size_t)b * 2 * P + t];
    const int p = t >> 1, comp = t & 1;
    int x = 0, rem = p;
    while (rem >= N - x) {
        rem -= N - x;
        ++x;
    }
    const int y = x + rem;
    const double v = s / n_gen;
    M[2 * (x * N + y) + comp] = v;
    if (x != y)
        M[2 * (y * N + x) + comp] = comp ? -v : v;  // M[y][x] = conj(M[x][y])
    else if (comp)
        M[2 * (x * N + x) + 1] = 0.0;               // the diagonal is real
}

int norm_grid(int num_sms) { return 2 * num_sms; }

}  // namespace

size_t norm_scratch_bytes(int n_waves, int num_sms)
{
    return (size_t)norm_grid(num_sms) * n_waves * (n_waves + 1) * sizeof(double);
}

cudaError_t launch_build_norm(const Planes &mc, double n_gen, double *M, double *scratch,
                              int num_sms, cudaStream_t s)
{
    const int grid = norm_grid(num_sms);
    const int64_t chunk = ((mc.n + grid - 1) / grid + kNormTile - 1) / kNormTile * kNormTile;
    norm_partial_kernel<<<grid, kNormThreads, 0, s>>>(mc.ptr, mc.pitch, mc.n, mc.n_waves, chunk,
                                                       scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const int P2 = mc.n_waves * (mc.n_waves + 1);
    norm_reduce_kernel<<<(P2 + 127) / 128, 128, 0, s>>>(scratch, grid, mc.n_waves, n_gen, M);
    return cudaGetLastError();
}

}  // namespace pwa
