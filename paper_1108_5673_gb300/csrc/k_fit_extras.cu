// What the paper's fitter takes besides the NLL and its gradient (Sec. 4, 5:
// FUMILI needs the gradient and an approximation of the Hessian; plots of the
// fit weight the accepted MC events with the fitted intensity).
//
// FUMILI's approximation of the NLL Hessian in the real parameters
// p = (Re V_0..Re V_{N-1}, Im V_0..): the second derivatives of the intensity
// are dropped in both terms of Eq. 3 (they cancel in expectation at the
// minimum), leaving
//   H = sum_i d_i d_i^T,   d_i = grad_p ln I_i = 2 (Re, Im) of conj(A_a(i)) S_i / I_i.
// Each thread forms d_i of one event (S by a compensated dot product with V
// as a float pair) into a shared-memory tile J of 256 events x 2NP columns
// (Re parts at 0..NP-1, Im parts at NP..2NP-1, zero-padded). The upper
// triangle of J^T J is cut into 4x4 blocks; each thread owns one to three
// (block, event group) items and accumulates 16 products per pair of float4
// loads. FP32 within a run of tiles, float-float across runs, FP64 across
// event groups and blocks, summed in a fixed order. This kernel serves
// samples of more than 20 waves (and PWA_HESS_KERNEL=generic); up to 20
// waves the tensor-core kernel of k_hess_tc.cu forms the same sum.
//
// Projection weights: w_j = I(Omega_j) / N_gen per accepted MC event (their
// sum is V^H M V), and fit fractions F_ab = Re(conj(V_a) M_ab V_b) / V^H M V.
#include "amp_kernel.cuh"
#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int kHT = 256;     // events per tile = threads per block
constexpr int kFlush = 8;    // tiles summed in FP32 before the float-float add

// Amplitudes of event i into ar, ai (zero for padded waves a >= N). Every
// load is unconditional (a padded wave re-reads wave 0, then is zeroed by a
// select) so that all 2NP loads are in flight together.
template <int NP>
__device__ __forceinline__ void load_event(const float *__restrict__ pl, int64_t pitch, int64_t i,
                                           int N, float *ar, float *ai)
{
#pragma unroll
    for (int w = 0; w < NP; ++w) {
        const int64_t o = (w < N ? 2 * w : 0) * pitch + i;
        const float x = __ldg(pl + o), y = __ldg(pl + o + pitch);
        ar[w] = w < N ? x : 0.f;
        ai[w] = w < N ? y : 0.f;
    }
}

// S = sum_a V_a A_a in FP32, in four independent FMA chains (waves a = c mod 4
// in chain c) joined pairwise. |S - S_exact| <= gamma_{N/4+3} sum_a |V_a A_a|
// per component, V rounded to float. Padded waves have A = 0 and V = 0.
template <int NP>
__device__ __forceinline__ void dot4(const float *ar, const float *ai, const float *vf, float &sr,
                                     float &si)
{
    float r[4] = {0.f, 0.f, 0.f, 0.f}, m[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int w = 0; w < NP; ++w) {
        const float x = ar[w], y = ai[w], vr = vf[2 * w], vi = vf[2 * w + 1];
        r[w & 3] = fmaf(x, vr, fmaf(-y, vi, r[w & 3]));
        m[w & 3] = fmaf(x, vi, fmaf(y, vr, m[w & 3]));
    }
    sr = (r[0] + r[1]) + (r[2] + r[3]);
    si = (m[0] + m[1]) + (m[2] + m[3]);
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// a + p into the pair (s, c): s the rounded sum, c collecting the TwoSum error
// and the product's rounding error pe.
__device__ __forceinline__ void acc2(float &s, float &c, float p, float pe)
{
    float t, te;
    two_sum(s, p, t, te);
    s = t;
    c += te + pe;
}

// S = sum_a (Vh + Vl)_a A_a, compensated (Dot2 of Ogita, Rump and Oishi: each
// product split exactly by FMA, TwoSum of the high parts) in four chains
// (waves a = c mod 4) joined by TwoSum; the Vl terms in plain FMA. The result
// is within about 2^-24 |S| + N^2 2^-48 sum_a |V_a A_a| of the exact sum.
template <int NP>
__device__ __forceinline__ void dot2x4(const float *ar, const float *ai, const float *vh,
                                       const float *vl, float &sr, float &si)
{
    float s0[4] = {0.f, 0.f, 0.f, 0.f}, c0[4] = {0.f, 0.f, 0.f, 0.f};
    float s1[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
    float l0 = 0.f, l1 = 0.f;
#pragma unroll
    for (int w = 0; w < NP; ++w) {
        const int j = w & 3;
        const float x = ar[w], y = ai[w], vr = vh[2 * w], vi = vh[2 * w + 1];
        float p;
        p = x * vr; acc2(s0[j], c0[j], p, fmaf(x, vr, -p));     // Re S += x vr - y vi
        p = -y * vi; acc2(s0[j], c0[j], p, fmaf(-y, vi, -p));
        p = x * vi; acc2(s1[j], c1[j], p, fmaf(x, vi, -p));     // Im S += x vi + y vr
        p = y * vr; acc2(s1[j], c1[j], p, fmaf(y, vr, -p));
        l0 = fmaf(x, vl[2 * w], fmaf(-y, vl[2 * w + 1], l0));
        l1 = fmaf(x, vl[2 * w + 1], fmaf(y, vl[2 * w], l1));
    }
#pragma unroll
    for (int j = 1; j < 4; ++j) {
        acc2(s0[0], c0[0], s0[j], c0[j]);
        acc2(s1[0], c1[0], s1[j], c1[j]);
    }
    sr = s0[0] + (c0[0] + l0);
    si = s1[0] + (c1[0] + l1);
}

__device__ __forceinline__ void load_v2(const double *V, int N, int np2, float *vh, float *vl)
{
    for (int c = threadIdx.x; c < np2; c += blockDim.x) {
        const double v = c < 2 * N ? V[c] : 0.0;
        vh[c] = __double2float_rn(v);
        vl[c] = __double2float_rn(v - (double)vh[c]);
    }
}

__device__ __forceinline__ void load_v(const double *V, int N, int np2, float *vf)
{
    for (int c = threadIdx.x; c < np2; c += blockDim.x)
        vf[c] = c < 2 * N ? __double2float_rn(V[c]) : 0.f;
}

// Work split of the Hessian kernel for NP padded waves.
template <int NP>
struct HessCfg {
    static constexpr int PP = 2 * NP;            // padded parameters
    static constexpr int B = PP / 4;             // 4-column blocks
    static constexpr int NB = B * (B + 1) / 2;   // upper-triangle 4x4 blocks
    // events handled by the busiest thread per tile with `it` items per thread,
    // plus `it` for the per-item overhead
    static constexpr int cost(int it)
    {
        return (it * kHT / NB) < 1 ? (1 << 20)
                                   : it * ((kHT + it * kHT / NB - 1) / (it * kHT / NB)) + it;
    }
    static constexpr int IT = (cost(1) <= cost(2) && cost(1) <= cost(3)) ? 1
                              : (cost(2) <= cost(3))                     ? 2
                                                                         : 3;
    static constexpr int EG0 = IT * kHT / NB;
    static constexpr int EG = EG0 > kHT ? kHT : EG0;  // event groups
    static constexpr int NI = NB * EG;                 // items
    static constexpr size_t SMEM = (size_t)kHT * PP * sizeof(float);
    static_assert(NI <= IT * kHT, "items exceed the threads' slots");
    static_assert((size_t)NB * 16 * sizeof(double) <= SMEM, "reduction does not fit the tile");
};

template <int NP>
__global__ void __launch_bounds__(kHT, 1)
    hess_kernel(const float *__restrict__ pl, int64_t pitch, int64_t n, int N, const double *V,
                double *partials, int *status)
{
    using C = HessCfg<NP>;
    extern __shared__ __align__(16) float J[];   // [kHT][PP]
    __shared__ float vh[2 * NP], vl[2 * NP];
    __shared__ int s_bad;
    float4 *J4 = reinterpret_cast<float4 *>(J);
    load_v2(V, N, 2 * NP, vh, vl);
    if (threadIdx.x == 0)
        s_bad = 0;

    int bx[C::IT], by[C::IT], grp[C::IT];
    bool live[C::IT];
#pragma unroll
    for (int k = 0; k < C::IT; ++k) {
        const int t = threadIdx.x + k * kHT;
        live[k] = t < C::NI;
        int blk = t % C::NB, x = 0;
        grp[k] = t / C::NB;
        while (blk >= C::B - x) {
            blk -= C::B - x;
            ++x;
        }
        bx[k] = x;
        by[k] = x + blk;
    }
    float s[C::IT][16];
    dfloat acc[C::IT][16];
#pragma unroll
    for (int k = 0; k < C::IT; ++k)
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            s[k][q] = 0.f;
            acc[k][q] = dfloat{0.f, 0.f};
        }
    __syncthreads();

    const int64_t n_tiles = (n + kHT - 1) / kHT;
    int bad = 0, run = 0;
    // this thread's event of the next tile, loaded while the current tile's
    // products run (events past n read event n - 1 and are dropped)
    float xr[NP], xi[NP];
    if (blockIdx.x < n_tiles)
        load_event<NP>(pl, pitch, min(blockIdx.x * (int64_t)kHT + threadIdx.x, n - 1), N, xr, xi);
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t i = tile * kHT + threadIdx.x;
        const int64_t left = n - tile * kHT;
        const int rows = left < kHT ? (int)left : kHT;
        {
            float rr = 0.f, ri = 0.f;
            if (i < n) {
                float sr, si;
                dot2x4<NP>(xr, xi, vh, vl, sr, si);
                const float I = fmaf(sr, sr, si * si);
                if (I > 0.f && I < INFINITY) {
                    rr = 2.f * sr / I;
                    ri = 2.f * si / I;
                } else {
                    bad = 1;
                }
            }
            // 2 Re(conj(A) S) / I and 2 Im(conj(A) S) / I (zero rows past n)
#pragma unroll
            for (int q = 0; q < NP / 4; ++q) {
                float4 re, im;
                re.x = fmaf(xr[4 * q], rr, xi[4 * q] * ri);
                re.y = fmaf(xr[4 * q + 1], rr, xi[4 * q + 1] * ri);
                re.z = fmaf(xr[4 * q + 2], rr, xi[4 * q + 2] * ri);
                re.w = fmaf(xr[4 * q + 3], rr, xi[4 * q + 3] * ri);
                im.x = fmaf(xr[4 * q], ri, -xi[4 * q] * rr);
                im.y = fmaf(xr[4 * q + 1], ri, -xi[4 * q + 1] * rr);
                im.z = fmaf(xr[4 * q + 2], ri, -xi[4 * q + 2] * rr);
                im.w = fmaf(xr[4 * q + 3], ri, -xi[4 * q + 3] * rr);
                J4[threadIdx.x * C::B + q] = re;
                J4[threadIdx.x * C::B + NP / 4 + q] = im;
            }
        }
        const int64_t next = tile + gridDim.x;
        if (next < n_tiles)
            load_event<NP>(pl, pitch, min(next * kHT + threadIdx.x, n - 1), N, xr, xi);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < C::IT; ++k) {
            if (!live[k])
                continue;
            const float4 *ja = J4 + bx[k], *jb = J4 + by[k];
#pragma unroll 2
            for (int e = grp[k]; e < rows; e += C::EG) {
                const float4 a = ja[e * C::B], b = jb[e * C::B];
                const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        s[k][4 * r + c] = fmaf(av[r], bv[c], s[k][4 * r + c]);
            }
        }
        if (++run == kFlush) {
            run = 0;
#pragma unroll
            for (int k = 0; k < C::IT; ++k)
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    acc[k][q] = df_add(acc[k][q], dfloat{s[k][q], 0.f});
                    s[k][q] = 0.f;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < C::IT; ++k)
#pragma unroll
        for (int q = 0; q < 16; ++q)
            acc[k][q] = df_add(acc[k][q], dfloat{s[k][q], 0.f});
    if (bad)
        s_bad = 1;

    // event groups -> one 4x4 block each, in group order (the tile is free now)
    double *red = reinterpret_cast<double *>(J);
    for (int q = threadIdx.x; q < C::NB * 16; q += kHT)
        red[q] = 0.0;
    for (int g = 0; g < C::EG; ++g) {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < C::IT; ++k) {
            if (live[k] && grp[k] == g) {
                const int blk = (threadIdx.x + k * kHT) % C::NB;
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    red[blk * 16 + q] += (double)acc[k][q].hi + (double)acc[k][q].lo;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_bad)
        atomicOr(status, FLAG_DOMAIN);
    double *out = partials + (size_t)blockIdx.x * C::NB * 16;
    for (int q = threadIdx.x; q < C::NB * 16; q += kHT)
        out[q] = red[q];
}

// H[r][c] over the real parameters (Re V at 0..N-1, Im V at N..2N-1): the sum
// of the block partials, one warp per entry (lane k adds blocks k, k + 32, ...
// in order, then a fixed shuffle tree), so the order is the same on every
// run; zero when a data intensity was not positive. With async_or set, the
// status bits of the call are also OR-ed into *async_or.
__global__ void hess_finalize(const double *partials, int grid, int NP, int N, const int *status,
                              double *H, int *async_or)
{
    if (async_or && blockIdx.x == 0 && threadIdx.x == 0 && *status)
        atomicOr(async_or, *status);
    const int B = NP / 2, NB = B * (B + 1) / 2, P = 2 * N;
    const int o = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (o >= P * P)
        return;
    const int r = o / P, c = o % P;
    const int pr = r < N ? r : NP + (r - N), pc = c < N ? c : NP + (c - N);
    int x = pr >> 2, y = pc >> 2, ii = pr & 3, jj = pc & 3;
    if (x > y) {
        const int t = x; x = y; y = t;
        const int u = ii; ii = jj; jj = u;
    }
    const int blk = x * B - x * (x - 1) / 2 + (y - x);
    const size_t stride = (size_t)NB * 16, at = (size_t)blk * 16 + ii * 4 + jj;
    double v = 0.0;
    for (int b = lane; b < grid; b += 32)
        v += partials[b * stride + at];
    v = warp_sum(v);
    if (lane == 0)
        H[o] = (*status & FLAG_DOMAIN) ? 0.0 : v;
}

// Blocks per SM the weights kernel is compiled for (the register cap that
// gave no spills per size).
constexpr int weights_min_blocks(int np) { return np == 16 ? 2 : np <= 24 ? 3 : 1; }

// One event per thread and iteration; its 2N loads are issued together (an L1
// prefetch of the next iteration's lines, as in the likelihood kernels, made
// this kernel slower: 190 -> 242 us at 5M events, three CTAs per SM).
template <int NP>
__global__ void __launch_bounds__(256, weights_min_blocks(NP))
    mc_weights_kernel(const float *__restrict__ pl, int64_t pitch, int64_t n, int N,
                      const double *V, float inv_ngen, float *__restrict__ w)
{
    __shared__ float vf[2 * NP];
    load_v(V, N, 2 * NP, vf);
    __syncthreads();
#pragma unroll 1
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float ar[NP], ai[NP], sr, si;
        load_event<NP>(pl, pitch, i, N, ar, ai);
        dot4<NP>(ar, ai, vf, sr, si);
        w[i] = fmaf(sr, sr, si * si) * inv_ngen;
    }
}

// F[a][b] = Re(conj(V_a) M_ab V_b) / V^H M V; the denominator is the sum of
// the numerators (M is Hermitian), summed in a fixed order.
__global__ void fit_fractions_kernel(const double *M, const double *V, int N, double *F)
{
    __shared__ double part[256];
    double mine = 0.0;
    for (int o = threadIdx.x; o < N * N; o += blockDim.x) {
        const int a = o / N, b = o % N;
        const double mr = M[2 * o], mi = M[2 * o + 1];
        const double pr = mr * V[2 * b] - mi * V[2 * b + 1], pi = mr * V[2 * b + 1] + mi * V[2 * b];
        const double num = V[2 * a] * pr + V[2 * a + 1] * pi;
        F[o] = num;
        mine += num;
    }
    part[threadIdx.x] = mine;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    const double nv = part[0];
    for (int o = threadIdx.x; o < N * N; o += blockDim.x)
        F[o] /= nv;
}

template <int NP>
cudaError_t hess_np(const Planes &d, const double *V, double *part, int grid, int *status,
                    double *H, int *async_or, cudaStream_t s)
{
    using C = HessCfg<NP>;
    cudaError_t e = cudaFuncSetAttribute(hess_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM);
    if (e != cudaSuccess)
        return e;
    hess_kernel<NP><<<grid, kHT, C::SMEM, s>>>(d.ptr, d.pitch, d.n, d.n_waves, V, part, status);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    const int P = 2 * d.n_waves;
    hess_finalize<<<(P * P + 7) / 8, 256, 0, s>>>(part, grid, NP, d.n_waves, status, H, async_or);
    return cudaGetLastError();
}

template <int NP>
cudaError_t weights_np(const Planes &mc, const double *V, float inv_ngen, float *w, int grid,
                       cudaStream_t s)
{
    mc_weights_kernel<NP><<<grid, 256, 0, s>>>(mc.ptr, mc.pitch, mc.n, mc.n_waves, V, inv_ngen, w);
    return cudaGetLastError();
}

int pad_np(int n)
{
    for (int p : {4, 8, 12, 16, 20, 24, 32, 40, 48})
        if (n <= p)
            return p;
    return -1;
}

}  // namespace

size_t hess_partials_doubles(int n_waves, int grid)
{
    const int B = pad_np(n_waves) / 2;
    return (size_t)grid * (B * (B + 1) / 2) * 16;
}

cudaError_t launch_hessian(const Planes &d, const double *V, double *partials, int grid, int *status,
                           double *H, int *async_or, cudaStream_t s)
{
    switch (pad_np(d.n_waves)) {
    case 4: return hess_np<4>(d, V, partials, grid, status, H, async_or, s);
    case 8: return hess_np<8>(d, V, partials, grid, status, H, async_or, s);
    case 12: return hess_np<12>(d, V, partials, grid, status, H, async_or, s);
    case 16: return hess_np<16>(d, V, partials, grid, status, H, async_or, s);
    case 20: return hess_np<20>(d, V, partials, grid, status, H, async_or, s);
    case 24: return hess_np<24>(d, V, partials, grid, status, H, async_or, s);
    case 32: return hess_np<32>(d, V, partials, grid, status, H, async_or, s);
    case 40: return hess_np<40>(d, V, partials, grid, status, H, async_or, s);
    case 48: return hess_np<48>(d, V, partials, grid, status, H, async_or, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_mc_weights(const Planes &mc, const double *V, double n_gen, float *w, int grid,
                              cudaStream_t s)
{
    const float ig = (float)(1.0 / n_gen);
    switch (pad_np(mc.n_waves)) {
    case 4: return weights_np<4>(mc, V, ig, w, grid, s);
    case 8: return weights_np<8>(mc, V, ig, w, grid, s);
    case 12: return weights_np<12>(mc, V, ig, w, grid, s);
    case 16: return weights_np<16>(mc, V, ig, w, grid, s);
    case 20: return weights_np<20>(mc, V, ig, w, grid, s);
    case 24: return weights_np<24>(mc, V, ig, w, grid, s);
    case 32: return weights_np<32>(mc, V, ig, w, grid, s);
    case 40: return weights_np<40>(mc, V, ig, w, grid, s);
    case 48: return weights_np<48>(mc, V, ig, w, grid, s);
    }
    return cudaErrorInvalidValue;
}

namespace {
__global__ void or_flags_kernel(const int *src, int *dst)
{
    if (*src)
        atomicOr(dst, *src);
}
}  // namespace

cudaError_t launch_or_flags(const int *src, int *dst, cudaStream_t s)
{
    or_flags_kernel<<<1, 1, 0, s>>>(src, dst);
    return cudaGetLastError();
}

namespace {
template <int N>
cudaError_t weights_tma_n(const CUtensorMap *map, const EvalArgs &a, int grid, cudaStream_t s)
{
    using C = AmpCfg<N, 2>;
    cudaError_t e = cudaFuncSetAttribute(nll_amp_kernel<N, 2, 1, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess)
        return e;
    const int n_tiles = (int)((a.n_events + C::TE - 1) / C::TE);
    nll_amp_kernel<N, 2, 1, true><<<grid, C::THREADS, C::SMEM, s>>>(*map, a, n_tiles, nullptr);
    return cudaGetLastError();
}
}  // namespace

// Projection weights through the TMA-fed direct-form kernel (its weights
// mode): map over the MC planes as for the data (the same box: 256 events,
// 192 from 40 waves on, x 2n rows), amax over the MC sample; S by the exact
// product split.
cudaError_t launch_mc_weights_tma(const CUtensorMap *map, const Planes &mc, const double *V,
                                  const float *amax, double n_gen, float *w, int *status, int grid,
                                  cudaStream_t s)
{
    EvalArgs a{};
    a.n_waves = mc.n_waves;
    a.n_events = mc.n;
    a.V = V;
    a.amax = amax;
    a.status = status;
    a.weights = w;
    a.inv_ngen = (float)(1.0 / n_gen);
    switch (pad_np(mc.n_waves)) {
    case 4: return weights_tma_n<4>(map, a, grid, s);
    case 8: return weights_tma_n<8>(map, a, grid, s);
    case 12: return weights_tma_n<12>(map, a, grid, s);
    case 16: return weights_tma_n<16>(map, a, grid, s);
    case 20: return weights_tma_n<20>(map, a, grid, s);
    case 24: return weights_tma_n<24>(map, a, grid, s);
    case 32: return weights_tma_n<32>(map, a, grid, s);
    case 40: return weights_tma_n<40>(map, a, grid, s);
    case 48: return weights_tma_n<48>(map, a, grid, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fit_fractions(const double *M, const double *V, int N, double *F, cudaStream_t s)
{
    fit_fractions_kernel<<<1, 256, 0, s>>>(M, V, N, F);
    return cudaGetLastError();
}

}  // namespace pwa
