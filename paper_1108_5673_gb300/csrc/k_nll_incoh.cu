// Direct form of Eq. 3 with an incoherent sum over L unobserved components
// (e.g. helicity states): each event carries L amplitude sets A_a^l and
//   I_i = sum_l |S_i^l|^2,  S_i^l = sum_a V_a A_a^l(i),
//   NLL = - sum_i ln I_i + V^H M V,
//   g_a = dNLL/dV*_a = - sum_i sum_l conj(A_a^l(i)) S_i^l / I_i + (M V)_a,
// with M summed over components as well (built from the MC sample viewed as
// L pseudo-events per event). The table form needs no kernel of its own: its
// per-event table is the sum over components of A_a^l conj(A_b^l).
//
// Store: 2 L N float planes, plane 2 (l N + a) = Re A_a^l, the next one Im,
// events contiguous; 8 L N bytes per event.
//
// One event per thread, grid-stride, in two passes over the components: S^l
// of every component first (the loads issued without branches), then the
// gradient, re-reading each component from L1. Each warp prefetches the lines
// of its next iteration into L1 while it computes the current one. S^l by the compensated dot product (Ogita,
// Rump and Oishi, Dot2) with V as a float pair, packed (Re, Im) in FP32x2
// registers, in four independent chains; ln I = e ln 2 + ln f with e summed
// as an integer and ln f in float-float; gradients in FP32 per thread,
// FP64 across warps and blocks. The last block (atomic ticket) adds the
// block partials in block order and the normalisation term in FP64, so the
// results are bitwise reproducible.
#include "amp_kernel.cuh"
#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int kIT = 256;         // threads per block
constexpr int kMaxLambda = 4;

__device__ __forceinline__ f2 splat(float v) { return pk2(v, v); }

__device__ __forceinline__ f2 two_sum2(f2 a, f2 b, f2 &err)
{
    const f2 s = add2(a, b);
    const f2 bb = sub2(s, a);
    err = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
    return s;
}

// Component l of event i: A_a^l for a < NP (padded waves re-read wave 0 and
// are zeroed by a select, so the loads are issued without branches).
template <int NP>
__device__ __forceinline__ void load_component(const float *__restrict__ pl, int64_t pitch,
                                               int64_t i, int N, int l, float *ar, float *ai)
{
#pragma unroll
    for (int w = 0; w < NP; ++w) {
        const int64_t o = (int64_t)(w < N ? 2 * (l * N + w) : 0) * pitch + i;
        const float x = __ldg(pl + o), y = __ldg(pl + o + pitch);
        ar[w] = w < N ? x : 0.f;
        ai[w] = w < N ? y : 0.f;
    }
}

__device__ __forceinline__ void prefetch_l1(const float *p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

struct IncohShared {
    // per wave: (vr, vi), (-vr, -vi), (-vi, vr), (vi, -vr) of the high part; low parts
    f2 va[kMaxWaves], van[kMaxWaves], vb[kMaxWaves], vbn[kMaxWaves], val[kMaxWaves],
        vbl[kMaxWaves];
};

template <int NP, int L>
__global__ void __launch_bounds__(kIT, 1)
    nll_incoh_kernel(const float *__restrict__ pl, int64_t pitch, const EvalArgs a)
{
    __shared__ IncohShared sh;
    __shared__ float red[kIT / 32][4 + 2 * NP];
    __shared__ int s_flags, s_last;
    const int N = a.n_waves;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int w = threadIdx.x; w < NP; w += kIT) {
        float vrh = 0.f, vrl = 0.f, vih = 0.f, vil = 0.f;
        if (w < N) {
            const double dr = a.V[2 * w], di = a.V[2 * w + 1];
            vrh = __double2float_rn(dr);
            vrl = __double2float_rn(dr - (double)vrh);
            vih = __double2float_rn(di);
            vil = __double2float_rn(di - (double)vih);
        }
        sh.va[w] = pk2(vrh, vih);
        sh.van[w] = pk2(-vrh, -vih);
        sh.vb[w] = pk2(-vih, vrh);
        sh.vbn[w] = pk2(vih, -vrh);
        sh.val[w] = pk2(vrl, vil);
        sh.vbl[w] = pk2(-vil, vrl);
    }
    if (threadIdx.x == 0)
        s_flags = 0;
    __syncthreads();

    f2 gv[NP];               // (Re, Im) of - sum conj(A_a^l) S^l / I
#pragma unroll
    for (int w = 0; w < NP; ++w)
        gv[w] = 0ull;
    dfloat acc = {0.f, 0.f};  // sum of ln f
    int eacc = 0;             // sum of exponents
    int bad = 0;
    const int64_t n = a.n_events;
    const int64_t stride = (int64_t)gridDim.x * kIT;
    for (int64_t i = (int64_t)blockIdx.x * kIT + threadIdx.x; i < n; i += stride) {
        // The warp's events of the next iteration fill one 128-byte line per
        // plane: lane k fetches the lines of planes k, k + 32, ... into L1,
        // so the loads of that iteration find them there.
        const int64_t nb = i - lane + stride;
        if (nb < n)
            for (int p = lane; p < 2 * L * N; p += 32)
                prefetch_l1(pl + p * pitch + nb);
        // the component loops are not unrolled (the V coefficients are re-read
        // from shared memory per component instead of held in registers); S^l
        // stays in registers through the selects
        float sr[L], si[L];
        float I = 0.f;
#pragma unroll 1
        for (int l = 0; l < L; ++l) {
            float ar[NP], ai[NP];
            load_component<NP>(pl, pitch, i, N, l, ar, ai);
            // (Sr, Si) += ar (vr, vi) + ai (-vi, vr), compensated, four chains
            f2 s[4] = {0ull, 0ull, 0ull, 0ull}, c[4] = {0ull, 0ull, 0ull, 0ull}, lo = 0ull;
#pragma unroll
            for (int w = 0; w < NP; ++w) {
                const f2 x = splat(ar[w]), y = splat(ai[w]);
                dot2_step(s[w & 3], c[w & 3], x, sh.va[w], sh.van[w]);
                dot2_step(s[w & 3], c[w & 3], y, sh.vb[w], sh.vbn[w]);
                lo = fma2(x, sh.val[w], fma2(y, sh.vbl[w], lo));
            }
            f2 e01, e23, e;
            const f2 s01 = two_sum2(s[0], s[1], e01), s23 = two_sum2(s[2], s[3], e23);
            const f2 st = two_sum2(s01, s23, e);
            const f2 ct = add2(add2(add2(c[0], c[1]), add2(c[2], c[3])), add2(add2(e01, e23), e));
            float xr, xi;
            upk2(add2(st, add2(ct, lo)), xr, xi);
            I = fmaf(xr, xr, fmaf(xi, xi, I));
#pragma unroll
            for (int k = 0; k < L; ++k)
                if (k == l) {
                    sr[k] = xr;
                    si[k] = xi;
                }
        }
        if (I > 0.f && I < INFINITY) {
            int ex;
            const float f = split_exponent(I, ex);
            eacc += ex;
            acc = df_add(acc, dfloat{logf(f), 0.f});
            const float rI = -__frcp_rn(I);
            // second pass over the components: this thread's own loads of a
            // moment ago, served from L1
#pragma unroll 1
            for (int l = 0; l < L; ++l) {
                float xr = sr[0], xi = si[0];
#pragma unroll
                for (int k = 1; k < L; ++k)
                    if (k == l) {
                        xr = sr[k];
                        xi = si[k];
                    }
                float ar[NP], ai[NP];
                load_component<NP>(pl, pitch, i, N, l, ar, ai);
                // conj(A) (wr + i wi) = (ar wr + ai wi) + i (ar wi - ai wr), w = -S / I
                const float wr = rI * xr, wi = rI * xi;
                const f2 W1 = pk2(wr, wi), W2 = pk2(wi, -wr);
#pragma unroll
                for (int w = 0; w < NP; ++w)
                    gv[w] = fma2(splat(ar[w]), W1, fma2(splat(ai[w]), W2, gv[w]));
            }
        } else {
            bad = 1;
        }
    }

    // ---- block reduction (fixed order) -------------------------------------
    const dfloat accw = warp_sum(acc);
    const long long ew = warp_sum((long long)eacc);
    if (lane == 0) {
        red[warp][0] = accw.hi;
        red[warp][1] = accw.lo;
        red[warp][2] = (float)(ew & 0xffffff);   // exact in float
        red[warp][3] = (float)(ew >> 24);
    }
#pragma unroll
    for (int w = 0; w < NP; ++w) {
        float x, y;
        upk2(gv[w], x, y);
        x = warp_sum(x);
        y = warp_sum(y);
        if (lane == 0) {
            red[warp][4 + 2 * w] = x;
            red[warp][5 + 2 * w] = y;
        }
    }
    if (bad)
        atomicOr(&s_flags, FLAG_DOMAIN);
    __syncthreads();
    const int P = 2 + 2 * N;
    double *out = a.partials + (size_t)blockIdx.x * P;
    for (int c = threadIdx.x; c < P; c += kIT) {
        double v = 0.0;
        if (c == 0) {
            for (int w = 0; w < kIT / 32; ++w)
                v += (double)red[w][0] + (double)red[w][1];
        } else if (c == 1) {
            for (int w = 0; w < kIT / 32; ++w)
                v += (double)red[w][2] + 16777216.0 * (double)red[w][3];
        } else {
            for (int w = 0; w < kIT / 32; ++w)
                v += (double)red[w][2 + c];
        }
        out[c] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_flags)
            atomicOr(a.status, s_flags);
        __threadfence();
        const unsigned t = atomicAdd(a.ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last)
        return;

    // ---- last block: block partials in block order, normalisation term -----
    __threadfence();
    __shared__ double fin[2 + 2 * kMaxWaves], mv[2 * kMaxWaves];
    const int nb = gridDim.x;
    for (int c = threadIdx.x; c < P; c += kIT) {
        double v = 0.0;
        for (int b = 0; b < nb; ++b)
            v += __ldcg(a.partials + (size_t)b * P + c);
        fin[c] = v;
    }
    // (M V)_row, one real component per thread
    for (int t = threadIdx.x; t < 2 * N; t += kIT) {
        const int row = t >> 1;
        double v = 0.0;
        for (int b = 0; b < N; ++b) {
            const double mr = a.M[2 * (row * N + b)], mi = a.M[2 * (row * N + b) + 1];
            const double vr = a.V[2 * b], vi = a.V[2 * b + 1];
            v = (t & 1) ? fma(mr, vi, fma(mi, vr, v)) : fma(mr, vr, fma(-mi, vi, v));
        }
        mv[t] = v;
    }
    __syncthreads();
    const bool dom = (*(volatile int *)a.status & FLAG_DOMAIN) != 0;
    if (threadIdx.x == 0) {
        double nv = 0.0;  // Re(V^H (M V))
        for (int row = 0; row < N; ++row)
            nv = fma(a.V[2 * row], mv[2 * row], fma(a.V[2 * row + 1], mv[2 * row + 1], nv));
        const double lnsum = 0.69314718055994530942 * fin[1] + fin[0];
        *a.nll = dom ? INFINITY : -lnsum + nv;
        *a.ticket = 0u;
        if (a.done)
            atomicAdd(a.done, 1);
    }
    if (a.grad)
        for (int c = threadIdx.x; c < 2 * N; c += kIT)
            a.grad[c] = dom ? 0.0 : fin[2 + c] + mv[c];
}

// Register budget: the L x NP amplitudes of an event stay in registers, so
// L * NP <= 48 (e.g. 2 components up to 24 waves, 4 up to 12).
constexpr int kMaxLanes = 48;

template <int NP, int L>
cudaError_t launch_nl(const float *pl, int64_t pitch, const EvalArgs &a, int grid, cudaStream_t s)
{
    if constexpr (NP * L > kMaxLanes) {
        return cudaErrorInvalidValue;
    } else {
        // shared memory is a few KB: leave the rest of the SM's array to L1,
        // which holds the prefetched lines of the next iteration
        cudaFuncSetAttribute(nll_incoh_kernel<NP, L>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             0);
        nll_incoh_kernel<NP, L><<<grid, kIT, 0, s>>>(pl, pitch, a);
        return cudaGetLastError();
    }
}

template <int NP>
cudaError_t launch_np(const float *pl, int64_t pitch, int L, const EvalArgs &a, int grid,
                      cudaStream_t s)
{
    switch (L) {
    case 1: return launch_nl<NP, 1>(pl, pitch, a, grid, s);
    case 2: return launch_nl<NP, 2>(pl, pitch, a, grid, s);
    case 3: return launch_nl<NP, 3>(pl, pitch, a, grid, s);
    case 4: return launch_nl<NP, 4>(pl, pitch, a, grid, s);
    }
    return cudaErrorInvalidValue;
}

int pad_np(int n)
{
    for (int p : {4, 8, 12, 16, 20, 24})
        if (n <= p)
            return p;
    return 1 << 20;
}

// ---- TMA-fed path: the direct-form kernel with L components per event ------
// (amp_kernel.cuh): tiles of 192 events x 2 L n rows streamed by TMA, the
// products split exactly against sigma (bounded over all components) and
// their high parts summed as integers, two events per thread in FP32x2, two
// groups of three consumer warps. It serves N_pad * L <= 48 (stages of
// 2 L N_pad x 192 floats in the 200 KB ring, owned by a group where two or
// more per group fit, shared by both groups otherwise).
template <int N, int L>
cudaError_t launch_tma_nl(const CUtensorMap *map, const EvalArgs &a, int grid, cudaStream_t s)
{
    if constexpr (N * L > kMaxLanes || L < 2) {
        return cudaErrorInvalidValue;
    } else {
        using C = AmpCfg<N, 2, L>;
        static_assert(C::FITS, "one stage per consumer group must fit");
        if (!finalize_fits<N, 2, L>(grid))
            return cudaErrorInvalidConfiguration;
        cudaError_t e = cudaFuncSetAttribute(nll_amp_kernel<N, 2, L>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess)
            return e;
        const int n_tiles = (int)((a.n_events + C::TE - 1) / C::TE);
        int *work_flags = amp_scratch(a.partials, grid).flags;
        nll_amp_kernel<N, 2, L><<<grid, C::THREADS, C::SMEM, s>>>(*map, a, n_tiles, work_flags);
        return cudaGetLastError();
    }
}

template <int N>
cudaError_t launch_tma_n(const CUtensorMap *map, int L, const EvalArgs &a, int grid,
                         cudaStream_t s)
{
    switch (L) {
    case 2: return launch_tma_nl<N, 2>(map, a, grid, s);
    case 3: return launch_tma_nl<N, 3>(map, a, grid, s);
    case 4: return launch_tma_nl<N, 4>(map, a, grid, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

bool incoh_tma_available(int n_waves, int n_lambda)
{
    return n_lambda >= 2 && n_lambda <= kMaxLambda && pad_np(n_waves) * n_lambda <= kMaxLanes;
}

int incoh_tma_box_events() { return AmpCfg<4, 2, 2>::TE; }

cudaError_t launch_nll_incoh_tma(const CUtensorMap *map, int n_lambda, const EvalArgs &a, int grid,
                                 cudaStream_t s)
{
    if (!incoh_tma_available(a.n_waves, n_lambda))
        return cudaErrorInvalidValue;
    switch (pad_np(a.n_waves)) {
    case 4: return launch_tma_n<4>(map, n_lambda, a, grid, s);
    case 8: return launch_tma_n<8>(map, n_lambda, a, grid, s);
    case 12: return launch_tma_n<12>(map, n_lambda, a, grid, s);
    case 16: return launch_tma_n<16>(map, n_lambda, a, grid, s);
    case 20: return launch_tma_n<20>(map, n_lambda, a, grid, s);
    case 24: return launch_tma_n<24>(map, n_lambda, a, grid, s);
    }
    return cudaErrorInvalidValue;
}

int incoh_max_components() { return kMaxLambda; }
int incoh_max_waves(int n_lambda)
{
    int best = 0;
    for (int p : {4, 8, 12, 16, 20, 24})
        if (p * n_lambda <= kMaxLanes)
            best = p;
    return best;
}

size_t incoh_partials_doubles(int n_waves, int grid) { return (size_t)grid * (2 + 2 * n_waves); }

cudaError_t launch_nll_incoh(const Planes &d, int n_lambda, const EvalArgs &a, int grid,
                             cudaStream_t s)
{
    const int N = a.n_waves;
    if (N < 1 || n_lambda < 1 || n_lambda > kMaxLambda || pad_np(N) * n_lambda > kMaxLanes ||
        d.n_waves != N * n_lambda)
        return cudaErrorInvalidValue;
    if (N <= 4)
        return launch_np<4>(d.ptr, d.pitch, n_lambda, a, grid, s);
    if (N <= 8)
        return launch_np<8>(d.ptr, d.pitch, n_lambda, a, grid, s);
    if (N <= 12)
        return launch_np<12>(d.ptr, d.pitch, n_lambda, a, grid, s);
    if (N <= 16)
        return launch_np<16>(d.ptr, d.pitch, n_lambda, a, grid, s);
    if (N <= 20)
        return launch_np<20>(d.ptr, d.pitch, n_lambda, a, grid, s);
    return launch_np<24>(d.ptr, d.pitch, n_lambda, a, grid, s);
}

}  // namespace pwa
