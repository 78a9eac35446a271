// Fused data-term kernel on the precomputed per-event table (Sec. 2, after
// Eq. 3: with masses and widths fixed, A_a A*_b can be formed once per event).
//
// Table layout (k_pack.cu): P = N^2 float planes t[p][i], p < N the real
// diagonal |A_a|^2, then for each pair a < b two planes Re(A_a conj A_b),
// Im(A_a conj A_b). With coefficients w (from V, per call)
//   w_a = |V_a|^2,  w_(a,b),re = 2 Re(V_a conj V_b),  w_(a,b),im = -2 Im(V_a conj V_b)
// the intensity of Eq. 1 is I_i = sum_p w_p t_p(i) (Eq. 3's double sum over
// the Hermitian table), and the data part of the gradient is
//   g_a = - sum_b V_b Ghat[b][a],  Ghat = sum_i T_i / I_i   (Hermitian),
// so the per-event work is one N^2-term sum and one N^2-term accumulation of
// t_p / I_i.
//
// Each CTA (persistent, one per SM) streams tiles of 32 events x P planes
// through a TMA/mbarrier ring. Lane = event everywhere, warp q owns the
// planes p = q, q + W, ...: the intensity pass and the gradient pass both
// read 32 consecutive floats of one plane per warp (conflict-free). Each
// w_p t_p is split exactly against sigma (as in the direct form, k_nll_amp.cu)
// so I_i is correct to one float rounding; the per-warp partial sums meet in
// shared memory. Every wait is bounded.
#include <stdlib.h>

#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr double kLn2 = 0.69314718055994530942;
constexpr int kBoxRows = 256;  // TMA box height limit

// Tiles of TE events: 64 (two per lane, packed in FP32x2 registers) where two
// stages of them fit in shared memory (N <= 20), else 32 (one per lane).
template <int N>
struct TabCfg {
    static constexpr int P = N * N;
    static constexpr int TE = N <= 20 ? 64 : 32;
    static constexpr int EPL = TE / 32;                      // events per lane
    static constexpr int W = (P <= 256) ? 8 : 16;            // consumer warps
    static constexpr int RPW = (P + W - 1) / W;              // planes per warp
    static constexpr uint32_t STAGE_BYTES = P * TE * 4;
    static constexpr int STAGES_RAW = (190 * 1024) / STAGE_BYTES;
    static constexpr int STAGES = STAGES_RAW < 2 ? 2 : (STAGES_RAW > 6 ? 6 : STAGES_RAW);
    static constexpr int THREADS = (W + 2) * 32;             // + producer warp + helper warp
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 2 * STAGES * sizeof(uint64_t) +
                                   (size_t)P * 3 * sizeof(float);  // w_hi, w_lo, |w|
    // with the static arrays (part_hi/part_lo 2 W TE words each) inside 227 KB
    static constexpr bool FITS = SMEM + (size_t)4 * W * TE * 4 + 4096 <= 227 * 1024;
};

// scratch: [G] int64 pairs (ln-integer part, exponents), [G][P + 1] float-float
// (ln remainders, Ghat planes), [2N+2] double (M V, V^H M V), flags
struct TabScratch {
    long long *pi;
    float2 *pf;
    double *mv;
    int *flags;
};

__host__ __device__ inline TabScratch tab_scratch(void *base, int grid, int P)
{
    char *p = static_cast<char *>(base);
    TabScratch s;
    s.pi = reinterpret_cast<long long *>(p);
    p += (size_t)grid * 2 * sizeof(long long);
    s.pf = reinterpret_cast<float2 *>(p);
    p += (size_t)grid * (P + 1) * sizeof(float2);
    s.mv = reinterpret_cast<double *>(p);
    p += (2 * kMaxWaves + 2) * sizeof(double);
    s.flags = reinterpret_cast<int *>(p);
    return s;
}

// Named barrier over the consumer warps only.
__device__ __forceinline__ void consumers_sync(int nthreads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

template <int N>
__global__ void __launch_bounds__(TabCfg<N>::THREADS, 1)
    nll_table_kernel(const __grid_constant__ CUtensorMap map, const EvalArgs a, const int n_tiles,
                     const float *__restrict__ tmax, const int box_rows, const int n_boxes)
{
    using C = TabCfg<N>;
    constexpr int P = C::P, W = C::W, STAGES = C::STAGES;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *tiles = reinterpret_cast<float *>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + (size_t)STAGES * C::STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    float *w_hi = reinterpret_cast<float *>(empty + STAGES);
    float *w_lo = w_hi + P;
    float *w_abs = w_lo + P;

    constexpr int TE = C::TE, EPL = C::EPL;
    __shared__ unsigned part_hi[2][W][TE];  // double-buffered by tile parity
    __shared__ float part_lo[2][W][TE];
    __shared__ float s_sigma, s_unit;
    __shared__ float red_g[W][C::RPW];
    __shared__ long long red_i[2];
    __shared__ float red_lf;
    __shared__ int s_flags, s_last;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Nw = a.n_waves;
    const int Pw = Nw * Nw;  // planes present (padded planes are zero)
    TabScratch sc = tab_scratch(a.partials, gridDim.x, P);
    const int n_my =
        (n_tiles > (int)blockIdx.x) ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    // every box is counted in full (rows past Pw arrive zero-filled)
    const int rows_loaded = box_rows * n_boxes;
    const uint32_t stage_tx = (uint32_t)rows_loaded * TE * 4u;
    const int n_first = n_my < STAGES ? n_my : STAGES;

    auto issue = [&](int j) {
        const int s = j % STAGES;
        float *dst = tiles + (size_t)s * P * TE;
        const int x = ((int)blockIdx.x + j * (int)gridDim.x) * TE;
        mbar_arrive_expect_tx(&full[s], stage_tx);
        for (int bx = 0; bx < n_boxes; ++bx)
            tma_load_2d(dst + (size_t)bx * box_rows * TE, &map, x, bx * box_rows, &full[s]);
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], W);
        }
        fence_barrier_init();
        s_flags = 0;
        red_i[0] = red_i[1] = 0;
        red_lf = 0.f;
        for (int j = 0; j < n_first; ++j)
            issue(j);
    }
    // planes past the loaded boxes (padded waves) are never written: zero them once
    for (int s = 0; s < STAGES; ++s)
        for (int i = rows_loaded * TE + threadIdx.x; i < P * TE; i += blockDim.x)
            tiles[(size_t)s * P * TE + i] = 0.f;
    // coefficients w_p as float pairs, from V in FP64
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        double w = 0.0;
        if (p < Nw) {
            w = a.V[2 * p] * a.V[2 * p] + a.V[2 * p + 1] * a.V[2 * p + 1];
        } else if (p < Pw) {
            // pair index q = (p - Nw) / 2 among x < y in row-major order
            int q = (p - Nw) >> 1, x = 0;
            while (q >= Nw - 1 - x) {
                q -= Nw - 1 - x;
                ++x;
            }
            const int y = x + 1 + q;
            const double xr = a.V[2 * x], xi = a.V[2 * x + 1], yr = a.V[2 * y], yi = a.V[2 * y + 1];
            w = ((p - Nw) & 1) ? -2.0 * (xi * yr - xr * yi)   // -2 Im(V_x conj V_y)
                               : 2.0 * (xr * yr + xi * yi);   //  2 Re(V_x conj V_y)
        }
        const float hi = __double2float_rn(w);
        w_hi[p] = hi;
        w_lo[p] = __double2float_rn(w - (double)hi);
        w_abs[p] = fabsf(__double2float_ru(fabs(w)));
    }
    __syncthreads();
    if (warp == 1) {
        // 2^(k-1) >= 1.25 sum_p |w_p| max_i |t_p(i)|
        float b = 0.f;
        for (int p = lane; p < Pw; p += 32)
            b = fmaf(w_abs[p], tmax[p], b);
        b = warp_sum(b);
        if (lane == 0) {
            const float target = 2.5f * b;
            int k = -100;
            if (target > 0.f)
                k = max(k, ((__float_as_int(target) >> 23) & 0xff) - 126);
            if (!(target < 1e30f))
                k = 100;
            s_sigma = 1.5f * ldexpf(1.0f, k);
            s_unit = ldexpf(1.0f, k - 23);
        }
    }
    __syncthreads();

    int flags = 0;
    if (warp == 0) {
        if (lane == 0) {
            int j = n_first;
            for (; j < n_my; ++j) {
                const int s = j % STAGES;
                const uint32_t u = j / STAGES;
                if (!mbar_wait(&empty[s], (u & 1) ^ 1)) {
                    flags |= FLAG_TIMEOUT;
                    break;
                }
                issue(j);
            }
            for (int q = (j > STAGES ? j - STAGES : 0); q < j; ++q)
                if (!mbar_wait(&full[q % STAGES], (q / STAGES) & 1))
                    flags |= FLAG_TIMEOUT;
        }
    } else if (warp <= W) {
        const int q = warp - 1;  // this warp's planes: q, q + W, ...
        const float sigma = s_sigma, unit = s_unit;
        const unsigned offset = (unsigned)P * __float_as_uint(sigma);
        float gacc[C::RPW];
#pragma unroll
        for (int r = 0; r < C::RPW; ++r)
            gacc[r] = 0.f;
        long long l_int = 0;
        int eacc = 0, bad = 0;
        float l_frac = 0.f;
        for (int j = 0; j < n_my; ++j) {
            const int s = j % STAGES;
            if (!mbar_wait(&full[s], (j / STAGES) & 1)) {
                flags |= FLAG_TIMEOUT;
                break;
            }
            const float *T = tiles + (size_t)s * P * TE + EPL * lane;
            // intensity: this warp's share of sum_p w_p t_p for the lane's EPL
            // events, split exactly
            unsigned hsum[EPL];
            float lsum[EPL];
            if constexpr (EPL == 2) {
                const f2 SG = pk2(sigma, sigma);
                unsigned h0 = 0, h1 = 0;
                f2 l2 = 0ull;
#pragma unroll
                for (int r = 0; r < C::RPW; ++r) {
                    const int p = q + r * W;
                    if (p < P) {
                        const f2 t = *reinterpret_cast<const f2 *>(T + p * TE);
                        const float wh = w_hi[p];
                        const f2 W2 = pk2(wh, wh);
                        const f2 x = fma2(W2, t, SG);
                        float x0, x1;
                        upk2(x, x0, x1);
                        h0 += __float_as_uint(x0);
                        h1 += __float_as_uint(x1);
                        l2 = add2(l2, fma2(W2, t, sub2(SG, x)));
                        const float wl = w_lo[p];
                        l2 = fma2(pk2(wl, wl), t, l2);
                    }
                }
                hsum[0] = h0;
                hsum[1] = h1;
                upk2(l2, lsum[0], lsum[1]);
            } else {
                unsigned h = 0;
                float l = 0.f;
#pragma unroll
                for (int r = 0; r < C::RPW; ++r) {
                    const int p = q + r * W;
                    if (p < P) {
                        const float t = T[p * TE];
                        const float wh = w_hi[p];
                        const float x = fmaf(wh, t, sigma);
                        h += __float_as_uint(x);
                        l += fmaf(wh, t, sigma - x);
                        l = fmaf(w_lo[p], t, l);
                    }
                }
                hsum[0] = h;
                lsum[0] = l;
            }
            // Every warp forms the TE intensities from the W partials (in the same
            // order, so to the same bits); warp 0 alone accumulates the log sums.
            // The partials are double-buffered by tile parity, so one barrier per
            // tile suffices: a warp past tile j's barrier writes buffer (j+1)&1
            // only after every warp has arrived there, i.e. finished reading it
            // for tile j-1.
            const int pb = j & 1;
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
                part_hi[pb][q][EPL * lane + e] = hsum[e];
                part_lo[pb][q][EPL * lane + e] = lsum[e];
            }
            consumers_sync(W * 32);
            float iv[EPL];
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
                iv[e] = 0.f;
                unsigned h = 0;
                float l = 0.f;
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    h += part_hi[pb][k][EPL * lane + e];
                    l += part_lo[pb][k][EPL * lane + e];
                }
                const float I = (float)(int)(h - offset) * unit + l;
                const int64_t ev =
                    (int64_t)((int)blockIdx.x + j * (int)gridDim.x) * TE + EPL * lane + e;
                if (ev < a.n_events) {
                    if (I > 0.f && I < INFINITY) {
                        iv[e] = __frcp_rn(I);
                        if (q == 0) {
                            int ex;
                            const float f = split_exponent(I, ex);
                            const float y = logf(f) * 8388608.0f;
                            const float tt = y + 12582912.0f;
                            l_int += __float_as_int(tt) - 0x4B400000;
                            l_frac += y - (tt - 12582912.0f);
                            eacc += ex;
                        }
                    } else {
                        bad = 1;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < C::RPW; ++r) {
                const int p = q + r * W;
                if (p < P) {
                    if constexpr (EPL == 2) {
                        const float2 t = *reinterpret_cast<const float2 *>(T + p * TE);
                        gacc[r] = fmaf(t.x, iv[0], fmaf(t.y, iv[1], gacc[r]));
                    } else {
                        gacc[r] = fmaf(T[p * TE], iv[0], gacc[r]);
                    }
                }
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&empty[s]);
        }
        if (bad)
            flags |= FLAG_DOMAIN;
#pragma unroll
        for (int r = 0; r < C::RPW; ++r) {
            const float v = warp_sum(gacc[r]);
            if (lane == 0)
                red_g[q][r] = v;
        }
        if (q == 0) {
            const long long li = warp_sum(l_int);
            const long long ei = warp_sum((long long)eacc);
            const float lf = warp_sum(l_frac);
            if (lane == 0) {
                red_i[0] = li;
                red_i[1] = ei;
                red_lf = lf;
            }
        }
    } else if (blockIdx.x == 0) {
        // helper warp of CTA 0: M V and V^H M V in FP64
        double nv = 0.0;
        for (int row = lane; row < Nw; row += 32) {
            double re = 0.0, im = 0.0;
            for (int b = 0; b < Nw; ++b) {
                const double mr = a.M[2 * (row * Nw + b)], mi = a.M[2 * (row * Nw + b) + 1];
                const double vr = a.V[2 * b], vi = a.V[2 * b + 1];
                re = fma(mr, vr, fma(-mi, vi, re));
                im = fma(mr, vi, fma(mi, vr, im));
            }
            sc.mv[2 * row] = re;
            sc.mv[2 * row + 1] = im;
            nv = fma(a.V[2 * row], re, fma(a.V[2 * row + 1], im, nv));
        }
        nv = warp_sum(nv);
        if (lane == 0)
            sc.mv[2 * kMaxWaves] = nv;
    }
    if (flags)
        atomicOr(&s_flags, flags);
    __syncthreads();

    // ---- CTA partials ------------------------------------------------------
    if (threadIdx.x < 2)
        sc.pi[2 * blockIdx.x + threadIdx.x] = red_i[threadIdx.x];
    for (int p = threadIdx.x; p < P + 1; p += blockDim.x) {
        float v;
        if (p == 0)
            v = red_lf;
        else
            v = red_g[(p - 1) % W][(p - 1) / W];
        sc.pf[(size_t)blockIdx.x * (P + 1) + p] = make_float2(v, 0.f);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_flags)
            atomicOr(sc.flags, s_flags);
        __threadfence();
        s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last)
        return;

    // ---- last CTA: fixed-order sums over CTAs, gradient from Ghat ----------
    const int G_ = gridDim.x;
    double *gh = reinterpret_cast<double *>(tiles);  // [P + 1] doubles
    __shared__ long long fin_i[2];
    // batches of 16 independent loads per thread: one L2 round trip per batch
    for (int p = threadIdx.x; p < P + 1; p += blockDim.x) {
        dfloat v = {0.f, 0.f};
        for (int b0 = 0; b0 < G_; b0 += 16) {
            float2 x[16];
#pragma unroll
            for (int k = 0; k < 16; ++k)
                x[k] = (b0 + k < G_) ? __ldcg(&sc.pf[(size_t)(b0 + k) * (P + 1) + p])
                                     : make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 16; ++k)
                v = df_add(v, dfloat{x[k].x, x[k].y});
        }
        gh[p] = (double)v.hi + (double)v.lo;
    }
    if (threadIdx.x < 2) {
        long long v = 0;
        for (int b0 = 0; b0 < G_; b0 += 16) {
            long long x[16];
#pragma unroll
            for (int k = 0; k < 16; ++k)
                x[k] = (b0 + k < G_) ? __ldcg(&sc.pi[2 * (b0 + k) + threadIdx.x]) : 0;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                v += x[k];
        }
        fin_i[threadIdx.x] = v;
    }
    __syncthreads();
    const int wf = __ldcg(sc.flags);
    const bool invalid = (wf & (FLAG_DOMAIN | FLAG_TIMEOUT)) != 0;
    // g_a = -sum_b V_b Ghat[b][a] + (M V)_a; Ghat from the plane sums gh[1 + p]
    if (a.grad) {
        for (int x = threadIdx.x; x < Nw; x += blockDim.x) {
            double re = 0.0, im = 0.0;
            for (int b = 0; b < Nw; ++b) {
                double hr, hi;
                if (b == x) {
                    hr = gh[1 + x];
                    hi = 0.0;
                } else {
                    const int lo = b < x ? b : x, up = b < x ? x : b;
                    const int pair = lo * Nw - lo * (lo + 1) / 2 + (up - lo - 1);
                    hr = gh[1 + Nw + 2 * pair];
                    hi = (b < x) ? gh[2 + Nw + 2 * pair] : -gh[2 + Nw + 2 * pair];
                }
                const double vr = a.V[2 * b], vi = a.V[2 * b + 1];
                re = fma(vr, hr, fma(-vi, hi, re));
                im = fma(vr, hi, fma(vi, hr, im));
            }
            a.grad[2 * x] = invalid ? 0.0 : __ldcg(&sc.mv[2 * x]) - re;
            a.grad[2 * x + 1] = invalid ? 0.0 : __ldcg(&sc.mv[2 * x + 1]) - im;
        }
    }
    if (threadIdx.x == 0) {
        const double lnsum =
            fma((double)fin_i[1], kLn2, ((double)fin_i[0] + gh[0]) * 0x1p-23);
        double nll = __ldcg(&sc.mv[2 * kMaxWaves]) - lnsum;
        if (wf & FLAG_DOMAIN)
            nll = INFINITY;
        if (wf & FLAG_TIMEOUT)
            nll = NAN;
        a.nll[0] = nll;
        if (wf)
            atomicOr(a.status, wf);
        if (a.done)
            atomicAdd(a.done, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *sc.flags = 0;
        *a.ticket = 0u;
    }
}

int pad_waves_table(int n)
{
    static const int pads[] = {4, 8, 12, 16, 20, 24};
    for (int p : pads)
        if (n <= p)
            return p;
    return -1;
}

template <int N>
cudaError_t configure_t()
{
    static_assert(TabCfg<N>::FITS, "table tile must fit in shared memory");
    return cudaFuncSetAttribute(nll_table_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TabCfg<N>::SMEM);
}

template <int N>
cudaError_t launch_t(const CUtensorMap *map, const EvalArgs &a, int grid, const float *tmax,
                     cudaStream_t s)
{
    const int n_tiles = (int)((a.n_events + TabCfg<N>::TE - 1) / TabCfg<N>::TE);
    const int Pw = a.n_waves * a.n_waves;
    const int n_boxes = (Pw + kBoxRows - 1) / kBoxRows;
    const int box_rows = (Pw + n_boxes - 1) / n_boxes;
    if (box_rows * n_boxes > TabCfg<N>::P)
        return cudaErrorInvalidValue;
    nll_table_kernel<N><<<grid, TabCfg<N>::THREADS, TabCfg<N>::SMEM, s>>>(*map, a, n_tiles, tmax,
                                                                          box_rows, n_boxes);
    return cudaGetLastError();
}

}  // namespace

int table_max_waves() { return 24; }  // tiles of N^2 planes must fit two stages
int table_box_events(int n_waves)
{
    switch (pad_waves_table(n_waves)) {
    case 4: return TabCfg<4>::TE;
    case 8: return TabCfg<8>::TE;
    case 12: return TabCfg<12>::TE;
    case 16: return TabCfg<16>::TE;
    case 20: return TabCfg<20>::TE;
    case 24: return TabCfg<24>::TE;
    }
    return 32;
}
int table_box_rows(int n_waves)
{
    const int Pw = n_waves * n_waves;
    const int n_boxes = (Pw + kBoxRows - 1) / kBoxRows;
    return (Pw + n_boxes - 1) / n_boxes;  // equal boxes, at most n_boxes - 1 rows past Pw
}

size_t table_scratch_bytes(int n_waves, int grid)
{
    const int P = pad_waves_table(n_waves) * pad_waves_table(n_waves);
    return (size_t)grid * 2 * sizeof(long long) + (size_t)grid * (P + 1) * sizeof(float2) +
           (2 * kMaxWaves + 2) * sizeof(double) + 64;
}

cudaError_t table_configure()
{
    cudaError_t e = cudaSuccess;
    for (cudaError_t r : {configure_t<4>(), configure_t<8>(), configure_t<12>(), configure_t<16>(),
                          configure_t<20>(), configure_t<24>()})
        if (r != cudaSuccess)
            e = r;
    return e;
}

cudaError_t launch_nll_table(int64_t n_events, int n_waves, const CUtensorMap *map,
                             const EvalArgs &a, const float *tmax, int grid, cudaStream_t s)
{
    (void)n_events;
    switch (pad_waves_table(n_waves)) {
    case 4: return launch_t<4>(map, a, grid, tmax, s);
    case 8: return launch_t<8>(map, a, grid, tmax, s);
    case 12: return launch_t<12>(map, a, grid, tmax, s);
    case 16: return launch_t<16>(map, a, grid, tmax, s);
    case 20: return launch_t<20>(map, a, grid, tmax, s);
    case 24: return launch_t<24>(map, a, grid, tmax, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pwa
