// NLL of Eq. 3 and its gradient when the masses and widths of R Breit-Wigner
// waves are free parameters. The paper's precomputation (Sec. 2: the MC sum
// and the per-event table) is only valid for fixed masses and widths; with
// them free, the amplitudes of the free waves are recomputed on every call
// and the normalisation term is the MC sum itself:
//   A_r(i) = BW(m_i; M_r, G_r) Y_r(i),  BW(m; M, G) = 1 / (M^2 - m^2 - i M G)
//   NLL = -sum_data ln |S_i|^2 + (1 / N_gen) sum_MC |S_j|^2,  S = sum_a V_a A_a
//   dNLL/dV*_a  = sum w_i conj(A_a(i)) S_i
//   dNLL/dM_r   = sum w_i 2 Re(conj(S_i) V_r Y_r dBW/dM),  dBW/dM = -(2M - iG) BW^2
//   dNLL/dG_r   = sum w_i 2 Re(conj(S_i) V_r Y_r dBW/dG),  dBW/dG = i M BW^2
// with w_i = -1 / I_i for data events and 1 / N_gen for MC events.
//
// Store: per sample one structure-of-arrays block of 1 + 2N planes of
// `pitch` floats: plane 0 = m, planes 1 + 2a, 2 + 2a = Re, Im of Y_a for the
// free waves a < R and of the fixed amplitude A_a for a >= R.
//
// One event per thread, complex values packed as (Re, Im) in FP32x2 registers.
// Precision:
//  * M^2, M G and (M G)^2 enter every event coherently, so they are carried
//    as float pairs (hi + lo), m^2 and D^2 are split exactly by FMA and the
//    denominator D^2 + (M G)^2 is kept as an exact pair through the
//    reciprocal: the Breit-Wigner is then correct to float roundings that vary
//    from event to event, with no error shared by all events near the peak;
//  * S uses the compensated dot product (Ogita, Rump and Oishi, Dot2) with V
//    as a float pair, in four independent chains joined by error-free sums,
//    so destructive interference does not cost digits;
//  * ln I = e ln 2 + ln f (e summed as an integer, ln f in float-float), the
//    MC sum of I in float-float, gradients in FP32 per thread and FP64 across
//    threads and blocks. Data and MC sums are kept apart (their weights
//    differ by ~N_gen) and combined in FP64 by the last block, in block order.
#include "pwa_internal.cuh"

namespace pwa {

namespace {

// threads per block: more warps where the register footprint allows it
__host__ __device__ constexpr int res_threads(int np) { return np <= 20 ? 384 : 256; }
constexpr int kMaxFree = 8;

struct ResShared {
    // per wave: (vr, vi), (-vr, -vi), (-vi, vr), (vi, -vr) of the high part; low parts
    f2 va[32], van[32], vb[32], vbn[32], val[32], vbl[32];
    float m2h[kMaxFree], m2l[kMaxFree];              // M^2
    float gh[kMaxFree], gl[kMaxFree];                // M G
    float g2h[kMaxFree], g2l[kMaxFree];              // (M G)^2
    float mf[kMaxFree], wf[kMaxFree];                // M, G
};

__device__ __forceinline__ f2 splat(float v) { return pk2(v, v); }

__device__ __forceinline__ void prefetch_l1(const float *p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Knuth's TwoSum on both halves: returns a + b rounded, err = the exact rest.
__device__ __forceinline__ f2 two_sum2(f2 a, f2 b, f2 &err)
{
    const f2 s = add2(a, b);
    const f2 bb = sub2(s, a);
    err = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
    return s;
}

__device__ __forceinline__ void split_pair(double v, float &h, float &l)
{
    h = __double2float_rn(v);
    l = __double2float_rn(v - (double)h);
}

template <int NP, int RP>
__global__ void __launch_bounds__(res_threads(NP), 1) nll_res_kernel(const ResArgs a)
{
    constexpr int kResThreads = res_threads(NP);
    __shared__ ResShared sh;
    __shared__ float red[kResThreads / 32][2 * 32 + 2 * kMaxFree + 4];
    __shared__ int s_flags, s_last;
    const int N = a.n_waves, R = a.n_free;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        const int w = threadIdx.x;
        float vrh = 0.f, vrl = 0.f, vih = 0.f, vil = 0.f;
        if (w < N) {
            split_pair(a.V[2 * w], vrh, vrl);
            split_pair(a.V[2 * w + 1], vih, vil);
        }
        sh.va[w] = pk2(vrh, vih);
        sh.van[w] = pk2(-vrh, -vih);
        sh.vb[w] = pk2(-vih, vrh);
        sh.vbn[w] = pk2(vih, -vrh);
        sh.val[w] = pk2(vrl, vil);
        sh.vbl[w] = pk2(-vil, vrl);
        if (w < kMaxFree) {
            const double M = w < R ? a.mass[w] : 1.0, G = w < R ? a.width[w] : 1.0;
            split_pair(M * M, sh.m2h[w], sh.m2l[w]);
            split_pair(M * G, sh.gh[w], sh.gl[w]);
            split_pair((M * G) * (M * G), sh.g2h[w], sh.g2l[w]);
            sh.mf[w] = (float)M;
            sh.wf[w] = (float)G;
        }
    }
    if (threadIdx.x == 0)
        s_flags = 0;
    __syncthreads();

    const int P = a.pstride;  // doubles per (block, phase) partial
    int bad = 0;
    for (int phase = 0; phase < 2; ++phase) {
        const float *base = phase == 0 ? a.data : a.mc;
        const int64_t pitch = phase == 0 ? a.data_pitch : a.mc_pitch;
        const int64_t n = phase == 0 ? a.n_data : a.n_mc;
        f2 gv[NP];                 // (Re, Im) of sum conj(A_a) w S
        float gm[RP], gw[RP];
#pragma unroll
        for (int w = 0; w < NP; ++w)
            gv[w] = 0ull;
#pragma unroll
        for (int r = 0; r < RP; ++r)
            gm[r] = gw[r] = 0.f;
        dfloat acc = {0.f, 0.f};  // data: sum ln f; MC: sum I
        int eacc = 0;             // data: sum of exponents
        const int64_t stride = (int64_t)gridDim.x * kResThreads;
        for (int64_t i = (int64_t)blockIdx.x * kResThreads + threadIdx.x; i < n; i += stride) {
            // the warp's events of the next iteration fill one 128-byte line per
            // plane: lane k prefetches planes k, k + 32, ... into L1
            const int64_t nb = i - lane + stride;
            if (nb < n)
                for (int p = lane; p < 1 + 2 * N; p += 32)
                    prefetch_l1(base + p * pitch + nb);
            float ar[NP], ai[NP], br[RP], bi[RP];
            const float m = __ldg(base + i);
            // unconditional loads (padded waves re-read wave 0, zeroed by a
            // select), so that no branch separates them
#pragma unroll
            for (int w = 0; w < NP; ++w) {
                const int64_t o = (int64_t)(w < N ? 1 + 2 * w : 1) * pitch + i;
                const float x = __ldg(base + o), y = __ldg(base + o + pitch);
                ar[w] = w < N ? x : 0.f;
                ai[w] = w < N ? y : 0.f;
            }
            // free waves: A = BW(m) Y
            const float mm = m * m;
            const float me = fmaf(m, m, -mm);  // m^2 = mm + me exactly
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                br[r] = bi[r] = 0.f;
                if (r < R) {
                    const float D = (sh.m2h[r] - mm) + (sh.m2l[r] - me);
                    // den = D^2 + (M G)^2 as an unevaluated pair dh + dl: D^2 = p + pe
                    // exactly, dh + e = (M G)^2_hi + p exactly (TwoSum). Near the peak
                    // many events share one dh, so rounding den or 1/dh to a float
                    // would give them all the same error; the Newton step below
                    // works against the full pair instead.
                    const float p = D * D, pe = fmaf(D, D, -p);
                    const float g2 = sh.g2h[r];
                    const float dh = g2 + p, bb = dh - g2;
                    const float dl = ((g2 - (dh - bb)) + (p - bb)) + pe + sh.g2l[r];
                    const float q0 = rcp_approx(dh);
                    const float q = fmaf(q0, fmaf(-dl, q0, fmaf(-dh, q0, 1.f)), q0);
                    br[r] = D * q;
                    bi[r] = fmaf(sh.gh[r], q, sh.gl[r] * q);
                    const float yr = ar[r], yi = ai[r];
                    ar[r] = fmaf(br[r], yr, -bi[r] * yi);
                    ai[r] = fmaf(br[r], yi, bi[r] * yr);
                }
            }
            // S = sum (Vh + Vl) A, compensated: (Sr, Si) += ar (vr, vi) + ai (-vi, vr),
            // in four independent chains (waves w mod 4) joined by error-free sums
            f2 s[4] = {0ull, 0ull, 0ull, 0ull}, c[4] = {0ull, 0ull, 0ull, 0ull}, l = 0ull;
#pragma unroll
            for (int w = 0; w < NP; ++w) {
                if (w < N) {
                    const f2 x = splat(ar[w]), y = splat(ai[w]);
                    dot2_step(s[w & 3], c[w & 3], x, sh.va[w], sh.van[w]);
                    dot2_step(s[w & 3], c[w & 3], y, sh.vb[w], sh.vbn[w]);
                    l = fma2(x, sh.val[w], fma2(y, sh.vbl[w], l));
                }
            }
            // (s0 + s1) + (s2 + s3) by TwoSum, the rounding errors join the corrections
            f2 e01, e23, e;
            const f2 s01 = two_sum2(s[0], s[1], e01), s23 = two_sum2(s[2], s[3], e23);
            const f2 st = two_sum2(s01, s23, e);
            const f2 ct = add2(add2(add2(c[0], c[1]), add2(c[2], c[3])), add2(add2(e01, e23), e));
            float sr, si;
            upk2(add2(st, add2(ct, l)), sr, si);
            const float I = fmaf(sr, sr, si * si);
            float wr = 0.f, wi = 0.f;
            if (phase == 0) {
                if (I > 0.f && I < INFINITY) {
                    int ex;
                    const float f = split_exponent(I, ex);
                    eacc += ex;
                    acc = df_add(acc, dfloat{logf(f), 0.f});
                    const float w = -__frcp_rn(I);
                    wr = w * sr;
                    wi = w * si;
                } else {
                    bad = 1;
                }
            } else {
                acc = df_add(acc, dfloat{I, 0.f});
                wr = sr;
                wi = si;
            }
            // gradient: conj(A) (wr + i wi) = (ar wr + ai wi) + i (ar wi - ai wr)
            const f2 W1 = pk2(wr, wi), W2 = pk2(wi, -wr);
#pragma unroll
            for (int w = 0; w < NP; ++w)
                if (w < N)
                    gv[w] = fma2(splat(ar[w]), W1, fma2(splat(ai[w]), W2, gv[w]));
            // masses and widths: c = conj(wS) V_r A_r BW_r, then
            // dM: 2 Re(c (-2M + iG)) = -4M Re c - 2G Im c;  dG: 2 Re(c i M) = -2M Im c
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                if (r < R) {
                    float vr, vi;
                    upk2(sh.va[r], vr, vi);
                    const float tr = fmaf(vr, ar[r], -vi * ai[r]), ti = fmaf(vr, ai[r], vi * ar[r]);
                    const float ur = fmaf(tr, br[r], -ti * bi[r]), ui = fmaf(tr, bi[r], ti * br[r]);
                    const float cr = fmaf(wr, ur, wi * ui), ci = fmaf(wr, ui, -wi * ur);
                    const float M = sh.mf[r], G = sh.wf[r];
                    gm[r] += -4.f * M * cr - 2.f * G * ci;
                    gw[r] += -2.f * M * ci;
                }
            }
        }
        // ---- block reduction (fixed order) ---------------------------------
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
            if (lane == 0 && w < N) {
                red[warp][4 + 2 * w] = x;
                red[warp][5 + 2 * w] = y;
            }
        }
#pragma unroll
        for (int r = 0; r < RP; ++r) {
            const float vm = warp_sum(gm[r]), vw = warp_sum(gw[r]);
            if (lane == 0 && r < R) {
                red[warp][4 + 2 * N + r] = vm;
                red[warp][4 + 2 * N + R + r] = vw;
            }
        }
        __syncthreads();
        double *out = a.partials + ((size_t)blockIdx.x * 2 + phase) * P;
        for (int c = threadIdx.x; c < P; c += kResThreads) {
            double v = 0.0;
            if (c == 0) {
                for (int w = 0; w < kResThreads / 32; ++w)
                    v += (double)red[w][0] + (double)red[w][1];
            } else if (c == 1) {
                for (int w = 0; w < kResThreads / 32; ++w)
                    v += (double)red[w][2] + 16777216.0 * (double)red[w][3];
            } else {
                for (int w = 0; w < kResThreads / 32; ++w)
                    v += (double)red[w][2 + c];
            }
            out[c] = v;
        }
        __syncthreads();
    }
    if (bad)
        atomicOr(&s_flags, FLAG_DOMAIN);
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
    // ---- last block: sums over blocks in block order, FP64 ------------------
    __threadfence();
    const int nb = gridDim.x;
    __shared__ double fin[2][2 + 2 * 32 + 2 * kMaxFree];
    for (int item = threadIdx.x; item < 2 * P; item += kResThreads) {
        const int phase = item / P, c = item % P;
        double v = 0.0;
        for (int b = 0; b < nb; ++b)
            v += __ldcg(a.partials + ((size_t)b * 2 + phase) * P + c);
        fin[phase][c] = v;
    }
    __syncthreads();
    const bool dom = (*(volatile int *)a.status & FLAG_DOMAIN) != 0;
    const double ig = a.inv_ngen;
    if (threadIdx.x == 0) {
        const double lnsum = 0.69314718055994530942 * fin[0][1] + fin[0][0];
        a.out[0] = dom ? INFINITY : -lnsum + ig * fin[1][0];
        *a.ticket = 0u;
        if (a.done)
            atomicAdd(a.done, 1);
    }
    for (int c = threadIdx.x; c < 2 * N + 2 * R; c += kResThreads)
        a.out[1 + c] = dom ? 0.0 : fin[0][2 + c] + ig * fin[1][2 + c];
}

template <int NP>
void launch_np(const ResArgs &a, int grid, cudaStream_t s)
{
    if (a.n_free <= 4)
        nll_res_kernel<NP, 4><<<grid, res_threads(NP), 0, s>>>(a);
    else
        nll_res_kernel<NP, kMaxFree><<<grid, res_threads(NP), 0, s>>>(a);
}

}  // namespace

int res_max_waves() { return 32; }
int res_max_free() { return kMaxFree; }

size_t res_partials_doubles(int n_waves, int n_free, int grid)
{
    return (size_t)grid * 2 * (2 + 2 * n_waves + 2 * n_free);
}

cudaError_t launch_nll_res(const ResArgs &args, int grid, cudaStream_t s)
{
    ResArgs a = args;
    a.pstride = 2 + 2 * a.n_waves + 2 * a.n_free;
    const int N = a.n_waves;
    if (N < 1 || N > 32 || a.n_free < 0 || a.n_free > kMaxFree || a.n_free > N)
        return cudaErrorInvalidValue;
    if (N <= 4)
        launch_np<4>(a, grid, s);
    else if (N <= 8)
        launch_np<8>(a, grid, s);
    else if (N <= 12)
        launch_np<12>(a, grid, s);
    else if (N <= 16)
        launch_np<16>(a, grid, s);
    else if (N <= 20)
        launch_np<20>(a, grid, s);
    else if (N <= 24)
        launch_np<24>(a, grid, s);
    else
        launch_np<32>(a, grid, s);
    return cudaGetLastError();
}

}  // namespace pwa
