// Fused data-term kernel of the direct form (see k_nll_amp.cu for the
// method): the kernel template, shared by the coherent launcher (k_nll_amp.cu,
// one component per event) and the incoherent one (k_nll_incoh.cu, L
// components per event: tiles of 2 L n rows, S^l of every component, I the
// sum of their squared moduli, the gradient summed over components).
#pragma once

#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr double kLn2 = 0.69314718055994530942;

// N padded waves, G consumer groups, L components per event (1: the coherent
// sum of Eq. 1; L > 1: an incoherent sum over L components, rows 2 (l n + a)
// of a tile holding component l of wave a for n loaded waves).
template <int N, int G, int L = 1>
struct AmpCfg {
    static constexpr int GROUPS = G;                   // consumer groups (tiles in turn)
    // warps per group: 4; 3 with several components or from 40 waves on, so
    // that a CTA of two groups keeps to eight warps and the register cap of
    // 255 (a larger CTA is allocated as twelve warps: 168 registers; the
    // per-component state, or at 40 and 48 waves the per-wave state, does
    // not fit). Measured on 1 GB samples: four-warp groups at 32 waves
    // (with the re-read of the amplitudes below) 14% faster than three, and
    // at 40 and 48 waves three-warp groups 1.7 and 1.6 times faster than four.
    static constexpr int GW = (L > 1 || N >= 40) ? 3 : 4;
    static constexpr int CW = GROUPS * GW;             // consumer warps
    static constexpr int TE = GW * 32 * 2;             // events per tile (2 per thread)
    static constexpr int ROWS = 2 * N * L;
    static constexpr uint32_t STAGE_BYTES = ROWS * TE * 4;
    // The ring. When two or more stages per group fit in 200 KB, each group
    // owns SPG of them (at most four): tile j goes to group j % G and to that
    // group's stage (j / G) % SPG, so a stage's successive uses belong to one
    // group and a waiter is never a whole phase behind. Otherwise (one stage
    // per group would fit), as many stages as fit are shared by the groups:
    // tile j sits in stage j % STAGES (a third stage at 32 waves, or for two
    // components of 20 waves, measured 8% and 21% faster than two; a fifth
    // shared 40 KB stage at 20 waves was slower than four owned ones). A
    // shared stage has two full barriers, for its even and its odd uses.
    // A group waiting for use u of a stage (tile j) waits on the barrier
    // whose previous phase was use u - 2 (tile j - 2 STAGES); with 2 STAGES a
    // multiple of G that tile was the same group's, consumed before, so the
    // parity wait (which only tells adjacent phases apart) cannot match an
    // older phase; and use u + 2 cannot complete before this group releases
    // use u (the refill for use u + 1 waits for that release).
    static constexpr int ST_RAW = (200 * 1024) / STAGE_BYTES;
    static constexpr int ST_CAP = ST_RAW < G ? G : (ST_RAW > 8 ? 8 : ST_RAW);
    static constexpr int pick_stages()
    {
        for (int st = ST_CAP; st > G; --st)
            if ((2 * st) % G == 0)
                return st;
        return G;
    }
    static constexpr int SPG_RAW = (200 * 1024) / (STAGE_BYTES * G);
    static constexpr bool SHARED = SPG_RAW < 2;
    static constexpr int SPG = SHARED ? 1 : (SPG_RAW > 4 ? 4 : SPG_RAW);
    static constexpr int STAGES = SHARED ? pick_stages() : G * SPG;
    // the shared ring's parity argument needs 2 STAGES to be a multiple of G
    // (and at least one stage per group)
    static_assert(!SHARED || ((2 * STAGES) % G == 0 && STAGES >= G), "shared ring shape");
    static constexpr int THREADS = (CW + 2) * 32;      // + producer warp + helper warp
    static constexpr int NF = 2 * N + 1;               // float partials: ln-fraction, gradient
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 3 * STAGES * sizeof(uint64_t);
    // dynamic shared memory must leave room for the static arrays (< 16 KB)
    static constexpr bool FITS = SMEM <= 210 * 1024;
};

// Layout of the per-launch scratch (EvalArgs::partials) for a grid of G CTAs
// (component-major, so that the final sum reads each component coalesced):
//   pi  [2][G] int64   per-CTA sum of round(2^23 ln f) and of exponents
//   pf  [2N+1][G]      per-CTA float-float sums: ln-f remainders, gradient
//   mv  [2 kMaxWaves + 1]  M V and then V^H M V (double), by CTA 0's helper warp
//   flags              status bits of this launch (reset by the last CTA)
struct AmpScratch {
    long long *pi;
    float2 *pf;
    double *mv;
    int *flags;
};

__host__ __device__ inline AmpScratch amp_scratch(void *base, int grid)
{
    char *p = static_cast<char *>(base);
    AmpScratch s;
    s.pi = reinterpret_cast<long long *>(p);
    p += (size_t)grid * 2 * sizeof(long long);
    s.pf = reinterpret_cast<float2 *>(p);
    p += (size_t)grid * (2 * kMaxWaves + 1) * sizeof(float2);
    s.mv = reinterpret_cast<double *>(p);
    p += (2 * kMaxWaves + 2) * sizeof(double);
    s.flags = reinterpret_cast<int *>(p);
    return s;
}



// Per-wave coefficients, each duplicated into both halves of a packed pair.
struct alignas(16) WaveCoef {
    f2 vr, vi;  // Vhi
    f2 lr, li;  // Vlo
};

__device__ __forceinline__ f2 lds2(const float *p) { return *reinterpret_cast<const f2 *>(p); }

// Split c*a for both events of the pair (see the file comment): returns the
// remainders and the bit patterns of t, whose sum gives the high parts.
__device__ __forceinline__ f2 extract(f2 c, f2 a, f2 sg, unsigned &t0, unsigned &t1)
{
    const f2 t = fma2(c, a, sg);
    float x0, x1;
    upk2(t, x0, x1);
    t0 = __float_as_uint(x0);
    t1 = __float_as_uint(x1);
    return fma2(c, a, sub2(sg, t));
}

// S = sum_w V_w A_w of two events, exact up to its final rounding (see the
// file comment); amp(w, ar, ai) gives wave w's amplitudes of both events.
// SG = (sigma, sigma), unit = u_k, im_offset = 2 N bits(sigma).
template <int N, class AmpOf>
__device__ __forceinline__ void exact_sum2(AmpOf amp, const WaveCoef *Vc, f2 SG, float unit,
                                           unsigned im_offset, float (&sr)[2], float (&si)[2])
{
    // Re S = vr ar - vi ai ; Im S = vr ai + vi ar
    unsigned hR0 = 0, hR1 = 0, hI0 = 0, hI1 = 0;  // high parts (units of u_k)
    const f2 Z = 0ull;
    f2 lR = Z, lRm = Z, lI = Z;                    // remainders; lRm is subtracted
#pragma unroll
    for (int w = 0; w < N; ++w) {
        f2 ar, ai;
        amp(w, ar, ai);
        const WaveCoef cf = Vc[w];
        unsigned x0, x1;
        lR = add2(lR, extract(cf.vr, ar, SG, x0, x1));
        hR0 += x0;
        hR1 += x1;
        lRm = add2(lRm, extract(cf.vi, ai, SG, x0, x1));
        hR0 -= x0;
        hR1 -= x1;
        lI = add2(lI, extract(cf.vr, ai, SG, x0, x1));
        hI0 += x0;
        hI1 += x1;
        lI = add2(lI, extract(cf.vi, ar, SG, x0, x1));
        hI0 += x0;
        hI1 += x1;
        lR = fma2(cf.lr, ar, lR);
        lRm = fma2(cf.li, ai, lRm);
        lI = fma2(cf.lr, ai, fma2(cf.li, ar, lI));
    }
    const f2 hR = pk2((float)(int)hR0 * unit, (float)(int)hR1 * unit);
    const f2 hI = pk2((float)(int)(hI0 - im_offset) * unit, (float)(int)(hI1 - im_offset) * unit);
    upk2(add2(hR, sub2(lR, lRm)), sr[0], sr[1]);
    upk2(add2(hI, lI), si[0], si[1]);
}

// Sums of P values over the 32 lanes of a warp, every lane ending with the
// total of value `lane` of each block of 32 (x[32 b + lane]); the rest of x
// is left undefined. At each of the five levels a lane keeps one half of its
// remaining values, sends the other half to its partner and adds what it
// receives: 31 shuffles per 32 values instead of 5 per value.
template <int P>
__device__ __forceinline__ void warp_transpose_sum(float (&x)[P], int lane)
{
    constexpr int B = (P + 31) / 32;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i)
            v[i] = (32 * b + i < P) ? x[32 * b + i] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < o; ++i) {
                const float send = upper ? v[i] : v[i + o];
                const float keep = upper ? v[i + o] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        x[32 * b] = v[0];
    }
}

// V as float pairs Vhi + Vlo, duplicated for packed use; waves w >= n_waves
// (padding) get V = 0. One thread per wave.
__device__ __forceinline__ void wave_coef(const double *V, int n_waves, int w, WaveCoef &c)
{
    const bool on = w < n_waves;
    const double dr = on ? V[2 * w] : 0.0, di = on ? V[2 * w + 1] : 0.0;
    const float vr = __double2float_rn(dr), vi = __double2float_rn(di);
    const float lr = __double2float_rn(dr - (double)vr), li = __double2float_rn(di - (double)vi);
    c.vr = pk2(vr, vr);
    c.vi = pk2(vi, vi);
    c.lr = pk2(lr, lr);
    c.li = pk2(li, li);
}

// sigma = 1.5 2^k and u_k = 2^(k-23) with 2^(k-1) >= 1.25 sum_a |V_a|_1
// max_i |A_a(i)|_1 (margin for rounding); called by one whole warp, lane 0
// writes the results.
__device__ __forceinline__ void exact_scale(const double *V, const float *amax, int n_waves,
                                            int lane, float *sigma, float *unit)
{
    float b = 0.f;
    for (int w = lane; w < n_waves; w += 32) {
        const float v1 = fabsf(__double2float_ru(fabs(V[2 * w]))) +
                         fabsf(__double2float_ru(fabs(V[2 * w + 1])));
        b = fmaf(v1, amax[w], b);
    }
    b = warp_sum(b);
    if (lane == 0) {
        const float target = 2.5f * b;
        int k = -100;  // floor keeps u_k normal
        if (target > 0.f)
            k = max(k, ((__float_as_int(target) >> 23) & 0xff) - 126);  // target < 2^k
        if (!(target < 1e30f))
            k = 100;   // non-finite bound: the results will flag the domain error
        *sigma = 1.5f * ldexpf(1.0f, k);
        *unit = ldexpf(1.0f, k - 23);
    }
}

// WEIGHTS: instead of the NLL, write I / N_gen of every event to a.weights
// (the projection weights of the accepted MC events; L = 1), with no sums.
template <int N, int G, int L = 1, bool WEIGHTS = false>
__global__ void __launch_bounds__(AmpCfg<N, G, L>::THREADS, 1)
    nll_amp_kernel(const __grid_constant__ CUtensorMap map, const EvalArgs a, const int n_tiles,
                   int *work_flags)
{
    static_assert(!WEIGHTS || L == 1, "projection weights of a coherent sample");
    using C = AmpCfg<N, G, L>;
    constexpr int TE = C::TE, ROWS = C::ROWS, STAGES = C::STAGES, CW = C::CW;
    constexpr int GROUPS = C::GROUPS, GW = C::GW;
    constexpr int NF = C::NF;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *tiles = reinterpret_cast<float *>(smem_raw);
    // full[s] (owned stages) or full[(u & 1) STAGES + s] (shared): use u of
    // stage s; empty[s]: its release
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + (size_t)STAGES * C::STAGE_BYTES);
    uint64_t *empty = full + 2 * STAGES;

    __shared__ WaveCoef Vc[N];
    __shared__ double sV[2 * N];   // the helper warp's copy of V
    __shared__ float s_sigma, s_unit;
    __shared__ long long red_i[CW][2];
    __shared__ float red_f[CW][NF];
    __shared__ int s_flags;
    __shared__ int s_last;
    AmpScratch sc = amp_scratch(a.partials, gridDim.x);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tiles of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...; tile j goes
    // to group j % GROUPS and to stage stage_of(j) (see AmpCfg)
    const int n_my =
        (n_tiles > (int)blockIdx.x) ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t stage_tx = 2u * (uint32_t)a.n_waves * L * TE * 4u;
    auto stage_of = [](int j) {
        return C::SHARED ? j % STAGES : (j % GROUPS) * C::SPG + (j / GROUPS) % C::SPG;
    };
    auto use_of = [](int j) {
        return (uint32_t)(C::SHARED ? j / STAGES : (j / GROUPS) / C::SPG);
    };
    auto full_of = [&](int j) {
        return &full[(C::SHARED ? (use_of(j) & 1) * STAGES : 0) + stage_of(j)];
    };
    auto full_parity = [&](int j) { return C::SHARED ? (use_of(j) >> 1) & 1u : use_of(j) & 1u; };
    // tiles the producer issues (none when the timeout path is being tested)
    const int n_issue = a.stall_ns ? 0 : n_my;
    const unsigned long long wait_ns = a.stall_ns ? a.stall_ns : kWaitLimitNs;
    const int n_first = n_issue < STAGES ? n_issue : STAGES;  // first use of every stage
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&full[STAGES + s], 1);
            mbar_init(&empty[s], GW);
        }
        fence_barrier_init();
        s_flags = 0;
        // start streaming before the prologue below (its global loads take ~1 us)
        for (int j = 0; j < n_first; ++j) {
            mbar_arrive_expect_tx(full_of(j), stage_tx);
            tma_load_2d(tiles + (size_t)stage_of(j) * ROWS * TE, &map,
                        ((int)blockIdx.x + j * (int)gridDim.x) * TE, 0, full_of(j));
        }
    }
    // Rows of padded waves (n_waves < N) are never written by TMA: zero them
    // once so that they contribute nothing (their V is zero as well).
    for (int s = 0; s < STAGES; ++s)
        for (int i = 2 * a.n_waves * L * TE + threadIdx.x; i < ROWS * TE; i += blockDim.x)
            tiles[(size_t)s * ROWS * TE + i] = 0.f;
    // V may sit in host memory: these reads and those of the helper warp are
    // its only ones (one round trip each, concurrent with the first tiles)
    if (threadIdx.x < N)
        wave_coef(a.V, a.n_waves, threadIdx.x, Vc[threadIdx.x]);
    if (warp == 1)
        exact_scale(a.V, a.amax, a.n_waves, lane, &s_sigma, &s_unit);
    __syncthreads();

    int flags = 0;
    long long l_int = 0;      // sum of round(2^23 ln f)
    int eacc = 0;             // sum of exponents
    float l_frac = 0.f;       // sum of the remainders (units of 2^-23)

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer: one thread issues the TMA copies ----------------
            int j = n_first;
            for (; j < n_issue; ++j) {
                const int s = stage_of(j);
                const uint32_t u = use_of(j);
                if (u > 0 && !mbar_wait(&empty[s], (u & 1) ^ 1)) {
                    flags |= FLAG_TIMEOUT;
                    break;
                }
                mbar_arrive_expect_tx(full_of(j), stage_tx);
                tma_load_2d(tiles + (size_t)s * ROWS * TE, &map,
                            ((int)blockIdx.x + j * (int)gridDim.x) * TE, 0, full_of(j));
            }
            // no copy may still be landing in shared memory when the CTA exits
            // (the last STAGES tiles issued are the latest use of every stage)
            for (int q = (j > STAGES ? j - STAGES : 0); q < j; ++q) {
                if (!mbar_wait(full_of(q), full_parity(q)))
                    flags |= FLAG_TIMEOUT;
            }
        }
    } else if (warp <= CW) {
        // ---- consumers: group grp takes tiles j = grp, grp + GROUPS, ... ---
        const int cw = warp - 1;
        const int grp = cw / GW;
        const int ct = (cw % GW) * 32 + lane;  // thread within its group
        const float sigma = s_sigma, unit = s_unit;
        const f2 SG = pk2(sigma, sigma);
        // bits(t) - bits(sigma) summed over the 2N terms of Im S: remove the offset once
        const unsigned im_offset = 2u * (unsigned)N * __float_as_uint(sigma);
        float gs[2 * N];
#pragma unroll
        for (int c = 0; c < 2 * N; ++c)
            gs[c] = 0.f;
        int bad = 0;
        for (int j = grp; j < n_my; j += GROUPS) {
            const int s = stage_of(j);
            if (!mbar_wait(full_of(j), full_parity(j), wait_ns)) {
                flags |= FLAG_TIMEOUT;
                break;
            }
            const float *T = tiles + (size_t)s * ROWS * TE + 2 * ct;
            const int64_t ev0 = (int64_t)((int)blockIdx.x + j * (int)gridDim.x) * TE + 2 * ct;

            // component l of wave w sits at rows 2 (l n + w), 2 (l n + w) + 1
            // (padded waves w >= n carry V = 0: their products are exactly 0)
            const int comp_rows = 2 * a.n_waves * TE;
            // S of the two events of this thread for the component at Tl
            auto component_sum = [&](const float *Tl, float (&sr)[2], float (&si)[2]) {
                exact_sum2<N>(
                    [&](int w, f2 &ar, f2 &ai) {
                        ar = lds2(Tl + (2 * w) * TE);
                        ai = lds2(Tl + (2 * w + 1) * TE);
                    },
                    Vc, SG, unit, im_offset, sr, si);
            };
            // gs += conj(A) r for the component at Tl, r = S / I of the two events
            auto component_grad = [&](const float *Tl, float r0, float r1, float i0, float i1) {
#pragma unroll
                for (int w = 0; w < N; ++w) {
                    float a0, a1, b0, b1;
                    upk2(lds2(Tl + (2 * w) * TE), a0, a1);
                    upk2(lds2(Tl + (2 * w + 1) * TE), b0, b1);
                    // conj(A) r = (ar rr + ai ri) + i (ar ri - ai rr)
                    gs[2 * w] = fmaf(a0, r0, fmaf(b0, i0, gs[2 * w]));
                    gs[2 * w] = fmaf(a1, r1, fmaf(b1, i1, gs[2 * w]));
                    gs[2 * w + 1] = fmaf(a0, i0, fmaf(-b0, r0, gs[2 * w + 1]));
                    gs[2 * w + 1] = fmaf(a1, i1, fmaf(-b1, r1, gs[2 * w + 1]));
                }
            };
            float Sr[L][2], Si[L][2], rr[L][2], ri[L][2];
            if constexpr (L == 1) {
                component_sum(T, Sr[0], Si[0]);
            } else {
                // not unrolled: unrolled, the compiler holds every wave's V
                // coefficients across the components and spills
#pragma unroll 1
                for (int l = 0; l < L; ++l) {
                    float sr[2], si[2];
                    component_sum(T + l * comp_rows, sr, si);
#pragma unroll
                    for (int k = 0; k < L; ++k)
                        if (k == l) {
                            Sr[k][0] = sr[0];
                            Sr[k][1] = sr[1];
                            Si[k][0] = si[0];
                            Si[k][1] = si[1];
                        }
                }
            }
            if constexpr (WEIGHTS) {
                const float w0 = fmaf(Sr[0][0], Sr[0][0], Si[0][0] * Si[0][0]) * a.inv_ngen;
                const float w1 = fmaf(Sr[0][1], Sr[0][1], Si[0][1] * Si[0][1]) * a.inv_ngen;
                if (ev0 + 1 < a.n_events)
                    *reinterpret_cast<float2 *>(a.weights + ev0) = make_float2(w0, w1);
                else if (ev0 < a.n_events)
                    a.weights[ev0] = w0;
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&empty[s]);
                continue;
            }
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                float I = fmaf(Sr[0][e], Sr[0][e], Si[0][e] * Si[0][e]);
#pragma unroll
                for (int l = 1; l < L; ++l)
                    I = I + fmaf(Sr[l][e], Sr[l][e], Si[l][e] * Si[l][e]);
                const bool in = (ev0 + e) < a.n_events;
                const bool ok = (I > 0.f) && (I < INFINITY);
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    rr[l][e] = 0.f;
                    ri[l][e] = 0.f;
                }
                if (in) {
                    if (ok) {
                        int ex;
                        const float f = split_exponent(I, ex);
                        // 2^23 ln f = k + r exactly: k integer (|k| < 2^22), |r| <= 1/2
                        const float y = logf(f) * 8388608.0f;
                        const float t = y + 12582912.0f;  // 1.5 * 2^23: rounds y to an integer
                        l_int += __float_as_int(t) - 0x4B400000;
                        l_frac += y - (t - 12582912.0f);
                        eacc += ex;
                        const float rI = __frcp_rn(I);
#pragma unroll
                        for (int l = 0; l < L; ++l) {
                            rr[l][e] = Sr[l][e] * rI;
                            ri[l][e] = Si[l][e] * rI;
                        }
                    } else {
                        bad = 1;
                    }
                }
            }
            if constexpr (L == 1) {
                // from 32 waves on, the amplitudes are read again from shared
                // memory rather than held from the pass for S (4N registers,
                // which spilled: 0.5 KB per thread at 32 waves with four-warp
                // groups, 1.4 KB at 48); below, holding them is faster (24
                // waves: 3% slower with the re-read)
                if constexpr (N >= 32)
                    asm volatile("" ::: "memory");
                component_grad(T, rr[0][0], rr[0][1], ri[0][0], ri[0][1]);
            } else {
#pragma unroll 1
                for (int l = 0; l < L; ++l) {
                    float r0 = rr[0][0], r1 = rr[0][1], i0 = ri[0][0], i1 = ri[0][1];
#pragma unroll
                    for (int k = 1; k < L; ++k)
                        if (k == l) {
                            r0 = rr[k][0];
                            r1 = rr[k][1];
                            i0 = ri[k][0];
                            i1 = ri[k][1];
                        }
                    component_grad(T + l * comp_rows, r0, r1, i0, i1);
                }
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&empty[s]);
        }
        if (bad)
            flags |= FLAG_DOMAIN;

        // ---- per-warp reduction of this thread's sums (fixed order) ------
        const long long li = warp_sum(l_int);
        const long long ei = warp_sum((long long)eacc);
        if (lane == 0) {
            red_i[cw][0] = li;
            red_i[cw][1] = ei;
        }
        float fv[NF];
        fv[0] = l_frac;
#pragma unroll
        for (int c = 0; c < 2 * N; ++c)
            fv[1 + c] = gs[c];
        warp_transpose_sum<NF>(fv, lane);
#pragma unroll
        for (int b = 0; b < (NF + 31) / 32; ++b)
            if (32 * b + lane < NF)
                red_f[cw][32 * b + lane] = fv[32 * b];
    } else if (warp == CW + 1 && blockIdx.x == 0 && !WEIGHTS) {
        // ---- helper warp of CTA 0: M V and V^H M V in FP64 -------------
        // One row per lane; this overlaps the streaming of the data.
        const int Nw = a.n_waves;
        for (int i = lane; i < 2 * Nw; i += 32)
            sV[i] = a.V[i];
        __syncwarp();
        double nv = 0.0;
        for (int row = lane; row < Nw; row += 32) {
            double re = 0.0, im = 0.0;
            for (int b = 0; b < Nw; ++b) {
                const double mr = a.M[2 * (row * Nw + b)], mi = a.M[2 * (row * Nw + b) + 1];
                const double vr = sV[2 * b], vi = sV[2 * b + 1];
                re = fma(mr, vr, fma(-mi, vi, re));
                im = fma(mr, vi, fma(mi, vr, im));
            }
            sc.mv[2 * row] = re;
            sc.mv[2 * row + 1] = im;
            nv = fma(sV[2 * row], re, fma(sV[2 * row + 1], im, nv));  // Re(conj(V) (M V))
        }
        nv = warp_sum(nv);
        if (lane == 0)
            sc.mv[2 * kMaxWaves] = nv;
    }
    if constexpr (WEIGHTS) {
        if (flags)
            atomicOr(a.status, flags);
        return;
    }
    if (flags)
        atomicOr(&s_flags, flags);
    __syncthreads();

    // ---- block partial, fixed order over warps -------------------------
    if (threadIdx.x < 2) {
        long long v = 0;
        for (int w = 0; w < CW; ++w)
            v += red_i[w][threadIdx.x];
        sc.pi[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = v;
    }
    for (int c = threadIdx.x; c < NF; c += blockDim.x) {
        dfloat v = {0.f, 0.f};
        for (int w = 0; w < CW; ++w)
            v = df_add(v, dfloat{red_f[w][c], 0.f});
        sc.pf[(size_t)c * gridDim.x + blockIdx.x] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_flags)
            atomicOr(work_flags, s_flags);
        __threadfence();
        const unsigned t = atomicAdd(a.ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last)
        return;

    // ---- last CTA: deterministic final sum + normalisation term ---------
    // One warp per component (2N+1 float-float ones, then the 2 integer
    // ones): lane l adds CTAs l, l + 32, ... (coalesced loads, all issued
    // before the adds, with M V and the launch's flags: one L2 round trip),
    // then a fixed shuffle tree. (The partials are read with L2 loads after
    // the ticket, so no further fence is needed.)
    const int Nw = a.n_waves;
    const int G_ = gridDim.x;
    constexpr int NWARPS = C::THREADS / 32;
    constexpr int CPW = (NF + 2 + NWARPS - 1) / NWARPS;  // components per warp
    constexpr int QB = 5;                                 // loads per lane and component in flight
    dfloat *tot_f = reinterpret_cast<dfloat *>(tiles);                  // [NF]
    long long *tot_i = reinterpret_cast<long long *>(tot_f + NF);       // [2]
    double *smv = reinterpret_cast<double *>(tot_i + 2);                // [2N] M V, V^H M V
    const double mv_i = threadIdx.x < 2 * Nw ? __ldcg(&sc.mv[threadIdx.x])
                                             : threadIdx.x == 2 * Nw ? __ldcg(&sc.mv[2 * kMaxWaves])
                                                                      : 0.0;
    const int wf = __ldcg(work_flags);
    {
        // a partial is 8 bytes either way: a float pair (hi in the low word)
        // or an integer
        const unsigned long long *pf64 = reinterpret_cast<const unsigned long long *>(sc.pf);
        const unsigned long long *pi64 = reinterpret_cast<const unsigned long long *>(sc.pi);
        dfloat acc[CPW];
        long long iacc[CPW];
#pragma unroll
        for (int k = 0; k < CPW; ++k) {
            acc[k] = dfloat{0.f, 0.f};
            iacc[k] = 0;
        }
        for (int b0 = 0; b0 < G_; b0 += 32 * QB) {
            unsigned long long r[CPW][QB];
#pragma unroll
            for (int k = 0; k < CPW; ++k) {
                const int comp = warp + k * NWARPS;
                const unsigned long long *src =
                    comp < NF ? pf64 + (size_t)comp * G_ : pi64 + (size_t)(comp - NF) * G_;
#pragma unroll
                for (int q = 0; q < QB; ++q) {
                    const int b = b0 + lane + 32 * q;
                    r[k][q] = (b < G_ && comp < NF + 2) ? __ldcg(src + b) : 0ull;
                }
            }
#pragma unroll
            for (int k = 0; k < CPW; ++k) {
                if (warp + k * NWARPS < NF) {
#pragma unroll
                    for (int q = 0; q < QB; ++q)
                        acc[k] = df_add(acc[k], dfloat{__uint_as_float((unsigned)r[k][q]),
                                                       __uint_as_float((unsigned)(r[k][q] >> 32))});
                } else {
#pragma unroll
                    for (int q = 0; q < QB; ++q)
                        iacc[k] += (long long)r[k][q];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < CPW; ++k) {
            const int comp = warp + k * NWARPS;
            if (comp < NF) {
                const dfloat v = warp_sum(acc[k]);
                if (lane == 0)
                    tot_f[comp] = v;
            } else if (comp < NF + 2) {
                const long long v = warp_sum(iacc[k]);
                if (lane == 0)
                    tot_i[comp - NF] = v;
            }
        }
    }
    if (threadIdx.x <= 2 * Nw)
        smv[threadIdx.x] = mv_i;
    __syncthreads();
    const bool invalid = (wf & (FLAG_DOMAIN | FLAG_TIMEOUT)) != 0;
    for (int c = threadIdx.x; c < 2 * Nw + 1; c += blockDim.x) {  // padded waves excluded
        const dfloat v = tot_f[c];
        if (c > 0) {
            // gradient: - sum_i conj(A) S / I + (M V)
            if (a.grad)
                a.grad[c - 1] = invalid ? 0.0 : (smv[c - 1] - (double)v.hi) - (double)v.lo;
        } else {
            // ln sum: integer part and exponents are exact; the rest is small
            const long long li = tot_i[0], ei = tot_i[1];
            const double lnsum =
                fma((double)ei, kLn2, ((double)li + ((double)v.hi + (double)v.lo)) * 0x1p-23);
            double nll = smv[2 * Nw] - lnsum;
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
    }
    if (a.host_flag)
        __threadfence_system();  // this thread's results reach the host before the flag
    __syncthreads();
    if (threadIdx.x == 0) {
        *work_flags = 0;
        *a.ticket = 0u;
        if (a.host_flag)
            *reinterpret_cast<volatile unsigned long long *>(a.host_flag) =
                ((unsigned long long)a.seq << 32) | (unsigned)wf;
    }
}

// The last CTA keeps its sub-sums in its (then idle) stage buffers.
template <int N, int G, int L = 1>
constexpr bool finalize_fits(int grid)
{
    (void)grid;
    return (size_t)(2 * N + 3) * 8 + 8 * (2 * N + 1) <= AmpCfg<N, G, L>::SMEM &&
           AmpCfg<N, G, L>::THREADS > 2 * N;
}

}  // namespace

}  // namespace pwa
