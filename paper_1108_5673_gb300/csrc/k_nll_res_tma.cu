// Free masses and widths (the same NLL and gradients as k_nll_res.cu), with
// the direct form's data movement and arithmetic:
//   A_r(i) = BW(m_i; M_r, G_r) Y_r(i),  BW(m; M, G) = 1 / (M^2 - m^2 - i M G),
//   NLL = -sum_data ln |S_i|^2 + (1 / N_gen) sum_MC |S_j|^2,  S = sum_a V_a A_a,
//   dNLL/dV*_a = sum w_i conj(A_a(i)) S_i,
//   dNLL/dM_r  = sum w_i 2 Re(conj(S_i) V_r Y_r dBW/dM),  dBW/dM = -(2M - iG) BW^2,
//   dNLL/dG_r  = sum w_i 2 Re(conj(S_i) V_r Y_r dBW/dG),  dBW/dG = i M BW^2,
// with w_i = -1 / I_i for data events and 1 / N_gen for MC events.
//
// One persistent CTA per SM streams tiles of 192 events x (1 + 2n) rows (m,
// then Re/Im of Y_r for the free waves r < R and of A_a for the fixed waves)
// from both samples, the data tiles first, into a ring of shared-memory
// stages with TMA; two groups of three consumer warps take tiles in turn, each
// thread two adjacent events packed in FP32x2 registers:
//  * BW_r per event with the exact-pair denominator of the per-event kernel
//    (M^2, M G, (M G)^2 as float pairs, m^2 and D^2 split by FMA, a Newton
//    step of the reciprocal against the pair), then A_r = BW_r Y_r;
//  * S by the exact product split of the direct form: each product c a is
//    split against sigma = 1.5 2^k into a multiple of u_k (its bits summed as
//    an integer) and an exact remainder (summed in FP32); 2^(k-1) bounds
//    1.25 sum_a |V_a|_1 max |A_a|_1 over both samples, with |BW_r| <= 1/(M_r G_r)
//    for the free waves;
//  * ln I = e ln 2 + ln f, e and round(2^23 ln f) summed as integers; the MC
//    sum of I and all gradients in FP32 per thread, float-float per warp and
//    block, FP64 across blocks in block order (the last CTA, atomic ticket).
// Every wait is bounded (FLAG_TIMEOUT) so a stalled pipeline returns.
#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int kMaxFreeT = 8;

template <int NP, int RP>
struct ResTmaCfg {
    static constexpr int G = 2;                     // consumer groups
    static constexpr int GW = 3;                    // warps per group (7 warps in all: the
                                                    // register cap is then 255, not 168)
    static constexpr int CW = G * GW;
    static constexpr int TE = GW * 32 * 2;          // events per tile
    static constexpr int ROWS = 1 + 2 * NP;
    static constexpr uint32_t STAGE_BYTES = ROWS * TE * 4;
    static constexpr int SPG_RAW = (200 * 1024) / (STAGE_BYTES * G);
    static constexpr int SPG = SPG_RAW < 1 ? 1 : (SPG_RAW > 4 ? 4 : SPG_RAW);
    static constexpr int STAGES = G * SPG;
    static constexpr int THREADS = (CW + 1) * 32;      // + the producer warp
    static constexpr int NR = 4 + 2 * NP + 2 * RP;  // per-warp float partials
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 2 * STAGES * sizeof(uint64_t);
    // dynamic shared memory must leave room for the static arrays (< 8 KB)
    static constexpr bool FITS = SMEM <= 210 * 1024;
};

struct ResWave {
    f2 vr, vi, lr, li;  // V high and low parts, duplicated for the two events
};

struct ResFree {
    f2 m2h, m2l, gh, gl, g2h, g2l;  // M^2, M G, (M G)^2 as pairs
    float mf, wf;                   // M, G
};

__device__ __forceinline__ f2 lds2r(const float *p) { return *reinterpret_cast<const f2 *>(p); }

__device__ __forceinline__ f2 extract2(f2 c, f2 a, f2 sg, unsigned &t0, unsigned &t1)
{
    const f2 t = fma2(c, a, sg);
    float x0, x1;
    upk2(t, x0, x1);
    t0 = __float_as_uint(x0);
    t1 = __float_as_uint(x1);
    return fma2(c, a, sub2(sg, t));
}

__device__ __forceinline__ f2 neg2(f2 a) { return a ^ 0x8000000080000000ull; }

__device__ __forceinline__ f2 rcp2(f2 a)
{
    float x0, x1;
    upk2(a, x0, x1);
    return pk2(rcp_approx(x0), rcp_approx(x1));
}

template <int NP, int RP>
__global__ void __launch_bounds__(ResTmaCfg<NP, RP>::THREADS, 1)
    nll_res_tma_kernel(const __grid_constant__ CUtensorMap dmap, const __grid_constant__ CUtensorMap mmap,
                       const ResArgs a, const float *amax, int tiles_d, int tiles_m)
{
    using C = ResTmaCfg<NP, RP>;
    constexpr int TE = C::TE, ROWS = C::ROWS, STAGES = C::STAGES, GW = C::GW, CW = C::CW, NR = C::NR;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *tiles = reinterpret_cast<float *>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + (size_t)STAGES * C::STAGE_BYTES);
    uint64_t *empty = full + STAGES;

    __shared__ ResWave Vc[NP];
    __shared__ ResFree Fr[RP];
    __shared__ float s_sigma, s_unit;
    __shared__ long long red_i[CW][2];
    __shared__ float red_f[2][CW][NR];
    __shared__ int s_flags, s_last;

    const int N = a.n_waves, R = a.n_free;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = tiles_d + tiles_m;
    const int n_my =
        (n_tiles > (int)blockIdx.x) ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t stage_tx = (uint32_t)(1 + 2 * N) * TE * 4u;
    auto stage_of = [](int j) { return (j % C::G) * C::SPG + (j / C::G) % C::SPG; };
    auto use_of = [](int j) { return (uint32_t)((j / C::G) / C::SPG); };
    auto issue = [&](int j, int s) {
        const int t = (int)blockIdx.x + j * (int)gridDim.x;
        mbar_arrive_expect_tx(&full[s], stage_tx);
        if (t < tiles_d)
            tma_load_2d(tiles + (size_t)s * ROWS * TE, &dmap, t * TE, 0, &full[s]);
        else
            tma_load_2d(tiles + (size_t)s * ROWS * TE, &mmap, (t - tiles_d) * TE, 0, &full[s]);
    };
    const int n_first = n_my < STAGES ? n_my : STAGES;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], GW);
        }
        fence_barrier_init();
        s_flags = 0;
        for (int j = 0; j < n_first; ++j)
            issue(j, stage_of(j));
    }
    // rows of padded waves are never written by TMA: zero them once
    for (int s = 0; s < STAGES; ++s)
        for (int i = (1 + 2 * N) * TE + threadIdx.x; i < ROWS * TE; i += blockDim.x)
            tiles[(size_t)s * ROWS * TE + i] = 0.f;
    if (threadIdx.x < NP) {
        const int w = threadIdx.x;
        const bool on = w < N;
        const double dr = on ? a.V[2 * w] : 0.0, di = on ? a.V[2 * w + 1] : 0.0;
        const float vr = __double2float_rn(dr), vi = __double2float_rn(di);
        const float lr = __double2float_rn(dr - (double)vr), li = __double2float_rn(di - (double)vi);
        Vc[w] = ResWave{pk2(vr, vr), pk2(vi, vi), pk2(lr, lr), pk2(li, li)};
    }
    if (threadIdx.x >= 32 && threadIdx.x < 32 + RP) {
        const int r = threadIdx.x - 32;
        const double M = r < R ? a.mass[r] : 1.0, G = r < R ? a.width[r] : 1.0;
        auto pr = [](double v, f2 &h, f2 &l) {
            const float x = __double2float_rn(v), y = __double2float_rn(v - (double)x);
            h = pk2(x, x);
            l = pk2(y, y);
        };
        ResFree f;
        pr(M * M, f.m2h, f.m2l);
        pr(M * G, f.gh, f.gl);
        pr((M * G) * (M * G), f.g2h, f.g2l);
        f.mf = (float)M;
        f.wf = (float)G;
        Fr[r] = f;
    }
    if (warp == 2) {
        // 2^(k-1) >= 1.25 sum_a |V_a|_1 max |A_a|_1 over both samples; for a free
        // wave max |A_r|_1 <= max |Y_r|_1 / (M_r G_r) (|BW| peaks at m = M)
        float b = 0.f;
        for (int w = lane; w < N; w += 32) {
            const float v1 = fabsf(__double2float_ru(fabs(a.V[2 * w]))) +
                             fabsf(__double2float_ru(fabs(a.V[2 * w + 1])));
            float am = amax[w];
            if (w < R)
                am = __double2float_ru((double)am / (a.mass[w] * a.width[w]) * 1.001);
            b = fmaf(v1, am, b);
        }
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
            // ---- producer -------------------------------------------------------
            int j = n_first;
            for (; j < n_my; ++j) {
                const int s = stage_of(j);
                const uint32_t u = use_of(j);
                if (u > 0 && !mbar_wait(&empty[s], (u & 1) ^ 1)) {
                    flags |= FLAG_TIMEOUT;
                    break;
                }
                issue(j, s);
            }
            for (int q = (j > STAGES ? j - STAGES : 0); q < j; ++q)
                if (!mbar_wait(&full[stage_of(q)], use_of(q) & 1))
                    flags |= FLAG_TIMEOUT;
        }
    } else if (warp <= CW) {
        // ---- consumers: group grp takes tiles j = grp, grp + G, ... ----------
        const int cw = warp - 1;
        const int grp = cw / GW;
        const int ct = (cw % GW) * 32 + lane;
        const float sigma = s_sigma, unit = s_unit;
        const f2 SG = pk2(sigma, sigma), Z = 0ull, ONE = pk2(1.f, 1.f);
        const unsigned im_offset = 2u * (unsigned)NP * __float_as_uint(sigma);
        float gs[2 * NP];
        f2 gm[RP], gw[RP];
        long long l_int = 0;
        int eacc = 0;
        dfloat acc = {0.f, 0.f};  // data: remainders of 2^23 ln f; MC: sum of I
        int bad = 0;
        auto reset = [&]() {
#pragma unroll
            for (int c = 0; c < 2 * NP; ++c)
                gs[c] = 0.f;
#pragma unroll
            for (int r = 0; r < RP; ++r)
                gm[r] = gw[r] = Z;
            l_int = 0;
            eacc = 0;
            acc = dfloat{0.f, 0.f};
        };
        // per-warp sums of this thread's accumulators for a phase (fixed order)
        auto flush = [&](int ph) {
            const dfloat aw = warp_sum(acc);
            const long long li = warp_sum(l_int), ei = warp_sum((long long)eacc);
            if (lane == 0) {
                red_f[ph][cw][0] = aw.hi;
                red_f[ph][cw][1] = aw.lo;
                if (ph == 0) {
                    red_i[cw][0] = li;
                    red_i[cw][1] = ei;
                }
            }
#pragma unroll
            for (int c = 0; c < 2 * NP; ++c) {
                const float v = warp_sum(gs[c]);
                if (lane == 0)
                    red_f[ph][cw][4 + c] = v;
            }
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                float m0, m1, w0, w1;
                upk2(gm[r], m0, m1);
                upk2(gw[r], w0, w1);
                const float vm = warp_sum(m0 + m1), vw = warp_sum(w0 + w1);
                if (lane == 0) {
                    red_f[ph][cw][4 + 2 * NP + r] = vm;
                    red_f[ph][cw][4 + 2 * NP + RP + r] = vw;
                }
            }
        };
        reset();
        int phase = 0;
        for (int j = grp; j < n_my; j += C::G) {
            const int t = (int)blockIdx.x + j * (int)gridDim.x;
            const int ph = t < tiles_d ? 0 : 1;
            if (ph != phase) {  // every data tile of this CTA precedes its MC tiles
                flush(0);
                reset();
                phase = 1;
            }
            const int s = stage_of(j);
            if (!mbar_wait(&full[s], use_of(j) & 1)) {
                flags |= FLAG_TIMEOUT;
                break;
            }
            const float *T = tiles + (size_t)s * ROWS * TE + 2 * ct;
            const int64_t ev0 = (int64_t)(ph ? t - tiles_d : t) * TE + 2 * ct;
            const int64_t n_ph = ph ? a.n_mc : a.n_data;

            // free waves: BW_r(m) for the two events, computed where needed (in
            // the S pass and again in the gradient pass) rather than held in
            // registers across the pass over the waves
            const f2 m = lds2r(T);
            const f2 mm = mul2(m, m), me = fma2(m, m, neg2(mm));  // m^2 = mm + me exactly
            auto bw = [&](int r, f2 &br, f2 &bi) {
                const ResFree &f = Fr[r];
                const f2 D = add2(sub2(f.m2h, mm), sub2(f.m2l, me));
                // den = D^2 + (M G)^2 as the pair dh + dl (see the per-event kernel)
                const f2 p = mul2(D, D), pe = fma2(D, D, neg2(p));
                const f2 dh = add2(f.g2h, p), bb = sub2(dh, f.g2h);
                const f2 dl = add2(add2(add2(sub2(f.g2h, sub2(dh, bb)), sub2(p, bb)), pe), f.g2l);
                const f2 q0 = rcp2(dh);
                const f2 q = fma2(q0, fma2(neg2(dl), q0, fma2(neg2(dh), q0, ONE)), q0);
                br = mul2(D, q);
                bi = fma2(f.gh, q, mul2(f.gl, q));
            };
            // amplitude pair of wave w: A_w from the tile, or BW_w Y_w for a free wave
            auto amp = [&](int w, f2 &ar, f2 &ai, f2 &br, f2 &bi) {
                ar = lds2r(T + (1 + 2 * w) * TE);
                ai = lds2r(T + (2 + 2 * w) * TE);
                if (w < RP && w < R) {
                    bw(w, br, bi);
                    const f2 yr = ar, yi = ai;
                    ar = fma2(br, yr, neg2(mul2(bi, yi)));
                    ai = fma2(br, yi, mul2(bi, yr));
                }
            };
            // S, exact product split (Re S = vr ar - vi ai, Im S = vr ai + vi ar)
            unsigned hR0 = 0, hR1 = 0, hI0 = 0, hI1 = 0;
            f2 lR = Z, lRm = Z, lI = Z;
#pragma unroll
            for (int w = 0; w < NP; ++w) {
                f2 ar, ai, br, bi;
                amp(w, ar, ai, br, bi);
                const ResWave cf = Vc[w];
                unsigned x0, x1;
                lR = add2(lR, extract2(cf.vr, ar, SG, x0, x1));
                hR0 += x0;
                hR1 += x1;
                lRm = add2(lRm, extract2(cf.vi, ai, SG, x0, x1));
                hR0 -= x0;
                hR1 -= x1;
                lI = add2(lI, extract2(cf.vr, ai, SG, x0, x1));
                hI0 += x0;
                hI1 += x1;
                lI = add2(lI, extract2(cf.vi, ar, SG, x0, x1));
                hI0 += x0;
                hI1 += x1;
                lR = fma2(cf.lr, ar, lR);
                lRm = fma2(cf.li, ai, lRm);
                lI = fma2(cf.lr, ai, fma2(cf.li, ar, lI));
            }
            float Sr[2], Si[2], wr[2], wi[2];
            {
                const f2 hR = pk2((float)(int)hR0 * unit, (float)(int)hR1 * unit);
                const f2 hI = pk2((float)(int)(hI0 - im_offset) * unit,
                                  (float)(int)(hI1 - im_offset) * unit);
                upk2(add2(hR, sub2(lR, lRm)), Sr[0], Sr[1]);
                upk2(add2(hI, lI), Si[0], Si[1]);
            }
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                wr[e] = wi[e] = 0.f;
                if (ev0 + e < n_ph) {
                    const float I = fmaf(Sr[e], Sr[e], Si[e] * Si[e]);
                    if (ph == 0) {
                        if (I > 0.f && I < INFINITY) {
                            int ex;
                            const float f = split_exponent(I, ex);
                            const float y = logf(f) * 8388608.0f;
                            const float tt = y + 12582912.0f;
                            l_int += __float_as_int(tt) - 0x4B400000;
                            acc = df_add(acc, dfloat{y - (tt - 12582912.0f), 0.f});
                            eacc += ex;
                            const float rI = -__frcp_rn(I);
                            wr[e] = Sr[e] * rI;
                            wi[e] = Si[e] * rI;
                        } else {
                            bad = 1;
                        }
                    } else {
                        acc = df_add(acc, dfloat{I, 0.f});
                        wr[e] = Sr[e];
                        wi[e] = Si[e];
                    }
                }
            }
            const f2 WR = pk2(wr[0], wr[1]), WI = pk2(wi[0], wi[1]);
#pragma unroll
            for (int w = 0; w < NP; ++w) {
                f2 ar, ai, br, bi;
                amp(w, ar, ai, br, bi);
                // gradient in V: conj(A) (wr + i wi) = (ar wr + ai wi) + i (ar wi - ai wr)
                float a0, a1, b0, b1;
                upk2(ar, a0, a1);
                upk2(ai, b0, b1);
                gs[2 * w] = fmaf(a0, wr[0], fmaf(b0, wi[0], gs[2 * w]));
                gs[2 * w] = fmaf(a1, wr[1], fmaf(b1, wi[1], gs[2 * w]));
                gs[2 * w + 1] = fmaf(a0, wi[0], fmaf(-b0, wr[0], gs[2 * w + 1]));
                gs[2 * w + 1] = fmaf(a1, wi[1], fmaf(-b1, wr[1], gs[2 * w + 1]));
                // masses and widths: c = conj(w S) (V_r A_r BW_r) per event, then
                // dM += -4 M Re c - 2 G Im c, dG += -2 M Im c
                if (w < RP && w < R) {
                    const ResWave cf = Vc[w];
                    const f2 tr = fma2(cf.vr, ar, neg2(mul2(cf.vi, ai)));
                    const f2 ti = fma2(cf.vr, ai, mul2(cf.vi, ar));
                    const f2 ur = fma2(tr, br, neg2(mul2(ti, bi)));
                    const f2 ui = fma2(tr, bi, mul2(ti, br));
                    const f2 cr = fma2(WR, ur, mul2(WI, ui)), ci = fma2(WR, ui, neg2(mul2(WI, ur)));
                    const float Mf = Fr[w].mf, Gf = Fr[w].wf;
                    gm[w] = fma2(pk2(-4.f * Mf, -4.f * Mf), cr,
                                 fma2(pk2(-2.f * Gf, -2.f * Gf), ci, gm[w]));
                    gw[w] = fma2(pk2(-2.f * Mf, -2.f * Mf), ci, gw[w]);
                }
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&empty[s]);
        }
        if (bad)
            flags |= FLAG_DOMAIN;
        if (phase == 0) {  // this group saw no MC tile: its MC sums are zero
            flush(0);
            reset();
        }
        flush(1);
    }
    if (flags)
        atomicOr(&s_flags, flags);
    __syncthreads();

    // ---- block partials in warp order: [2][P] doubles per CTA ---------------
    const int P = a.pstride;  // 2 + 2N + 2R
    for (int item = threadIdx.x; item < 2 * P; item += blockDim.x) {
        const int ph = item / P, c = item % P;
        double v = 0.0;
        if (c == 0) {
            for (int w = 0; w < CW; ++w)
                v += (double)red_f[ph][w][0] + (double)red_f[ph][w][1];
            if (ph == 0) {
                long long li = 0;
                for (int w = 0; w < CW; ++w)
                    li += red_i[w][0];
                v = ((double)li + v) * 0x1p-23;   // sum of ln f
            }
        } else if (c == 1) {
            if (ph == 0) {
                long long ei = 0;
                for (int w = 0; w < CW; ++w)
                    ei += red_i[w][1];
                v = (double)ei;                    // sum of exponents
            }
        } else {
            const int k = c - 2;  // gradient V (2N), then dM (R), dG (R)
            const int col = k < 2 * N ? 4 + k : (k < 2 * N + R ? 4 + 2 * NP + (k - 2 * N)
                                                               : 4 + 2 * NP + RP + (k - 2 * N - R));
            for (int w = 0; w < CW; ++w)
                v += (double)red_f[ph][w][col];
        }
        a.partials[((size_t)blockIdx.x * 2 + ph) * P + c] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_flags)
            atomicOr(a.status, s_flags);
        __threadfence();
        const unsigned tk = atomicAdd(a.ticket, 1u);
        s_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last)
        return;
    // ---- last CTA: sums over CTAs in block order, FP64 -----------------------
    __threadfence();
    double *fin = reinterpret_cast<double *>(tiles);   // the ring is idle now
    for (int item = threadIdx.x; item < 2 * P; item += blockDim.x) {
        const int ph = item / P, c = item % P;
        double v = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b)
            v += __ldcg(a.partials + ((size_t)b * 2 + ph) * P + c);
        fin[item] = v;
    }
    __syncthreads();
    const int st = *(volatile int *)a.status;
    const bool dom = (st & FLAG_DOMAIN) != 0, tmo = (st & FLAG_TIMEOUT) != 0;
    const double ig = a.inv_ngen;
    if (threadIdx.x == 0) {
        const double lnsum = 0.69314718055994530942 * fin[1] + fin[0];
        a.out[0] = tmo ? NAN : dom ? INFINITY : -lnsum + ig * fin[P + 0];
        *a.ticket = 0u;
        if (a.done)
            atomicAdd(a.done, 1);
    }
    for (int c = threadIdx.x; c < 2 * N + 2 * R; c += blockDim.x)
        a.out[1 + c] = (dom || tmo) ? 0.0 : fin[2 + c] + ig * fin[P + 2 + c];
}

template <int NP, int RP>
cudaError_t launch_nr(const CUtensorMap *dmap, const CUtensorMap *mmap, const ResArgs &a,
                      const float *amax, int grid, cudaStream_t s)
{
    using C = ResTmaCfg<NP, RP>;
    static_assert(C::FITS, "the ring must fit");
    static_assert((size_t)2 * (2 + 2 * NP + 2 * RP) * 8 <= C::SMEM, "final sums must fit the ring");
    cudaError_t e = cudaFuncSetAttribute(nll_res_tma_kernel<NP, RP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess)
        return e;
    const int td = (int)((a.n_data + C::TE - 1) / C::TE), tm = (int)((a.n_mc + C::TE - 1) / C::TE);
    nll_res_tma_kernel<NP, RP><<<grid, C::THREADS, C::SMEM, s>>>(*dmap, *mmap, a, amax, td, tm);
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch_np(const CUtensorMap *dmap, const CUtensorMap *mmap, const ResArgs &a,
                      const float *amax, int grid, cudaStream_t s)
{
    if (a.n_free <= 4)
        return launch_nr<NP, 4>(dmap, mmap, a, amax, grid, s);
    return launch_nr<NP, kMaxFreeT>(dmap, mmap, a, amax, grid, s);
}

}  // namespace

int res_tma_box_events() { return ResTmaCfg<4, 4>::TE; }

bool res_tma_available(int n_waves, int n_free)
{
    return n_waves >= 1 && n_waves <= 32 && n_free >= 1 && n_free <= kMaxFreeT && n_free <= n_waves;
}

cudaError_t launch_nll_res_tma(const CUtensorMap *dmap, const CUtensorMap *mmap, const ResArgs &args,
                               const float *amax, int grid, cudaStream_t s)
{
    ResArgs a = args;
    a.pstride = 2 + 2 * a.n_waves + 2 * a.n_free;
    if (!res_tma_available(a.n_waves, a.n_free))
        return cudaErrorInvalidValue;
    const int N = a.n_waves;
    if (N <= 4)
        return launch_np<4>(dmap, mmap, a, amax, grid, s);
    if (N <= 8)
        return launch_np<8>(dmap, mmap, a, amax, grid, s);
    if (N <= 12)
        return launch_np<12>(dmap, mmap, a, amax, grid, s);
    if (N <= 16)
        return launch_np<16>(dmap, mmap, a, amax, grid, s);
    if (N <= 20)
        return launch_np<20>(dmap, mmap, a, amax, grid, s);
    if (N <= 24)
        return launch_np<24>(dmap, mmap, a, amax, grid, s);
    return launch_np<32>(dmap, mmap, a, amax, grid, s);
}

}  // namespace pwa
