// FUMILI's Hessian approximation (Sec. 4, 5) on the tensor cores:
//   H = sum_i d_i d_i^T,  d_i = grad_p ln I_i = 2 (Re, Im) of conj(A_a(i)) S_i / I_i
// over p = (Re V_0..Re V_{N-1}, Im V_0..Im V_{N-1}), i.e. the contraction
// H = J^T J over the events of the event x parameter matrix J of the d_i.
//
// Per CTA (persistent, one per SM), tiles of 128 events stream in by TMA.
// Consumer groups (two warps, one tile each in turn) form S of two events per
// thread exactly as the direct form does (high parts of the products V_a A_a
// summed as integers, remainders in FP32), then d of both events, and split
// every entry into three BF16 terms d = b1 + b2 + b3 (8 + 8 + 8 significant
// bits; each remainder is exact in FP32, so the split leaves at most the last
// bits of b3). The tile is stored K-major (events along K, 64 per 128-byte
// swizzled row): rows 0..R-1 hold b1 of the R = 2 NW padded parameters (Re
// parts at rows 0..NW-1, Im parts at NW..2NW-1), rows R..2R-1 b2, rows
// 2R..3R-1 b3. One elected thread issues tcgen05.mma (kind::f16, BF16
// operands, FP32 accumulation in tensor memory) with M = 128 (A = rows 0..127
// of the tile, the rows past 3R unused), N = 2R (B = rows 0..2R-1: b1 and
// b2), K = 128 events:
//   D[m][n] = sum_i A_m(i) B_n(i),  A = [b1; b2; b3], B = [b1; b2],
// so that, with T[m][q] = D[m][q] + D[m][R + q] for m < 2R and D[m][q] else,
//   sum_i d_p d_q = T[p][q] + T[R + p][q] + T[2R + p][q] + T[2R + q][p]
// up to the dropped products b2 b3, b3 b2, b3 b3 (below 2^-23 |d_p d_q|).
// The accumulator (two of them, alternating tiles) is drained after every
// tile by four warps, one per lane quarter of tensor memory, into float-float
// sums per CTA; the tensor core's FP32 sums thus span 128 events. A second
// kernel adds the CTAs' sums in FP64 in a fixed order and assembles H.
//
// Buffers: the TMA stages belong to the consumer groups (two per group), so
// that a stage's successive uses are one group's tiles in order; the J
// buffers (two) are shared by the groups in tile order, tile j in buffer
// j % 2. A group may write tile j's J once the products of tile j - 2 are
// done: a drain warp publishes the count of finished tiles in shared memory
// (a count, unlike a barrier phase, cannot be mistaken for an older one when
// a group runs ahead).
//
// Padded waves (n_waves < NW) have zero rows in the tile (never written by
// TMA) and V = 0, hence d = 0. Events past the sample read the TMA fill value
// zero and get d = 0.
#include "amp_kernel.cuh"
#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int kHTE = 128;                                  // events per tile
constexpr int kHGroups = 4;                                // consumer groups
constexpr int kHGW = 2;                                    // warps per group
constexpr int kHDrain = 4;                                 // drain warps (lane quarters)
constexpr int kHFirstDrain = 2;                            // warp 0: TMA, warp 1: MMA
constexpr int kHFirstCons = kHFirstDrain + kHDrain;
constexpr int kHThreads = (kHFirstCons + kHGroups * kHGW) * 32;
constexpr uint32_t kHAccCols = 128;                        // column of the second accumulator
constexpr uint32_t kHTmemCols = 256;
constexpr int kHJB = 2;                                    // J buffers (tile j: j % kHJB)

template <int NW>
struct HessTcCfg {
    static constexpr int R = 2 * NW;                       // padded parameters
    static constexpr int AROWS = 3 * R;                    // b1, b2, b3 rows
    static constexpr int NMMA = 2 * R;                     // N of the MMA: the b1 and b2 rows
    static constexpr uint32_t KA = AROWS * 128;            // one K-atom: 64 events of every row
    // a tile's J buffer: two K-atoms, plus the rows past AROWS that the MMA
    // reads from the second atom (A has 128 rows)
    static constexpr uint32_t JBYTES = 2 * KA + (128 - AROWS) * 128;
    static constexpr uint32_t STAGE_BYTES = 2 * NW * kHTE * 4;
    // TMA stages per consumer group, as many as fit beside the J buffers (up
    // to three)
    static constexpr size_t smem_for(int spg)
    {
        return (size_t)kHGroups * spg * STAGE_BYTES + (size_t)kHJB * JBYTES + 1024;
    }
    static constexpr size_t kMax = 223 * 1024;
    static constexpr int SPG = smem_for(3) <= kMax ? 3 : smem_for(2) <= kMax ? 2 : 1;
    static constexpr int STAGES = kHGroups * SPG;
    static constexpr size_t SMEM = smem_for(SPG);
    static_assert(AROWS <= 128, "three BF16 terms of the parameters exceed M = 128");
    static_assert(NMMA % 16 == 0 && NMMA <= 128, "N of the MMA");
    static_assert(R % 8 == 0, "drain in 8-column steps");
    static_assert(KA % 1024 == 0 && STAGE_BYTES % 1024 == 0 && JBYTES % 1024 == 0,
                  "swizzle atoms must stay 1 KB aligned");
    static_assert(SMEM <= kMax, "shared memory");
};

// Byte offset of (row, byte b of the row) in a K-major operand with 128-byte
// swizzle: 128-byte rows in 8-row (1 KB) atoms, the 16-byte chunk index
// XOR-ed with the row within the atom.
__device__ __forceinline__ uint32_t sw128_off(int row, uint32_t b)
{
    return (uint32_t)(row >> 3) * 1024 + (uint32_t)(row & 7) * 128 +
           ((((b >> 4) ^ (uint32_t)(row & 7)) & 7) << 4) + (b & 15);
}

// Two floats (events e, e + 1) to a packed BF16 pair, event e in the low half
// (the lower address, i.e. the smaller K index).
__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ f2 bf16x2_to_f2(uint32_t b)
{
    return pk2(__uint_as_float(b << 16), __uint_as_float(b & 0xffff0000u));
}

__device__ __forceinline__ void sts32(uint32_t addr, uint32_t v)
{
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// d of both events at row `row` of the K-atom at `atom` (shared address):
// b1 at row, b2 at R + row, b3 at 2R + row; `cb` = this lane's byte in the row.
template <int R>
__device__ __forceinline__ void store_split(uint32_t atom, int row, uint32_t cb, f2 x)
{
    float x0, x1;
    upk2(x, x0, x1);
    uint32_t b = bf16x2_rn(x0, x1);
    f2 r = sub2(x, bf16x2_to_f2(b));
    sts32(atom + sw128_off(row, cb), b);
    upk2(r, x0, x1);
    b = bf16x2_rn(x0, x1);
    r = sub2(r, bf16x2_to_f2(b));
    sts32(atom + sw128_off(R + row, cb), b);
    upk2(r, x0, x1);
    sts32(atom + sw128_off(2 * R + row, cb), bf16x2_rn(x0, x1));
}

// (hi, lo) += x for two float-float sums at once (TwoSum of Knuth).
__device__ __forceinline__ void two_sum_acc2(f2 &hi, f2 &lo, f2 x)
{
    const f2 s = add2(hi, x);
    const f2 bb = sub2(s, hi);
    lo = add2(lo, add2(sub2(hi, sub2(s, bb)), sub2(x, bb)));
    hi = s;
}

// Wait until *count >= target (a count written by one thread of the CTA with
// release semantics); gives up after kWaitLimitNs and returns false.
__device__ __forceinline__ bool wait_count(const int *count, int target)
{
    const uint32_t a = smem_u32(count);
    int v;
    asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    if (v >= target)
        return true;
    const unsigned long long t0 = global_timer_ns();
    for (;;) {
        __nanosleep(64);
        asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
        if (v >= target)
            return true;
        if (global_timer_ns() - t0 > kWaitLimitNs)
            return false;
    }
}

template <int NW>
__global__ void __launch_bounds__(kHThreads, 1)
    hess_tc_kernel(const __grid_constant__ CUtensorMap map, const float *__restrict__ amax,
                   const double *__restrict__ V, int n_waves, int64_t n_events, int n_tiles,
                   double *__restrict__ part, int *status)
{
    using C = HessTcCfg<NW>;
    static_assert((size_t)C::AROWS * (C::R + 1) * 8 <= (size_t)kHJB * C::JBYTES,
                  "the CTA's sums fit in the J buffers");
    constexpr int R = C::R, STAGES = C::STAGES, SPG = C::SPG;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    float *tiles = reinterpret_cast<float *>(base);
    const uint32_t jbase = smem_u32(base) + (uint32_t)STAGES * C::STAGE_BYTES;
    __shared__ uint64_t full[STAGES], empty[STAGES], jfull[kHJB];
    __shared__ uint64_t accfull[2], accempty[2], g_done;
    __shared__ WaveCoef Vc[NW];
    __shared__ float s_sigma, s_unit;
    __shared__ uint32_t tmem_base;
    __shared__ int s_flags;
    __shared__ int s_done;    // tiles whose products are complete

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tiles of this CTA: blockIdx.x + j gridDim.x, j = 0 .. n_my - 1; tile j
    // goes to group j % kHGroups, to that group's stage and to J buffer j % kHJB
    const int n_my =
        (n_tiles > (int)blockIdx.x) ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t stage_tx = 2u * (uint32_t)n_waves * kHTE * 4u;
    auto stage_of = [](int j) { return (j % kHGroups) * SPG + (j / kHGroups) % SPG; };
    auto use_of = [](int j) { return (uint32_t)((j / kHGroups) / SPG); };
    const int n_first = n_my < STAGES ? n_my : STAGES;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kHGW);
        }
        for (int b = 0; b < kHJB; ++b)
            mbar_init(&jfull[b], kHGW);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accfull[b], 1);
            mbar_init(&accempty[b], kHDrain);
        }
        mbar_init(&g_done, 1);
        fence_barrier_init();
        s_flags = 0;
        s_done = 0;
        for (int j = 0; j < n_first; ++j) {
            mbar_arrive_expect_tx(&full[stage_of(j)], stage_tx);
            tma_load_2d(tiles + (size_t)stage_of(j) * (C::STAGE_BYTES / 4), &map,
                        ((int)blockIdx.x + j * (int)gridDim.x) * kHTE, 0, &full[stage_of(j)]);
        }
    }
    // rows of padded waves are never written by TMA: zero them once
    for (int s = 0; s < STAGES; ++s)
        for (int i = 2 * n_waves * kHTE + threadIdx.x; i < 2 * NW * kHTE; i += blockDim.x)
            tiles[(size_t)s * (C::STAGE_BYTES / 4) + i] = 0.f;
    if (threadIdx.x < NW)
        wave_coef(V, n_waves, threadIdx.x, Vc[threadIdx.x]);
    if (warp == 1)
        tmem_alloc(&tmem_base, kHTmemCols);
    if (warp == kHFirstDrain)
        exact_scale(V, amax, n_waves, lane, &s_sigma, &s_unit);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    int flags = 0;

    if (warp == 0) {
        // ---- producer: one thread issues the TMA copies --------------------
        if (lane == 0) {
            int j = n_first;
            for (; j < n_my; ++j) {
                const int s = stage_of(j);
                const uint32_t u = use_of(j);
                if (u > 0 && !mbar_wait(&empty[s], (u & 1) ^ 1)) {
                    flags |= FLAG_TIMEOUT;
                    break;
                }
                mbar_arrive_expect_tx(&full[s], stage_tx);
                tma_load_2d(tiles + (size_t)s * (C::STAGE_BYTES / 4), &map,
                            ((int)blockIdx.x + j * (int)gridDim.x) * kHTE, 0, &full[s]);
            }
            // no copy may still be landing in shared memory when the CTA exits
            for (int q = (j > STAGES ? j - STAGES : 0); q < j; ++q)
                if (!mbar_wait(&full[stage_of(q)], use_of(q) & 1))
                    flags |= FLAG_TIMEOUT;
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----------------------------------------------------
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_bf16(128, C::NMMA, 0, 0);
            const uint64_t dK = umma_desc_sw128(0, 16, 1024);
            bool ok = true;
            for (int j = 0; j < n_my; ++j) {
                const int b = j % kHJB, ab = j & 1;
                if (!mbar_wait(&jfull[b], (uint32_t)(j / kHJB) & 1)) {
                    ok = false;
                    break;
                }
                // accumulator ab is free once tile j - 2 has been drained
                if (j >= 2 && !mbar_wait(&accempty[ab], (uint32_t)((j >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t jb = jbase + (uint32_t)b * C::JBYTES;
#pragma unroll
                for (int ks = 0; ks < kHTE / 16; ++ks) {
                    // 16 events (32 bytes) per step, four steps per K-atom
                    const uint32_t a = jb + (uint32_t)(ks >> 2) * C::KA + (uint32_t)(ks & 3) * 32;
                    umma_bf16(tmem + (uint32_t)ab * kHAccCols, dK + (a >> 4), dK + (a >> 4), idesc,
                              ks > 0 ? 1u : 0u);
                }
                // on completion tile j's J buffer is free and its accumulator full
                umma_commit(&accfull[ab]);
            }
            umma_commit(&g_done);
            // tensor memory is released only after every product has finished
            if (!mbar_wait(&g_done, 0))
                ok = false;
            if (!ok)
                flags |= FLAG_TIMEOUT;
        }
    } else if (warp < kHFirstCons) {
        // ---- drain: lane quarter q of tensor memory, rows m = 32 q + lane ---
        const int q = warp & 3, m = q * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        f2 hi[R / 2], lo[R / 2];
#pragma unroll
        for (int c = 0; c < R / 2; ++c)
            hi[c] = lo[c] = 0ull;
        for (int j = 0; j < n_my; ++j) {
            const int ab = j & 1;
            if (!mbar_wait(&accfull[ab], (uint32_t)(j >> 1) & 1)) {
                flags |= FLAG_TIMEOUT;
                break;
            }
            if (warp == kHFirstDrain && lane == 0)  // tile j's J buffer may be rewritten
                asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_done)),
                             "r"(j + 1)
                             : "memory");
            tc_fence_after();
            const uint32_t acc = tmem + lane_addr + (uint32_t)ab * kHAccCols;
#pragma unroll
            for (int c0 = 0; c0 < R; c0 += 8) {
                uint32_t v1[8], v2[8];
                tmem_ld8(acc + c0, v1);
                tmem_ld8(acc + R + c0, v2);
                tmem_ld_wait();
                if (c0 + 8 >= R) {
                    // the last columns are in registers: the accumulator may be reused
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0)
                        mbar_arrive(&accempty[ab]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    f2 x = pk2(__uint_as_float(v1[2 * i]), __uint_as_float(v1[2 * i + 1]));
                    if (m < 2 * R)
                        x = add2(x, pk2(__uint_as_float(v2[2 * i]), __uint_as_float(v2[2 * i + 1])));
                    two_sum_acc2(hi[c0 / 2 + i], lo[c0 / 2 + i], x);
                }
            }
        }
        // ---- this CTA's share of H -------------------------------------
        // The rows T[m] go through shared memory (the J buffers are free once
        // the last tile is drained), then every entry p <= q of H takes its
        // four terms: T[p][q] + T[R + p][q] + T[2R + p][q] + T[2R + q][p]
        // (row indices of the J layout), summed in FP64 and stored with the
        // CTA index innermost.
        double *Td = reinterpret_cast<double *>(base + (size_t)STAGES * C::STAGE_BYTES);
        constexpr int RP = R + 1;  // padded row stride: rows in different banks
        if (m < C::AROWS) {
#pragma unroll
            for (int c = 0; c < R / 2; ++c) {
                float h0, h1, l0, l1;
                upk2(hi[c], h0, h1);
                upk2(lo[c], l0, l1);
                Td[m * RP + 2 * c] = (double)h0 + (double)l0;
                Td[m * RP + 2 * c + 1] = (double)h1 + (double)l1;
            }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kHDrain * 32) : "memory");
        const int P = 2 * n_waves;
        for (int rc = (warp - kHFirstDrain) * 32 + lane; rc < P * P; rc += kHDrain * 32) {
            const int r = rc / P, c = rc % P;
            if (r > c)
                continue;
            const int e = r * P - r * (r - 1) / 2 + (c - r);  // row-major upper triangle
            const int jp = r < n_waves ? r : NW + (r - n_waves);
            const int jq = c < n_waves ? c : NW + (c - n_waves);
            part[(size_t)e * gridDim.x + blockIdx.x] =
                (Td[jp * RP + jq] + Td[(R + jp) * RP + jq]) +
                (Td[(2 * R + jp) * RP + jq] + Td[(2 * R + jq) * RP + jp]);
        }
    } else {
        // ---- consumers: group grp takes tiles j = grp, grp + kHGroups, ... --
        const int cw = warp - kHFirstCons, grp = cw / kHGW, wg = cw % kHGW;
        const int ct = wg * 32 + lane;                     // thread of the group: events 2 ct, 2 ct + 1
        const float sigma = s_sigma, unit = s_unit;
        const f2 SG = pk2(sigma, sigma);
        const unsigned im_offset = 2u * (unsigned)NW * __float_as_uint(sigma);
        // this warp's K-atom of a J buffer, this lane's 4 bytes of a row
        const uint32_t atom0 = jbase + (uint32_t)wg * C::KA;
        const uint32_t cb = (uint32_t)lane * 4;
        int bad = 0;
        for (int j = grp; j < n_my; j += kHGroups) {
            const int s = stage_of(j);
            if (!mbar_wait(&full[s], use_of(j) & 1)) {
                flags |= FLAG_TIMEOUT;
                break;
            }
            const float *T = tiles + (size_t)s * (C::STAGE_BYTES / 4) + 2 * ct;
            f2 ar[NW], ai[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                ar[w] = lds2(T + (2 * w) * kHTE);
                ai[w] = lds2(T + (2 * w + 1) * kHTE);
            }
            // the amplitudes are in registers: the stage may be refilled
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&empty[s]);
            float sr[2], si[2];
            exact_sum2<NW>(
                [&](int w, f2 &x, f2 &y) {
                    x = ar[w];
                    y = ai[w];
                },
                Vc, SG, unit, im_offset, sr, si);
            const int64_t ev0 = (int64_t)((int)blockIdx.x + j * (int)gridDim.x) * kHTE + 2 * ct;
            float r[2] = {0.f, 0.f}, im[2] = {0.f, 0.f};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float I = fmaf(sr[e], sr[e], si[e] * si[e]);
                if (ev0 + e < n_events) {
                    if (I > 0.f && I < INFINITY) {
                        const float q = 2.f / I;
                        r[e] = sr[e] * q;
                        im[e] = si[e] * q;
                    } else {
                        bad = 1;
                    }
                }
            }
            const f2 rr = pk2(r[0], r[1]), ri = pk2(im[0], im[1]), nrr = pk2(-r[0], -r[1]);
            // J buffer j % kHJB is free once the products of tile j - kHJB are done
            if (j >= kHJB && !wait_count(&s_done, j - kHJB + 1)) {
                flags |= FLAG_TIMEOUT;
                break;
            }
            const uint32_t atom = atom0 + (uint32_t)(j % kHJB) * C::JBYTES;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                // 2 conj(A) S / I = (ar rr + ai ri) + i (ar ri - ai rr), rr + i ri = 2 S / I
                store_split<R>(atom, w, cb, fma2(ar[w], rr, mul2(ai[w], ri)));
                store_split<R>(atom, NW + w, cb, fma2(ar[w], ri, mul2(ai[w], nrr)));
            }
            // generic-proxy writes become visible to the tensor core, then signal
            fence_async_smem();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&jfull[j % kHJB]);
        }
        if (bad)
            flags |= FLAG_DOMAIN;
    }
    if (flags)
        atomicOr(&s_flags, flags);
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && s_flags)
        atomicOr(status, s_flags);
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kHTmemCols);
    }
}

// H[r][c] over the real parameters (Re V at 0..N-1, Im V at N..2N-1), one
// warp per entry of the upper triangle, written to both (r, c) and (c, r):
// lane k adds the CTAs k, k + 32, ... in order (all of its loads issued
// before the adds), then a fixed shuffle tree; zero when a data intensity
// was not positive. With async_or set, the status bits of the call are also
// OR-ed into *async_or.
constexpr int kFinMaxRounds = 8;   // CTAs up to 32 x 8

__global__ void hess_tc_finalize(const double *__restrict__ part, int grid, int N, const int *status,
                                 double *H, int *async_or)
{
    if (async_or && blockIdx.x == 0 && threadIdx.x == 0 && *status)
        atomicOr(async_or, *status);
    const int P = 2 * N;
    const int e = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (e >= P * (P + 1) / 2)
        return;
    int o = e, r = 0;
    while (o >= P - r) {
        o -= P - r;
        ++r;
    }
    const int c = r + o;
    const double *pe = part + (size_t)e * grid;
    double x[kFinMaxRounds];
#pragma unroll
    for (int k = 0; k < kFinMaxRounds; ++k) {
        const int b = lane + 32 * k;
        x[k] = b < grid ? pe[b] : 0.0;
    }
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < kFinMaxRounds; ++k)
        v += x[k];
    v = warp_sum(v);
    if (lane == 0) {
        const double h = (*status & FLAG_DOMAIN) ? 0.0 : v;
        H[(size_t)r * P + c] = h;
        H[(size_t)c * P + r] = h;
    }
}

template <int NW>
cudaError_t hess_tc_nw(const CUtensorMap *map, const Planes &d, const double *V, const float *amax,
                       double *partials, int grid, int *status, double *H, int *async_or,
                       cudaStream_t s)
{
    using C = HessTcCfg<NW>;
    const int n_tiles = (int)((d.n + kHTE - 1) / kHTE);
    if (grid > n_tiles)
        grid = n_tiles;
    if (grid > 32 * kFinMaxRounds)
        grid = 32 * kFinMaxRounds;
    cudaError_t e = cudaFuncSetAttribute(hess_tc_kernel<NW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess)
        return e;
    hess_tc_kernel<NW><<<grid, kHThreads, C::SMEM, s>>>(*map, amax, V, d.n_waves, d.n, n_tiles,
                                                        partials, status);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    const int P = 2 * d.n_waves, entries = P * (P + 1) / 2;
    hess_tc_finalize<<<(entries + 7) / 8, 256, 0, s>>>(partials, grid, d.n_waves, status, H,
                                                       async_or);
    return cudaGetLastError();
}

int hess_tc_nw_of(int n_waves)
{
    for (int p : {4, 8, 12, 16, 20})
        if (n_waves <= p)
            return p;
    return -1;
}

}  // namespace

bool hess_tc_available(int n_waves) { return n_waves >= 1 && hess_tc_nw_of(n_waves) > 0; }

int hess_tc_box_events() { return kHTE; }

size_t hess_tc_partials_doubles(int n_waves, int grid)
{
    const int P = 2 * n_waves;
    return hess_tc_nw_of(n_waves) > 0 ? (size_t)grid * (P * (P + 1) / 2) : 0;
}

cudaError_t launch_hessian_tc(const CUtensorMap *map, const Planes &d, const double *V,
                              const float *amax, double *partials, int grid, int *status, double *H,
                              int *async_or, cudaStream_t s)
{
    if (d.n < 1)
        return cudaErrorInvalidValue;
    switch (hess_tc_nw_of(d.n_waves)) {
    case 4: return hess_tc_nw<4>(map, d, V, amax, partials, grid, status, H, async_or, s);
    case 8: return hess_tc_nw<8>(map, d, V, amax, partials, grid, status, H, async_or, s);
    case 12: return hess_tc_nw<12>(map, d, V, amax, partials, grid, status, H, async_or, s);
    case 16: return hess_tc_nw<16>(map, d, V, amax, partials, grid, status, H, async_or, s);
    case 20: return hess_tc_nw<20>(map, d, V, amax, partials, grid, status, H, async_or, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace pwa
