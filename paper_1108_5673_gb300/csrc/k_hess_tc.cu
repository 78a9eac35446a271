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
    // TMA stages per consumer group (a stage's successive uses belong to one group)
    static constexpr int SPG =
        (kHGroups * (2 * STAGE_BYTES + JBYTES) + 1024 <= 210 * 1024) ? 2 : 1;
    static constexpr int STAGES = kHGroups * SPG;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + (size_t)kHGroups * JBYTES + 1024;
    static_assert(AROWS <= 128, "three BF16 terms of the parameters exceed M = 128");
    static_assert(NMMA % 16 == 0 && NMMA <= 128, "N of the MMA");
    static_assert(R % 8 == 0, "drain in 8-column steps");
    static_assert(KA % 1024 == 0 && STAGE_BYTES % 1024 == 0 && JBYTES % 1024 == 0,
                  "swizzle atoms must stay 1 KB aligned");
    static_assert(SMEM <= 220 * 1024, "shared memory");
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

__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x)
{
    const float s = hi + x;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

template <int NW>
__global__ void __launch_bounds__(kHThreads, 1)
    hess_tc_kernel(const __grid_constant__ CUtensorMap map, const float *__restrict__ amax,
                   const double *__restrict__ V, int n_waves, int64_t n_events, int n_tiles,
                   float2 *__restrict__ part, int *status)
{
    using C = HessTcCfg<NW>;
    constexpr int R = C::R, STAGES = C::STAGES, SPG = C::SPG;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    float *tiles = reinterpret_cast<float *>(base);
    const uint32_t jbase = smem_u32(base) + (uint32_t)STAGES * C::STAGE_BYTES;
    __shared__ uint64_t full[STAGES], empty[STAGES], jfull[kHGroups], jempty[kHGroups];
    __shared__ uint64_t accfull[2], accempty[2], g_done;
    __shared__ WaveCoef Vc[NW];
    __shared__ float s_sigma, s_unit;
    __shared__ uint32_t tmem_base;
    __shared__ int s_flags;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tiles of this CTA: blockIdx.x + j gridDim.x, j = 0 .. n_my - 1; tile j
    // goes to group j % kHGroups, to that group's stage and to its J buffer
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
        for (int g = 0; g < kHGroups; ++g) {
            mbar_init(&jfull[g], kHGW);
            mbar_init(&jempty[g], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accfull[b], 1);
            mbar_init(&accempty[b], kHDrain);
        }
        mbar_init(&g_done, 1);
        fence_barrier_init();
        s_flags = 0;
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
                const int g = j % kHGroups, ab = j & 1;
                if (!mbar_wait(&jfull[g], (uint32_t)(j / kHGroups) & 1)) {
                    ok = false;
                    break;
                }
                // accumulator ab is free once tile j - 2 has been drained
                if (j >= 2 && !mbar_wait(&accempty[ab], (uint32_t)((j >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t jb = jbase + (uint32_t)g * C::JBYTES;
#pragma unroll
                for (int ks = 0; ks < kHTE / 16; ++ks) {
                    // 16 events (32 bytes) per step, four steps per K-atom
                    const uint32_t a = jb + (uint32_t)(ks >> 2) * C::KA + (uint32_t)(ks & 3) * 32;
                    umma_bf16(tmem + (uint32_t)ab * kHAccCols, dK + (a >> 4), dK + (a >> 4), idesc,
                              ks > 0 ? 1u : 0u);
                }
                umma_commit(&jempty[g]);
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
        float hi[R], lo[R];
#pragma unroll
        for (int c = 0; c < R; ++c)
            hi[c] = lo[c] = 0.f;
        for (int j = 0; j < n_my; ++j) {
            const int ab = j & 1;
            if (!mbar_wait(&accfull[ab], (uint32_t)(j >> 1) & 1)) {
                flags |= FLAG_TIMEOUT;
                break;
            }
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
                for (int i = 0; i < 8; ++i) {
                    const float x1 = __uint_as_float(v1[i]), x2 = __uint_as_float(v2[i]);
                    two_sum_acc(hi[c0 + i], lo[c0 + i], m < 2 * R ? x1 + x2 : x1);
                }
            }
        }
        if (m < C::AROWS) {
            float2 *out = part + ((size_t)blockIdx.x * C::AROWS + m) * R;
#pragma unroll
            for (int c = 0; c < R; ++c)
                out[c] = make_float2(hi[c], lo[c]);
        }
    } else {
        // ---- consumers: group grp takes tiles j = grp, grp + kHGroups, ... --
        const int cw = warp - kHFirstCons, grp = cw / kHGW, wg = cw % kHGW;
        const int ct = wg * 32 + lane;                     // thread of the group: events 2 ct, 2 ct + 1
        const float sigma = s_sigma, unit = s_unit;
        const f2 SG = pk2(sigma, sigma);
        const unsigned im_offset = 2u * (unsigned)NW * __float_as_uint(sigma);
        // this warp's K-atom of the group's J buffer, this lane's 4 bytes of a row
        const uint32_t atom = jbase + (uint32_t)grp * C::JBYTES + (uint32_t)wg * C::KA;
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
            // the group's J buffer is free once the MMAs of its previous tile are done
            const uint32_t ju = (uint32_t)(j / kHGroups);
            if (ju > 0 && !mbar_wait(&jempty[grp], (ju - 1) & 1)) {
                flags |= FLAG_TIMEOUT;
                break;
            }
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
                mbar_arrive(&jfull[grp]);
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

// H[r][c] over the real parameters (Re V at 0..N-1, Im V at N..2N-1): one
// warp per entry, lane k adding the CTAs k, k + 32, ... in order, then a
// fixed shuffle tree. Entries (r, c) and (c, r) take the same terms (the pair
// ordered), so H is exactly symmetric; zero when a data intensity was not
// positive.
__global__ void hess_tc_finalize(const float2 *__restrict__ part, int grid, int NW, int N,
                                 const int *status, double *H)
{
    const int R = 2 * NW, AR = 3 * R, P = 2 * N;
    const int o = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (o >= P * P)
        return;
    int r = o / P, c = o % P;
    if (r > c) {
        const int t = r;
        r = c;
        c = t;
    }
    const int jp = r < N ? r : NW + (r - N), jq = c < N ? c : NW + (c - N);
    const size_t stride = (size_t)AR * R;
    const size_t i1 = (size_t)jp * R + jq, i2 = (size_t)(R + jp) * R + jq;
    const size_t i3 = (size_t)(2 * R + jp) * R + jq, i4 = (size_t)(2 * R + jq) * R + jp;
    double v = 0.0;
    for (int b = lane; b < grid; b += 32) {
        const float2 *pb = part + (size_t)b * stride;
        const float2 x1 = pb[i1], x2 = pb[i2], x3 = pb[i3], x4 = pb[i4];
        v += (((double)x1.x + x1.y) + ((double)x2.x + x2.y)) +
             (((double)x3.x + x3.y) + ((double)x4.x + x4.y));
    }
    v = warp_sum(v);
    if (lane == 0)
        H[o] = (*status & FLAG_DOMAIN) ? 0.0 : v;
}

template <int NW>
cudaError_t hess_tc_nw(const CUtensorMap *map, const Planes &d, const double *V, const float *amax,
                       double *partials, int grid, int *status, double *H, cudaStream_t s)
{
    using C = HessTcCfg<NW>;
    const int n_tiles = (int)((d.n + kHTE - 1) / kHTE);
    if (grid > n_tiles)
        grid = n_tiles;
    cudaError_t e = cudaFuncSetAttribute(hess_tc_kernel<NW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess)
        return e;
    float2 *part = reinterpret_cast<float2 *>(partials);
    hess_tc_kernel<NW><<<grid, kHThreads, C::SMEM, s>>>(*map, amax, V, d.n_waves, d.n, n_tiles,
                                                        part, status);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    const int P = 2 * d.n_waves;
    hess_tc_finalize<<<(P * P + 7) / 8, 256, 0, s>>>(part, grid, NW, d.n_waves, status, H);
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
    const int NW = hess_tc_nw_of(n_waves);
    return NW > 0 ? (size_t)grid * (6 * NW) * (2 * NW) : 0;
}

cudaError_t launch_hessian_tc(const CUtensorMap *map, const Planes &d, const double *V,
                              const float *amax, double *partials, int grid, int *status, double *H,
                              cudaStream_t s)
{
    if (d.n < 1)
        return cudaErrorInvalidValue;
    switch (hess_tc_nw_of(d.n_waves)) {
    case 4: return hess_tc_nw<4>(map, d, V, amax, partials, grid, status, H, s);
    case 8: return hess_tc_nw<8>(map, d, V, amax, partials, grid, status, H, s);
    case 12: return hess_tc_nw<12>(map, d, V, amax, partials, grid, status, H, s);
    case 16: return hess_tc_nw<16>(map, d, V, amax, partials, grid, status, H, s);
    case 20: return hess_tc_nw<20>(map, d, V, amax, partials, grid, status, H, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace pwa
