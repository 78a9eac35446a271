// MC normalisation matrix on the tensor cores (the inner bracket of the
// second term of Eq. 3, built once per sample as Sec. 2 says it can be when
// masses and widths are fixed):
//
//   M[a][b] = (1/N_gen) sum_{j in accepted MC} conj(A_a(j)) A_b(j).
//
// With the real rows x_p(j), p = 2a (Re A_a) and 2a + 1 (Im A_a), this is the
// symmetric contraction over the events G = X X^T, G[p][q] = sum_j x_p(j)
// x_q(j), and Re M_ab = G[2a][2b] + G[2a+1][2b+1], Im M_ab = G[2a][2b+1] -
// G[2a+1][2b].
//
// Exact digits. Each wave a gets one power of two 2^r_a > 2 max_j (|Re A_a| +
// |Im A_a|) for the whole sample. Every float x of rows 2a, 2a+1 is written
// as five fixed-point digits x = sum_{s=1..5} t_s + rest, t_s = c_s 2^(r_a -
// 8s) with integers |c_s| <= 128 and |rest| <= 2^(r_a - 41): digit s is x's
// remainder rounded to the nearest multiple of 2^(r_a - 8s) (by adding and
// subtracting 1.5 2^(r_a - 8s + 23)), an exact float operation, and t_s has
// at most 8 significant bits, so it is an exact BF16 value. Any x with |x| >=
// 2^(r_a - 17) is a multiple of 2^(r_a - 40) and has rest = 0. A product of
// digits s and t of rows p and q is c c' 2^(r_p + r_q - 8(s + t)): within one
// accumulator entry (p, q) of one digit pair all products are integer
// multiples of one quantum and at most 2^14 of it, so the tensor cores' FP32
// sum over 512 events (at most 2^23 quanta) is exact.
//
// Digit blocks D_st[p][q] = sum_j t_s(p, j) t_t(q, j). The main MMA takes A =
// rows [X1; X2; X3] (digits 1-3 of every row, 3R <= 128 rows) and B = rows
// [X1; ...; X5] (5R columns): the blocks s <= 3, t <= 5, exact, drained every
// 512 events into float-float sums per CTA. The blocks with s >= 4, t <= 3
// are their transposes (D_ts[q][p] = D_st[p][q], exactly). A second MMA takes
// A = [X4; X5] and B = X4: the blocks (4,4) and (5,4) (and (4,5) as the
// transpose of (5,4)), below 2^-36 of the leading ones, accumulated in FP32
// over the whole launch (one-sided roundings of at most 2^-12 of their size
// per CTA). Every pair but (5,5) is kept: per event and real entry of G the
// error is at most 2^-41 (|x_p| 2^r_q [|x_q| < 2^(r_q - 17)] + |x_q| 2^r_p
// [|x_p| < 2^(r_p - 17)]) + 2^(r_p + r_q - 61), with unbiased signs apart
// from the last term.
//
// Per CTA (persistent, one per SM): a TMA warp streams 64-event tiles of the
// 2N MC planes; four consumer warps (tile j to warp j % 4, each with two TMA
// stages and one digit buffer of its own) write the digits K-major with
// 128-byte swizzle (rows (s - 1) R + p, one 64-event K-atom); one thread
// issues the two MMAs (kind::f16, M = 128, K = 16; four steps per tile), the
// main one into one of two accumulators in tensor memory (alternating every
// eight tiles); eight drain warps (two per lane quarter, half of the columns
// each) add the main accumulator into float-float sums. The CTA's share of M
// goes to global memory with the CTA index innermost; norm_tc_finalize adds
// the CTAs in a fixed order, divides by N_gen and fills the Hermitian matrix.
#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int kNTE = 64;         // events per tile (one K-atom)
constexpr int kNCons = 4;        // consumer warps
constexpr int kNSPC = 2;         // TMA stages per consumer warp
constexpr int kNDrain = 8;       // drain warps (warps 4..11: lane quarter = warp % 4)
constexpr int kNFirstDrain = 4;
constexpr int kNWarps = 14;      // 0 TMA, 1 MMA, 2-3 and 12-13 consumers, 4-11 drain
constexpr int kNThreads = kNWarps * 32;
constexpr int kNDigits = 5;
constexpr int kNPeriod = 8;      // tiles per accumulation period (512 events: sums < 2^23)
constexpr uint32_t kNTmemCols = 512;
constexpr int kNFinMaxRounds = 8;    // CTAs up to 32 x 8

__device__ __forceinline__ int consumer_index(int warp)
{
    return warp < kNFirstDrain ? warp - 2 : warp - (kNFirstDrain + kNDrain) + 2;
}

constexpr int round_up16(int x) { return (x + 15) / 16 * 16; }
constexpr int round_up32(int x) { return (x + 31) / 32 * 32; }
constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <int NW>
struct NormTcCfg {
    static constexpr int R = 2 * NW;                    // real rows (padded waves)
    static constexpr int N1 = round_up16(kNDigits * R); // main MMA: B = digits 1-5
    static constexpr int N2 = round_up16(R);            // second MMA: B = digit 4
    // buffer rows: the digits, the main B operand's padding, and the 128 rows
    // the second MMA's A operand reads from row 3R on
    static constexpr int BUFROWS = cmax(cmax(N1, 3 * R + 128), 128);
    static constexpr uint32_t JBYTES = BUFROWS * 128;   // one 64-event K-atom of every row
    static constexpr uint32_t STAGE_BYTES = R * kNTE * 4;
    static constexpr int STAGES = kNCons * kNSPC;
    static constexpr uint32_t ACC1 = round_up32(N1);    // column of the second main accumulator
    static constexpr uint32_t ACCX = 2 * ACC1;          // column of the small-block accumulator
    static constexpr size_t SMEM = (size_t)kNCons * JBYTES + (size_t)STAGES * STAGE_BYTES + 1024;
    // the CTA's sums as doubles, T[3R][R], U[3R][R] and X[2R][R], reuse the digit buffers
    static constexpr size_t SUMS_BYTES = (size_t)8 * R * R * sizeof(double);
    static_assert(3 * R <= 128, "digits 1-3 of every row fill M = 128");
    static_assert(N1 <= 256 && N2 <= 256, "N of the MMA");
    static_assert(ACCX + N2 <= kNTmemCols, "tensor memory");
    static_assert(NW % 4 == 0, "drain in 4-column steps");
    static_assert(JBYTES % 1024 == 0 && STAGE_BYTES % 1024 == 0 && (3 * R) % 8 == 0,
                  "swizzle atoms stay 1 KB aligned");
    static_assert(SMEM <= 227 * 1024, "shared memory");
    static_assert(SUMS_BYTES <= (size_t)kNCons * JBYTES, "sums fit in the digit buffers");
};

// Byte offset of (row, byte b of the row) in a K-major operand with 128-byte
// swizzle: 128-byte rows in 8-row (1 KB) atoms, the 16-byte chunk index
// XOR-ed with the row within the atom.
__device__ __forceinline__ uint32_t sw128(int row, uint32_t b)
{
    return (uint32_t)(row >> 3) * 1024 + (uint32_t)(row & 7) * 128 +
           ((((b >> 4) ^ (uint32_t)(row & 7)) & 7) << 4) + (b & 15);
}

// Two floats (events e, e + 1) to a packed BF16 pair, event e in the low
// half (the smaller K index). The inputs are exact BF16 values here.
__device__ __forceinline__ uint32_t to_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ f2 lds2_f2(const float *p) { return *reinterpret_cast<const f2 *>(p); }

__device__ __forceinline__ void st_shared_u32(uint32_t addr, uint32_t v)
{
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}

// (hi, lo) += x for two float-float sums at once (Knuth's TwoSum).
__device__ __forceinline__ void two_sum2(f2 &hi, f2 &lo, f2 x)
{
    const f2 s = add2(hi, x);
    const f2 bb = sub2(s, hi);
    lo = add2(lo, add2(sub2(hi, sub2(s, bb)), sub2(x, bb)));
    hi = s;
}

// The scale of wave a's digits: r = floor(log2 amax) + 2 (so that every |x| <
// 2^(r - 1)), clamped below at -35 (the quanta of the exact digit pairs stay
// normal floats: r_p + r_q - 48 >= -118); a wave that is zero throughout gets
// r = 0. Returns 1.5 2^(r + 15), the rounding constant of the first digit.
__device__ __forceinline__ float first_digit_constant(float amax)
{
    int r = 0;
    if (amax > 0.f) {
        const int ex = ((__float_as_int(amax) >> 23) & 0xff) - 127;  // subnormal: -127
        r = max(ex + 2, -35);
    }
    return 1.5f * ldexpf(1.0f, r + 15);
}

// NW columns (this thread's half of a block) of its lane's row at `taddr`.
template <int NW>
__device__ __forceinline__ void tmem_row_half(uint32_t taddr, uint32_t (&v)[NW])
{
#pragma unroll
    for (int c4 = 0; c4 < NW / 4; ++c4) {
        uint32_t r4[4];
        tmem_ld4(taddr + (uint32_t)(4 * c4), r4);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            v[4 * c4 + i] = r4[i];
    }
}

template <int NW>
__global__ void __launch_bounds__(kNThreads, 1)
    norm_tc_kernel(const __grid_constant__ CUtensorMap map, const float *__restrict__ amax,
                   int n_waves, int n_tiles, double *__restrict__ part, int *status)
{
    using C = NormTcCfg<NW>;
    constexpr int R = C::R, STAGES = C::STAGES;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const uint32_t jbase = smem_u32(base);
    float *stages = reinterpret_cast<float *>(base + (size_t)kNCons * C::JBYTES);
    __shared__ uint64_t full[STAGES], empty[STAGES], jfull[kNCons], jempty[kNCons];
    __shared__ uint64_t accfull[2], accempty[2], g_done;
    __shared__ float s_sig[R];
    __shared__ uint32_t tmem_base;
    __shared__ int s_flags;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tiles of this CTA: blockIdx.x + j gridDim.x, j < n_my; tile j goes to
    // consumer j % kNCons, to its stage (j / kNCons) % kNSPC and its buffer
    const int n_my =
        (n_tiles > (int)blockIdx.x) ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t stage_tx = 2u * (uint32_t)n_waves * kNTE * 4u;
    auto stage_of = [](int j) { return (j % kNCons) * kNSPC + (j / kNCons) % kNSPC; };
    auto use_of = [](int j) { return (uint32_t)((j / kNCons) / kNSPC); };
    const int n_first = n_my < STAGES ? n_my : STAGES;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int c = 0; c < kNCons; ++c) {
            mbar_init(&jfull[c], 1);
            mbar_init(&jempty[c], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accfull[b], 1);
            mbar_init(&accempty[b], kNDrain);
        }
        mbar_init(&g_done, 1);
        fence_barrier_init();
        s_flags = 0;
        for (int j = 0; j < n_first; ++j) {
            mbar_arrive_expect_tx(&full[stage_of(j)], stage_tx);
            tma_load_2d(stages + (size_t)stage_of(j) * (C::STAGE_BYTES / 4), &map,
                        ((int)blockIdx.x + j * (int)gridDim.x) * kNTE, 0, &full[stage_of(j)]);
        }
    }
    // rows of padded waves are never written by TMA: zero them once; so are
    // the buffer rows past the digits, which the MMAs read as padding
    for (int s = 0; s < STAGES; ++s)
        for (int i = 2 * n_waves * kNTE + threadIdx.x; i < R * kNTE; i += blockDim.x)
            stages[(size_t)s * (C::STAGE_BYTES / 4) + i] = 0.f;
    for (int c = 0; c < kNCons; ++c)
        for (uint32_t i = kNDigits * R * 32 + threadIdx.x; i < C::JBYTES / 4; i += blockDim.x)
            reinterpret_cast<uint32_t *>(base + (size_t)c * C::JBYTES)[i] = 0u;
    if (threadIdx.x < R)
        s_sig[threadIdx.x] =
            (threadIdx.x / 2 < n_waves) ? first_digit_constant(amax[threadIdx.x / 2]) : 1.5f * 32768.f;
    if (warp == 1)
        tmem_alloc(&tmem_base, kNTmemCols);
    fence_async_smem();
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
                tma_load_2d(stages + (size_t)s * (C::STAGE_BYTES / 4), &map,
                            ((int)blockIdx.x + j * (int)gridDim.x) * kNTE, 0, &full[s]);
            }
            // no copy may still be landing in shared memory when the CTA exits
            for (int q = (j > STAGES ? j - STAGES : 0); q < j; ++q)
                if (!mbar_wait(&full[stage_of(q)], use_of(q) & 1))
                    flags |= FLAG_TIMEOUT;
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----------------------------------------------------
        if (lane == 0) {
            const uint32_t id1 = umma_idesc_bf16(128, C::N1, 0, 0);
            const uint32_t id2 = umma_idesc_bf16(128, C::N2, 0, 0);
            const uint64_t dK = umma_desc_sw128(0, 16, 1024);
            const uint32_t row4 = 3u * R * 128u;  // byte offset of digit 4's rows
            bool ok = true;
            for (int j = 0; j < n_my; ++j) {
                const int c = j % kNCons;
                if (!mbar_wait(&jfull[c], (uint32_t)(j / kNCons) & 1)) {
                    ok = false;
                    break;
                }
                const int P = j / kNPeriod, ab = P & 1;
                const bool first = (j % kNPeriod) == 0;
                // accumulator ab is free once period P - 2 has been drained
                if (first && P >= 2 && !mbar_wait(&accempty[ab], (uint32_t)((P >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t jb = jbase + (uint32_t)c * C::JBYTES;
#pragma unroll
                for (int ks = 0; ks < kNTE / 16; ++ks) {
                    const uint32_t a = jb + (uint32_t)ks * 32;  // 16 events = 32 bytes of a row
                    umma_bf16(tmem + (uint32_t)ab * C::ACC1, dK + (a >> 4), dK + (a >> 4), id1,
                              (first && ks == 0) ? 0u : 1u);
                    umma_bf16(tmem + C::ACCX, dK + ((a + row4) >> 4), dK + ((a + row4) >> 4), id2,
                              (j == 0 && ks == 0) ? 0u : 1u);
                }
                // on completion the consumer's buffer is free again
                umma_commit(&jempty[c]);
                if ((j % kNPeriod) == kNPeriod - 1 || j == n_my - 1)
                    umma_commit(&accfull[ab]);
            }
            umma_commit(&g_done);
            // tensor memory is released only after every product has finished
            if (!mbar_wait(&g_done, 0))
                ok = false;
            if (!ok)
                flags |= FLAG_TIMEOUT;
        }
    } else if (warp >= kNFirstDrain && warp < kNFirstDrain + kNDrain) {
        // ---- drain: lane quarter q, rows m = 32 q + lane, columns half h ----
        // Row m < 3R is digit s = m / R + 1 of row p = m % R. T1 sums the
        // blocks t = 1..3 (columns (t - 1) R ...), T2 the blocks t = 4, 5.
        const int q = warp & 3, h = (warp - kNFirstDrain) >> 2, m = q * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        constexpr int HC = NW / 2;  // packed column pairs per thread and block (NW columns)
        f2 h1[HC], l1[HC], h2[HC], l2[HC];
#pragma unroll
        for (int c = 0; c < HC; ++c)
            h1[c] = l1[c] = h2[c] = l2[c] = 0ull;
        const int n_periods = (n_my + kNPeriod - 1) / kNPeriod;
        for (int P = 0; P < n_periods; ++P) {
            const int ab = P & 1;
            if (!mbar_wait(&accfull[ab], (uint32_t)(P >> 1) & 1)) {
                flags |= FLAG_TIMEOUT;
                break;
            }
            tc_fence_after();
            const uint32_t acc = tmem + lane_addr + (uint32_t)ab * C::ACC1 + (uint32_t)(h * NW);
#pragma unroll
            for (int t = 1; t <= kNDigits; ++t) {
                uint32_t v[NW];
                tmem_row_half<NW>(acc + (uint32_t)((t - 1) * R), v);
                tmem_ld_wait();
                if (t == kNDigits) {
                    // every column is in registers: the accumulator may be reused
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0)
                        mbar_arrive(&accempty[ab]);
                }
#pragma unroll
                for (int c = 0; c < HC; ++c) {
                    const f2 x = pk2(__uint_as_float(v[2 * c]), __uint_as_float(v[2 * c + 1]));
                    if (t <= 3)
                        two_sum2(h1[c], l1[c], x);
                    else
                        two_sum2(h2[c], l2[c], x);
                }
            }
        }
        // ---- this CTA's share of M -----------------------------------------
        // T[s][p][q] = sum_{t <= 5} D_st[p][q], U[s][p][q] = sum_{t = 4, 5}
        // D_st[p][q] (s <= 3) and X[s - 4][p][q] = D_s4[p][q] (s = 4, 5) go
        // through shared memory (the digit buffers are free once the last
        // period is drained: every MMA has completed); then
        //   G[p][q] = sum_s T[s][p][q] + sum_s U[s][q][p]
        //           + X[0][p][q] + X[1][p][q] + X[1][q][p].
        double *Ts = reinterpret_cast<double *>(base);
        double *Us = Ts + 3 * R * R;
        double *Xs = Us + 3 * R * R;
        if (m < 3 * R) {
#pragma unroll
            for (int c = 0; c < HC; ++c) {
                float a0, a1, b0, b1, c0, c1, d0, d1;
                upk2(h1[c], a0, a1);
                upk2(l1[c], b0, b1);
                upk2(h2[c], c0, c1);
                upk2(l2[c], d0, d1);
                const int col = h * NW + 2 * c;
                const double u0 = (double)c0 + (double)d0, u1 = (double)c1 + (double)d1;
                Ts[m * R + col] = ((double)a0 + (double)b0) + u0;
                Ts[m * R + col + 1] = ((double)a1 + (double)b1) + u1;
                Us[m * R + col] = u0;
                Us[m * R + col + 1] = u1;
            }
        }
        {
            // the small blocks, accumulated over the whole launch
            uint32_t v[NW];
            tmem_row_half<NW>(tmem + lane_addr + C::ACCX + (uint32_t)(h * NW), v);
            tmem_ld_wait();
            if (m < 2 * R) {
#pragma unroll
                for (int c = 0; c < NW; ++c)
                    Xs[m * R + h * NW + c] = (double)__uint_as_float(v[c]);
            }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kNDrain * 32) : "memory");
        // entries e of the upper triangle (a <= b) of M, real and imaginary parts
        const int E = n_waves * (n_waves + 1) / 2;
        for (int ec = (warp - kNFirstDrain) * 32 + lane; ec < 2 * E; ec += kNDrain * 32) {
            const int e = ec >> 1, comp = ec & 1;
            int a = 0, o = e;
            while (o >= n_waves - a) {
                o -= n_waves - a;
                ++a;
            }
            const int b = a + o;
            auto G = [&](int p, int r) {
                double v = Xs[p * R + r] + (Xs[(R + p) * R + r] + Xs[(R + r) * R + p]);
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    v += Ts[(d * R + p) * R + r] + Us[(d * R + r) * R + p];
                return v;
            };
            const double v = comp == 0 ? G(2 * a, 2 * b) + G(2 * a + 1, 2 * b + 1)
                                       : G(2 * a, 2 * b + 1) - G(2 * a + 1, 2 * b);
            part[(size_t)ec * gridDim.x + blockIdx.x] = v;
        }
    } else {
        // ---- consumers: warp c takes tiles j = c, c + kNCons, ... ----------
        const int c = consumer_index(warp);
        const uint32_t jb = jbase + (uint32_t)c * C::JBYTES;
        const uint32_t cb = (uint32_t)lane * 4;  // this lane's events 2 lane, 2 lane + 1
        const f2 STEP = pk2(0x1p-8f, 0x1p-8f);
        for (int j = c; j < n_my; j += kNCons) {
            const int st = stage_of(j);
            if (!mbar_wait(&full[st], use_of(j) & 1)) {
                flags |= FLAG_TIMEOUT;
                break;
            }
            const float *T = stages + (size_t)st * (C::STAGE_BYTES / 4) + 2 * lane;
            f2 x[R];
#pragma unroll
            for (int p = 0; p < R; ++p)
                x[p] = lds2_f2(T + p * kNTE);
            // the amplitudes are in registers: the stage may be refilled
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&empty[st]);
            // this warp's buffer is free once the products of its previous tile are done
            const int k = j / kNCons;
            if (k > 0 && !mbar_wait(&jempty[c], (uint32_t)(k - 1) & 1)) {
                flags |= FLAG_TIMEOUT;
                break;
            }
#pragma unroll
            for (int p = 0; p < R; ++p) {
                f2 z = x[p];
                f2 S = pk2(s_sig[p], s_sig[p]);
#pragma unroll
                for (int d = 0; d < kNDigits; ++d) {
                    const f2 t = sub2(add2(z, S), S);  // z rounded to a multiple of 2^(r - 8(d+1))
                    z = sub2(z, t);                    // exact remainder
                    float t0, t1;
                    upk2(t, t0, t1);
                    st_shared_u32(jb + sw128(d * R + p, cb), to_bf16x2(t0, t1));
                    S = mul2(S, STEP);
                }
            }
            // generic-proxy writes become visible to the tensor core, then signal
            fence_async_smem();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&jfull[c]);
        }
    }
    if (flags)
        atomicOr(&s_flags, flags);
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && s_flags)
        atomicOr(status, s_flags);
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kNTmemCols);
    }
}

// M from the CTAs' shares: one warp per (entry, part) of the upper triangle;
// lane k adds CTAs k, k + 32, ... (all loads issued first), then a fixed
// shuffle tree; divided by N_gen, written to (a, b) and conjugated to (b, a),
// the diagonal's imaginary part zero. With a timeout flagged, M is NaN.
__global__ void norm_tc_finalize(const double *__restrict__ part, int grid, int N, double n_gen,
                                 const int *status, double *__restrict__ M)
{
    const int ec = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int E = N * (N + 1) / 2;
    if (ec >= 2 * E)
        return;
    const int e = ec >> 1, comp = ec & 1;
    int a = 0, o = e;
    while (o >= N - a) {
        o -= N - a;
        ++a;
    }
    const int b = a + o;
    const double *pe = part + (size_t)ec * grid;
    double x[kNFinMaxRounds];
#pragma unroll
    for (int k = 0; k < kNFinMaxRounds; ++k) {
        const int g = lane + 32 * k;
        x[k] = g < grid ? pe[g] : 0.0;
    }
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < kNFinMaxRounds; ++k)
        v += x[k];
    v = warp_sum(v);
    if (lane == 0) {
        double r = v / n_gen;
        if (*status & FLAG_TIMEOUT)
            r = NAN;
        if (a == b) {
            M[2 * (a * N + a) + comp] = comp ? 0.0 : r;
        } else {
            M[2 * (a * N + b) + comp] = r;
            M[2 * (b * N + a) + comp] = comp ? -r : r;
        }
    }
}

template <int NW>
cudaError_t norm_tc_nw(const CUtensorMap *map, const Planes &mc, const float *amax, double n_gen,
                       double *part, int grid, int *status, double *M, cudaStream_t s)
{
    using C = NormTcCfg<NW>;
    const int n_tiles = (int)((mc.n + kNTE - 1) / kNTE);
    if (grid > n_tiles)
        grid = n_tiles;
    if (grid > 32 * kNFinMaxRounds)
        grid = 32 * kNFinMaxRounds;
    cudaError_t e = cudaFuncSetAttribute(norm_tc_kernel<NW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess)
        return e;
    norm_tc_kernel<NW><<<grid, kNThreads, C::SMEM, s>>>(*map, amax, mc.n_waves, n_tiles, part,
                                                        status);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    const int E2 = mc.n_waves * (mc.n_waves + 1);
    norm_tc_finalize<<<(E2 + 7) / 8, 256, 0, s>>>(part, grid, mc.n_waves, n_gen, status, M);
    return cudaGetLastError();
}

int norm_tc_nw_of(int n_waves)
{
    for (int p : {4, 8, 12, 16, 20})
        if (n_waves <= p)
            return p;
    return -1;
}

}  // namespace

bool norm_tc_available(int n_waves) { return n_waves >= 1 && norm_tc_nw_of(n_waves) > 0; }

int norm_tc_box_events() { return kNTE; }

bool norm_tc_scale_ok(float amax)
{
    // every kept quantum a normal float and every accumulator below 2^127:
    // 2^r <= 2^55, i.e. amax < 2^53 (and finite)
    return amax >= 0.f && amax < 0x1p53f;
}

size_t norm_tc_partials_doubles(int n_waves, int grid)
{
    return (size_t)grid * n_waves * (n_waves + 1);
}

cudaError_t launch_build_norm_tc(const CUtensorMap *map, const Planes &mc, const float *amax,
                                 double n_gen, double *partials, int grid, int *status, double *M,
                                 cudaStream_t s)
{
    if (mc.n < 1)
        return cudaErrorInvalidValue;
    switch (norm_tc_nw_of(mc.n_waves)) {
    case 4: return norm_tc_nw<4>(map, mc, amax, n_gen, partials, grid, status, M, s);
    case 8: return norm_tc_nw<8>(map, mc, amax, n_gen, partials, grid, status, M, s);
    case 12: return norm_tc_nw<12>(map, mc, amax, n_gen, partials, grid, status, M, s);
    case 16: return norm_tc_nw<16>(map, mc, amax, n_gen, partials, grid, status, M, s);
    case 20: return norm_tc_nw<20>(map, mc, amax, n_gen, partials, grid, status, M, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace pwa
