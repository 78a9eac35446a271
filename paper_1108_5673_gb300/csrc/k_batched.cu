// Batched evaluation of NLL and gradient for K parameter sets on the
// tensor cores (tcgen05, BF16 operands, FP32 accumulation in tensor memory).
//
// The paper runs thousands of fits from different starting parameters and
// models (Sec. 2); evaluating K parameter sets against the same events turns
// the direct form into two chained products per tile of 128 events:
//   S[e][(k,re/im)] = sum_f X[e][f] W[(k,re/im)][f]            (GEMM 1)
//   I = Sre^2 + Sim^2,  ln I,  R = S / I                      (epilogue)
//   G[(k,re/im)][f] += sum_e R[e][(k,re/im)] X[e][f]           (GEMM 2)
// where X holds the amplitudes as features f = (Re A_a, Im A_a) and W the
// parameter sets (row (k,re): vr on Re A_a, -vi on Im A_a; row (k,im): vi on
// Re A_a, vr on Im A_a). The gradient is g_a = -(G[(k,re)][2a] +
// G[(k,im)][2a+1]) - i (G[(k,im)][2a] - G[(k,re)][2a+1]) + (M V)_a.
//
// Operands: the amplitudes are a BF16 structure-of-arrays copy (the values
// this path consumes are the BF16-rounded amplitudes); V is split into two
// BF16 pieces (16 significant bits) and the NLL is corrected to first order
// for the remainder, 2 Re(g^H dV), in double in the final kernel; R is one
// BF16 piece. Products are exact in FP32 and accumulate in FP32.
//
// Layout in shared memory (all 128-byte swizzled, 1 KB aligned):
//  X tile  [2 blocks of 64 events][F feature rows][128 B]: for GEMM 1 the
//          MN-major A operand (events contiguous), for GEMM 2 the K-major B
//          operand (K = events) -- the same bytes serve both products.
//  W       [chunk][piece][F/64 blocks][128 rows][128 B], K-major B of GEMM 1.
//  R^T     [2 blocks of 64 events][128 rows][128 B], K-major A of GEMM 2,
//          written by the epilogue threads.
// Tensor memory (512 columns): two S buffers of 128 columns, then the G^T
// accumulators of every chunk (F columns each) for the whole launch.
//
// Warps: 0-7 epilogue (warp w reads TMEM lane quarter w%4 and half w/4 of
// each chunk's columns), 8 producer (TMA), 9 MMA issuer (one thread), 10
// helper (M V and V^H M V in FP64). Every wait is bounded.
#include <cuda_bf16.h>

#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int kBM = 128;       // events per tile
constexpr int kKC = 64;        // parameter sets per chunk (2 kKC = 128 S columns)
constexpr int kXS = 3;         // X stages
constexpr int kPieces = 2;     // BF16 pieces of V
constexpr int kEpiWarps = 8;
constexpr int kThreads = (kEpiWarps + 3) * 32;
constexpr double kLn2 = 0.69314718055994530942;

// The V pieces, shared by the main and the final kernel.
__host__ __device__ inline void split_bf16(double v, float &hi, float &lo)
{
    const __nv_bfloat16 h = __double2bfloat16(v);
    hi = __bfloat162float(h);
    lo = __bfloat162float(__double2bfloat16(v - (double)hi));
}

struct BatchArgs {
    int n_waves, F, K, n_chunks;
    int64_t n_events;
    const double *V;      // [K][N] complex
    const double *M;      // [N][N] complex
    float *gpart;         // [grid][n_chunks][128][F]
    float2 *lpart;        // [grid][4][n_chunks * 64] float-float ln sums
    unsigned *kflags;     // [n_chunks * 2] domain bits per parameter set (OR)
    double *mv;           // [K][2N + 1]: M V and V^H M V
    int *status;
};

struct Smem {
    uint32_t w_off, x_off, r_off, bytes;
};

__host__ __device__ inline Smem batch_smem(int F, int n_chunks)
{
    const int kb = (F + 63) / 64;
    Smem s;
    s.w_off = 0;
    s.x_off = s.w_off + (uint32_t)n_chunks * kPieces * kb * 128 * 128;
    s.r_off = s.x_off + (uint32_t)kXS * 2 * F * 128;
    s.bytes = s.r_off + 2 * 128 * 128 + 1024;  // + alignment slack
    return s;
}

__device__ __forceinline__ uint32_t sw128(int row, int byte_in_row)
{
    return (row >> 3) * 1024 + (row & 7) * 128 + ((((byte_in_row >> 4) ^ (row & 7)) & 7) << 4) +
           (byte_in_row & 15);
}

__device__ __forceinline__ unsigned pack_bf16x2(float lo, float hi)
{
    unsigned r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

template <int F>
__global__ void __launch_bounds__(kThreads, 1)
    batched_kernel(const __grid_constant__ CUtensorMap xmap, const BatchArgs a, const int n_tiles)
{
    constexpr int KB = (F + 63) / 64;
    extern __shared__ unsigned char smem_dyn[];
    __shared__ uint64_t x_full[kXS], x_empty[kXS], s_full[2], s_free[2], r_full, r_free, g_done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_flags;
    __shared__ unsigned s_kflags[2 * 8];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NCH = a.n_chunks;
    const Smem L = batch_smem(F, NCH);
    unsigned char *base = smem_dyn + ((1024 - (smem_u32(smem_dyn) & 1023)) & 1023);
    unsigned char *sW = base + L.w_off;
    unsigned char *sX = base + L.x_off;
    unsigned char *sR = base + L.r_off;
    const uint32_t x_bytes = 2 * F * 128;
    const int n_my =
        (n_tiles > (int)blockIdx.x) ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kXS; ++s) {
            mbar_init(&x_full[s], 1);
            mbar_init(&x_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&s_full[b], 1);
            mbar_init(&s_free[b], kEpiWarps);
        }
        mbar_init(&r_full, kEpiWarps);
        mbar_init(&r_free, 1);
        mbar_init(&g_done, 1);
        fence_barrier_init();
        s_flags = 0;
    }
    if (threadIdx.x < 16)
        s_kflags[threadIdx.x] = 0;
    // W pieces from V: row r = 2k' + t of chunk c, feature f = 2 a + u
    {
        const int rows_total = NCH * 128;
        for (int idx = threadIdx.x; idx < rows_total * F; idx += blockDim.x) {
            const int row_g = idx / F, f = idx - row_g * F;
            const int c = row_g >> 7, r = row_g & 127;
            const int k = c * kKC + (r >> 1), t = r & 1, w = f >> 1, u = f & 1;
            float hi = 0.f, lo = 0.f;
            if (k < a.K && w < a.n_waves) {
                const double vr = a.V[2 * (k * a.n_waves + w)], vi = a.V[2 * (k * a.n_waves + w) + 1];
                const double coef = t == 0 ? (u == 0 ? vr : -vi) : (u == 0 ? vi : vr);
                split_bf16(coef, hi, lo);
            }
            const uint32_t rb = sw128(r, (f & 63) * 2);
            for (int p = 0; p < kPieces; ++p) {
                unsigned char *piece = sW + ((size_t)(c * kPieces + p) * KB + (f >> 6)) * 128 * 128;
                *reinterpret_cast<__nv_bfloat16 *>(piece + rb) = __float2bfloat16_rn(p == 0 ? hi : lo);
            }
        }
        // feature padding inside a 128-byte row block (F not a multiple of 64)
        if (F % 64) {
            for (int idx = threadIdx.x; idx < NCH * kPieces * 128 * (64 - F % 64); idx += blockDim.x) {
                const int pad = 64 - F % 64;
                const int cp = idx / (128 * pad), rem = idx - cp * 128 * pad;
                const int r = rem / pad, f = F % 64 + rem % pad;
                unsigned char *piece = sW + ((size_t)cp * KB + (KB - 1)) * 128 * 128;
                *reinterpret_cast<__nv_bfloat16 *>(piece + sw128(r, f * 2)) = __float2bfloat16_rn(0.f);
            }
        }
    }
    fence_async_smem();
    if (warp == kEpiWarps + 1)
        tmem_alloc(&tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    int flags = 0;

    if (warp == kEpiWarps) {
        // ---- producer ------------------------------------------------------
        if (lane == 0) {
            int j = 0;
            for (; j < n_my; ++j) {
                const int s = j % kXS;
                const uint32_t u = j / kXS;
                if (u > 0 && !mbar_wait(&x_empty[s], (u & 1) ^ 1)) {
                    flags |= FLAG_TIMEOUT;
                    break;
                }
                const int e0 = ((int)blockIdx.x + j * (int)gridDim.x) * kBM;
                mbar_arrive_expect_tx(&x_full[s], x_bytes);
                tma_load_2d(sX + (size_t)s * x_bytes, &xmap, e0, 0, &x_full[s]);
                tma_load_2d(sX + (size_t)s * x_bytes + F * 128, &xmap, e0 + 64, 0, &x_full[s]);
            }
            for (int q = (j > kXS ? j - kXS : 0); q < j; ++q)
                if (!mbar_wait(&x_full[q % kXS], (q / kXS) & 1))
                    flags |= FLAG_TIMEOUT;
        }
    } else if (warp == kEpiWarps + 1) {
        // ---- MMA issuer -------------------------------------------------------
        if (lane == 0) {
            const uint32_t id1 = umma_idesc_bf16(128, 128, 1, 0);
            const uint32_t id2 = umma_idesc_bf16(128, F, 0, 0);
            const uint32_t xbase = smem_u32(sX), wbase = smem_u32(sW), rbase = smem_u32(sR);
            const int total = n_my * NCH;
            // GEMM 2 of chunk q (pipelined one chunk behind GEMM 1)
            auto gemm2 = [&](int q) -> bool {
                const int j = q / NCH, c = q % NCH, s = j % kXS;
                if (!mbar_wait(&r_full, q & 1))
                    return false;
                tc_fence_after();
                const uint32_t xs = xbase + s * x_bytes;
                for (int ks = 0; ks < kBM / 16; ++ks) {
                    const uint32_t blk = ks >> 2, off = (ks & 3) * 32;
                    const uint64_t da = umma_desc_sw128(rbase + blk * 128 * 128 + off, 16, 1024);
                    const uint64_t db = umma_desc_sw128(xs + blk * F * 128 + off, 16, 1024);
                    umma_bf16(tmem + 256 + c * F, da, db, id2, (j > 0 || ks > 0) ? 1u : 0u);
                }
                umma_commit(&r_free);
                if (c == NCH - 1)
                    umma_commit(&x_empty[s]);
                return true;
            };
            bool ok = true;
            for (int q = 0; q < total && ok; ++q) {
                const int j = q / NCH, c = q % NCH, s = j % kXS, b = q & 1;
                if (c == 0 && !mbar_wait(&x_full[s], (j / kXS) & 1)) {
                    ok = false;
                    break;
                }
                if (q >= 2 && !mbar_wait(&s_free[b], ((q >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // GEMM 1: S[b] = X (MN-major) . W_c^T, both V pieces
                const uint32_t xs = xbase + s * x_bytes;
                for (int p = 0; p < kPieces; ++p)
                    for (int ks = 0; ks < F / 16; ++ks) {
                        const uint64_t da = umma_desc_sw128(xs + ks * 2048, F * 128, 1024);
                        const uint32_t wp = wbase + ((c * kPieces + p) * KB + (ks >> 2)) * 128 * 128;
                        const uint64_t db = umma_desc_sw128(wp + (ks & 3) * 32, 16, 1024);
                        umma_bf16(tmem + b * 128, da, db, id1, (p > 0 || ks > 0) ? 1u : 0u);
                    }
                umma_commit(&s_full[b]);
                if (q >= 1)
                    ok = gemm2(q - 1);
            }
            if (ok && total > 0)
                ok = gemm2(total - 1);
            umma_commit(&g_done);
            // tensor memory is released only after every product has finished
            if (!mbar_wait(&g_done, 0))
                ok = false;
            if (!ok)
                flags |= FLAG_TIMEOUT;
        }
    } else if (warp < kEpiWarps) {
        // ---- epilogue -----------------------------------------------------------
        const int qq = warp & 3, h = warp >> 2;
        const int lane_row = qq * 32 + lane;          // TMEM lane = event row of the tile
        const uint32_t lane_addr = (uint32_t)(qq * 32) << 16;
        dfloat acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        unsigned kbad[4] = {0u, 0u, 0u, 0u};
        const int blk = lane_row >> 6, e64 = lane_row & 63;
        bool ok = true;
        for (int q = 0; q < n_my * NCH && ok; ++q) {
            const int j = q / NCH, c = q % NCH, b = q & 1;
            if (!mbar_wait(&s_full[b], (q >> 1) & 1)) {
                ok = false;
                break;
            }
            tc_fence_after();
            uint32_t v[2][32];
            tmem_ld32(tmem + lane_addr + b * 128 + 64 * h, v[0]);
            tmem_ld32(tmem + lane_addr + b * 128 + 64 * h + 32, v[1]);
            tmem_ld_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&s_free[b]);
            const int64_t ev = (int64_t)((int)blockIdx.x + j * (int)gridDim.x) * kBM + lane_row;
            const bool valid = ev < a.n_events;
            float ln[32];
            unsigned rpk[32];  // bf16 (re, im) of R for the 32 parameter sets of this half
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const float re = __uint_as_float(v[k >> 4][(2 * k) & 31]);
                const float im = __uint_as_float(v[k >> 4][(2 * k + 1) & 31]);
                const float I = fmaf(re, re, im * im);
                float l = 0.f, rr = 0.f, ri = 0.f;
                if (valid) {
                    if (I > 0.f && I < INFINITY) {
                        int ex;
                        const float f = split_exponent(I, ex);
                        l = fmaf((float)ex, 0.693147180559945f, __logf(f));
                        const float inv = __frcp_rn(I);
                        rr = re * inv;
                        ri = im * inv;
                    } else {
                        kbad[c] |= 1u << k;
                    }
                }
                ln[k] = l;
                rpk[k] = pack_bf16x2(rr, ri);
            }
            // reduce-scatter the 32 log values over the 32 lanes: lane k ends
            // with the sum over the warp's events for parameter set k
#pragma unroll
            for (int width = 16; width >= 1; width >>= 1) {
                const bool upper = (lane & width) != 0;
#pragma unroll
                for (int k = 0; k < width; ++k) {
                    const float send = upper ? ln[k] : ln[k + width];
                    const float keep = upper ? ln[k + width] : ln[k];
                    ln[k] = keep + __shfl_xor_sync(0xffffffffu, send, width);
                }
            }
            // lane L now holds, in ln[0], the sum for parameter set L of this half
            acc[c] = df_add(acc[c], dfloat{ln[0], 0.f});
            // R^T may be overwritten once GEMM 2 of the previous chunk is done
            if (q >= 1 && !mbar_wait(&r_free, (q - 1) & 1)) {
                ok = false;
                break;
            }
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int row = 64 * h + 2 * k;
                unsigned char *rb = sR + blk * 128 * 128;
                *reinterpret_cast<unsigned short *>(rb + sw128(row, e64 * 2)) = (unsigned short)(rpk[k] & 0xffff);
                *reinterpret_cast<unsigned short *>(rb + sw128(row + 1, e64 * 2)) = (unsigned short)(rpk[k] >> 16);
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&r_full);
        }
        if (!ok)
            flags |= FLAG_TIMEOUT;
        // parameter-set bits and log partials
        for (int c = 0; c < NCH; ++c) {
            const unsigned m = __reduce_or_sync(0xffffffffu, kbad[c]);
            if (lane == 0 && m)
                atomicOr(&s_kflags[2 * c + h], m);
        }
        for (int c = 0; c < NCH; ++c)
            a.lpart[((size_t)blockIdx.x * 4 + qq) * (NCH * kKC) + c * kKC + 32 * h + lane] =
                make_float2(acc[c].hi, acc[c].lo);
        // G^T of every chunk: rows = this warp's lane quarter, half the columns
        if (ok && mbar_wait(&g_done, 0)) {
            tc_fence_after();
            // F/2 is a multiple of 8: eight-column loads cover it exactly
            for (int c = 0; c < NCH; ++c) {
                for (int c0 = h * (F / 2); c0 < (h + 1) * (F / 2); c0 += 8) {
                    uint32_t g[8];
                    tmem_ld8(tmem + lane_addr + 256 + c * F + c0, g);
                    tmem_ld_wait();
                    float4 *dst = reinterpret_cast<float4 *>(
                        a.gpart + (((size_t)blockIdx.x * NCH + c) * 128 + lane_row) * F + c0);
                    dst[0] = make_float4(__uint_as_float(g[0]), __uint_as_float(g[1]),
                                         __uint_as_float(g[2]), __uint_as_float(g[3]));
                    dst[1] = make_float4(__uint_as_float(g[4]), __uint_as_float(g[5]),
                                         __uint_as_float(g[6]), __uint_as_float(g[7]));
                }
            }
        } else {
            flags |= FLAG_TIMEOUT;
        }
    } else if (warp == kEpiWarps + 2) {
        // ---- helper: M V and V^H M V for the sets k = blockIdx.x, + grid, ... --
        const int Nw = a.n_waves;
        for (int k = blockIdx.x; k < a.K; k += gridDim.x) {
            const double *V = a.V + 2 * (size_t)k * Nw;
            double nv = 0.0;
            for (int row = lane; row < Nw; row += 32) {
                double re = 0.0, im = 0.0;
                for (int bb = 0; bb < Nw; ++bb) {
                    const double mr = a.M[2 * (row * Nw + bb)], mi = a.M[2 * (row * Nw + bb) + 1];
                    re = fma(mr, V[2 * bb], fma(-mi, V[2 * bb + 1], re));
                    im = fma(mr, V[2 * bb + 1], fma(mi, V[2 * bb], im));
                }
                a.mv[(size_t)k * (2 * Nw + 1) + 2 * row] = re;
                a.mv[(size_t)k * (2 * Nw + 1) + 2 * row + 1] = im;
                nv = fma(V[2 * row], re, fma(V[2 * row + 1], im, nv));
            }
            nv = warp_sum(nv);
            if (lane == 0)
                a.mv[(size_t)k * (2 * Nw + 1) + 2 * Nw] = nv;
        }
    }
    if (flags)
        atomicOr(&s_flags, flags);
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 2 * NCH && s_kflags[threadIdx.x])
        atomicOr(&a.kflags[threadIdx.x], s_kflags[threadIdx.x]);
    if (threadIdx.x == 0 && s_flags)
        atomicOr(a.status, s_flags);
    if (warp == kEpiWarps + 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// Final sums over CTAs (fixed order, float-float), M V, first-order
// correction for the V remainder; one block per parameter set.
__global__ void batched_finalize(const BatchArgs a, int grid, int *done, double *nll, double *grad)
{
    const int k = blockIdx.x, Nw = a.n_waves, F = a.F, NCH = a.n_chunks;
    const int c = k / kKC, kl = k % kKC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ double s_corr[2];
    __shared__ double s_ln;
    const bool bad = (a.kflags[2 * c + (kl >> 5)] >> (kl & 31)) & 1u;
    double corr = 0.0;
    for (int w = threadIdx.x; w < Nw; w += blockDim.x) {
        // Re conj(A) r = G[(k,re)][2w] + G[(k,im)][2w+1];  Im = G[(k,im)][2w] - G[(k,re)][2w+1]
        dfloat s_re = {0.f, 0.f}, s_im = {0.f, 0.f};
        const size_t cta_stride = (size_t)NCH * 128 * F;
        const float *g0 = a.gpart + (size_t)c * 128 * F;
        for (int b0 = 0; b0 < grid; b0 += 16) {
            float2 re_row[16], im_row[16];  // (G[(k,re)][2w], G[(k,re)][2w+1]), same for im
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const float *g = g0 + (size_t)(b0 + t) * cta_stride;
                const bool in = b0 + t < grid;
                re_row[t] = in ? *reinterpret_cast<const float2 *>(g + (2 * kl) * F + 2 * w)
                               : make_float2(0.f, 0.f);
                im_row[t] = in ? *reinterpret_cast<const float2 *>(g + (2 * kl + 1) * F + 2 * w)
                               : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                s_re = df_add(s_re, df_add(dfloat{re_row[t].x, 0.f}, dfloat{im_row[t].y, 0.f}));
                s_im = df_add(s_im, df_add(dfloat{im_row[t].x, 0.f}, dfloat{-re_row[t].y, 0.f}));
            }
        }
        const double gre = -((double)s_re.hi + (double)s_re.lo);
        const double gim = -((double)s_im.hi + (double)s_im.lo);
        const double *V = a.V + 2 * ((size_t)k * Nw + w);
        float h0, l0, h1, l1;
        split_bf16(V[0], h0, l0);
        split_bf16(V[1], h1, l1);
        const double dvr = V[0] - ((double)h0 + (double)l0), dvi = V[1] - ((double)h1 + (double)l1);
        corr += 2.0 * (gre * dvr + gim * dvi);
        const double *mv = a.mv + (size_t)k * (2 * Nw + 1);
        if (grad) {
            grad[2 * ((size_t)k * Nw + w)] = bad ? 0.0 : gre + mv[2 * w];
            grad[2 * ((size_t)k * Nw + w) + 1] = bad ? 0.0 : gim + mv[2 * w + 1];
        }
    }
    corr = warp_sum(corr);
    if (lane == 0)
        s_corr[warp] = corr;
    if (warp == 0) {
        dfloat l = {0.f, 0.f};
        for (int i0 = lane; i0 < grid * 4; i0 += 32 * 8) {
            float2 p[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int i = i0 + 32 * t;
                p[t] = i < grid * 4 ? a.lpart[(size_t)i * (NCH * kKC) + k] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int t = 0; t < 8; ++t)
                l = df_add(l, dfloat{p[t].x, p[t].y});
        }
        l = warp_sum(l);
        if (lane == 0)
            s_ln = (double)l.hi + (double)l.lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double nv = a.mv[(size_t)k * (2 * Nw + 1) + 2 * Nw];
        double v = -s_ln + nv + s_corr[0] + (blockDim.x > 32 ? s_corr[1] : 0.0);
        if (bad)
            v = INFINITY;
        nll[k] = v;
        if (done)
            atomicAdd(done, 1);
    }
}

constexpr int kMaxSmem = 215 * 1024;

template <int F>
cudaError_t configure_f()
{
    return cudaFuncSetAttribute(batched_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kMaxSmem);
}

}  // namespace

int batched_features(int n_waves) { return (2 * n_waves + 15) / 16 * 16; }

int batched_max_k(int n_waves)
{
    const int F = batched_features(n_waves);
    int nch = 4;
    while (nch > 0 && (256 + nch * F > 512 || batch_smem(F, nch).bytes > kMaxSmem))
        --nch;
    return nch * kKC;
}

size_t batched_scratch_bytes(int n_waves, int K, int grid)
{
    const int F = batched_features(n_waves), nch = (K + kKC - 1) / kKC;
    return (size_t)grid * nch * 128 * F * 4 + (size_t)grid * 4 * nch * kKC * 8 + (size_t)nch * 2 * 4 +
           (size_t)K * (2 * n_waves + 1) * 8 + 256;
}

cudaError_t batched_configure()
{
    cudaError_t e = cudaSuccess;
    for (cudaError_t r : {configure_f<16>(), configure_f<32>(), configure_f<48>(), configure_f<64>(),
                          configure_f<80>(), configure_f<96>()})
        if (r != cudaSuccess)
            e = r;
    return e;
}

// K <= batched_max_k(n_waves) parameter sets; scratch >= batched_scratch_bytes.
cudaError_t launch_batched(const CUtensorMap *xmap, int64_t n_events, int n_waves, const double *V,
                           int K, const double *M, void *scratch, int grid, int *status, int *done,
                           double *nll, double *grad, cudaStream_t s)
{
    const int F = batched_features(n_waves), nch = (K + kKC - 1) / kKC;
    BatchArgs a{};
    a.n_waves = n_waves;
    a.F = F;
    a.K = K;
    a.n_chunks = nch;
    a.n_events = n_events;
    a.V = V;
    a.M = M;
    char *p = static_cast<char *>(scratch);
    a.gpart = reinterpret_cast<float *>(p);
    p += (size_t)grid * nch * 128 * F * 4;
    a.lpart = reinterpret_cast<float2 *>(p);
    p += (size_t)grid * 4 * nch * kKC * 8;
    a.kflags = reinterpret_cast<unsigned *>(p);
    p += (size_t)nch * 2 * 4;
    p = reinterpret_cast<char *>(((uintptr_t)p + 7) & ~(uintptr_t)7);
    a.mv = reinterpret_cast<double *>(p);
    a.status = status;
    cudaError_t e = cudaMemsetAsync(a.kflags, 0, nch * 2 * 4, s);
    if (e != cudaSuccess)
        return e;
    const int n_tiles = (int)((n_events + kBM - 1) / kBM);
    const uint32_t smem = batch_smem(F, nch).bytes;
    switch (F) {
    case 16: batched_kernel<16><<<grid, kThreads, smem, s>>>(*xmap, a, n_tiles); break;
    case 32: batched_kernel<32><<<grid, kThreads, smem, s>>>(*xmap, a, n_tiles); break;
    case 48: batched_kernel<48><<<grid, kThreads, smem, s>>>(*xmap, a, n_tiles); break;
    case 64: batched_kernel<64><<<grid, kThreads, smem, s>>>(*xmap, a, n_tiles); break;
    case 80: batched_kernel<80><<<grid, kThreads, smem, s>>>(*xmap, a, n_tiles); break;
    case 96: batched_kernel<96><<<grid, kThreads, smem, s>>>(*xmap, a, n_tiles); break;
    default: return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    batched_finalize<<<K, 64, 0, s>>>(a, grid, done, nll, grad);
    return cudaGetLastError();
}

}  // namespace pwa
