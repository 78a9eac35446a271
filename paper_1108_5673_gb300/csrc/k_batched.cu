// Batched evaluation of NLL and gradient for K parameter sets on the
// tensor cores (tcgen05, BF16 operands, FP32 accumulation in tensor memory).
//
// The paper runs a great many fits from different starting parameters and
// models (Sec. 2); evaluating K parameter sets against the same events turns
// the direct form into two chained products per tile of 128 events:
//   S[e][(k,re/im)] = sum_f A[e][f] W[(k,re/im)][f]            (GEMM 1)
//   I = Sre^2 + Sim^2,  ln I,  R = S / I                      (epilogue)
//   G[(k,re/im)][f] += sum_e R[e][(k,re/im)] A[e][f]           (GEMM 2)
// with features f = (Re A_a, Im A_a) and W the parameter sets (row (k,re):
// vr on Re A_a, -vi on Im A_a; row (k,im): vi on Re A_a, vr on Im A_a). The
// data part of the gradient is g_a = -(G[(k,re)][2a] + G[(k,im)][2a+1])
// - i (G[(k,im)][2a] - G[(k,re)][2a+1]); M V is added in the final kernel.
//
// Exact sums on the tensor cores. The FP32 accumulation of the tensor cores
// does not round to nearest when it adds products of different exponents, and
// the error it leaves is one-sided: summed over a million events it shifts the
// NLL far beyond its tolerance. This path therefore makes every tensor-core
// sum an exact integer sum:
//  * amplitudes (features of event i): A = 2^(E_i - 8) (x0 + x1 / 256) with a
//    shared exponent E_i per event and integer slices |x0| <= 256,
//    |x1| <= 128 (16-bit block floating point, XS = 2) or A = 2^(E_i - 8) x0
//    (8-bit, XS = 1): these are the values this path consumes;
//  * parameter set k: W = 2^(T_k - 8) (w0 + w1 / 2^8 + w2 / 2^16), shared
//    exponent T_k per set, integer slices |w0| <= 256, |w1|, |w2| <= 128; the
//    remainder V - V_r (below 2^-24 |V|) is accounted for to first order,
//    2 Re(g^H (V - V_r)), in the final kernel.
// Integers of at most 9 bits are exact in BF16, their products exact in FP32,
// and the accumulators (one per power of 2^-8)
//   acc0 = x0 w0,  acc1 = x0 w1 + x1 w0,  acc2 = x0 w2 + x1 w1,  acc3 = x1 w2
// (sums over features; the x1 terms only for XS = 2) stay below 2^23 for
// F <= 96 features, so each is exact whatever the accumulation order or
// rounding, and S = 2^(E_i + T_k - 16) Q with
// Q = acc0 + (acc1 + (acc2 + acc3 / 2^8) / 2^8) / 2^8 (FP32 roundings to nearest).
// ln I = ln 2 (2 (E_i + T_k - 16) + log2 |Q|^2): the exponent parts are summed
// exactly once per call; log2 |Q|^2 is evaluated with a polynomial of
// max error 8e-10 (log2_poly.py) and summed as fixed point with resolution
// 2^-19 in 32-bit integer warp sums and 64-bit per-set accumulators, so the
// NLL sum is exact and independent of order. For the gradient
// R A = 2^(8 - T_k) (Q / |Q|^2) (x0 + x1 / 256): GEMM 2 multiplies
// R' = Q / |Q|^2, rounded to BF16, by both slices (N = XS F columns).
//
// Layout in shared memory (128-byte swizzled, 1 KB aligned):
//  W   [chunk][half][F/64 blocks][slice w0,w1,w2][64 rows][128 B]: K-major B
//      operands of GEMM 1 (the three slices of a block are adjacent, so one
//      product covers w0|w1|w2 as 192 columns), copied once per launch from an
//      image the prep kernel builds.
//  X   [stage][2 blocks of 64 events][XS F rows (x0 then x1)][128 B]: MN-major
//      A operand of GEMM 1 (events contiguous) and K-major B operand of GEMM 2
//      (K = events) -- the same bytes serve both products. The data store in
//      global memory holds every 128-event tile in exactly this byte order, so
//      a tile arrives with one contiguous bulk copy (a 2D tensor copy of 64
//      events x XS F rows reads XS F separate 128-byte pieces, far apart).
//  R'  [2 blocks of 64 rows (k,re/im)][128 events][128 B]: MN-major A operand
//      of GEMM 2, written by the epilogue (each thread stores its event's row).
// Tensor memory (512 columns): acc0..acc3 of one half chunk (32 sets, 64
// columns each), then the G^T accumulators of every chunk (XS F columns each)
// for the whole launch.
//
// Warps: 0-15 epilogue (warp w reads TMEM lane quarter w%4 and the 8 sets
// w/4 of each half chunk), 16 producer (TMA), 17 MMA issuer (one thread),
// 18 helper (M V and V^H M V in FP64). Every wait is bounded.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int kBM = 128;        // events per tile
constexpr int kKC = 64;         // parameter sets per chunk (GEMM 2: M = 2 kKC = 128)
constexpr int kHS = 32;         // parameter sets per half chunk (one GEMM 1 / epilogue step)
constexpr int kXSMax = 6;       // X stages at most (as many as shared memory takes, at least 2)
constexpr int kMaxSmem = 226 * 1024;
constexpr int kMaxChunks = 4;
constexpr int kEpiWarps = 16;
constexpr int kThreads = (kEpiWarps + 3) * 32;
constexpr uint32_t kWBlock = 64 * 128;      // 64 rows x 64 BF16 features
constexpr uint32_t kRBytes = 2 * 128 * 128;
constexpr int kWSlices = 3;                 // BF16 slices of V
// tensor-memory columns: accumulators acc0..acc3 at 64 j, then G^T
__host__ __device__ constexpr int s_cols(int xs) { return xs == 2 ? 256 : 192; }
constexpr double kLn2 = 0.69314718055994530942;
constexpr int kFixBits = 19;                // fixed-point resolution of log2 sums

// Integer slices of v * 2^(8 - T): v ~ 2^(T-8) (w0 + w1 / 2^8 + w2 / 2^16).
__host__ __device__ inline void split_slices(double v, int T, double (&w)[kWSlices])
{
    double x = ldexp(v, 8 - T);
    for (int p = 0; p < kWSlices; ++p) {
        w[p] = rint(x);
        x = (x - w[p]) * 256.0;
    }
}

__host__ __device__ inline double round_slices(double v, int T)
{
    double w[kWSlices];
    split_slices(v, T, w);
    return ldexp(w[0] + (w[1] + w[2] / 256.0) / 256.0, T - 8);
}

struct BatchArgs {
    int n_waves, F, XS, K, n_chunks;
    const unsigned char *xg;    // the data store: n_tiles tiles of 2 XS F 128 bytes
    int64_t n_events;
    const double *V;            // [K][N] complex
    const double *M;            // [N][N] complex
    const long long *sum_e;     // sum over events of the event exponents
    unsigned char *wimg;        // W image (byte-identical to shared memory)
    int *T;                     // [K] set exponents
    float *gpart;               // [grid][n_chunks][128][F]
    long long *lpart;           // [grid][4][n_chunks * 64] fixed-point log2 sums (zeroed per launch)
    unsigned *kflags;           // [n_chunks * 2] domain bits per half chunk
    double *mv;                 // [K][2N + 1]: M V and V^H M V
    int *status;
    int nxs_req;                // X stages asked for (0: as many as fit)
};

struct Smem {
    uint32_t w_off, x_off, r_off, w_bytes, bytes;
    int nxs;   // X stages
};

// Bytes of the W image of n_chunks chunks (both halves of each), as built in
// global memory by the prep kernel.
__host__ __device__ inline uint32_t w_image_bytes(int F, int n_chunks)
{
    return (uint32_t)n_chunks * 2 * kWSlices * ((F + 63) / 64) * kWBlock;
}

// Shared memory of a launch for K sets: the W image of the hpt half chunks
// that hold sets (its first part), then as many X stages as fit (2..kXSMax),
// then R'. Small K leave room for a deeper X pipeline, which their short
// per-tile work needs to hide the loads.
__host__ __device__ inline Smem batch_smem(int F, int xs, int hpt, int nxs_req = 0)
{
    const int kb = (F + 63) / 64;
    Smem s;
    s.w_bytes = (uint32_t)hpt * kWSlices * kb * kWBlock;
    const uint32_t stage = 2u * xs * F * 128;
    const int64_t room = (int64_t)kMaxSmem - 1024 - kRBytes - (int64_t)s.w_bytes;
    const int fit = room > 0 ? (int)(room / stage) : 0;
    s.nxs = fit < 2 ? 2 : (fit > kXSMax ? kXSMax : fit);
    if (nxs_req >= 2 && nxs_req < s.nxs)
        s.nxs = nxs_req;
    s.w_off = 0;
    s.x_off = s.w_bytes;
    s.r_off = s.x_off + (uint32_t)s.nxs * stage;
    s.bytes = s.r_off + kRBytes + 1024;  // + alignment slack
    return s;
}

__host__ __device__ inline int batch_hpt(int K) { return (K + kHS - 1) / kHS; }

__host__ __device__ inline uint32_t sw128(int row, int byte_in_row)
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

// Fixed-point 2^19 log2(1 + z) for two values, z in [sqrt(1/2) - 1, sqrt(2) - 1];
// the last step adds 1.5 * 2^23 so that the float's low bits hold the
// rounded-to-nearest integer. Coefficients: log2_poly.py (a_j * 2^19).
__device__ __forceinline__ f2 log2_fixed2(f2 z)
{
    f2 p = pk2(4.891085156e+04f, 4.891085156e+04f);
    p = fma2(p, z, pk2(-8.236935156e+04f, -8.236935156e+04f));
    p = fma2(p, z, pk2(8.752553125e+04f, 8.752553125e+04f));
    p = fma2(p, z, pk2(-9.489117188e+04f, -9.489117188e+04f));
    p = fma2(p, z, pk2(1.081302109e+05f, 1.081302109e+05f));
    p = fma2(p, z, pk2(-1.260154688e+05f, -1.260154688e+05f));
    p = fma2(p, z, pk2(1.512498594e+05f, 1.512498594e+05f));
    p = fma2(p, z, pk2(-1.890981094e+05f, -1.890981094e+05f));
    p = fma2(p, z, pk2(2.521303281e+05f, 2.521303281e+05f));
    p = fma2(p, z, pk2(-3.781938438e+05f, -3.781938438e+05f));
    p = fma2(p, z, pk2(7.563876875e+05f, 7.563876875e+05f));
    return fma2(p, z, pk2(12582912.0f, 12582912.0f));
}

// A work item of the model batch: tiles [tile0, tile0 + n_tiles) of a model,
// partial sums at `slot` among that model's.
struct BatchItem {
    int model, tile0, n_tiles, slot;
};

// ---- per-call preparation: W image and set exponents ------------------------
// One block per (chunk, half, slice).
__device__ __forceinline__ void batched_prep_block(const BatchArgs &a, const int blk)
{
    const int p = blk % kWSlices, h = (blk / kWSlices) & 1, c = blk / (2 * kWSlices);
    const int Nw = a.n_waves, KB = (a.F + 63) / 64;
    __shared__ int s_T[kHS];
    if (threadIdx.x < kHS) {
        const int k = c * kKC + h * kHS + threadIdx.x;
        int e = 0;
        if (k < a.K) {
            double m = 0.0;
            bool finite = true;
            for (int w = 0; w < Nw; ++w) {
                const double vr = a.V[2 * ((size_t)k * Nw + w)], vi = a.V[2 * ((size_t)k * Nw + w) + 1];
                finite = finite && isfinite(vr) && isfinite(vi);
                m = fmax(m, fmax(fabs(vr), fabs(vi)));
            }
            if (finite && m > 0.0)
                frexp(m, &e);
            if (p == 0) {
                a.T[k] = e;
                if (!finite)  // every intensity of this set is undefined
                    atomicOr(&a.kflags[c * 2 + h], 1u << threadIdx.x);
            }
        }
        s_T[threadIdx.x] = e;
    }
    __syncthreads();
    unsigned char *out = a.wimg + (size_t)(c * 2 + h) * KB * kWSlices * kWBlock + (size_t)p * kWBlock;
    for (int idx = threadIdx.x; idx < KB * 64 * 64; idx += blockDim.x) {
        const int kb = idx >> 12, r = (idx >> 6) & 63, fb = idx & 63;
        const int f = kb * 64 + fb, sl = r >> 1, t = r & 1;
        const int k = c * kKC + h * kHS + sl;
        float val = 0.f;
        if (k < a.K && f < 2 * Nw) {
            const int w = f >> 1, u = f & 1;
            const double vr = a.V[2 * ((size_t)k * Nw + w)], vi = a.V[2 * ((size_t)k * Nw + w) + 1];
            const double coef = t == 0 ? (u == 0 ? vr : -vi) : (u == 0 ? vi : vr);
            double ws[kWSlices];
            split_slices(coef, s_T[sl], ws);
            val = isfinite(coef) ? (float)ws[p] : 0.f;
        }
        *reinterpret_cast<__nv_bfloat16 *>(out + kb * kWSlices * kWBlock + sw128(r, fb * 2)) =
            __float2bfloat16_rn(val);
    }
}

__global__ void batched_prep(const BatchArgs a) { batched_prep_block(a, blockIdx.x); }

// The preparation of every model of a batch: blocks_per_model blocks each.
__global__ void batched_items_prep(const BatchArgs *__restrict__ models, int blocks_per_model)
{
    batched_prep_block(models[blockIdx.x / blocks_per_model], blockIdx.x % blocks_per_model);
}

// ---- main kernel ----------------------------------------------------------------
// The CTA's share of one launch: tiles tile0 + j stride for j < n_tiles of
// one sample, with its partial sums at `slot` of the sample's scratch; the
// helper warp forms M V for the sets mv_k0, mv_k0 + mv_kstride, ...
struct TileRange {
    int tile0, n_tiles, stride, slot;
    int mv_k0, mv_kstride;
};

// The CTA's barriers and small state (declared once per kernel, so that the
// several instantiations of the body in one kernel share them).
struct BatchShared {
    uint64_t w_full, x_full[kXSMax], x_empty[kXSMax], s_full, s_free, r_full, r_free, g_done;
    uint32_t tmem_base;
    int s_flags;
    unsigned s_kflags[2 * kMaxChunks];
};

template <int F, int XS>
__device__ __forceinline__ void batched_body(const BatchArgs &a,
                                             const TileRange &tr, unsigned char *smem_dyn,
                                             BatchShared &sh)
{
    constexpr int KB = (F + 63) / 64;
    constexpr int kGCol = s_cols(XS);
    constexpr uint32_t kXBlk = XS * F * 128;    // one 64-event block: x0 (and x1) rows
    constexpr uint32_t kXBytes = 2 * kXBlk;     // one stage
    uint64_t &w_full = sh.w_full, &s_full = sh.s_full, &s_free = sh.s_free, &r_full = sh.r_full,
             &r_free = sh.r_free, &g_done = sh.g_done;
    uint64_t *x_full = sh.x_full, *x_empty = sh.x_empty;
    uint32_t &tmem_base = sh.tmem_base;
    int &s_flags = sh.s_flags;
    unsigned *s_kflags = sh.s_kflags;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NCH = a.n_chunks;
    // half chunks per tile that hold parameter sets (a last half past K is skipped)
    const int HPT = batch_hpt(a.K);
    const Smem L = batch_smem(F, XS, HPT, a.nxs_req);
    const int NXS = L.nxs;
    unsigned char *base = smem_dyn + ((1024 - (smem_u32(smem_dyn) & 1023)) & 1023);
    unsigned char *sW = base + L.w_off;
    unsigned char *sX = base + L.x_off;
    unsigned char *sR = base + L.r_off;
    const int n_my = tr.n_tiles;
    const int steps = n_my * HPT;

    if (threadIdx.x == 0) {
        mbar_init(&w_full, 1);
        for (int s = 0; s < NXS; ++s) {
            mbar_init(&x_full[s], 1);
            mbar_init(&x_empty[s], 1);
        }
        mbar_init(&s_full, 1);
        mbar_init(&s_free, kEpiWarps);
        mbar_init(&r_full, kEpiWarps);
        mbar_init(&r_free, 1);
        mbar_init(&g_done, 1);
        fence_barrier_init();
        s_flags = 0;
    }
    if (threadIdx.x < 2 * kMaxChunks)
        s_kflags[threadIdx.x] = 0;
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
            mbar_arrive_expect_tx(&w_full, L.w_bytes);
            bulk_load(sW, a.wimg, L.w_bytes, &w_full);
            int j = 0;
            for (; j < n_my; ++j) {
                const int s = j % NXS;
                const uint32_t u = j / NXS;
                if (u > 0 && !mbar_wait(&x_empty[s], (u & 1) ^ 1)) {
                    flags |= FLAG_TIMEOUT;
                    break;
                }
                const int64_t tile = tr.tile0 + (int64_t)j * tr.stride;
                mbar_arrive_expect_tx(&x_full[s], kXBytes);
                bulk_load(sX + (size_t)s * kXBytes, a.xg + tile * kXBytes, kXBytes, &x_full[s]);
            }
            // copies still in flight complete before the block may exit
            for (int q = (j > NXS ? j - NXS : 0); q < j; ++q)
                if (!mbar_wait(&x_full[q % NXS], (q / NXS) & 1))
                    flags |= FLAG_TIMEOUT;
            if (!mbar_wait(&w_full, 0))
                flags |= FLAG_TIMEOUT;
        }
    } else if (warp == kEpiWarps + 1) {
        // ---- MMA issuer ---------------------------------------------------
        if (lane == 0) {
            const uint32_t id64 = umma_idesc_bf16(128, 64, 1, 0);
            const uint32_t id128 = umma_idesc_bf16(128, 128, 1, 0);
            const uint32_t id192 = umma_idesc_bf16(128, 192, 1, 0);
            const uint32_t id2 = umma_idesc_bf16(128, XS * F, 1, 0);
            const uint32_t xbase = smem_u32(sX), wbase = smem_u32(sW), rbase = smem_u32(sR);
            // descriptors without their start address (added as address / 16 below)
            const uint64_t dA = umma_desc_sw128(0, kXBlk, 1024);      // X, MN-major
            const uint64_t dR = umma_desc_sw128(0, 128 * 128, 1024);  // R', MN-major
            const uint64_t dK = umma_desc_sw128(0, 16, 1024);         // K-major operands
            // GEMM 2 of chunk step cq (its R' complete: r_full phase cq)
            auto gemm2 = [&](int cq) {
                const int j = cq / NCH, c = cq % NCH, s = j % NXS;
                tc_fence_after();
                const uint32_t xs = xbase + s * kXBytes;
#pragma unroll
                for (int ks = 0; ks < kBM / 16; ++ks) {
                    const uint32_t ra = rbase + ks * 2048;
                    const uint32_t xa = xs + (ks >> 2) * kXBlk + (ks & 3) * 32;
                    umma_bf16(tmem + kGCol + c * XS * F, dR + (ra >> 4), dK + (xa >> 4), id2,
                              (j > 0 || ks > 0) ? 1u : 0u);
                }
                umma_commit(&r_free);
                if (c == NCH - 1)
                    umma_commit(&x_empty[s]);
            };
            // GEMM 2 does not wait in line behind GEMM 1: while the thread
            // waits for a barrier (bar, parity), it issues the GEMM 2 of each
            // chunk step whose R' is complete, in order, and returns once the
            // barrier's phase is complete and at least `need` GEMM 2s are
            // issued (bar = null: the barrier part holds). It polls without
            // sleeping: a suspended thread was measured to resume up to ~1300
            // cycles after the phase completed, on the critical path of GEMM 1.
            // GEMM 1 of the first half of
            // chunk step cq needs the GEMM 2 of cq - 2 issued: its completion,
            // seen by the epilogue as s_full, then implies that r_free has
            // passed phase cq - 2, so the epilogue's parity wait for phase
            // cq - 1 cannot match an older phase. Bounded as mbar_wait.
            int g2 = 0, g2_ready = 0;   // next GEMM 2; chunk steps whose GEMM 1s are issued
            auto serve = [&](uint64_t *bar, uint32_t parity, int need) -> bool {
                const unsigned long long t0 = global_timer_ns();
                for (unsigned it = 1;; ++it) {
                    if (g2 < g2_ready && mbar_test(&r_full, g2 & 1)) {
                        gemm2(g2++);
                        continue;
                    }
                    if (g2 >= need && (!bar || mbar_test(bar, parity)))
                        return true;
                    if ((it & 255) == 0 && global_timer_ns() - t0 > kWaitLimitNs)
                        return false;
                }
            };
            bool ok = mbar_wait(&w_full, 0);
            for (int q = 0; q < steps && ok; ++q) {
                const int j = q / HPT, ch = q % HPT, c = ch >> 1, h = ch & 1, s = j % NXS;
                const int need = h == 0 ? j * NCH + c - 1 : 0;
                if (ch == 0 && !serve(&x_full[s], (j / NXS) & 1, need)) {
                    ok = false;
                    break;
                }
                if (q >= 1 && !serve(&s_free, (q - 1) & 1, need)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t xs = xbase + s * kXBytes;
                const uint32_t wb = wbase + (uint32_t)(c * 2 + h) * KB * kWSlices * kWBlock;
                // accumulator j (64 columns at 64 j) collects the slice products x_i w_p, i + p = j
#pragma unroll
                for (int ks = 0; ks < F / 16; ++ks) {
                    const uint32_t x0a = xs + ks * 2048;
                    const uint32_t wa = wb + (ks >> 2) * kWSlices * kWBlock + (ks & 3) * 32;
                    const uint32_t acc = ks > 0 ? 1u : 0u;
                    if (XS == 2) {
                        // x0 [w0|w1|w2] into acc0..2 and x1 [w0|w1|w2] into acc1..3:
                        // two N = 192 products per K step; in the first, acc3
                        // is started by x1 w2 alone (one accumulate flag per MMA)
                        const uint32_t x1a = x0a + F * 128;
                        umma_bf16(tmem, dA + (x0a >> 4), dK + (wa >> 4), id192, acc);        // acc0..2 x0 [w0|w1|w2]
                        if (ks == 0) {
                            umma_bf16(tmem + 192, dA + (x1a >> 4), dK + ((wa + 2 * kWBlock) >> 4), id64,
                                      0u);                                                   // acc3    x1 w2
                            umma_bf16(tmem + 64, dA + (x1a >> 4), dK + (wa >> 4), id128, 1u);  // acc1..2 x1 [w0|w1]
                        } else {
                            umma_bf16(tmem + 64, dA + (x1a >> 4), dK + (wa >> 4), id192, 1u);  // acc1..3 x1 [w0|w1|w2]
                        }
                    } else {
                        umma_bf16(tmem, dA + (x0a >> 4), dK + (wa >> 4), id192, acc);        // acc0..2 x0 [w0|w1|w2]
                    }
                }
                umma_commit(&s_full);
                if (h == 1 || ch == HPT - 1)  // the chunk step's last GEMM 1
                    g2_ready = j * NCH + c + 1;
            }
            if (ok && !serve(nullptr, 0, g2_ready))
                ok = false;
            umma_commit(&g_done);
            // tensor memory is released only after every product has finished
            if (!mbar_wait(&g_done, 0))
                ok = false;
            if (!ok)
                flags |= FLAG_TIMEOUT;
        }
    } else if (warp < kEpiWarps) {
        // ---- epilogue -------------------------------------------------------
        const int qq = warp & 3, sg = warp >> 2;
        const int e = qq * 32 + lane;                  // event row of the tile = TMEM lane
        const uint32_t lane_addr = (uint32_t)(qq * 32) << 16;
        // per-thread constants: R' store offsets, the atomic partials of this lane
        const uint32_t st0 = sw128(e, 32 * sg), st1 = sw128(e, 32 * sg + 16);
        unsigned long long *lp = reinterpret_cast<unsigned long long *>(
            a.lpart + ((size_t)tr.slot * 4 + qq) * (NCH * kKC) + 8 * sg + lane);
        const f2 c8 = pk2(1.0f / 256.0f, 1.0f / 256.0f), one2 = pk2(1.0f, 1.0f);
        int64_t ev = (int64_t)tr.tile0 * kBM + e;          // this thread's event in tile j
        const int64_t ev_step = (int64_t)tr.stride * kBM;
        bool ok = true;
        int j = 0, ch = 0;                                 // tile, half chunk (q = j HPT + ch)
        for (int q = 0; q < steps && ok; ++q) {
            const int h = ch & 1, cq = j * NCH + (ch >> 1);
            const bool last_half = h == 1 || ch == HPT - 1;
            if (!mbar_wait(&s_full, q & 1)) {
                ok = false;
                break;
            }
            tc_fence_after();
            // a warp whose 8 sets all lie past K (padding of the last half
            // chunk) keeps to the barriers and does no work: its rows of R'
            // feed only the G^T rows of those sets, which are never read
            const int nvs = a.K - (ch >> 1) * kKC - h * kHS - 8 * sg;
            const bool idle = nvs <= 0;
            // Q = acc0 + (acc1 + (acc2 + acc3 / 2^8) / 2^8) / 2^8 of this warp's
            // 8 sets, as (re, im) pairs
            f2 qv[8];
            if (!idle) {
                uint32_t v0[16], v1[16], v2[16], v3[16];
                tmem_ld16(tmem + lane_addr + 16 * sg, v0);
                tmem_ld16(tmem + lane_addr + 64 + 16 * sg, v1);
                tmem_ld16(tmem + lane_addr + 128 + 16 * sg, v2);
                if (XS == 2)
                    tmem_ld16(tmem + lane_addr + 192 + 16 * sg, v3);
                tmem_ld_wait();
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    f2 u = pk2(__uint_as_float(v2[2 * t]), __uint_as_float(v2[2 * t + 1]));
                    if (XS == 2)
                        u = fma2(pk2(__uint_as_float(v3[2 * t]), __uint_as_float(v3[2 * t + 1])), c8, u);
                    u = fma2(u, c8, pk2(__uint_as_float(v1[2 * t]), __uint_as_float(v1[2 * t + 1])));
                    qv[t] = fma2(u, c8, pk2(__uint_as_float(v0[2 * t]), __uint_as_float(v0[2 * t + 1])));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&s_free);
            uint32_t rpk[8];
            int l[8];
            if (!idle && ev < a.n_events) {
                float zz[8];
                int kk[8];
                unsigned mn = 0xffffffffu;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    float qr, qi;
                    upk2(qv[t], qr, qi);
                    const float I = fmaf(qr, qr, qi * qi);
                    const int bits = __float_as_int(I);
                    mn = min(mn, (unsigned)bits);
                    const float r = rcp_approx(I);
                    float rr, ri;
                    upk2(mul2(qv[t], pk2(r, r)), rr, ri);
                    rpk[t] = pack_bf16x2(rr, ri);
                    // I = 2^k (1 + z), 1 + z in [sqrt(1/2), sqrt(2)): km = k 2^23
                    // (the arithmetic shift's low bits cleared)
                    const int km = (bits - 0x3F3504F3) & (int)0xFF800000;
                    zz[t] = __int_as_float(bits - km);
                    kk[t] = km >> (23 - kFixBits);
                }
#pragma unroll
                for (int t = 0; t < 8; t += 2) {
                    float y0, y1;
                    upk2(log2_fixed2(sub2(pk2(zz[t], zz[t + 1]), one2)), y0, y1);
                    l[t] = __float_as_int(y0) - 0x4B400000 + kk[t];
                    l[t + 1] = __float_as_int(y1) - 0x4B400000 + kk[t + 1];
                }
                if (mn == 0u) {  // some Q = 0 (rare): record the parameter sets, if real
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        float qr, qi;
                        upk2(qv[t], qr, qi);
                        if (t < nvs && fmaf(qr, qr, qi * qi) == 0.f)
                            atomicOr(&s_kflags[ch], 1u << (8 * sg + t));
                    }
                }
            } else {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    rpk[t] = 0u;
                    l[t] = 0;
                }
            }
            // fixed-point log2 sums over the warp's 32 events; lane t keeps set t
            if (!idle) {
                int mine = 0;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int sum = __reduce_add_sync(0xffffffffu, l[t]);
                    mine = lane == t ? sum : mine;
                }
                if (lane < 8)  // no return value: a fire-and-forget reduction
                    atomicAdd(lp + ch * kHS, (unsigned long long)(long long)mine);
            }
            // R' may be overwritten once GEMM 2 of the previous chunk step is done
            if (h == 0 && cq >= 1 && !mbar_wait(&r_free, (cq - 1) & 1)) {
                ok = false;
                break;
            }
            unsigned char *rrow = sR + h * (128 * 128);
            if (!idle) {
                *reinterpret_cast<uint4 *>(rrow + st0) = make_uint4(rpk[0], rpk[1], rpk[2], rpk[3]);
                *reinterpret_cast<uint4 *>(rrow + st1) = make_uint4(rpk[4], rpk[5], rpk[6], rpk[7]);
            }
            if (last_half) {
                fence_async_smem();
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&r_full);
            }
            if (++ch == HPT) {
                ch = 0;
                ++j;
                ev += ev_step;
            }
        }
        if (!ok)
            flags |= FLAG_TIMEOUT;
        // G^T of every chunk: rows = this warp's lane quarter, 8-column groups
        if (ok && mbar_wait(&g_done, 0)) {
            tc_fence_after();
            for (int c = 0; c < NCH; ++c) {
                for (int c0 = 8 * sg; c0 < F; c0 += 32) {
                    uint32_t g[8], g1[8];
                    if (n_my > 0) {
                        tmem_ld8(tmem + lane_addr + kGCol + c * XS * F + c0, g);
                        if (XS == 2)
                            tmem_ld8(tmem + lane_addr + kGCol + c * XS * F + F + c0, g1);
                        tmem_ld_wait();
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            g[i] = g1[i] = 0u;
                    }
                    float gv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        gv[i] = XS == 2 ? fmaf(__uint_as_float(g1[i]), 1.0f / 256.0f, __uint_as_float(g[i]))
                                        : __uint_as_float(g[i]);
                    float4 *dst = reinterpret_cast<float4 *>(
                        a.gpart + (((size_t)tr.slot * NCH + c) * 128 + e) * F + c0);
                    dst[0] = make_float4(gv[0], gv[1], gv[2], gv[3]);
                    dst[1] = make_float4(gv[4], gv[5], gv[6], gv[7]);
                }
            }
        } else {
            flags |= FLAG_TIMEOUT;
        }
    } else if (warp == kEpiWarps + 2) {
        // ---- helper: M V and V^H M V for the sets mv_k0, + mv_kstride, ... --
        const int Nw = a.n_waves;
        for (int k = tr.mv_k0; k < a.K; k += tr.mv_kstride) {
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

// One sample, a persistent grid: CTA b takes tiles b, b + grid, ...
template <int F, int XS>
__global__ void __launch_bounds__(kThreads, 1)
    batched_kernel(const BatchArgs a, const int n_tiles)
{
    extern __shared__ unsigned char smem_dyn[];
    __shared__ BatchShared sh;
    TileRange tr;
    tr.tile0 = blockIdx.x;
    tr.stride = gridDim.x;
    tr.n_tiles = (n_tiles > (int)blockIdx.x) ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    tr.slot = blockIdx.x;
    tr.mv_k0 = blockIdx.x;
    tr.mv_kstride = gridDim.x;
    batched_body<F, XS>(a, tr, smem_dyn, sh);
}

// Many samples (the uneven model batch) in one launch: CTA b is the work item
// items[b], a contiguous range of one model's tiles; its partials go to the
// item's slot among the model's, and the model's first item forms M V. The
// hardware starts an item's CTA as an SM frees up; the items and the order
// in which the final kernel adds their partials are fixed, so the results
// do not depend on that schedule. The body is instantiated per feature
// count F (the tile shape of each wave-count bucket).
template <int XS>
__global__ void __launch_bounds__(kThreads, 1)
    batched_items_kernel(const BatchItem *__restrict__ items, const BatchArgs *__restrict__ models)
{
    extern __shared__ unsigned char smem_dyn[];
    __shared__ BatchShared sh;
    const BatchItem it = items[blockIdx.x];
    const BatchArgs &a = models[it.model];
    TileRange tr;
    tr.tile0 = it.tile0;
    tr.n_tiles = it.n_tiles;
    tr.stride = 1;
    tr.slot = it.slot;
    tr.mv_k0 = it.slot == 0 ? 0 : a.K;    // the model's first item forms M V
    tr.mv_kstride = 1;
    switch (a.F) {
    case 16: batched_body<16, XS>(a, tr, smem_dyn, sh); break;
    case 32: batched_body<32, XS>(a, tr, smem_dyn, sh); break;
    case 48: batched_body<48, XS>(a, tr, smem_dyn, sh); break;
    case 64: batched_body<64, XS>(a, tr, smem_dyn, sh); break;
    case 80: batched_body<80, XS>(a, tr, smem_dyn, sh); break;
    case 96: batched_body<96, XS>(a, tr, smem_dyn, sh); break;
    default: break;
    }
}

// Final sums over the n_slots partial slots of a sample (fixed order), M V,
// the first-order correction for V - V_r; one block per parameter set.
__device__ __forceinline__ void batched_finalize_set(const BatchArgs &a, int k, int n_slots,
                                                     int *done, double *nll, double *grad)
{
    const int grid = n_slots;
    const int Nw = a.n_waves, F = a.F, NCH = a.n_chunks;
    const int c = k / kKC, kl = k % kKC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ double s_corr[2];
    __shared__ long long s_l;
    const bool bad = (a.kflags[2 * c + (kl >> 5)] >> (kl & 31)) & 1u;
    const int T = a.T[k];
    const double gscale = ldexp(1.0, 8 - T);
    double corr = 0.0;
    for (int w = threadIdx.x; w < Nw; w += blockDim.x) {
        // Re conj(A) r = G[(k,re)][2w] + G[(k,im)][2w+1];  Im = G[(k,im)][2w] - G[(k,re)][2w+1]
        dfloat s_re = {0.f, 0.f}, s_im = {0.f, 0.f};
        const size_t cta_stride = (size_t)NCH * 128 * F;
        const float *g0 = a.gpart + (size_t)c * 128 * F;
        for (int b0 = 0; b0 < grid; b0 += 16) {
            float2 re_row[16], im_row[16];
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
        const double gre = -gscale * ((double)s_re.hi + (double)s_re.lo);
        const double gim = -gscale * ((double)s_im.hi + (double)s_im.lo);
        const double *V = a.V + 2 * ((size_t)k * Nw + w);
        const double dvr = V[0] - round_slices(V[0], T), dvi = V[1] - round_slices(V[1], T);
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
        long long l = 0;
        for (int i = lane; i < grid * 4; i += 32)
            l += a.lpart[(size_t)i * (NCH * kKC) + k];
        l = warp_sum(l);
        if (lane == 0)
            s_l = l;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long ex = 2 * *a.sum_e + 2 * a.n_events * (long long)(T - 16);
        const double lnsum = kLn2 * ((double)ex + ldexp((double)s_l, -kFixBits));
        const double nv = a.mv[(size_t)k * (2 * Nw + 1) + 2 * Nw];
        double v = -lnsum + nv + s_corr[0] + (blockDim.x > 32 ? s_corr[1] : 0.0);
        if (bad) {
            v = INFINITY;
            atomicOr(a.status, FLAG_DOMAIN);
        }
        nll[k] = v;
        if (done)
            atomicAdd(done, 1);
    }
}

__global__ void batched_finalize(const BatchArgs a, int grid, int *done, double *nll, double *grad)
{
    batched_finalize_set(a, blockIdx.x, grid, done, nll, grad);
}

// The final sums of every model of a batch: block b is set b % K of model b / K.
__global__ void batched_items_finalize(const BatchArgs *__restrict__ models, const int *n_slots,
                                       int K, int *const *done, double *const *nll,
                                       double *const *grad)
{
    const int m = blockIdx.x / K, k = blockIdx.x % K;
    batched_finalize_set(models[m], k, n_slots[m], done[m], nll[m], grad[m]);
}

// ---- block-floating-point encoding of the data (once per load) ---------------
// One thread per event: shared exponent E = exponent of the largest |feature|
// (max = m 2^E, m in [1/2, 1)), slices x0 = rint(A 2^(8-E)) and, for XS = 2,
// x1 = rint((A 2^(8-E) - x0) 256). Written in the tile order the kernel's
// shared memory uses: event i sits in 64-event block i / 64 (xs F 128 bytes,
// consecutive blocks), row r (x0 rows, then x1 rows) at 128-byte pitch with
// the 128-byte swizzle, at byte 2 (i % 64) of its row.
__global__ void batched_encode_kernel(const float *__restrict__ planes, int64_t pitch, int64_t n,
                                      int rows_in, int F, int xs, unsigned char *__restrict__ out,
                                      long long *sum_e)
{
    long long es = 0;
    const size_t blk_bytes = (size_t)xs * F * 128;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < pitch;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool valid = i < n;
        float m = 0.f;
        if (valid)
            for (int r = 0; r < rows_in; ++r)
                m = fmaxf(m, fabsf(planes[(int64_t)r * pitch + i]));
        int E = 0;
        if (m > 0.f)
            frexpf(m, &E);
        unsigned char *blk = out + (size_t)(i >> 6) * blk_bytes;
        const int byte = 2 * (int)(i & 63);
        for (int r = 0; r < F; ++r) {
            float x0 = 0.f, x1 = 0.f;
            if (valid && r < rows_in) {
                const float x = ldexpf(planes[(int64_t)r * pitch + i], 8 - E);
                x0 = rintf(x);
                x1 = rintf((x - x0) * 256.f);
            }
            *reinterpret_cast<__nv_bfloat16 *>(blk + sw128(r, byte)) = __float2bfloat16_rn(x0);
            if (xs == 2)
                *reinterpret_cast<__nv_bfloat16 *>(blk + sw128(F + r, byte)) = __float2bfloat16_rn(x1);
        }
        if (valid)
            es += E;
    }
    es = warp_sum(es);
    __shared__ long long s_e[8];
    if ((threadIdx.x & 31) == 0)
        s_e[threadIdx.x >> 5] = es;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            t += s_e[w];
        atomicAdd(reinterpret_cast<unsigned long long *>(sum_e), (unsigned long long)t);
    }
}

template <int F, int XS>
cudaError_t configure_f()
{
    return cudaFuncSetAttribute(batched_kernel<F, XS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kMaxSmem);
}

template <int XS>
cudaError_t configure_xs()
{
    cudaError_t e = cudaSuccess;
    for (cudaError_t r : {configure_f<16, XS>(), configure_f<32, XS>(), configure_f<48, XS>(),
                          configure_f<64, XS>(), configure_f<80, XS>(), configure_f<96, XS>(),
                          cudaFuncSetAttribute(batched_items_kernel<XS>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               kMaxSmem)})
        if (r != cudaSuccess)
            e = r;
    return e;
}

template <int XS>
cudaError_t launch_main(int F, int grid, uint32_t smem, cudaStream_t s, const BatchArgs &a,
                        int n_tiles)
{
    switch (F) {
    case 16: batched_kernel<16, XS><<<grid, kThreads, smem, s>>>(a, n_tiles); break;
    case 32: batched_kernel<32, XS><<<grid, kThreads, smem, s>>>(a, n_tiles); break;
    case 48: batched_kernel<48, XS><<<grid, kThreads, smem, s>>>(a, n_tiles); break;
    case 64: batched_kernel<64, XS><<<grid, kThreads, smem, s>>>(a, n_tiles); break;
    case 80: batched_kernel<80, XS><<<grid, kThreads, smem, s>>>(a, n_tiles); break;
    case 96: batched_kernel<96, XS><<<grid, kThreads, smem, s>>>(a, n_tiles); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

struct ScratchLayout {
    size_t wimg, gpart, lpart, mv, T, kflags, total;
};

ScratchLayout scratch_layout(int F, int xs, int n_waves, int K, int grid)
{
    const int nch = (K + kKC - 1) / kKC;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    ScratchLayout s;
    s.wimg = 0;
    s.gpart = up(s.wimg + w_image_bytes(F, nch));
    s.lpart = up(s.gpart + (size_t)grid * nch * 128 * F * 4);
    s.mv = up(s.lpart + (size_t)grid * 4 * nch * kKC * 8);
    s.T = up(s.mv + (size_t)K * (2 * n_waves + 1) * 8);
    s.kflags = up(s.T + (size_t)K * 4);
    s.total = up(s.kflags + (size_t)nch * 2 * 4);
    return s;
}

}  // namespace

int batched_features(int n_waves) { return (2 * n_waves + 15) / 16 * 16; }

int batched_max_k(int n_waves, int xs)
{
    const int F = batched_features(n_waves);
    int nch = kMaxChunks;
    while (nch > 0 &&
           (s_cols(xs) + nch * xs * F > 512 ||
            (int)batch_smem(F, xs, batch_hpt(nch * kKC)).bytes > kMaxSmem))
        --nch;
    return nch * kKC;
}

int batched_max_x_stages(int n_waves, int xs, int K)
{
    return batch_smem(batched_features(n_waves), xs, batch_hpt(K)).nxs;
}

size_t batched_scratch_bytes(int n_waves, int xs, int K, int grid)
{
    return scratch_layout(batched_features(n_waves), xs, n_waves, K, grid).total;
}

cudaError_t batched_configure()
{
    const cudaError_t e1 = configure_xs<1>(), e2 = configure_xs<2>();
    return e1 != cudaSuccess ? e1 : e2;
}

cudaError_t launch_batched_encode(const float *planes, int64_t pitch, int64_t n, int n_waves, int xs,
                                  void *out, long long *sum_e, cudaStream_t s)
{
    if (xs != 1 && xs != 2)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(sum_e, 0, sizeof(long long), s);
    if (e != cudaSuccess)
        return e;
    const int blocks = (int)std::min<int64_t>((pitch + 255) / 256, 4096);
    batched_encode_kernel<<<blocks, 256, 0, s>>>(planes, pitch, n, 2 * n_waves,
                                                 batched_features(n_waves), xs,
                                                 static_cast<unsigned char *>(out), sum_e);
    return cudaGetLastError();
}

// K <= batched_max_k(n_waves, xs) parameter sets; scratch >= batched_scratch_bytes.
cudaError_t launch_batched(const void *xbf, int64_t n_events, int n_waves, int xs,
                           const long long *sum_e, const double *V, int K, const double *M,
                           void *scratch, int grid, int *status, int *done, double *nll,
                           double *grad, cudaStream_t s, int nxs)
{
    const int F = batched_features(n_waves), nch = (K + kKC - 1) / kKC;
    if ((xs != 1 && xs != 2) || K < 1 || K > batched_max_k(n_waves, xs) || grid < 1)
        return cudaErrorInvalidValue;
    const ScratchLayout sl = scratch_layout(F, xs, n_waves, K, grid);
    char *p = static_cast<char *>(scratch);
    BatchArgs a{};
    a.n_waves = n_waves;
    a.F = F;
    a.XS = xs;
    a.K = K;
    a.n_chunks = nch;
    a.xg = static_cast<const unsigned char *>(xbf);
    a.n_events = n_events;
    a.V = V;
    a.M = M;
    a.sum_e = sum_e;
    a.wimg = reinterpret_cast<unsigned char *>(p + sl.wimg);
    a.gpart = reinterpret_cast<float *>(p + sl.gpart);
    a.lpart = reinterpret_cast<long long *>(p + sl.lpart);
    a.mv = reinterpret_cast<double *>(p + sl.mv);
    a.T = reinterpret_cast<int *>(p + sl.T);
    a.kflags = reinterpret_cast<unsigned *>(p + sl.kflags);
    a.status = status;
    a.nxs_req = nxs;
    cudaError_t e = cudaMemsetAsync(a.kflags, 0, nch * 2 * 4, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(a.lpart, 0, (size_t)grid * 4 * nch * kKC * 8, s);
    if (e != cudaSuccess)
        return e;
    batched_prep<<<nch * 2 * kWSlices, 256, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const int n_tiles = (int)((n_events + kBM - 1) / kBM);
    const uint32_t smem = batch_smem(F, xs, batch_hpt(K), nxs).bytes;
    e = xs == 2 ? launch_main<2>(F, grid, smem, s, a, n_tiles)
                : launch_main<1>(F, grid, smem, s, a, n_tiles);
    if (e != cudaSuccess)
        return e;
    batched_finalize<<<K, 64, 0, s>>>(a, grid, done, nll, grad);
    return cudaGetLastError();
}

// ---- the uneven model batch in one launch -------------------------------------
// Plan buffer (device, one allocation), in this order: BatchArgs[n_models],
// BatchItem[n_items], int
// n_slots[n_models], the per-model output pointers (done, nll, grad), then
// per model its scratch: W image, G^T partials, log partials, M V, set
// exponents, domain flags. The log partials and domain flags of all models
// are contiguous, so one memset clears them per call.
namespace {

struct PlanLayout {
    size_t args, items, nslots, pdone, pnll, pgrad, zero, zero_bytes, scratch, total;
    std::vector<size_t> wimg, gpart, lpart, mv, T, kflags;
    std::vector<BatchItem> items_h;
    std::vector<int> slots;
};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

PlanLayout plan_layout(const BatchModelDesc *m, int n_models, int xs, int K, int num_sms,
                       int items_per_sm)
{
    PlanLayout p;
    const int nch = (K + kKC - 1) / kKC;
    // work items: about num_sms * items_per_sm in all, of equal estimated
    // cost (tiles x (F + 32): the MMAs grow with F, the epilogue does not)
    std::vector<double> cost(n_models);
    double total = 0.0;
    for (int i = 0; i < n_models; ++i) {
        const int64_t tiles = (m[i].n_events + kBM - 1) / kBM;
        cost[i] = (double)tiles * (batched_features(m[i].n_waves) + 32);
        total += cost[i];
    }
    const double target = total / std::max(1, num_sms * items_per_sm);
    p.slots.resize(n_models);
    for (int i = 0; i < n_models; ++i) {
        const int tiles = (int)((m[i].n_events + kBM - 1) / kBM);
        int n_it = (int)std::lround(cost[i] / target);
        n_it = std::max(1, std::min(n_it, tiles));
        p.slots[i] = n_it;
        for (int k = 0; k < n_it; ++k) {
            const int t0 = (int)((int64_t)tiles * k / n_it), t1 = (int)((int64_t)tiles * (k + 1) / n_it);
            p.items_h.push_back({i, t0, t1 - t0, k});
        }
    }
    // largest items first: the hardware hands out CTAs in block order
    std::stable_sort(p.items_h.begin(), p.items_h.end(), [&](const BatchItem &x, const BatchItem &y) {
        return (double)x.n_tiles * (batched_features(m[x.model].n_waves) + 32) >
               (double)y.n_tiles * (batched_features(m[y.model].n_waves) + 32);
    });
    size_t o = 0;
    p.args = o;
    o = up256(o + sizeof(BatchArgs) * n_models);
    p.items = o;
    o = up256(o + sizeof(BatchItem) * p.items_h.size());
    p.nslots = o;
    o = up256(o + sizeof(int) * n_models);
    p.pdone = o;
    o = up256(o + sizeof(void *) * n_models);
    p.pnll = o;
    o = up256(o + sizeof(void *) * n_models);
    p.pgrad = o;
    o = up256(o + sizeof(void *) * n_models);
    p.zero = o;
    p.lpart.resize(n_models);
    p.kflags.resize(n_models);
    for (int i = 0; i < n_models; ++i) {
        p.lpart[i] = o;
        o = up256(o + (size_t)p.slots[i] * 4 * nch * kKC * 8);
        p.kflags[i] = o;
        o = up256(o + (size_t)nch * 2 * 4);
    }
    p.zero_bytes = o - p.zero;
    p.scratch = o;
    p.wimg.resize(n_models);
    p.gpart.resize(n_models);
    p.mv.resize(n_models);
    p.T.resize(n_models);
    for (int i = 0; i < n_models; ++i) {
        const int F = batched_features(m[i].n_waves);
        p.wimg[i] = o;
        o = up256(o + w_image_bytes(F, nch));
        p.gpart[i] = o;
        o = up256(o + (size_t)p.slots[i] * nch * 128 * F * 4);
        p.mv[i] = o;
        o = up256(o + (size_t)K * (2 * m[i].n_waves + 1) * 8);
        p.T[i] = o;
        o = up256(o + (size_t)K * 4);
    }
    p.total = o;
    return p;
}

}  // namespace

size_t batched_plan_bytes(const BatchModelDesc *models, int n_models, int xs, int K, int num_sms,
                          int items_per_sm, int *n_items)
{
    const PlanLayout p = plan_layout(models, n_models, xs, K, num_sms, items_per_sm);
    if (n_items)
        *n_items = (int)p.items_h.size();
    return p.total;
}

cudaError_t batched_plan_build(void *plan, const BatchModelDesc *models, int n_models, int xs,
                               int K, int num_sms, int items_per_sm, int nxs, cudaStream_t s)
{
    if ((xs != 1 && xs != 2) || K < 1 || n_models < 1)
        return cudaErrorInvalidValue;
    const PlanLayout p = plan_layout(models, n_models, xs, K, num_sms, items_per_sm);
    char *d = static_cast<char *>(plan);
    std::vector<char> h(p.scratch, 0);
    const int nch = (K + kKC - 1) / kKC;
    for (int i = 0; i < n_models; ++i) {
        const BatchModelDesc &m = models[i];
        if (K > batched_max_k(m.n_waves, xs))
            return cudaErrorInvalidValue;
        BatchArgs a{};
        a.n_waves = m.n_waves;
        a.F = batched_features(m.n_waves);
        a.XS = xs;
        a.K = K;
        a.n_chunks = nch;
        a.xg = static_cast<const unsigned char *>(m.xbf);
        a.n_events = m.n_events;
        a.V = m.V;
        a.M = m.M;
        a.sum_e = m.sum_e;
        a.wimg = reinterpret_cast<unsigned char *>(d + p.wimg[i]);
        a.gpart = reinterpret_cast<float *>(d + p.gpart[i]);
        a.lpart = reinterpret_cast<long long *>(d + p.lpart[i]);
        a.mv = reinterpret_cast<double *>(d + p.mv[i]);
        a.T = reinterpret_cast<int *>(d + p.T[i]);
        a.kflags = reinterpret_cast<unsigned *>(d + p.kflags[i]);
        a.status = m.status;
        a.nxs_req = nxs;
        memcpy(&h[p.args + i * sizeof(BatchArgs)], &a, sizeof a);
        memcpy(&h[p.nslots + i * sizeof(int)], &p.slots[i], sizeof(int));
        memcpy(&h[p.pdone + i * sizeof(void *)], &m.done, sizeof(void *));
        memcpy(&h[p.pnll + i * sizeof(void *)], &m.nll, sizeof(void *));
        memcpy(&h[p.pgrad + i * sizeof(void *)], &m.grad, sizeof(void *));
    }
    memcpy(&h[p.items], p.items_h.data(), p.items_h.size() * sizeof(BatchItem));
    // the host vector is staged through a synchronous copy: it goes away here
    cudaError_t e = cudaMemcpyAsync(d, h.data(), p.scratch, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    return e;
}

cudaError_t launch_batched_items(void *plan, const BatchModelDesc *models, int n_models, int xs,
                                 int K, int num_sms, int items_per_sm, int nxs, cudaStream_t s)
{
    const PlanLayout p = plan_layout(models, n_models, xs, K, num_sms, items_per_sm);
    char *d = static_cast<char *>(plan);
    const int nch = (K + kKC - 1) / kKC;
    uint32_t smem = 0;
    for (int i = 0; i < n_models; ++i)
        smem = std::max(smem,
                        batch_smem(batched_features(models[i].n_waves), xs, batch_hpt(K), nxs).bytes);
    cudaError_t e = cudaMemsetAsync(d + p.zero, 0, p.zero_bytes, s);
    if (e != cudaSuccess)
        return e;
    const BatchArgs *args = reinterpret_cast<const BatchArgs *>(d + p.args);
    const int bpm = nch * 2 * kWSlices;
    batched_items_prep<<<n_models * bpm, 256, 0, s>>>(args, bpm);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    const BatchItem *items = reinterpret_cast<const BatchItem *>(d + p.items);
    const int n_items = (int)p.items_h.size();
    if (xs == 2)
        batched_items_kernel<2><<<n_items, kThreads, smem, s>>>(items, args);
    else
        batched_items_kernel<1><<<n_items, kThreads, smem, s>>>(items, args);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    batched_items_finalize<<<n_models * K, 64, 0, s>>>(
        args, reinterpret_cast<const int *>(d + p.nslots), K,
        reinterpret_cast<int *const *>(d + p.pdone), reinterpret_cast<double *const *>(d + p.pnll),
        reinterpret_cast<double *const *>(d + p.pgrad));
    return cudaGetLastError();
}

}  // namespace pwa
