// Internal declarations shared by the CUDA translation units of libpwa.
// Device helpers here are thin inline-PTX wrappers for sm_103a: mbarrier,
// TMA (cp.async.bulk.tensor) and a bounded wait built on %globaltimer.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pwa.h"

namespace pwa {

// Device-side status bits, OR-ed into a status word by the kernels.
enum : int {
    FLAG_DOMAIN = 1,   // an intensity was <= 0 or not finite
    FLAG_TIMEOUT = 2,  // a bounded wait gave up
};

// Upper bound on any single device-side wait (nanoseconds).
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

constexpr int kMaxWaves = 48;

// --------------------------------------------------------------------------
// PTX wrappers
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_timer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One test of the phase; the thread may sleep until the phase completes, for
// at most about kSuspendNs (a hint), instead of spinning on the issue slots.
constexpr uint32_t kSuspendNs = 100000;

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// Non-blocking test of the phase (never suspends the thread): for loops that
// poll several barriers.
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete; gives up after
// limit_ns (default kWaitLimitNs) and returns false (the caller records
// FLAG_TIMEOUT).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitLimitNs)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = global_timer_ns();
    for (;;) {
        for (int i = 0; i < 4; ++i)
            if (mbar_try_wait(bar, parity))
                return true;
        if (global_timer_ns() - t0 > limit_ns)
            return false;
    }
}

// 2D tiled TMA load global -> shared, completion signalled on `bar`.
// x is the innermost coordinate (elements); x * sizeof(elem) must be a
// multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// ---- tcgen05 (5th-generation tensor cores) --------------------------------
// Shared-memory matrix descriptor for a 128-byte-swizzled operand: start
// address, leading and stride byte offsets (16-byte units), version 1,
// layout SWIZZLE_128B. K-major: rows 128 B apart in 8-row (1 KB) atoms, SBO =
// 1 KB, LBO unused. MN-major: 64 M/N elements per 128-B row, rows = K, SBO =
// 1 KB between 8-row groups along K, LBO = byte stride between 64-element
// blocks along M/N. Swizzle atoms must be 1 KB aligned in shared memory.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr, uint32_t lbo_bytes,
                                                    uint32_t sbo_bytes)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16 with BF16 operands and FP32 accumulation.
__device__ __forceinline__ uint32_t umma_idesc_bf16(int M, int N, int a_mn_major, int b_mn_major)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn_major << 15) |
           ((uint32_t)b_mn_major << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once every tcgen05 operation issued so far by this thread is done.
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Contiguous global -> shared copy by the bulk-copy engine (addresses 16-byte
// aligned, bytes a multiple of 16), completion signalled on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Approximate reciprocal (special-function unit), flush-to-zero.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Split x > 0 (finite, possibly subnormal) as x = f * 2^e with
// f in [1/sqrt(2), sqrt(2)], so that ln x = e ln 2 + ln f with |ln f| <= 0.35.
__device__ __forceinline__ float split_exponent(float x, int &e)
{
    int bits = __float_as_int(x);
    int ex = (bits >> 23) & 0xff;
    int adj = 0;
    if (ex == 0) {  // subnormal: scale into the normal range first
        x *= 16777216.0f;
        bits = __float_as_int(x);
        ex = (bits >> 23) & 0xff;
        adj = -24;
    }
    int k = ex - 127;
    float f = __int_as_float((bits & 0x007fffff) | 0x3f800000);
    if (f > 1.41421356f) {
        f *= 0.5f;
        k += 1;
    }
    e = k + adj;
    return f;
}

// ---- packed FP32 pairs (two events per 64-bit register pair) -------------
// Blackwell executes these as one instruction for both halves.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk2(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(f2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// One step of the compensated dot product (Ogita, Rump and Oishi, "Accurate
// sum and dot product", SIAM J. Sci. Comput. 26 (2005), algorithm Dot2):
// (s, c) += x * y with the product split exactly by FMA (TwoProduct) and the
// sum by Knuth's TwoSum. yn must equal -y. Uses hn = x * yn = -(x*y rounded),
// r = fma(x, y, hn) = the exact product error.
__device__ __forceinline__ void dot2_step(f2 &s, f2 &c, f2 x, f2 y, f2 yn)
{
    const f2 hn = mul2(x, yn);
    const f2 r = fma2(x, y, hn);
    const f2 t = sub2(s, hn);           // s + h
    const f2 bb = sub2(t, s);
    const f2 err = sub2(sub2(s, sub2(t, bb)), add2(hn, bb));
    s = t;
    c = add2(c, add2(err, r));
}

// ---- float-float ("double-float") sums on the FP32 pipe -------------------
// FP64 throughput on this part is ~1% of FP32, so reductions that need more
// than float precision carry an unevaluated sum hi + lo of two floats
// (Knuth's TwoSum for the high parts).
struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    const float h = s + e;
    return {h, e - (h - s)};
}

__device__ __forceinline__ dfloat warp_sum(dfloat v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dfloat w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    return v;
}

__device__ __forceinline__ long long warp_sum(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// --------------------------------------------------------------------------
// Host-side launch interfaces between translation units
// --------------------------------------------------------------------------

// Per-launch arguments of the fused data-term kernels (both forms).
struct EvalArgs {
    int n_waves;
    int64_t n_events;
    const double *V;   // [n_waves] complex128 (device), the parameter set
    const double *M;   // [n_waves][n_waves] complex128 (device)
    const float *amax; // [n_waves] max over data events of |Re A_a| + |Im A_a|
    double *partials;  // scratch [grid][stride] doubles
    unsigned *ticket;  // zero on entry; reset to zero by the last block
    int *status;       // status bits are OR-ed here
    int *done;         // incremented by the last block (may be null)
    double *nll;       // [1] output
    double *grad;      // [n_waves] complex output (null: NLL only)
    float *weights;    // projection weights I / N_gen per event (the weights mode)
    float inv_ngen;    // 1 / N_gen (the weights mode)
    // Results straight to (mapped, pinned) host memory: when set, nll, grad
    // and V may be host addresses, and the last CTA, once every result is
    // visible to the host, stores (seq << 32) | status bits here.
    unsigned long long *host_flag;
    unsigned seq;
    // Test of the timeout path (direct form): with stall_ns > 0 the producer
    // issues no copies and the consumers wait at most stall_ns for a tile, so
    // their waits run out with nothing in flight and the call reports
    // FLAG_TIMEOUT. Zero in normal use.
    unsigned long long stall_ns;
};

// Structure-of-arrays store: plane 2a holds Re A_a, plane 2a+1 holds Im A_a,
// each plane `pitch` floats long with events contiguous.
struct Planes {
    float *ptr;
    int64_t pitch;  // floats per plane (multiple of 256)
    int64_t n;      // valid events
    int n_waves;
};

// Encode a 2D tensor map over `rows` planes of `pitch` floats with a box of
// box_x events x box_y planes. Returns cudaSuccess or an error.
cudaError_t encode_planes_map(CUtensorMap *map, const float *base, int64_t n, int64_t pitch,
                              int rows, int box_x, int box_y);

// k_pack.cu
cudaError_t launch_pack(const void *src, int dtype, int64_t n, int n_waves, float *planes,
                        int64_t pitch, cudaStream_t s);
cudaError_t launch_table_build(const Planes &amp, float *table, int64_t table_pitch,
                               cudaStream_t s);
// amax[a] = max_i |Re A_a(i)| + |Im A_a(i)| (amax must be zeroed first)
cudaError_t launch_amp_max(const Planes &amp, float *amax, cudaStream_t s);
// out[r] = max_i |planes[r][i]| for r < rows (out must be zeroed first)
cudaError_t launch_plane_absmax(const float *planes, int64_t pitch, int64_t n, int rows, float *out,
                                cudaStream_t s);

// k_batched.cu
// xs = number of BF16 slices of the amplitudes (1: 8-bit, 2: 16-bit block
// floating point).
int batched_features(int n_waves);        // 2 N rounded up to a multiple of 16
int batched_max_k(int n_waves, int xs);   // parameter sets per launch
size_t batched_scratch_bytes(int n_waves, int xs, int K, int grid);
cudaError_t batched_configure();
// Block-floating-point copy of the data planes for the tensor-core form:
// xs F rows of BF16 per event (slice x0 rows 0..F-1, slice x1 rows F..2F-1;
// rows past 2 n_waves and events past n are zero) in 64-event blocks of
// xs F 128 bytes, each laid out as the kernel's shared memory holds it (out:
// 2 xs F pitch bytes); *sum_e (zeroed here) receives the sum over events of
// the event exponents.
cudaError_t launch_batched_encode(const float *planes, int64_t pitch, int64_t n, int n_waves, int xs,
                                  void *out, long long *sum_e, cudaStream_t s);
// nxs: X pipeline stages (0: as many as shared memory takes; the autotuner
// may ask for fewer, from 2 up to batched_max_x_stages)
cudaError_t launch_batched(const void *xbf, int64_t n_events, int n_waves, int xs,
                           const long long *sum_e, const double *V, int K, const double *M,
                           void *scratch, int grid, int *status, int *done, double *nll,
                           double *grad, cudaStream_t s, int nxs = 0);
int batched_max_x_stages(int n_waves, int xs, int K);

// The uneven model batch in one launch (k_batched.cu): work items, each a
// contiguous range of one model's 128-event tiles, about num_sms *
// items_per_sm in all with equal estimated cost; one kernel takes them all
// (one CTA per item), a prep kernel and a final kernel serve every model.
struct BatchModelDesc {
    const void *xbf;           // the model's BF16 store (launch_batched_encode)
    int64_t n_events;
    int n_waves;
    const long long *sum_e;    // the sum of its event exponents
    const double *M;           // [N][N] complex
    const double *V;           // [K][N] complex, device
    double *nll;               // [K]
    double *grad;              // [K][N] complex, may be null
    int *status;               // status bits OR-ed here
    int *done;                 // incremented once per set, may be null
};
// Bytes of the plan (device buffer) and its number of work items.
size_t batched_plan_bytes(const BatchModelDesc *models, int n_models, int xs, int K, int num_sms,
                          int items_per_sm, int *n_items);
// Writes the plan (arguments, tensor maps, items, output pointers) into the
// device buffer `plan`; synchronises the stream. Each model: K <= its
// batched_max_k.
cudaError_t batched_plan_build(void *plan, const BatchModelDesc *models, int n_models, int xs,
                               int K, int num_sms, int items_per_sm, int nxs, cudaStream_t s);
// One evaluation of every model (the plan built for the same arguments).
cudaError_t launch_batched_items(void *plan, const BatchModelDesc *models, int n_models, int xs,
                                 int K, int num_sms, int items_per_sm, int nxs, cudaStream_t s);

// k_nll_res.cu: free Breit-Wigner masses and widths
struct ResArgs {
    int n_waves, n_free, pstride;
    const float *data;   // [1 + 2N][data_pitch] (+ padding): m, then Re/Im of Y_r or A_a
    int64_t data_pitch, n_data;
    const float *mc;
    int64_t mc_pitch, n_mc;
    double inv_ngen;
    const double *V, *mass, *width;  // device
    double *partials;    // [grid][2][pstride]
    unsigned *ticket;    // zero on entry, left at zero
    int *status;         // status bits OR-ed here
    int *done;           // incremented once (may be null)
    double *out;         // [1 + 2N + 2R]: nll, dNLL/dV*, dNLL/dM, dNLL/dG
};
int res_max_waves();
int res_max_free();
size_t res_partials_doubles(int n_waves, int n_free, int grid);
cudaError_t launch_nll_res(const ResArgs &a, int grid, cudaStream_t s);
// k_nll_res_tma.cu: the same evaluation, TMA-fed (maps over the [1 + 2N]
// planes of each sample with a box of res_tma_box_events() events x 1 + 2N
// rows); amax[a] >= max over both samples of |Re| + |Im| of Y_a (free waves)
// or A_a (fixed waves). Scratch as launch_nll_res with grid = one CTA per SM.
int res_tma_box_events();
bool res_tma_available(int n_waves, int n_free);
cudaError_t launch_nll_res_tma(const CUtensorMap *dmap, const CUtensorMap *mmap, const ResArgs &a,
                               const float *amax, int grid, cudaStream_t s);

// k_ampgen.cu: amplitudes BW(m; M, G) Y_l^m(theta, phi) from per-event
// kinematics kin [n][3] = (m, cos theta, phi) (device), FP64, rounded to float;
// out as SoA planes (Re A_a at plane 2a of `pitch` floats) or, soa = false,
// event-major complex64 [n][N].
struct GenWave {
    double mass, width, norm;  // norm = sqrt((2l + 1)/(4 pi) (l - |m|)!/(l + |m|)!)
    int l, m;
};
int ampgen_max_l();
cudaError_t launch_amp_gen(const double *kin, int64_t n, int N, const GenWave *waves, int max_m,
                           float *out, bool soa, int64_t pitch, int grid, cudaStream_t s);

// k_ampgen_cov.cu: covariant tensor amplitudes of J/psi -> gamma X, X -> K+ K-
// from p3 [n][9] (photon, K+, K- 3-momenta, device), 4 incoherent components
// per event; out as event-major [n][4][N] complex64 or, soa, the planes of an
// incoherent sample (plane 2 (l N + a) = Re A_a^l of `pitch` floats).
struct CovWave {
    double mass, width;
    int spin;  // 0 or 2
};
cudaError_t launch_cov_amp_gen(const double *p3, int64_t n, int N, const CovWave *waves, float *out,
                               bool soa, int64_t pitch, int grid, cudaStream_t s);

// k_nll_incoh.cu: direct form with an incoherent sum over n_lambda components;
// d holds 2 n_lambda N planes (plane 2 (l N + a) = Re A_a^l). Same scratch,
// ticket and outputs as the direct-form kernel (EvalArgs, one parameter set).
int incoh_max_components();
int incoh_max_waves(int n_lambda);  // largest N the direct kernel takes for n_lambda
size_t incoh_partials_doubles(int n_waves, int grid);
cudaError_t launch_nll_incoh(const Planes &d, int n_lambda, const EvalArgs &a, int grid,
                             cudaStream_t s);
// TMA-fed incoherent direct form (n_waves padded x n_lambda <= 48): map over
// the 2 n_lambda n_waves planes with a box of incoh_tma_box_events() events x
// all rows; a.amax[a] >= max over components and events of |Re| + |Im| of A_a.
bool incoh_tma_available(int n_waves, int n_lambda);
int incoh_tma_box_events();
cudaError_t launch_nll_incoh_tma(const CUtensorMap *map, int n_lambda, const EvalArgs &a, int grid,
                                 cudaStream_t s);
// table of the incoherent sum: T[a][b] = sum_l A_a^l conj(A_b^l), layout as
// launch_table_build, from planes of n_lambda * N waves
cudaError_t launch_table_build_incoh(const Planes &amp, int n_lambda, float *table,
                                     int64_t table_pitch, cudaStream_t s);

// k_fit_extras.cu
// FUMILI Hessian of the NLL over (Re V, Im V), sum_i grad ln I_i grad ln I_i^T:
// H [2N][2N] doubles (device); partials: hess_partials_doubles(n_waves, grid)
// doubles of scratch.
size_t hess_partials_doubles(int n_waves, int grid);
// async_or (may be null): the call's status bits are OR-ed into it as well.
cudaError_t launch_hessian(const Planes &d, const double *V, double *partials, int grid, int *status,
                           double *H, int *async_or, cudaStream_t s);
// k_hess_tc.cu
// The same Hessian on the tensor cores (n_waves <= 20): map over the data
// planes with box hess_tc_box_events() x 2 n_waves rows, amax[a] >= max over
// the data of |Re A_a| + |Im A_a|, partials: hess_tc_partials_doubles(n_waves,
// grid) doubles. Returns cudaErrorNotSupported for more waves.
bool hess_tc_available(int n_waves);
int hess_tc_box_events();
size_t hess_tc_partials_doubles(int n_waves, int grid);
cudaError_t launch_hessian_tc(const CUtensorMap *map, const Planes &d, const double *V,
                              const float *amax, double *partials, int grid, int *status, double *H,
                              int *async_or, cudaStream_t s);
// w[j] = |sum_a V_a A_a(j)|^2 / n_gen for the accepted MC events (float, device).
cudaError_t launch_mc_weights(const Planes &mc, const double *V, double n_gen, float *w, int grid,
                              cudaStream_t s);
// w[j] = |S_j|^2 / n_gen through the TMA-fed kernel: map over the MC planes
// (box amp_box_events() x 2 n_waves rows), amax[a] >= max over the MC sample
// of |Re A_a| + |Im A_a|; a timeout is OR-ed into *status.
cudaError_t launch_mc_weights_tma(const CUtensorMap *map, const Planes &mc, const double *V,
                                  const float *amax, double n_gen, float *w, int *status, int grid,
                                  cudaStream_t s);
// *dst |= *src on the stream (status words)
cudaError_t launch_or_flags(const int *src, int *dst, cudaStream_t s);
// F[a][b] = Re(conj(V_a) M_ab V_b) / V^H M V (device doubles).
cudaError_t launch_fit_fractions(const double *M, const double *V, int N, double *F, cudaStream_t s);
// dst[i] = (float)src[i] (round to nearest)
cudaError_t launch_to_float(const double *src, int64_t n, float *dst, cudaStream_t s);

// k_nll_table.cu
int table_max_waves();
int table_box_events(int n_waves);
int table_box_rows(int n_waves);
size_t table_scratch_bytes(int n_waves, int grid);
cudaError_t table_configure();
cudaError_t launch_nll_table(int64_t n_events, int n_waves, const CUtensorMap *map,
                             const EvalArgs &a, const float *tmax, int grid, cudaStream_t s);

// k_norm.cu
size_t norm_scratch_bytes(int n_waves, int num_sms);
cudaError_t launch_build_norm(const Planes &mc, double n_gen, double *M, double *scratch,
                              int num_sms, cudaStream_t s);
// k_norm_tc.cu: the same M on the tensor cores (n_waves <= 20) from exact
// fixed-point digits of the amplitudes. map: over the MC planes with a box of
// norm_tc_box_events() events x 2 n_waves rows; amax[a] = max over the MC of
// |Re A_a| + |Im A_a| (each must pass norm_tc_scale_ok); partials:
// norm_tc_partials_doubles(n_waves, grid) doubles; a timeout is OR-ed into
// *status (zero on entry) and M is then NaN.
bool norm_tc_available(int n_waves);
int norm_tc_box_events();
bool norm_tc_scale_ok(float amax);
size_t norm_tc_partials_doubles(int n_waves, int grid);
cudaError_t launch_build_norm_tc(const CUtensorMap *map, const Planes &mc, const float *amax,
                                 double n_gen, double *partials, int grid, int *status, double *M,
                                 cudaStream_t s);

// k_nll_amp.cu
int amp_grid(int n_waves, int num_sms);
size_t amp_partials_doubles(int n_waves, int num_sms);
// groups: consumer groups per CTA (2 or 3; 0 = the default rule or the
// PWA_AMP_GROUPS environment override). 3 only where amp_groups3_available.
cudaError_t launch_nll_amp(const Planes &amp, const CUtensorMap *map, const EvalArgs &a,
                           int num_sms, cudaStream_t s, int groups = 0);
bool amp_groups3_available(int n_waves);
int amp_box_events(int n_waves);
// Same launch with an explicit persistent grid. EvalArgs::partials must hold
// amp_scratch_bytes_for_grid(grid) bytes; the kernel's work-flag word sits at
// byte amp_flags_offset(grid) of it and, like the ticket, must be zero on
// entry (the last CTA leaves both at zero).
cudaError_t launch_nll_amp_grid(const Planes &amp, const CUtensorMap *map, const EvalArgs &a,
                                int grid, cudaStream_t s, int groups = 0);
size_t amp_flags_offset(int grid);
size_t amp_scratch_bytes_for_grid(int grid);
cudaError_t amp_configure();  // once per device: opt in to large shared memory
int amp_box_rows(int n_waves);

}  // namespace pwa
