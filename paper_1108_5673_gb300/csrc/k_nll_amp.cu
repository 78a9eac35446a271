// Fused data-term kernel, direct amplitude form (Eq. 1 and the first sum of
// Eq. 3), followed in the same launch by the deterministic FP64 final sum
// and the normalisation term (Sec. 4: single precision per event, double
// precision final sum).
//
// Per event i (each consumer thread handles two adjacent events of a tile,
// packed in the two halves of FP32x2 registers):
//   S_i = sum_a (Vhi_a + Vlo_a) A_a(i)   FP32, error-free extraction (below)
//   I_i = |S_i|^2                         FP32
//   ln I_i = e_i ln 2 + ln f_i            f_i in [2^-1/2, 2^1/2], e_i summed exactly
//   r_i = S_i / I_i,  g_a += conj(A_a(i)) r_i
// Per-thread sums stay off the FP64 pipe (a small fraction of the FP32 rate on
// this part): ln f_i is scaled by 2^23 and split into its integer part, summed
// exactly in an int32, and its fraction, summed in FP32; both become doubles
// once per thread for the block reduction.
//
// Accuracy of S. A plain FP32 sum of the 4N real products loses digits where
// the waves interfere destructively (|S_i| much smaller than
// B_i = sum_a |V_a|_1 |A_a(i)|_1); over 1M events those losses add up to
// several 1e-3 in the NLL. Instead every product p = c * a is split exactly
// against sigma = 1.5 * 2^k, with 2^(k-1) >= max_i B_i fixed per call:
//     t = fma(c, a, sigma)    lies in [2^k, 2^(k+1)]: c*a rounded to a
//                             multiple of u_k = 2^(k-23)
//     bits(t) - bits(sigma) = q / u_k, the high part of c*a as an integer
//     r = fma(c, a, sigma - t)   the remainder c*a - q (sigma - t is exact)
// The high parts are summed exactly as 32-bit integers (on the integer
// pipe, wrapping harmlessly since the final sum is below 2^23), the
// remainders in FP32 with an error ~2^-48 sigma. S = hi + lo is then correct
// to about one float rounding however small it is relative to B_i (the
// guarantee of a doubled-precision dot product, at well under its cost).
// sigma comes from V and the per-wave maxima of |A| over the sample, so no
// per-event pre-pass is needed. V is carried as a float pair Vhi + Vlo; the
// products Vlo A are ~2^-24 of the leading ones and go straight into the
// low sums.
//
// Data movement: a persistent grid (one CTA per SM) streams tiles of 256
// events x 2N planes (192 events from 40 waves on) from the structure-of-
// arrays store into a ring of shared-memory stages with TMA
// (cp.async.bulk.tensor.2d); one producer thread issues the copies; GROUPS
// groups of four consumer warps (three from 40 waves on) take tiles in turn,
// each group cycling through its own stages of the ring, or the groups
// sharing the stages where one per group would fit. Every wait is bounded
// (FLAG_TIMEOUT) so a stalled pipeline returns instead of hanging.
//
// Reductions avoid the FP64 pipe (about 1% of the FP32 rate on this part):
// integer parts of the log sum are added exactly as integers, the rest as
// float-float pairs. Each CTA writes its partials; the last CTA to finish
// (atomic ticket) adds them in block order, so results are bitwise
// reproducible from run to run. M V and V^H M V, the only double-precision
// arithmetic, are formed at the start by a helper warp of CTA 0, off the
// critical path; the last CTA only converts its float-float and integer
// sums to double once.
#include <stdlib.h>

#include "pwa_internal.cuh"
#include "amp_kernel.cuh"

namespace pwa {

namespace {

// The NLL-only call runs the same kernel and discards the gradient sums (the
// extra FMAs hide under the HBM time).

template <int N>
cudaError_t configure_n()
{
    static_assert(AmpCfg<N, 2>::FITS, "two consumer groups must fit for every N");
    cudaError_t e = cudaFuncSetAttribute(nll_amp_kernel<N, 2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)AmpCfg<N, 2>::SMEM);
    if constexpr (AmpCfg<N, 3>::FITS) {
        cudaError_t f = cudaFuncSetAttribute(nll_amp_kernel<N, 3>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)AmpCfg<N, 3>::SMEM);
        if (e == cudaSuccess)
            e = f;
    }
    return e;
}

// Consumer groups per CTA: 2 (10 warps, up to 168 registers per thread; 8
// warps and 255 registers from 40 waves on) or 3 (14 warps, 128 registers;
// 11 warps and 168 registers from 40 waves on). PWA_AMP_GROUPS overrides the
// default.
int amp_groups()
{
    static const int g = [] {
        const char *v = getenv("PWA_AMP_GROUPS");
        return (v && atoi(v) == 3) ? 3 : (v && atoi(v) == 2) ? 2 : 0;
    }();
    return g;
}


template <int N>
cudaError_t launch_n(const CUtensorMap *map, const EvalArgs &a, int grid, int n_tiles,
                     int *work_flags, cudaStream_t s, int groups)
{
    if (!finalize_fits<N, 2>(grid))
        return cudaErrorInvalidConfiguration;
    const int g = groups ? groups : amp_groups() ? amp_groups() : (N <= 12 ? 3 : 2);
    if constexpr (AmpCfg<N, 3>::FITS) {
        if (g == 3 && finalize_fits<N, 3>(grid)) {
            nll_amp_kernel<N, 3><<<grid, AmpCfg<N, 3>::THREADS, AmpCfg<N, 3>::SMEM, s>>>(
                *map, a, n_tiles, work_flags);
            return cudaGetLastError();
        }
    }
    nll_amp_kernel<N, 2><<<grid, AmpCfg<N, 2>::THREADS, AmpCfg<N, 2>::SMEM, s>>>(
        *map, a, n_tiles, work_flags);
    return cudaGetLastError();
}

int pad_waves(int n)
{
    static const int pads[] = {4, 8, 12, 16, 20, 24, 32, 40, 48};
    for (int p : pads)
        if (n <= p)
            return p;
    return -1;
}

}  // namespace

// Events per tile (the tensor map's box), the same for both group counts.
int amp_box_events(int n_waves)
{
    static_assert(AmpCfg<40, 2>::TE == AmpCfg<40, 3>::TE && AmpCfg<20, 2>::TE == AmpCfg<20, 3>::TE,
                  "a tile's events do not depend on the group count");
    switch (pad_waves(n_waves)) {
    case 4: return AmpCfg<4, 2>::TE;
    case 8: return AmpCfg<8, 2>::TE;
    case 12: return AmpCfg<12, 2>::TE;
    case 16: return AmpCfg<16, 2>::TE;
    case 20: return AmpCfg<20, 2>::TE;
    case 24: return AmpCfg<24, 2>::TE;
    case 32: return AmpCfg<32, 2>::TE;
    case 40: return AmpCfg<40, 2>::TE;
    case 48: return AmpCfg<48, 2>::TE;
    }
    return -1;
}

int amp_box_rows(int n_waves) { return 2 * n_waves; }

cudaError_t amp_configure()
{
    cudaError_t e = cudaSuccess;
    for (cudaError_t r : {configure_n<4>(), configure_n<8>(), configure_n<12>(), configure_n<16>(),
                          configure_n<20>(), configure_n<24>(), configure_n<32>(), configure_n<40>(),
                          configure_n<48>()})
        if (r != cudaSuccess)
            e = r;
    return e;
}

// One persistent CTA per SM; PWA_AMP_GRID overrides it (a tuning knob, and a
// test's way to give each CTA many tiles). It serves the TMA-fed incoherent
// launches as well, whose scratch has the same layout.
int amp_grid(int n_waves, int num_sms)
{
    (void)n_waves;
    static const int forced = [] {
        const char *v = getenv("PWA_AMP_GRID");
        return v ? atoi(v) : 0;
    }();
    return (forced > 0 && forced <= 4 * num_sms) ? forced : num_sms;
}

size_t amp_flags_offset(int grid)
{
    return (size_t)grid * 2 * sizeof(long long) + (size_t)grid * (2 * kMaxWaves + 1) * sizeof(float2) +
           (2 * kMaxWaves + 2) * sizeof(double);
}

size_t amp_scratch_bytes_for_grid(int grid) { return amp_flags_offset(grid) + 64; }

size_t amp_partials_doubles(int n_waves, int num_sms)
{
    return amp_scratch_bytes_for_grid(amp_grid(n_waves, num_sms)) / sizeof(double) + 8;
}

cudaError_t launch_nll_amp(const Planes &amp, const CUtensorMap *map, const EvalArgs &a,
                           int num_sms, cudaStream_t s, int groups)
{
    return launch_nll_amp_grid(amp, map, a, amp_grid(amp.n_waves, num_sms), s, groups);
}

template <int N>
bool groups3_fit()
{
    if constexpr (AmpCfg<N, 3>::FITS)
        return true;
    return false;
}

bool amp_groups3_available(int n_waves)
{
    switch (pad_waves(n_waves)) {
    case 4: return groups3_fit<4>();
    case 8: return groups3_fit<8>();
    case 12: return groups3_fit<12>();
    case 16: return groups3_fit<16>();
    case 20: return groups3_fit<20>();
    case 24: return groups3_fit<24>();
    case 32: return groups3_fit<32>();
    case 40: return groups3_fit<40>();
    case 48: return groups3_fit<48>();
    }
    return false;
}

cudaError_t launch_nll_amp_grid(const Planes &amp, const CUtensorMap *map, const EvalArgs &a,
                                int grid, cudaStream_t s, int groups)
{
    const int te = amp_box_events(amp.n_waves);
    if (te <= 0)
        return cudaErrorInvalidValue;
    const int n_tiles = (int)((amp.n + te - 1) / te);
    int *work_flags = amp_scratch(a.partials, grid).flags;
    switch (pad_waves(amp.n_waves)) {
    case 4: return launch_n<4>(map, a, grid, n_tiles, work_flags, s, groups);
    case 8: return launch_n<8>(map, a, grid, n_tiles, work_flags, s, groups);
    case 12: return launch_n<12>(map, a, grid, n_tiles, work_flags, s, groups);
    case 16: return launch_n<16>(map, a, grid, n_tiles, work_flags, s, groups);
    case 20: return launch_n<20>(map, a, grid, n_tiles, work_flags, s, groups);
    case 24: return launch_n<24>(map, a, grid, n_tiles, work_flags, s, groups);
    case 32: return launch_n<32>(map, a, grid, n_tiles, work_flags, s, groups);
    case 40: return launch_n<40>(map, a, grid, n_tiles, work_flags, s, groups);
    case 48: return launch_n<48>(map, a, grid, n_tiles, work_flags, s, groups);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pwa
