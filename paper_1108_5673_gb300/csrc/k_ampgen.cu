// Amplitudes on the device (Sec. 4: the framework computes its amplitudes on
// the GPU), for the amplitude model of the samples here:
//   A_a(Omega) = BW(m; M_a, G_a) Y_{l_a}^{m_a}(theta, phi),
//   BW(m; M, G) = 1 / (M^2 - m^2 - i M G) = (D + i M G) / (D^2 + (M G)^2), D = M^2 - m^2,
//   Y_l^m = N_lm P_l^m(cos theta) e^{i m phi} for m >= 0 (Condon-Shortley phase
//   in P_l^m), Y_l^{-m} = (-1)^m conj(Y_l^m).
// Evaluated in FP64 and rounded once to float (as the host generator does),
// so that the stored amplitudes are the floats nearest to the model's values.
// This runs once per sample, not per fit iteration, so the FP64 pipe's low
// rate costs milliseconds; a per-event FP32 evaluation would move the phase
// of e^{i m phi} by ~1e-6 at m phi ~ 8 pi.
//
// One event per thread; the wave table (mass, width, l, m, N_lm) sits in
// shared memory. e^{i k phi} for k = 1 .. max |m| comes from one sincos and
// complex products; P_l^m by the upward recurrence in l (its divisions by
// l - m as products with a table of 1/k); one division per Breit-Wigner.
#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int kGenThreads = 256;
constexpr int kMaxL = 16;

// 1 / k for the recurrence's divisor l - m (k = 1 .. kMaxL), rounded to double
__constant__ double c_inv[kMaxL + 1] = {
    0.0, 1.0, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8, 1.0 / 9, 1.0 / 10,
    1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16};

__global__ void __launch_bounds__(kGenThreads)
    amp_gen_kernel(const double *__restrict__ kin, int64_t n, int N, const GenWave *__restrict__ waves,
                   int max_m, float *__restrict__ out, int64_t s_wave, int64_t s_event,
                   int64_t s_imag)
{
    __shared__ GenWave w[kMaxWaves];
    for (int a = threadIdx.x; a < N; a += blockDim.x)
        w[a] = waves[a];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double m = kin[3 * i], x = kin[3 * i + 1], phi = kin[3 * i + 2];
        const double s = sqrt(fmax(0.0, 1.0 - x * x));
        // e^{i k phi}, k = 0 .. max_m
        double er[kMaxL + 1], ei[kMaxL + 1];
        er[0] = 1.0;
        ei[0] = 0.0;
        double c1, s1;
        sincos(phi, &s1, &c1);
        for (int k = 1; k <= max_m; ++k) {
            er[k] = er[k - 1] * c1 - ei[k - 1] * s1;
            ei[k] = er[k - 1] * s1 + ei[k - 1] * c1;
        }
        float *o = out + i * s_event;
        for (int a = 0; a < N; ++a) {
            const int l = w[a].l, mm = w[a].m, am = mm < 0 ? -mm : mm;
            // P_l^am(x), Condon-Shortley phase
            double pmm = 1.0;
            for (int k = 1; k <= am; ++k)
                pmm *= -(2.0 * k - 1.0) * s;
            double p = pmm;
            if (l > am) {
                double p2 = pmm, p1 = x * (2.0 * am + 1.0) * pmm;
                for (int ll = am + 2; ll <= l; ++ll) {
                    const double q =
                        ((2.0 * ll - 1.0) * x * p1 - (ll + am - 1.0) * p2) * c_inv[ll - am];
                    p2 = p1;
                    p1 = q;
                }
                p = p1;
            }
            const double y = w[a].norm * p;
            double yr = y * er[am], yi = y * ei[am];
            if (mm < 0) {
                const double sign = (am & 1) ? -1.0 : 1.0;
                yr *= sign;
                yi *= -sign;
            }
            const double D = w[a].mass * w[a].mass - m * m, G = w[a].mass * w[a].width;
            const double rden = 1.0 / (D * D + G * G);
            const double br = D * rden, bi = G * rden;
            o[a * s_wave] = __double2float_rn(br * yr - bi * yi);
            o[a * s_wave + s_imag] = __double2float_rn(br * yi + bi * yr);
        }
    }
}

}  // namespace

int ampgen_max_l() { return kMaxL; }

cudaError_t launch_amp_gen(const double *kin, int64_t n, int N, const GenWave *waves, int max_m,
                           float *out, bool soa, int64_t pitch, int grid, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    if (N < 1 || N > kMaxWaves || max_m < 0 || max_m > kMaxL)
        return cudaErrorInvalidValue;
    // SoA planes: Re A_a at plane 2a, Im at 2a + 1; event-major complex64: (i N + a) 2 + {0, 1}
    const int64_t s_wave = soa ? 2 * pitch : 2, s_event = soa ? 1 : 2 * (int64_t)N,
                  s_imag = soa ? pitch : 1;
    amp_gen_kernel<<<grid, kGenThreads, 0, s>>>(kin, n, N, waves, max_m, out, s_wave, s_event,
                                                s_imag);
    return cudaGetLastError();
}

}  // namespace pwa
