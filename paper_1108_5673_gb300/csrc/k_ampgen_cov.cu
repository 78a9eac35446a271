// Covariant tensor amplitudes on the device (Sec. 4: the framework builds its
// amplitudes on the GPU in the covariant tensor formalism), for the radiative
// decay J/psi -> gamma X, X -> K+ K-:
//   4-vectors in the J/psi rest frame, metric (+,-,-,-); per event the
//   photon q and the kaons k1, k2 (from their 3-momenta, mK = 0.493677 GeV),
//   p = k1 + k2, r = k1 - k2, rt = r - (r.p / p.p) p;
//   unobserved components l = 2 (M index) + (photon polarization index):
//   J/psi helicity M = +1, -1 along z, psi(+1) = (0, -1, -i, 0)/sqrt2,
//   psi(-1) = (0, 1, -i, 0)/sqrt2; photon e1 = (0, z x q / |z x q|) (x when q
//   lies along z), e2 = (0, q/|q| x e1);
//   spin 0: A = BW(p.p) psi.e;
//   spin 2: A = BW(p.p) B2(Q) [(psi.rt)(e.rt) - (1/3)(rt.rt)(psi.e - (psi.p)(e.p)/p.p)],
//     Q^2 = p.p/4 - mK^2, B2 = sqrt(13 / (Q^4 + 3 Q^2 Q0^2 + 9 Q0^4)), Q0 = 0.197327 GeV;
//   BW(s) = 1 / (M^2 - s - i M G).
// Evaluated in FP64 and rounded once to float, so that the stored amplitudes
// are the floats nearest to the formalism's values; once per sample.
//
// One event per thread: the 4 components' contractions (the spin-0 and the
// spin-2 one, each complex) first, then one Breit-Wigner and 4 complex
// products per wave; the wave table sits in shared memory. Output: event-
// major [n][4][N] complex64, or the planes of an incoherent sample (plane
// 2 (l N + a) = Re A_a^l, `pitch` floats each).
#include <algorithm>

#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int kCovThreads = 256;

__device__ __forceinline__ double mdot(const double (&a)[4], const double (&b)[4])
{
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

__global__ void __launch_bounds__(kCovThreads)
    cov_amp_kernel(const double *__restrict__ p3, int64_t n, int N, const CovWave *__restrict__ waves,
                   float *__restrict__ out, bool soa, int64_t pitch)
{
    __shared__ CovWave w[kMaxWaves];
    for (int a = threadIdx.x; a < N; a += blockDim.x)
        w[a] = waves[a];
    __syncthreads();
    const double mK = 0.493677, Q0 = 0.197327, isq2 = 0.70710678118654752440;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double *v = p3 + 9 * i;
        double q[4], k1[4], k2[4], p[4], r[4], rt[4];
        q[1] = v[0];
        q[2] = v[1];
        q[3] = v[2];
        const double qq = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        q[0] = qq;
        k1[0] = sqrt(mK * mK + v[3] * v[3] + v[4] * v[4] + v[5] * v[5]);
        k2[0] = sqrt(mK * mK + v[6] * v[6] + v[7] * v[7] + v[8] * v[8]);
        for (int c = 0; c < 3; ++c) {
            k1[c + 1] = v[3 + c];
            k2[c + 1] = v[6 + c];
        }
        for (int c = 0; c < 4; ++c) {
            p[c] = k1[c] + k2[c];
            r[c] = k1[c] - k2[c];
        }
        const double pp = mdot(p, p), rp = mdot(r, p);
        for (int c = 0; c < 4; ++c)
            rt[c] = r[c] - rp / pp * p[c];
        const double rr = mdot(rt, rt);
        const double Q2 = pp / 4.0 - mK * mK;
        const double b2 = sqrt(13.0 / (Q2 * Q2 + 3.0 * Q2 * Q0 * Q0 + 9.0 * Q0 * Q0 * Q0 * Q0));
        double e[2][4];
        const double ux = -q[2], uy = q[1];  // z x q
        const double un = sqrt(ux * ux + uy * uy);
        e[0][0] = 0.0;
        e[0][3] = 0.0;
        if (un > 1e-12 * qq) {
            e[0][1] = ux / un;
            e[0][2] = uy / un;
        } else {
            e[0][1] = 1.0;
            e[0][2] = 0.0;
        }
        const double qh0 = q[1] / qq, qh1 = q[2] / qq, qh2 = q[3] / qq;
        e[1][0] = 0.0;
        e[1][1] = qh1 * e[0][3] - qh2 * e[0][2];
        e[1][2] = qh2 * e[0][1] - qh0 * e[0][3];
        e[1][3] = qh0 * e[0][2] - qh1 * e[0][1];
        // the contractions, real and imaginary parts of psi apart: [l][spin 0/2][re/im]
        double cpl[4][2][2];
#pragma unroll
        for (int im = 0; im < 2; ++im) {
            const double psr[4] = {0.0, im == 0 ? -isq2 : isq2, 0.0, 0.0};
            const double psi[4] = {0.0, 0.0, -isq2, 0.0};
#pragma unroll
            for (int il = 0; il < 2; ++il) {
                const double(&ww)[4] = e[il];
                const double s0r = mdot(psr, ww), s0i = mdot(psi, ww);
                const double prw = mdot(ww, rt), pwp = mdot(ww, p);
                const double ar = mdot(psr, rt), ai = mdot(psi, rt);
                const double apr = mdot(psr, p), api = mdot(psi, p);
                const int l = 2 * im + il;
                cpl[l][0][0] = s0r;
                cpl[l][0][1] = s0i;
                cpl[l][1][0] = b2 * (ar * prw - rr / 3.0 * (s0r - apr * pwp / pp));
                cpl[l][1][1] = b2 * (ai * prw - rr / 3.0 * (s0i - api * pwp / pp));
            }
        }
        for (int a = 0; a < N; ++a) {
            const double D = w[a].mass * w[a].mass - pp, G = w[a].mass * w[a].width;
            const double inv = 1.0 / (D * D + G * G);
            const double br = D * inv, bi = G * inv;
            const bool s2 = w[a].spin == 2;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const double cr = s2 ? cpl[l][1][0] : cpl[l][0][0];
                const double ci = s2 ? cpl[l][1][1] : cpl[l][0][1];
                const float re = __double2float_rn(br * cr - bi * ci);
                const float im = __double2float_rn(br * ci + bi * cr);
                if (soa) {
                    out[(int64_t)(2 * (l * N + a)) * pitch + i] = re;
                    out[(int64_t)(2 * (l * N + a) + 1) * pitch + i] = im;
                } else {
                    float *o = out + ((i * 4 + l) * N + a) * 2;
                    o[0] = re;
                    o[1] = im;
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_cov_amp_gen(const double *p3, int64_t n, int N, const CovWave *waves, float *out,
                               bool soa, int64_t pitch, int grid, cudaStream_t s)
{
    if (n < 1 || N < 1 || N > kMaxWaves)
        return cudaErrorInvalidValue;
    const int64_t need = (n + kCovThreads - 1) / kCovThreads;
    const int g = (int)std::min<int64_t>(need, grid > 0 ? grid : 1024);
    cov_amp_kernel<<<g, kCovThreads, 0, s>>>(p3, n, N, waves, out, soa, pitch);
    return cudaGetLastError();
}

}  // namespace pwa
