/*
 * FP64 CPU oracle for the partial wave analysis likelihood.
 *
 * TEST INFRASTRUCTURE, not part of the library: only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark load it. It shares no code,
 * header or table with the CUDA path. Every function is a plain, slow,
 * literal statement of the paper's definitions in double precision with
 * Neumaier-compensated sums, so that it can be checked against the paper by
 * eye:
 *
 *   Eq. 1   I(Omega) = | sum_alpha V_alpha A_alpha(Omega) |^2
 *   Eq. 3   -ln L = - sum_i ln( sum_{alpha,alpha'} V_alpha V*_alpha' A_alpha(i) A*_alpha'(i) )
 *                   + sum_{alpha,alpha'} V_alpha V*_alpha' (1/N_gen) sum_{j in Acc} A_alpha(j) A*_alpha'(j)
 *   Sec. 2 (after Eq. 3): with masses and widths fixed, the MC bracket and
 *           the per-event products A_alpha A*_alpha' can be precomputed
 *           (the "table form").
 *
 * Conventions (one reading of Eq. 3, fixed here):
 *   M[a][b] = (1/N_gen) sum_j conj(A_a(j)) A_b(j), so that the normalisation
 *   term equals V^H M V = (1/N_gen) sum_j |S_j|^2 with S_j = sum_a V_a A_a(j).
 *   This is the paper's double sum in Eq. 3 written with the conjugate on the
 *   other index pair; both give the same real number because the double sum
 *   is a Hermitian form.
 *   The gradient is the Wirtinger derivative g_a = dNLL/dV*_a
 *     = - sum_i conj(A_a(i)) S_i / I_i + (M V)_a.
 *   An intensity that is not positive and finite makes the evaluation
 *   undefined: the call reports status 1, NLL = +inf and a zero gradient.
 *
 * Beyond the likelihood itself (the fitter's needs, Sec. 4 and 5):
 *   FUMILI's approximation of the Hessian of the NLL in the real parameters
 *   p = (Re V, Im V): the second derivatives of the intensity are dropped in
 *   both terms of Eq. 3 (-sum_i d^2 I_i / I_i in the data term, d^2(V^H M V)
 *   in the MC term; at the minimum they cancel in expectation), leaving
 *     H = sum_i grad(ln I_i) grad(ln I_i)^T,
 *   grad(ln I_i) = 2 (Re, Im) of conj(A_a(i)) S_i / I_i per wave a;
 *   per-MC-event weights w_j = I(Omega_j) / N_gen (their sum is V^H M V) for
 *   projections, and the fit fractions F_ab = Re(conj(V_a) M_ab V_b) / V^H M V.
 *
 * Incoherent sum over L unobserved components (e.g. helicity states of an
 * undetected photon polarisation): each event carries amplitudes A_a^l(i),
 * l < L, and Eq. 1 becomes I = sum_l |sum_a V_a A_a^l|^2. Eq. 3 keeps its
 * form with the per-event products summed over l, A_a A*_b -> sum_l A_a^l
 * conj(A_b^l), in the data term (the table) and in the MC bracket alike;
 * g_a = - sum_i sum_l conj(A_a^l(i)) S_i^l / I_i + (M V)_a.
 *
 * The amplitude model the samples here use (the paper computes its amplitudes
 * on the GPU, Sec. 4; its covariant tensor library is not given, so this is
 * the model of the synthetic samples): A_a(Omega) = BW(m; M_a, G_a) Y_{l_a}^{m_a}
 * (theta, phi) with BW(m; M, G) = 1 / (M^2 - m^2 - i M G) and Y_l^m the
 * orthonormal spherical harmonic with the Condon-Shortley phase.
 *
 * Layouts: complex numbers are interleaved (re, im) doubles.
 *   Amplitudes: event-major A[(i*N + a)*2 + {0,1}]; with L components
 *   A[((i*L + l)*N + a)*2 + {0,1}].
 *   Table: event-major T[i*N*N + p] with p = a for the real diagonal
 *   |A_a|^2, then for each pair a < b in row-major order the two reals
 *   Re(A_a conj A_b), Im(A_a conj A_b).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- Neumaier summation ---------------------------------------------- */
typedef struct { double s, c; } nsum;

static void nadd(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nval(const nsum *a) { return a->s + a->c; }

/* complex helpers on interleaved doubles */
static void cmul(double ar, double ai, double br, double bi, double *r, double *i)
{
    *r = ar * br - ai * bi;
    *i = ar * bi + ai * br;
}

/* ---- Eq. 1: coherent intensity per event ------------------------------ */
/* I[i] = |sum_a V_a A_a(i)|^2 for one parameter set V. */
void oracle_intensity(const double *A, int64_t n, int N, const double *V, double *I)
{
    for (int64_t i = 0; i < n; ++i) {
        nsum sr = {0, 0}, si = {0, 0};
        for (int a = 0; a < N; ++a) {
            double pr, pi;
            cmul(V[2 * a], V[2 * a + 1], A[(i * N + a) * 2], A[(i * N + a) * 2 + 1], &pr, &pi);
            nadd(&sr, pr);
            nadd(&si, pi);
        }
        double r = nval(&sr), im = nval(&si);
        I[i] = r * r + im * im;
    }
}

/* ---- Normalisation matrix (Eq. 3, inner bracket of the second term) --- */
/* M[a][b] = (1/n_gen) sum_{j < n_acc} conj(A_a(j)) A_b(j), all N x N entries. */
int oracle_norm_matrix(const double *A, int64_t n_acc, int N, double n_gen, double *M)
{
    if (N <= 0 || n_acc < 0 || !(n_gen > 0))
        return -1;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            nsum re = {0, 0}, im = {0, 0};
            for (int64_t j = 0; j < n_acc; ++j) {
                double xr = A[(j * N + a) * 2], xi = -A[(j * N + a) * 2 + 1];
                double yr = A[(j * N + b) * 2], yi = A[(j * N + b) * 2 + 1];
                double pr, pi;
                cmul(xr, xi, yr, yi, &pr, &pi);
                nadd(&re, pr);
                nadd(&im, pi);
            }
            M[(a * N + b) * 2] = nval(&re) / n_gen;
            M[(a * N + b) * 2 + 1] = nval(&im) / n_gen;
        }
    return 0;
}

/* Normalisation term V^H M V (real part; the imaginary part of a Hermitian
 * form vanishes) and the vector M V. */
void oracle_norm_term(const double *M, int N, const double *V, double *nv, double *MV)
{
    nsum q = {0, 0};
    for (int a = 0; a < N; ++a) {
        nsum r = {0, 0}, im = {0, 0};
        for (int b = 0; b < N; ++b) {
            double pr, pi;
            cmul(M[(a * N + b) * 2], M[(a * N + b) * 2 + 1], V[2 * b], V[2 * b + 1], &pr, &pi);
            nadd(&r, pr);
            nadd(&im, pi);
        }
        double mr = nval(&r), mi = nval(&im);
        if (MV) {
            MV[2 * a] = mr;
            MV[2 * a + 1] = mi;
        }
        /* conj(V_a) * (M V)_a, real part */
        nadd(&q, V[2 * a] * mr + V[2 * a + 1] * mi);
    }
    *nv = nval(&q);
}

/* ---- Eq. 3, amplitude form -------------------------------------------- */
/* For each of K parameter sets V[k][N]: nll[k] and, if grad != NULL,
 * grad[k][N] (complex) = dNLL/dV*. Returns the number of parameter sets
 * whose evaluation hit a non-positive or non-finite intensity. */
int oracle_nll_amp(const double *A, int64_t n, int N, const double *M,
                   const double *V, int K, double *nll, double *grad)
{
    int bad_sets = 0;
    nsum *gr = (nsum *)malloc(sizeof(nsum) * 2 * (size_t)N);
    double *mv = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    for (int k = 0; k < K; ++k) {
        const double *v = V + (size_t)k * 2 * N;
        nsum lnsum = {0, 0};
        int bad = 0;
        memset(gr, 0, sizeof(nsum) * 2 * (size_t)N);
        for (int64_t i = 0; i < n && !bad; ++i) {
            nsum sr = {0, 0}, si = {0, 0};
            for (int a = 0; a < N; ++a) {
                double pr, pi;
                cmul(v[2 * a], v[2 * a + 1], A[(i * N + a) * 2], A[(i * N + a) * 2 + 1], &pr, &pi);
                nadd(&sr, pr);
                nadd(&si, pi);
            }
            double s_r = nval(&sr), s_i = nval(&si);
            double I = s_r * s_r + s_i * s_i;
            if (!(I > 0) || !isfinite(I)) {
                bad = 1;
                break;
            }
            nadd(&lnsum, log(I));
            if (grad) {
                /* conj(A_a) * S / I */
                double rr = s_r / I, ri = s_i / I;
                for (int a = 0; a < N; ++a) {
                    double xr = A[(i * N + a) * 2], xi = -A[(i * N + a) * 2 + 1];
                    double pr, pi;
                    cmul(xr, xi, rr, ri, &pr, &pi);
                    nadd(&gr[2 * a], pr);
                    nadd(&gr[2 * a + 1], pi);
                }
            }
        }
        double nv;
        oracle_norm_term(M, N, v, &nv, mv);
        if (bad) {
            ++bad_sets;
            nll[k] = INFINITY;
            if (grad)
                memset(grad + (size_t)k * 2 * N, 0, sizeof(double) * 2 * (size_t)N);
            continue;
        }
        nll[k] = -nval(&lnsum) + nv;
        if (grad)
            for (int c = 0; c < 2 * N; ++c)
                grad[(size_t)k * 2 * N + c] = -nval(&gr[c]) + mv[c];
    }
    free(gr);
    free(mv);
    return bad_sets;
}

/* ---- Precomputed per-event table (Sec. 2, after Eq. 3) ---------------- */
int oracle_table(const double *A, int64_t n, int N, double *T)
{
    const int64_t P = (int64_t)N * N;
    for (int64_t i = 0; i < n; ++i) {
        double *t = T + i * P;
        for (int a = 0; a < N; ++a) {
            double ar = A[(i * N + a) * 2], ai = A[(i * N + a) * 2 + 1];
            t[a] = ar * ar + ai * ai;
        }
        int p = N;
        for (int a = 0; a < N; ++a)
            for (int b = a + 1; b < N; ++b) {
                double pr, pi;
                cmul(A[(i * N + a) * 2], A[(i * N + a) * 2 + 1],
                     A[(i * N + b) * 2], -A[(i * N + b) * 2 + 1], &pr, &pi);
                t[p++] = pr;
                t[p++] = pi;
            }
    }
    return 0;
}

/* Element [a][b] of the Hermitian per-event matrix T_ab = A_a conj(A_b),
 * read back from the stored upper triangle. */
static void table_entry(const double *t, int N, int a, int b, double *re, double *im)
{
    if (a == b) {
        *re = t[a];
        *im = 0;
        return;
    }
    int lo = a < b ? a : b, hi = a < b ? b : a;
    /* position of pair (lo, hi) among the row-major pairs lo < hi */
    int idx = lo * N - lo * (lo + 1) / 2 + (hi - lo - 1);
    double r = t[N + 2 * idx], i = t[N + 2 * idx + 1];
    *re = r;
    *im = (a < b) ? i : -i;
}

/* Eq. 3 evaluated on the table: I_i = sum_{a,b} V_a conj(V_b) T_i[a][b],
 * g_a = - sum_i (1/I_i) sum_b V_b T_i[b][a] + (M V)_a. */
int oracle_nll_table(const double *T, int64_t n, int N, const double *M,
                     const double *V, int K, double *nll, double *grad)
{
    const int64_t P = (int64_t)N * N;
    int bad_sets = 0;
    nsum *gr = (nsum *)malloc(sizeof(nsum) * 2 * (size_t)N);
    double *mv = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    for (int k = 0; k < K; ++k) {
        const double *v = V + (size_t)k * 2 * N;
        nsum lnsum = {0, 0};
        int bad = 0;
        memset(gr, 0, sizeof(nsum) * 2 * (size_t)N);
        for (int64_t i = 0; i < n && !bad; ++i) {
            const double *t = T + i * P;
            nsum Is = {0, 0};
            for (int a = 0; a < N; ++a)
                for (int b = 0; b < N; ++b) {
                    double tr, ti, pr, pi, qr, qi;
                    table_entry(t, N, a, b, &tr, &ti);
                    cmul(v[2 * a], v[2 * a + 1], v[2 * b], -v[2 * b + 1], &pr, &pi);
                    cmul(pr, pi, tr, ti, &qr, &qi);
                    nadd(&Is, qr);
                }
            double I = nval(&Is);
            if (!(I > 0) || !isfinite(I)) {
                bad = 1;
                break;
            }
            nadd(&lnsum, log(I));
            if (grad)
                for (int a = 0; a < N; ++a)
                    for (int b = 0; b < N; ++b) {
                        double tr, ti, pr, pi;
                        table_entry(t, N, b, a, &tr, &ti);
                        cmul(v[2 * b], v[2 * b + 1], tr, ti, &pr, &pi);
                        nadd(&gr[2 * a], pr / I);
                        nadd(&gr[2 * a + 1], pi / I);
                    }
        }
        double nv;
        oracle_norm_term(M, N, v, &nv, mv);
        if (bad) {
            ++bad_sets;
            nll[k] = INFINITY;
            if (grad)
                memset(grad + (size_t)k * 2 * N, 0, sizeof(double) * 2 * (size_t)N);
            continue;
        }
        nll[k] = -nval(&lnsum) + nv;
        if (grad)
            for (int c = 0; c < 2 * N; ++c)
                grad[(size_t)k * 2 * N + c] = -nval(&gr[c]) + mv[c];
    }
    free(gr);
    free(mv);
    return bad_sets;
}

/* ---- Free resonance parameters ----------------------------------------- */
/* When masses and widths are fit parameters the precompute of Sec. 2 no
 * longer holds: the amplitudes of the free waves are re-evaluated from the
 * event's mass and the MC term is summed directly each call.
 *
 * Waves 0..R-1 are free: A_r(i) = BW(m_i; mass_r, width_r) * Y_r(i) with
 * BW(m; M, G) = 1 / (M^2 - m^2 - i M G). Waves R..N-1 are fixed:
 * A_{R+f}(i) = Afix[i][f]. Y is [n][R] complex, Afix is [n][N-R] complex.
 *
 * NLL(V, mass, width) = - sum_i ln I_i + (1/n_gen) sum_{j in MC} I_j.
 * Outputs: nll, gV[N] complex (dNLL/dV*), gM[R], gW[R] (real derivatives). */
static void bw_and_derivs(double m, double M, double G, double *bw, double *dM, double *dG)
{
    /* BW = 1/(M^2 - m^2 - i M G);  dBW/dM = -(2M - i G) BW^2;  dBW/dG = i M BW^2 */
    double dr = M * M - m * m, di = -M * G;
    double den = dr * dr + di * di;
    double br = dr / den, bi = -di / den;
    double b2r, b2i;
    cmul(br, bi, br, bi, &b2r, &b2i);
    bw[0] = br;
    bw[1] = bi;
    double pr, pi;
    cmul(-2.0 * M, G, b2r, b2i, &pr, &pi);
    dM[0] = pr;
    dM[1] = pi;
    cmul(0.0, M, b2r, b2i, &pr, &pi);
    dG[0] = pr;
    dG[1] = pi;
}

static void res_amp(int64_t i, int N, int R, const double *m, const double *Y, const double *Afix,
                    const double *mass, const double *width, double *A, double *dAM, double *dAG)
{
    for (int r = 0; r < R; ++r) {
        double bw[2], dM[2], dG[2];
        bw_and_derivs(m[i], mass[r], width[r], bw, dM, dG);
        double yr = Y[(i * R + r) * 2], yi = Y[(i * R + r) * 2 + 1];
        cmul(bw[0], bw[1], yr, yi, &A[2 * r], &A[2 * r + 1]);
        cmul(dM[0], dM[1], yr, yi, &dAM[2 * r], &dAM[2 * r + 1]);
        cmul(dG[0], dG[1], yr, yi, &dAG[2 * r], &dAG[2 * r + 1]);
    }
    for (int f = 0; f < N - R; ++f) {
        A[2 * (R + f)] = Afix[(i * (N - R) + f) * 2];
        A[2 * (R + f) + 1] = Afix[(i * (N - R) + f) * 2 + 1];
    }
}

/* One pass over a sample: accumulates sum ln I (if lnsum), or sum I (if isum),
 * and the derivative sums. weight multiplies each event's contribution to the
 * gradients: -1/I_i for data, +1/n_gen for MC. */
static int res_pass(int64_t n, int N, int R, const double *m, const double *Y, const double *Afix,
                    const double *mass, const double *width, const double *V, int data,
                    nsum *acc, nsum *gV, nsum *gM, nsum *gW)
{
    double *A = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    double *dAM = (double *)malloc(sizeof(double) * 2 * (size_t)(R > 0 ? R : 1));
    double *dAG = (double *)malloc(sizeof(double) * 2 * (size_t)(R > 0 ? R : 1));
    int bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        res_amp(i, N, R, m, Y, Afix, mass, width, A, dAM, dAG);
        nsum sr = {0, 0}, si = {0, 0};
        for (int a = 0; a < N; ++a) {
            double pr, pi;
            cmul(V[2 * a], V[2 * a + 1], A[2 * a], A[2 * a + 1], &pr, &pi);
            nadd(&sr, pr);
            nadd(&si, pi);
        }
        double s_r = nval(&sr), s_i = nval(&si);
        double I = s_r * s_r + s_i * s_i;
        double w;
        if (data) {
            if (!(I > 0) || !isfinite(I)) {
                bad = 1;
                break;
            }
            nadd(acc, log(I));
            w = -1.0 / I;
        } else {
            nadd(acc, I);
            w = 1.0;
        }
        /* dI/dV*_a = conj(A_a) S ; dI/dp = 2 Re(conj(S) V_r dA_r/dp) */
        for (int a = 0; a < N; ++a) {
            double pr, pi;
            cmul(A[2 * a], -A[2 * a + 1], s_r, s_i, &pr, &pi);
            nadd(&gV[2 * a], w * pr);
            nadd(&gV[2 * a + 1], w * pi);
        }
        for (int r = 0; r < R; ++r) {
            double vr, vi, pr, pi;
            cmul(V[2 * r], V[2 * r + 1], dAM[2 * r], dAM[2 * r + 1], &vr, &vi);
            cmul(s_r, -s_i, vr, vi, &pr, &pi);
            nadd(&gM[r], w * 2.0 * pr);
            cmul(V[2 * r], V[2 * r + 1], dAG[2 * r], dAG[2 * r + 1], &vr, &vi);
            cmul(s_r, -s_i, vr, vi, &pr, &pi);
            nadd(&gW[r], w * 2.0 * pr);
        }
    }
    free(A);
    free(dAM);
    free(dAG);
    return bad;
}

int oracle_nll_res(int N, int R,
                   const double *m_d, const double *Y_d, const double *Afix_d, int64_t n_d,
                   const double *m_mc, const double *Y_mc, const double *Afix_mc, int64_t n_mc,
                   double n_gen, const double *V, const double *mass, const double *width,
                   double *nll, double *gV, double *gM, double *gW)
{
    if (R < 0 || R > N || !(n_gen > 0))
        return -1;
    nsum *gVd = (nsum *)calloc(2 * (size_t)N, sizeof(nsum));
    nsum *gVm = (nsum *)calloc(2 * (size_t)N, sizeof(nsum));
    nsum *gMd = (nsum *)calloc((size_t)R + 1, sizeof(nsum));
    nsum *gMm = (nsum *)calloc((size_t)R + 1, sizeof(nsum));
    nsum *gWd = (nsum *)calloc((size_t)R + 1, sizeof(nsum));
    nsum *gWm = (nsum *)calloc((size_t)R + 1, sizeof(nsum));
    nsum lnsum = {0, 0}, isum = {0, 0};
    int bad = res_pass(n_d, N, R, m_d, Y_d, Afix_d, mass, width, V, 1, &lnsum, gVd, gMd, gWd);
    res_pass(n_mc, N, R, m_mc, Y_mc, Afix_mc, mass, width, V, 0, &isum, gVm, gMm, gWm);
    if (bad) {
        *nll = INFINITY;
        memset(gV, 0, sizeof(double) * 2 * (size_t)N);
        memset(gM, 0, sizeof(double) * (size_t)R);
        memset(gW, 0, sizeof(double) * (size_t)R);
    } else {
        *nll = -nval(&lnsum) + nval(&isum) / n_gen;
        for (int c = 0; c < 2 * N; ++c)
            gV[c] = nval(&gVd[c]) + nval(&gVm[c]) / n_gen;
        for (int r = 0; r < R; ++r) {
            gM[r] = nval(&gMd[r]) + nval(&gMm[r]) / n_gen;
            gW[r] = nval(&gWd[r]) + nval(&gWm[r]) / n_gen;
        }
    }
    free(gVd); free(gVm); free(gMd); free(gMm); free(gWd); free(gWm);
    return bad;
}

/* ---- FUMILI Hessian (Sec. 4, 5) ---------------------------------------- */
/* H = sum_i grad ln I_i grad ln I_i^T, [2N][2N] row-major in
 * p = (Re V_0..Re V_{N-1}, Im V_0..Im V_{N-1}).
 * Returns 1 (and leaves H zero) if an intensity is not positive and finite. */
int oracle_hessian(const double *A, int64_t n, int N, const double *V, double *H)
{
    const int P = 2 * N;
    nsum *h = (nsum *)calloc((size_t)P * P, sizeof(nsum));
    double *d = (double *)malloc(sizeof(double) * (size_t)P);
    int bad = 0;
    for (int64_t i = 0; i < n && !bad; ++i) {
        const double *Ai = A + (size_t)i * N * 2;
        nsum sr = {0, 0}, si = {0, 0};
        for (int a = 0; a < N; ++a) {
            double pr, pi;
            cmul(V[2 * a], V[2 * a + 1], Ai[2 * a], Ai[2 * a + 1], &pr, &pi);
            nadd(&sr, pr);
            nadd(&si, pi);
        }
        const double s_r = nval(&sr), s_i = nval(&si), I = s_r * s_r + s_i * s_i;
        if (!(I > 0) || !isfinite(I)) {
            bad = 1;
            break;
        }
        /* d/dRe V_a ln I = 2 Re(conj(A_a) S) / I,  d/dIm V_a ln I = 2 Im(conj(A_a) S) / I */
        for (int a = 0; a < N; ++a) {
            double pr, pi;
            cmul(Ai[2 * a], -Ai[2 * a + 1], s_r, s_i, &pr, &pi);
            d[a] = 2.0 * pr / I;
            d[N + a] = 2.0 * pi / I;
        }
        for (int x = 0; x < P; ++x)
            for (int y = 0; y < P; ++y)
                nadd(&h[x * P + y], d[x] * d[y]);
    }
    for (int x = 0; x < P; ++x)
        for (int y = 0; y < P; ++y)
            H[x * P + y] = bad ? 0.0 : nval(&h[x * P + y]);
    free(h);
    free(d);
    return bad;
}

/* ---- projection weights and fit fractions ------------------------------ */
/* w[j] = |sum_a V_a A_a(j)|^2 / N_gen over the accepted MC events. */
void oracle_mc_weights(const double *A, int64_t n, int N, const double *V, double n_gen, double *w)
{
    oracle_intensity(A, n, N, V, w);
    for (int64_t j = 0; j < n; ++j)
        w[j] /= n_gen;
}

/* F[a][b] = Re(conj(V_a) M_ab V_b) / V^H M V (the diagonal: the waves' fit
 * fractions; off-diagonal pairs F_ab + F_ba: their interference). */
void oracle_fit_fractions(const double *M, int N, const double *V, double *F)
{
    double nv;
    oracle_norm_term(M, N, V, &nv, NULL);
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            double pr, pi, qr, qi;
            cmul(M[(a * N + b) * 2], M[(a * N + b) * 2 + 1], V[2 * b], V[2 * b + 1], &pr, &pi);
            cmul(V[2 * a], -V[2 * a + 1], pr, pi, &qr, &qi);
            F[a * N + b] = qr / nv;
        }
}

/* ---- Incoherent sum over L components ---------------------------------- */
/* M[a][b] = (1/n_gen) sum_{j < n_acc} sum_{l < L} conj(A_a^l(j)) A_b^l(j). */
int oracle_norm_incoh(const double *A, int64_t n_acc, int L, int N, double n_gen, double *M)
{
    if (N <= 0 || L <= 0 || n_acc < 0 || !(n_gen > 0))
        return -1;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            nsum re = {0, 0}, im = {0, 0};
            for (int64_t j = 0; j < n_acc; ++j)
                for (int l = 0; l < L; ++l) {
                    const double *x = A + ((j * L + l) * N) * 2;
                    double pr, pi;
                    cmul(x[2 * a], -x[2 * a + 1], x[2 * b], x[2 * b + 1], &pr, &pi);
                    nadd(&re, pr);
                    nadd(&im, pi);
                }
            M[(a * N + b) * 2] = nval(&re) / n_gen;
            M[(a * N + b) * 2 + 1] = nval(&im) / n_gen;
        }
    return 0;
}

/* Per-event table of the incoherent sum, T_i[a][b] = sum_l A_a^l conj(A_b^l),
 * stored like oracle_table (real diagonal, then Re/Im of the pairs a < b). */
int oracle_table_incoh(const double *A, int64_t n, int L, int N, double *T)
{
    const int64_t P = (int64_t)N * N;
    for (int64_t i = 0; i < n; ++i) {
        double *t = T + i * P;
        for (int a = 0; a < N; ++a) {
            nsum d = {0, 0};
            for (int l = 0; l < L; ++l) {
                const double *x = A + ((i * L + l) * N) * 2;
                nadd(&d, x[2 * a] * x[2 * a] + x[2 * a + 1] * x[2 * a + 1]);
            }
            t[a] = nval(&d);
        }
        int p = N;
        for (int a = 0; a < N; ++a)
            for (int b = a + 1; b < N; ++b) {
                nsum re = {0, 0}, im = {0, 0};
                for (int l = 0; l < L; ++l) {
                    const double *x = A + ((i * L + l) * N) * 2;
                    double pr, pi;
                    cmul(x[2 * a], x[2 * a + 1], x[2 * b], -x[2 * b + 1], &pr, &pi);
                    nadd(&re, pr);
                    nadd(&im, pi);
                }
                t[p++] = nval(&re);
                t[p++] = nval(&im);
            }
    }
    return 0;
}

/* Eq. 3 with the incoherent intensity I_i = sum_l |S_i^l|^2,
 * S_i^l = sum_a V_a A_a^l(i), for K parameter sets; returns and outputs as
 * oracle_nll_amp. */
int oracle_nll_incoh(const double *A, int64_t n, int L, int N, const double *M,
                     const double *V, int K, double *nll, double *grad)
{
    int bad_sets = 0;
    nsum *gr = (nsum *)malloc(sizeof(nsum) * 2 * (size_t)N);
    double *mv = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    double *s = (double *)malloc(sizeof(double) * 2 * (size_t)L);
    for (int k = 0; k < K; ++k) {
        const double *v = V + (size_t)k * 2 * N;
        nsum lnsum = {0, 0};
        int bad = 0;
        memset(gr, 0, sizeof(nsum) * 2 * (size_t)N);
        for (int64_t i = 0; i < n && !bad; ++i) {
            nsum I = {0, 0};
            for (int l = 0; l < L; ++l) {
                const double *x = A + ((i * L + l) * N) * 2;
                nsum sr = {0, 0}, si = {0, 0};
                for (int a = 0; a < N; ++a) {
                    double pr, pi;
                    cmul(v[2 * a], v[2 * a + 1], x[2 * a], x[2 * a + 1], &pr, &pi);
                    nadd(&sr, pr);
                    nadd(&si, pi);
                }
                s[2 * l] = nval(&sr);
                s[2 * l + 1] = nval(&si);
                nadd(&I, s[2 * l] * s[2 * l] + s[2 * l + 1] * s[2 * l + 1]);
            }
            const double Iv = nval(&I);
            if (!(Iv > 0) || !isfinite(Iv)) {
                bad = 1;
                break;
            }
            nadd(&lnsum, log(Iv));
            if (grad)
                for (int l = 0; l < L; ++l) {
                    const double *x = A + ((i * L + l) * N) * 2;
                    const double rr = s[2 * l] / Iv, ri = s[2 * l + 1] / Iv;
                    for (int a = 0; a < N; ++a) {
                        double pr, pi;
                        cmul(x[2 * a], -x[2 * a + 1], rr, ri, &pr, &pi);  /* conj(A) S / I */
                        nadd(&gr[2 * a], pr);
                        nadd(&gr[2 * a + 1], pi);
                    }
                }
        }
        double nv;
        oracle_norm_term(M, N, v, &nv, mv);
        if (bad) {
            ++bad_sets;
            nll[k] = INFINITY;
            if (grad)
                memset(grad + (size_t)k * 2 * N, 0, sizeof(double) * 2 * (size_t)N);
            continue;
        }
        nll[k] = -nval(&lnsum) + nv;
        if (grad)
            for (int c = 0; c < 2 * N; ++c)
                grad[(size_t)k * 2 * N + c] = -nval(&gr[c]) + mv[c];
    }
    free(gr);
    free(mv);
    free(s);
    return bad_sets;
}

/* ---- Amplitude model: Breit-Wigner x spherical harmonic ----------------- */
/* Associated Legendre function P_l^m(x), 0 <= m <= l, with the Condon-Shortley
 * phase: P_m^m = (-1)^m (2m - 1)!! (1 - x^2)^(m/2), P_{m+1}^m = x (2m + 1) P_m^m,
 * (l - m) P_l^m = (2l - 1) x P_{l-1}^m - (l + m - 1) P_{l-2}^m. */
static double legendre_p(int l, int m, double x)
{
    const double s = sqrt(fmax(0.0, 1.0 - x * x));
    double pmm = 1.0;
    for (int k = 1; k <= m; ++k)
        pmm *= -(2.0 * k - 1.0) * s;
    if (l == m)
        return pmm;
    double p1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1)
        return p1;
    double p2 = pmm;
    for (int ll = m + 2; ll <= l; ++ll) {
        const double p = ((2.0 * ll - 1.0) * x * p1 - (ll + m - 1.0) * p2) / (ll - m);
        p2 = p1;
        p1 = p;
    }
    return p1;
}

/* Y_l^m(theta, phi) = sqrt((2l + 1)/(4 pi) (l - m)!/(l + m)!) P_l^m(cos theta)
 * e^{i m phi} for m >= 0; Y_l^{-m} = (-1)^m conj(Y_l^m). */
static void sph_harm(int l, int m, double costh, double phi, double *re, double *im)
{
    const int am = m < 0 ? -m : m;
    double ratio = 1.0;  /* (l - am)! / (l + am)! */
    for (int k = l - am + 1; k <= l + am; ++k)
        ratio /= k;
    const double pi = 3.14159265358979323846;
    const double norm = sqrt((2.0 * l + 1.0) / (4.0 * pi) * ratio);
    const double p = norm * legendre_p(l, am, costh);
    double r = p * cos(am * phi), i = p * sin(am * phi);
    if (m < 0) {
        const double sign = (am & 1) ? -1.0 : 1.0;
        r *= sign;
        i *= -sign;
    }
    *re = r;
    *im = i;
}

/* A[i][a] = BW(m_i; mass_a, width_a) Y_{l_a}^{mm_a}(costh_i, phi_i) for
 * kin[i] = (m, cos theta, phi); BW = 1 / (M^2 - m^2 - i M G) written as
 * (D + i M G) / (D^2 + (M G)^2) with D = M^2 - m^2. Returns -1 for a wave
 * with |mm| > l or l < 0. */
int oracle_amplitudes(const double *kin, int64_t n, int N, const double *mass, const double *width,
                      const int *l, const int *mm, double *A)
{
    for (int a = 0; a < N; ++a)
        if (l[a] < 0 || mm[a] > l[a] || -mm[a] > l[a])
            return -1;
    for (int64_t i = 0; i < n; ++i) {
        const double m = kin[3 * i], c = kin[3 * i + 1], ph = kin[3 * i + 2];
        for (int a = 0; a < N; ++a) {
            const double D = mass[a] * mass[a] - m * m, G = mass[a] * width[a];
            const double den = D * D + G * G;
            const double br = D / den, bi = G / den;
            double yr, yi;
            sph_harm(l[a], mm[a], c, ph, &yr, &yi);
            A[(i * N + a) * 2] = br * yr - bi * yi;
            A[(i * N + a) * 2 + 1] = br * yi + bi * yr;
        }
    }
    return 0;
}

/* ---- Covariant tensor amplitudes: J/psi -> gamma X, X -> K+ K- -------------
 * Paper Sec. 4: the framework builds its amplitudes on the GPU in the
 * covariant tensor formalism. Written here from that formalism: 4-vectors in
 * the J/psi rest frame, metric (+,-,-,-), a.b = a0 b0 - a.b(3).
 *   p3[i] = (q, k1, k2): 3-momenta (GeV) of the photon, K+ and K-.
 *   q = (|q|, q), k = (sqrt(mK^2 + |k|^2), k), p = k1 + k2, m^2 = p.p,
 *   r = k1 - k2, rt = r - (r.p / p.p) p  (the relative momentum orthogonal to p).
 * Unobserved: the J/psi helicity M = +1, -1 along the beam (z) axis,
 *   psi(+1) = (0, -1, -i, 0)/sqrt2, psi(-1) = (0, 1, -i, 0)/sqrt2,
 * and the photon's linear polarization lam = 1, 2, real and transverse,
 *   e1 = (0, z x q / |z x q|) (x when q is along z), e2 = (0, q/|q| x e1).
 * Component l = 2 (M index) + (lam index), M index 0 for +1.
 * Wave a (mass M_a, width G_a, spin s_a):
 *   s = 0: A = BW(m^2) psi.e
 *   s = 2: A = BW(m^2) B2(Q) t(psi, e),
 *          t(u, w) = (u.rt)(w.rt) - (1/3)(rt.rt)(u.w - (u.p)(w.p)/p.p),
 *          the contraction of psi and e with the symmetric, traceless tensor
 *          of rank 2 orthogonal to p built from rt;
 *          Q^2 = m^2/4 - mK^2, B2 = sqrt(13 / (Q^4 + 3 Q^2 Q0^2 + 9 Q0^4)),
 *          Q0 = 0.197327 GeV (an interaction radius of 1 fm);
 *   BW(m^2) = 1 / (M^2 - m^2 - i M G).
 * out[((i * 4 + l) * N + a) * 2 + {0, 1}]. Returns -1 for a spin other than
 * 0 or 2. */
static double mdot(const double *a, const double *b)
{
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

int oracle_cov_amplitudes(const double *p3, int64_t n, int N, const double *mass,
                          const double *width, const int *spin, double *out)
{
    const double mK = 0.493677, Q0 = 0.197327, isq2 = 0.70710678118654752440;
    for (int a = 0; a < N; ++a)
        if (spin[a] != 0 && spin[a] != 2)
            return -1;
    for (int64_t i = 0; i < n; ++i) {
        const double *v = p3 + 9 * i;
        double q[4], k1[4], k2[4], p[4], r[4], rt[4];
        const double qq = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        q[0] = qq;
        k1[0] = sqrt(mK * mK + v[3] * v[3] + v[4] * v[4] + v[5] * v[5]);
        k2[0] = sqrt(mK * mK + v[6] * v[6] + v[7] * v[7] + v[8] * v[8]);
        for (int c = 0; c < 3; ++c) {
            q[c + 1] = v[c];
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
        /* photon polarizations */
        double e[2][4];
        double ux = -q[2], uy = q[1];           /* z x q */
        double un = sqrt(ux * ux + uy * uy);
        if (un > 1e-12 * qq) {
            e[0][1] = ux / un;
            e[0][2] = uy / un;
        } else {
            e[0][1] = 1.0;
            e[0][2] = 0.0;
        }
        e[0][0] = 0.0;
        e[0][3] = 0.0;
        const double qh[3] = {q[1] / qq, q[2] / qq, q[3] / qq};
        e[1][0] = 0.0;
        e[1][1] = qh[1] * e[0][3] - qh[2] * e[0][2];
        e[1][2] = qh[2] * e[0][1] - qh[0] * e[0][3];
        e[1][3] = qh[0] * e[0][2] - qh[1] * e[0][1];
        /* psi polarizations: real and imaginary parts */
        const double psr[2][4] = {{0.0, -isq2, 0.0, 0.0}, {0.0, isq2, 0.0, 0.0}};
        const double psi[2][4] = {{0.0, 0.0, -isq2, 0.0}, {0.0, 0.0, -isq2, 0.0}};
        for (int im = 0; im < 2; ++im)
            for (int il = 0; il < 2; ++il) {
                const int l = 2 * im + il;
                const double *w = e[il];
                /* the contractions are linear in psi: real and imaginary parts apart */
                const double s0r = mdot(psr[im], w), s0i = mdot(psi[im], w);
                const double prw = mdot(w, rt), pwp = mdot(w, p);
                const double ar = mdot(psr[im], rt), ai = mdot(psi[im], rt);
                const double apr = mdot(psr[im], p), api = mdot(psi[im], p);
                const double t_r = ar * prw - rr / 3.0 * (s0r - apr * pwp / pp);
                const double t_i = ai * prw - rr / 3.0 * (s0i - api * pwp / pp);
                for (int a = 0; a < N; ++a) {
                    const double D = mass[a] * mass[a] - pp, G = mass[a] * width[a];
                    const double den = D * D + G * G;
                    const double br = D / den, bi = G / den;
                    double cr, ci;
                    if (spin[a] == 0) {
                        cr = s0r;
                        ci = s0i;
                    } else {
                        cr = b2 * t_r;
                        ci = b2 * t_i;
                    }
                    double *o = out + ((i * 4 + l) * N + a) * 2;
                    o[0] = br * cr - bi * ci;
                    o[1] = br * ci + bi * cr;
                }
            }
    }
    return 0;
}
