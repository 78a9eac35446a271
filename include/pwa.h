/*
 * pwa.h -- C ABI of the GB300 partial wave analysis likelihood library.
 *
 * The library evaluates the extended negative log-likelihood of Eq. 3 of
 * Berger, "Partial wave analysis at BES III harnessing the power of GPUs":
 *
 *   NLL(V) = - sum_{i in data} ln I(Omega_i) + V^H M V,
 *   I(Omega) = | sum_alpha V_alpha A_alpha(Omega) |^2                  (Eq. 1)
 *   M[a][b]  = (1/N_MC^Gen) sum_{j in accepted MC} conj(A_a(j)) A_b(j)
 *
 * and its Wirtinger gradient g_a = dNLL/dV*_a
 *   = - sum_i conj(A_a(i)) S_i / I_i + (M V)_a,  S_i = sum_b V_b A_b(i).
 * The real-parameter gradient is dNLL/dRe V_a = 2 Re g_a and
 * dNLL/dIm V_a = 2 Im g_a.
 *
 * As in Sec. 2 (after Eq. 3), amplitudes are fixed once loaded and the MC
 * bracket M is built once; per call only the parameters go in and the
 * likelihood and gradient come out (Sec. 5: transfers are restricted to the
 * fit parameters and the results).
 *
 * Conventions shared by every call:
 *  - Complex numbers are interleaved (re, im) pairs.
 *  - Amplitudes are event-major: element (i, a) of an [n][n_waves] array.
 *  - V for K parameter sets is [K][n_waves] complex128 (double pairs).
 *  - Every function returns a status code (PWA_OK = 0 or a negative error);
 *    pwa_last_error() gives a human-readable message for the last failure on
 *    that context. No function aborts, traps or throws across the ABI.
 *  - A context is bound to one device and one CUDA stream and must not be
 *    used from two host threads at once.
 */
#ifndef PWA_H
#define PWA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PWA_OK 0
#define PWA_EINVAL -1   /* bad argument (null pointer, size, K out of range) */
#define PWA_ENOMEM -2   /* a device or pinned allocation failed */
#define PWA_ECUDA -3    /* a CUDA runtime/driver call failed */
#define PWA_ESTATE -4   /* call out of order (e.g. pwa_nll before pwa_build_norm) */
#define PWA_EDOMAIN -5  /* some data intensity I_i was <= 0 or not finite for a
                           parameter set: that set's nll is +inf and its gradient 0 */
#define PWA_ETIMEOUT -6 /* a device-side bounded wait gave up; results invalid */
#define PWA_ENOTSUP -7  /* configuration not supported by this build */

/* ---- forms of the data term (Sec. 2, after Eq. 3) ----------------------- */
#define PWA_FORM_AMP 1   /* direct: S_i = sum_a V_a A_a(i), I_i = |S_i|^2 */
#define PWA_FORM_TABLE 2 /* precomputed per-event table A_a A*_b (upper triangle) */
#define PWA_FORM_TC 4    /* batched K parameter sets on the tensor cores (the thousands
                            of restarts of Sec. 2 evaluated together): amplitudes in
                            block floating point (one exponent per event, see
                            PWA_PREC_*), V in 24-bit block floating point per set plus
                            a first-order correction, BF16 integer operands whose FP32
                            tensor-core sums are exact */

/* ---- amplitude encoding of the tensor-core form (pwa_config.precision) --- */
#define PWA_PREC_DEFAULT 0 /* PWA_PREC_BFP16 */
#define PWA_PREC_BFP16 1   /* A = 2^(E-8) (x0 + x1/256), |x0| <= 256, |x1| <= 128 integers:
                              16 bits below the event's largest component. Against
                              FP64 amplitudes (1M events x 20 waves) this moves the
                              NLL by ~0.04 and a fitted V by < 0.01 of its error */
#define PWA_PREC_BFP8 2    /* A = 2^(E-8) x0: 8 bits below the event's largest
                              component; about half the tensor-core work. A coarser
                              sample: the NLL moves by ~500 and a fitted V by tens of
                              its errors at the same size, so it ranks starting
                              points; a final fit takes an FP32 form */

/* ---- amplitude element types ------------------------------------------- */
#define PWA_C64 1  /* float pairs: used as given */
#define PWA_C128 2 /* double pairs: rounded to nearest float on load */

typedef struct pwa_ctx pwa_ctx;

typedef struct pwa_config {
    int n_waves;   /* number of partial waves N, 1 <= N <= 48 */
    int forms;     /* bitmask of PWA_FORM_* stores built by pwa_load_events;
                      0 means PWA_FORM_AMP; PWA_FORM_TABLE needs n_waves <= 24 */
    int precision; /* PWA_PREC_*: amplitude encoding of the tensor-core form
                      (ignored by the other forms) */
    int max_k;     /* largest K accepted by the evaluation calls (>= 1) */
    void *stream;  /* cudaStream_t to run on; NULL = a stream the context owns */
} pwa_config;

/* Create a context on CUDA device `device`. On success *out owns all device
 * memory the library allocates for it; release it with pwa_destroy.
 * Errors: PWA_EINVAL (null out/cfg, n_waves or max_k out of range),
 * PWA_ECUDA (device not usable), PWA_ENOMEM. */
int pwa_create(pwa_ctx **out, int device, const pwa_config *cfg);

/* Free everything the context owns. Null is accepted. */
int pwa_destroy(pwa_ctx *ctx);

/* Load the data sample and the accepted MC sample (Eq. 2/3 and the text after
 * Eq. 2: the normalisation integral is a sum over the N_MC^Acc accepted events
 * divided by the number generated, N_MC^Gen).
 *   data_amp: [n_data][n_waves] complex, host or device pointer (detected)
 *   mc_amp:   [n_mc_acc][n_waves] complex, host or device pointer
 *   n_mc_gen: number of generated MC events, n_mc_gen >= n_mc_acc
 *   amp_dtype: PWA_C64 or PWA_C128 (C128 is rounded to float on the device)
 * The library copies the amplitudes into its own structure-of-arrays store
 * (one float plane per real and imaginary part of each wave, events
 * contiguous), and builds the per-event table if PWA_FORM_TABLE was
 * requested; the caller keeps ownership of its buffers. Device inputs (here
 * and in every call that loads or generates from caller buffers) are read
 * after all work already issued to the device has completed, whichever
 * stream produced them (the call synchronises the device first). Loading again
 * replaces the sample and invalidates the normalisation matrix.
 * Errors: PWA_EINVAL (n_data < 1, n_mc_acc < 1, n_mc_gen < n_mc_acc, null
 * pointers, bad dtype), PWA_ENOMEM, PWA_ECUDA. */
int pwa_load_events(pwa_ctx *ctx, const void *data_amp, int64_t n_data,
                    const void *mc_amp, int64_t n_mc_acc, double n_mc_gen,
                    int amp_dtype);

/* ---- amplitudes on the device ---------------------------------------------
 * The framework of the paper computes its amplitudes on the GPU (Sec. 4).
 * Two amplitude models: the covariant tensor amplitudes of the radiative
 * decay J/psi -> gamma X, X -> K+ K- (pwa_compute_covariant_amplitudes,
 * pwa_load_events_covariant, below the incoherent loader), and a model with
 * one angle pair that serves the coherent samples:
 *   A_a(Omega) = BW(m; M_a, G_a) Y_{l_a}^{m_a}(theta, phi),
 *   BW(m; M, G) = 1 / (M^2 - m^2 - i M G)   (fixed-width Breit-Wigner),
 *   Y_l^m the orthonormal spherical harmonic with the Condon-Shortley phase,
 * in double precision, each amplitude rounded once to float. */
typedef struct pwa_wave {
    double mass;   /* M > 0 (GeV) */
    double width;  /* G > 0 (GeV) */
    int l;         /* 0 <= l <= 16 */
    int m;         /* -l <= m <= l */
} pwa_wave;

/* Amplitudes of n events for the context's n_waves waves.
 *   waves: host [n_waves];  kin: [n][3] doubles (m, cos theta, phi), host or
 *   device pointer;  out: [n][n_waves] complex64 (float pairs), host or device.
 * Does not touch the loaded sample. Errors: PWA_EINVAL (null pointer, n out
 * of [1, 2^31 - 1024], a wave with |m| > l, l > 16, or a non-positive mass or
 * width), PWA_ENOMEM, PWA_ECUDA. */
int pwa_compute_amplitudes(pwa_ctx *ctx, const pwa_wave *waves, const double *kin, int64_t n,
                           void *out);

/* Load a data and an accepted-MC sample given by their kinematics: the
 * amplitudes are generated on the device straight into the library's store
 * (no host amplitude arrays, no amplitude transfer), then everything
 * pwa_load_events does follows (table, tensor-core store as configured).
 *   data_kin [n_data][3], mc_kin [n_mc_acc][3]: (m, cos theta, phi) doubles,
 *   host or device pointers; n_mc_gen as in pwa_load_events.
 * Errors as pwa_compute_amplitudes and pwa_load_events. */
int pwa_load_events_generated(pwa_ctx *ctx, const pwa_wave *waves, const double *data_kin,
                              int64_t n_data, const double *mc_kin, int64_t n_mc_acc,
                              double n_mc_gen);

/* Load a sample whose intensity is an incoherent sum over n_lambda
 * unobserved components per event (e.g. helicity states of an undetected
 * polarisation), I(Omega) = sum_l |sum_a V_a A_a^l(Omega)|^2. Eq. 3 keeps its
 * form with the per-event products A_a A*_b of its data term and of its MC
 * bracket summed over the components: M[a][b] = (1/N_MC^Gen) sum_j sum_l
 * conj(A_a^l(j)) A_b^l(j), g_a = - sum_i sum_l conj(A_a^l(i)) S_i^l / I_i +
 * (M V)_a with S_i^l = sum_b V_b A_b^l(i). (The paper writes the coherent
 * sum, Eq. 1; this is the reading of Eq. 3 for several components, which
 * leaves the table form's cost unchanged.)
 *   data_amp: [n_data][n_lambda][n_waves] complex, host or device pointer
 *   mc_amp:   [n_mc_acc][n_lambda][n_waves] complex, host or device pointer
 *   n_lambda: 1 <= n_lambda <= 4 (1 is pwa_load_events)
 * Afterwards pwa_build_norm, pwa_nll, pwa_nll_grad(_async), pwa_set_form
 * and pwa_fit_fractions work as for a coherent sample; the direct form
 * (PWA_FORM_AMP) reads 8 n_lambda n_waves bytes per event and takes up to 24
 * waves at n_lambda = 2, 16 at 3, 12 at 4; the table form reads 4 n_waves^2
 * bytes per event whatever n_lambda. Errors as pwa_load_events, plus
 * PWA_EINVAL (n_lambda out of range, n_mc_acc * n_lambda >= 2^31 - 1024) and
 * PWA_ENOTSUP (a context with PWA_FORM_TC, or n_waves above the direct
 * form's limit for n_lambda); pwa_hessian and pwa_mc_weights return
 * PWA_ENOTSUP on such a sample. */
int pwa_load_events_incoherent(pwa_ctx *ctx, int n_lambda, const void *data_amp, int64_t n_data,
                               const void *mc_amp, int64_t n_mc_acc, double n_mc_gen,
                               int amp_dtype);

/* Covariant tensor amplitudes of J/psi -> gamma X, X -> K+ K- (Sec. 4: the
 * amplitudes are built on the GPU in the covariant tensor formalism), per
 * event four unobserved components l = 2 iM + ie: the J/psi helicity
 * M = +1 (iM = 0) or -1 (iM = 1) along z, and the photon's linear
 * polarization e1 (ie = 0) or e2 (ie = 1) (the photon and the J/psi spin
 * states are not observed, so the intensity is the incoherent sum over
 * them, pwa_load_events_incoherent with n_lambda = 4). In the J/psi rest
 * frame, metric (+,-,-,-), mK = 0.493677 GeV:
 *   q the photon, k1 = K+, k2 = K-, p = k1 + k2, r = k1 - k2,
 *   rt = r - (r.p / p.p) p;
 *   psi(+1) = (0, -1, -i, 0)/sqrt2, psi(-1) = (0, 1, -i, 0)/sqrt2;
 *   e1 = (0, z x q / |z x q|) (the x axis when q is along z),
 *   e2 = (0, q/|q| x e1);
 *   spin 0: A = BW(p.p) (psi.e);
 *   spin 2: A = BW(p.p) B2(Q) [(psi.rt)(e.rt) - (1/3)(rt.rt)(psi.e - (psi.p)(e.p)/p.p)]
 *     with Q^2 = p.p/4 - mK^2, B2(Q) = sqrt(13 / (Q^4 + 3 Q^2 Q0^2 + 9 Q0^4)),
 *     Q0 = 0.197327 GeV (the spin-2 Blatt-Weisskopf barrier);
 *   BW(s) = 1 / (M^2 - s - i M G).
 * Evaluated in double precision, each amplitude rounded once to float. */
typedef struct pwa_cov_wave {
    double mass;   /* M > 0 (GeV) */
    double width;  /* G > 0 (GeV) */
    int spin;      /* 0 or 2 */
} pwa_cov_wave;

/* Covariant amplitudes of n events for the context's n_waves waves.
 *   waves: host [n_waves];  p3: [n][9] doubles, the 3-momenta (GeV) of the
 *   photon, the K+ and the K- in the J/psi rest frame, host or device
 *   pointer;  out: [n][4][n_waves] complex64 (component l, then wave), host
 *   or device pointer.
 * Does not touch the loaded sample. Errors: PWA_EINVAL (null pointer, n out
 * of [1, 2^31 - 1024], a spin other than 0 or 2, a non-positive mass or
 * width), PWA_ENOMEM, PWA_ECUDA. */
int pwa_compute_covariant_amplitudes(pwa_ctx *ctx, const pwa_cov_wave *waves, const double *p3,
                                     int64_t n, void *out);

/* Load a data and an accepted-MC sample of J/psi -> gamma K+ K- events given
 * by their 3-momenta: the covariant amplitudes are generated on the device
 * (as pwa_compute_covariant_amplitudes) and loaded as an incoherent sample
 * with n_lambda = 4, without host amplitude arrays.
 *   data_p3 [n_data][9], mc_p3 [n_mc_acc][9], host or device pointers;
 *   n_mc_gen as in pwa_load_events.
 * Errors as pwa_compute_covariant_amplitudes and pwa_load_events_incoherent
 * (the direct form takes up to 12 waves at n_lambda = 4). */
int pwa_load_events_covariant(pwa_ctx *ctx, const pwa_cov_wave *waves, const double *data_p3,
                              int64_t n_data, const double *mc_p3, int64_t n_mc_acc,
                              double n_mc_gen);

/* Build the MC normalisation matrix M (the inner bracket of the second term
 * of Eq. 3), once per loaded sample. If M_out is not NULL it receives M as
 * [n_waves][n_waves] complex128, row-major, M_out[a][b] as defined above.
 * Errors: PWA_ESTATE (no events loaded), PWA_ECUDA. */
int pwa_build_norm(pwa_ctx *ctx, double *M_out);

/* Select which store evaluates the data term: PWA_FORM_AMP (default),
 * PWA_FORM_TABLE or PWA_FORM_TC. The first two give the same NLL up to
 * rounding; PWA_FORM_TC evaluates the BF16-rounded amplitudes (a different
 * sample at the 1e-3 level) with FP32 accumulation and is meant for many
 * parameter sets per call.
 * Errors: PWA_EINVAL (unknown form), PWA_ESTATE (store not built). */
int pwa_set_form(pwa_ctx *ctx, int form);

/* Negative log-likelihood of Eq. 3 for K parameter sets.
 *   V:   host [K][n_waves] complex128
 *   nll: host [K]
 * Returns PWA_EDOMAIN if any set had a non-positive intensity (its nll is
 * +inf; the others are valid). Errors: PWA_EINVAL (K < 1 or K > max_k, null
 * pointers), PWA_ESTATE (before pwa_build_norm), PWA_ECUDA, PWA_ETIMEOUT. */
int pwa_nll(pwa_ctx *ctx, const double *V, int K, double *nll);

/* NLL and its Wirtinger gradient dNLL/dV* for K parameter sets.
 *   grad: host [K][n_waves] complex128
 * Otherwise as pwa_nll; a set with PWA_EDOMAIN gets a zero gradient. */
int pwa_nll_grad(pwa_ctx *ctx, const double *V, int K, double *nll, double *grad);

/* Stream-ordered variant with device pointers: d_V [K][n_waves] complex128,
 * d_nll [K], d_grad [K][n_waves] complex128 (d_grad may be NULL for the NLL
 * alone). Returns after enqueueing. Device-side status (domain, timeout)
 * accumulates in the context until pwa_sync. */
int pwa_nll_grad_async(pwa_ctx *ctx, const double *d_V, int K, double *d_nll, double *d_grad);

/* Wait for the context's stream and return the status accumulated by the
 * asynchronous calls since the previous pwa_sync (PWA_OK, PWA_EDOMAIN or
 * PWA_ETIMEOUT), then clear it. */
int pwa_sync(pwa_ctx *ctx);

/* ---- free Breit-Wigner masses and widths (Sec. 2) ------------------------
 * The precomputed normalisation matrix and per-event table assume fixed
 * masses and widths (Sec. 2, after Eq. 3). With the masses and widths of the
 * first n_free waves free, their amplitudes A_r = BW(m; M_r, G_r) Y_r(Omega),
 * BW(m; M, G) = 1 / (M^2 - m^2 - i M G), are recomputed on every call and the
 * normalisation term of Eq. 3 is the MC sum (1 / n_mc_gen) sum_j |S_j|^2.
 *
 * Load both samples (copied by the library; host or device pointers):
 *   n_free       R, 1 <= R <= 8 and R <= n_waves; needs n_waves <= 32
 *   m_data       [n_data] double, the mass variable m of each event (rounded
 *                to the nearest float on load)
 *   Y_data       [n_data][R] angular factors of the free waves, interleaved
 *                complex of amp_dtype (PWA_C64 or PWA_C128, rounded to float)
 *   Afix_data    [n_data][n_waves - R] amplitudes of the fixed waves (NULL
 *                when R = n_waves)
 *   m_mc, Y_mc, Afix_mc, n_mc_acc: the same for the accepted MC events;
 *   n_mc_gen >= n_mc_acc generated MC events.
 * Independent of pwa_load_events. Errors: PWA_EINVAL (null pointer, sizes),
 * PWA_ENOTSUP (n_waves > 32 or n_free > 8), PWA_ENOMEM, PWA_ECUDA. */
int pwa_load_resonance_events(pwa_ctx *ctx, int n_free, const double *m_data, const void *Y_data,
                              const void *Afix_data, int64_t n_data, const double *m_mc,
                              const void *Y_mc, const void *Afix_mc, int64_t n_mc_acc,
                              double n_mc_gen, int amp_dtype);

/* NLL of Eq. 3 and its gradients with free masses and widths (host pointers):
 *   V       [n_waves] complex128
 *   mass    [n_free] double; width [n_free] double
 *   nll     [1]; gV [n_waves] complex128, dNLL/dV* (may be NULL);
 *   gM, gW  [n_free] double, dNLL/dM_r and dNLL/dG_r (may be NULL)
 * Returns PWA_EDOMAIN (nll = +inf, gradients 0) if a data intensity was not
 * positive and finite; PWA_ESTATE before pwa_load_resonance_events;
 * PWA_EINVAL for null V, mass, width or nll; PWA_ECUDA, PWA_ETIMEOUT. */
int pwa_nll_grad_res(pwa_ctx *ctx, const double *V, const double *mass, const double *width,
                     double *nll, double *gV, double *gM, double *gW);

/* pwa_nll_grad_res with device pointers, stream-ordered, returning after
 * enqueueing: d_V [n_waves] complex128, d_mass and d_width [n_free] double in;
 * d_out [1 + 2 n_waves + 2 n_free] double out: nll, dNLL/dV* (complex128),
 * dNLL/dM, dNLL/dG (nll = +inf and gradients 0 on a domain error, reported by
 * pwa_sync with the other asynchronous calls' status). */
int pwa_nll_grad_res_async(pwa_ctx *ctx, const double *d_V, const double *d_mass,
                           const double *d_width, double *d_out);

/* ---- what the fitter and the plots take besides the NLL -------------------
 * FUMILI Hessian (Sec. 4 fits with FUMILI on analytic gradients and Hessian;
 * Sec. 5 returns the Hessian to the host each iteration). FUMILI's
 * approximation of the Hessian of Eq. 3 over the real parameters
 * p = (Re V_0 .. Re V_{N-1}, Im V_0 .. Im V_{N-1}) drops the second
 * derivatives of the intensity in both terms (-sum_i d^2 I_i / I_i in the data
 * term, d^2(V^H M V) in the MC term; at the minimum they cancel in
 * expectation), leaving
 *   H = sum_{i in data} d_i d_i^T,  d_i = grad_p ln I_i,
 *   (d_i)_a = 2 Re(conj(A_a(i)) S_i) / I_i,  (d_i)_{N+a} = 2 Im(...) / I_i.
 * H is positive semi-definite with the global phase direction
 * (-Im V, Re V) in its null space: fix one phase before solving with it.
 *   V: host [n_waves] complex128;  H: host [2 n_waves][2 n_waves] double,
 *   row-major, symmetric.
 * Uses the context's direct-form store (the data planes loaded by
 * pwa_load_events); any form may be current. Up to 20 waves the sum runs on
 * the tensor cores (each d_i split into three BF16 terms, FP32 sums over
 * 128-event tiles, float-float and FP64 beyond), otherwise (or with the
 * environment variable PWA_HESS_KERNEL=generic) on the FP32 pipe; either way
 * max |H - H_exact| <= 3e-6 max |H_exact|, and the result of a given sample
 * and V is the same on every call. Returns PWA_EDOMAIN (H all
 * zero) if a data intensity was not positive and finite; PWA_ESTATE before
 * pwa_load_events; PWA_EINVAL for null pointers; PWA_ENOTSUP for an
 * incoherent sample; PWA_ENOMEM, PWA_ECUDA. */
int pwa_hessian(pwa_ctx *ctx, const double *V, double *H);

/* pwa_hessian with device pointers (d_V [n_waves] complex128, d_H
 * [2 n_waves][2 n_waves] double), stream-ordered, returning after enqueueing;
 * a domain error zeroes d_H and is reported, with the other asynchronous
 * calls' status, by pwa_sync. Errors as pwa_hessian (before any work). */
int pwa_hessian_async(pwa_ctx *ctx, const double *d_V, double *d_H);

/* Projection weights (the "Plots" step of Table 1): the fitted intensity of
 * each accepted MC event divided by the number generated,
 *   w[j] = |sum_a V_a A_a(j)|^2 / n_mc_gen,  j < n_mc_acc,
 * so that sum_j w[j] = V^H M V, the predicted number of events.
 *   V: host [n_waves] complex128;  w: [n_mc_acc] float, host or device
 *   pointer (detected; a host buffer is filled through a device copy).
 * Errors: PWA_ESTATE (no events loaded), PWA_EINVAL, PWA_ENOMEM, PWA_ECUDA. */
int pwa_mc_weights(pwa_ctx *ctx, const double *V, float *w);

/* Fit fractions: F[a][b] = Re(conj(V_a) M_ab V_b) / V^H M V (host [n_waves]
 * [n_waves] double). The diagonal holds each wave's fraction of the
 * predicted yield; F[a][b] + F[b][a] is the interference of waves a and b;
 * all entries sum to one. Errors: PWA_ESTATE before pwa_build_norm,
 * PWA_EINVAL, PWA_ECUDA. */
int pwa_fit_fractions(pwa_ctx *ctx, const double *V, double *F);

/* ---- uneven model batch (Sec. 2: various trial models are fitted) --------
 * A batch of n_models independent models, each with its own number of waves,
 * data sample and MC sample, evaluated for K parameter sets per model in one
 * CUDA-graph launch (captured on the first call for a given K and replayed;
 * the models' batched tensor-core evaluations run on several streams inside
 * the graph, so small models overlap). Each model uses the tensor-core form.
 *
 *   pwa_batch_create: n_waves[n_models] (each 1..48), max_k per model (1..
 *                     the tensor-core limit for the largest model), precision
 *                     PWA_PREC_*, stream as in pwa_config (NULL: owned).
 *   pwa_batch_load_model: loads model m's samples exactly as pwa_load_events
 *                     and builds its normalisation matrix.
 *   pwa_batch_nll_grad: V_all host, models concatenated: model m's [K][n_waves[m]]
 *                     complex128 block follows model m-1's. nll host [n_models][K];
 *                     grad host, laid out like V_all (may be NULL).
 * Returns PWA_EDOMAIN if some set of some model had a non-positive intensity
 * (that set's nll is +inf, its gradient 0), PWA_ESTATE if a model is not
 * loaded, PWA_EINVAL for bad sizes or pointers, PWA_ENOTSUP if max_k exceeds
 * the tensor-core limit of a model's size, PWA_ENOMEM, PWA_ECUDA,
 * PWA_ETIMEOUT. pwa_batch_last_error gives the message. */
typedef struct pwa_batch pwa_batch;
int pwa_batch_create(pwa_batch **out, int device, int n_models, const int *n_waves, int max_k,
                     int precision, void *stream);
int pwa_batch_destroy(pwa_batch *b);
int pwa_batch_load_model(pwa_batch *b, int model, const void *data_amp, int64_t n_data,
                         const void *mc_amp, int64_t n_mc_acc, double n_mc_gen, int amp_dtype);
int pwa_batch_nll_grad(pwa_batch *b, const double *V_all, int K, double *nll, double *grad);
const char *pwa_batch_last_error(const pwa_batch *b);

/* Direct-form NLL and gradient that allocates no device memory.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate: code whose device memory is all owned by another
 * framework's pool or held to a fixed budget, and latency-critical loops
 * that cannot afford cudaMalloc/cudaFree (which may synchronize the device).
 * It evaluates the same quantity with the same kernel as pwa_nll_grad_async
 * for one parameter set, but without a context: the caller passes every
 * input and output in device memory, and the kernel's scratch (per-CTA
 * partial sums, a completion ticket, status words; about 200 KB) lives in a
 * file-scope device array of the library, which every GPU that loads the
 * library holds until the process exits.
 *
 *   d_planes     structure-of-arrays amplitudes, float: plane 2a holds Re A_a,
 *                plane 2a+1 holds Im A_a, event i of plane p at
 *                d_planes[p * plane_pitch + i]; 16-byte aligned
 *   plane_pitch  floats per plane, >= n_events and a multiple of 4
 *   n_events     data events, 1 <= n_events <= 2^31 - 1024
 *   n_waves      1 <= n_waves <= 48
 *   d_amax       [n_waves] floats, d_amax[a] >= max_i |Re A_a(i)| + |Im A_a(i)|
 *                (the kernel sizes its exact splitting of the products from
 *                it; a value below the true maximum gives wrong results)
 *   d_M          [n_waves][n_waves] complex128, the normalisation matrix as
 *                returned by pwa_build_norm
 *   d_V          [n_waves] complex128
 *   d_nll        [1] double, receives the NLL (+inf on a non-positive
 *                intensity, NaN if a device-side wait timed out)
 *   d_grad       [n_waves] complex128, receives dNLL/dV* (may be NULL)
 *   d_status     [1] int or NULL: status bits are OR-ed into it (1: an
 *                intensity was not positive and finite, 2: a wait timed out)
 *   stream       cudaStream_t to run on (NULL: the legacy default stream)
 * The call is stream-ordered and returns after enqueueing. It works on the
 * current device. Its first call on a device does the set-up (looks up the
 * array's device address and sets the kernel's shared-memory limit), so make
 * that first call before any stream capture. Every call shares the one
 * array: calls whose kernels overlap on the GPU (other streams, other host
 * threads) race and corrupt each other's sums; order them on one stream.
 * Returns PWA_OK, PWA_EINVAL (null pointer, size or alignment out of range),
 * PWA_ENOTSUP (scratch too small for this GPU) or PWA_ECUDA. It calls no
 * cudaMalloc, cudaFree or allocating library routine. */
int pwa_nll_grad_noalloc(const float *d_planes, int64_t plane_pitch, int64_t n_events,
                         int n_waves, const float *d_amax, const double *d_M, const double *d_V,
                         double *d_nll, double *d_grad, int *d_status, void *stream);

/* Autotuner. Times the launch variants of the context's current form on its
 * loaded sample (a few evaluations of a fixed parameter set each, CUDA events
 * on the context's stream), and of the free-resonance kernel if resonance
 * samples are loaded; applies the fastest; records each choice in a JSON
 * cache file, one line per key (device name, SM count, form, n_waves, and
 * for the tensor-core form max_k and the precision), and applies a cached
 * choice instead of timing when the key is present. The variants: the
 * direct form's consumer groups per block (2 or 3 groups of four warps,
 * three from 40 waves on, where both fit); the tensor-core form's tile parameters for max_k sets per
 * call, the sets per launch (multiples of 64 up to the launch's tensor- and
 * shared-memory limit) and the X pipeline stages (2 up to what shared memory
 * takes); the free-resonance kernel's blocks per SM (1 to 3). The table
 * form has one launch shape (set by its shared-memory budget) and is
 * reported as such.
 *   cache_path  file to read and update (NULL: time every call, no file)
 *   choice      receives a one-line summary (may be NULL), choice_len bytes
 * Results of the evaluation calls do not depend on the choice beyond float
 * summation order. Errors: PWA_ESTATE (nothing loaded), PWA_ECUDA, PWA_EINVAL
 * (an unreadable or unwritable cache file). */
int pwa_autotune(pwa_ctx *ctx, const char *cache_path, char *choice, int choice_len);

/* Launch-shape autotuner of a model batch (the one-launch form; Sec. 2: many
 * trial models are fitted to one data set): times the batch's evaluation for
 * max_k sets with 4, 8, 16 or 32 work items per SM (16 without tuning) and
 * 2 up to the most X pipeline stages shared memory takes, applies the
 * fastest and records it
 * in the JSON cache (cache_path as for pwa_autotune; a cached key is applied
 * without timing). The key holds the device name, SM count, number of
 * models, total waves and events, max_k and the precision. Results do not
 * depend on the choice beyond float summation order. With
 * PWA_BATCH_MODE=graph (per-model launches) there is nothing to tune.
 * Errors: PWA_ESTATE (a model not loaded), PWA_ECUDA, PWA_EINVAL (cache). */
int pwa_batch_autotune(pwa_batch *b, const char *cache_path, char *choice, int choice_len);

/* Message describing the last error on ctx ("" if none); valid until the
 * next call on ctx. A NULL ctx gives the message of the last failed
 * pwa_create on this thread. */
const char *pwa_last_error(const pwa_ctx *ctx);

/* Host-only size query: bytes of the per-event table for n_events events of
 * n_waves waves (n_waves^2 floats per event: n_waves real diagonal entries
 * and n_waves(n_waves-1)/2 complex off-diagonal ones; Sec. 2 sizes the table
 * as about 1.5 GB per million events at 20 waves). Errors: PWA_EINVAL. */
int pwa_table_bytes(int n_waves, int64_t n_events, int64_t *bytes);

/* Library version as an integer MAJOR*10000 + MINOR*100 + PATCH. */
int pwa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PWA_H */
