/*
 * amp4d -- GPU hot path of the four-dimensional B0 -> J/psi K+ pi- amplitude fit
 * (Sur, Cristella, Di Florio, Mastrapasqua, "A GPU based multidimensional
 * amplitude analysis to search for tetraquark candidates").
 *
 * C ABI.  Plain pointers and sizes only; no exceptions cross it.  Every call
 * returns an amp4d_status (0 = AMP4D_OK, < 0 = error); amp4d_last_error()
 * returns a message for the last failure on a model.
 *
 * What is computed (Methodology section):
 *   A^R(m)      lineshape, Eq. 2 with the running width of Eq. 3 and ratio-form
 *               Blatt-Weisskopf barrier factors, or the LASS S-wave of Eq. 7-8;
 *   B_k,xi(e)   basis column k = (resonance R, helicity l) for muon helicity xi:
 *               K*  A^R(m_Kpi) d^J_{l0}(theta_K*) e^{i l phi} d^1_{l xi}(theta_psi)   (Eq. 4)
 *               Z   A^Z(m_psipi) d^J_{0l'}(theta_Z) e^{i l' phi~} d^1_{l' xi}(theta~_psi)
 *                   e^{i xi alpha}, with l' = +-1 tied by H_{-l'} = eta H_{l'}     (Eq. 10, 11)
 *   S(e)        sum_xi |sum_k c_k B_k,xi(e)|^2                         (Eq. 5, Eq. 9, Eq. 12)
 *   I           (V / N_mc) sum_n w_n S(x_n), the numerical normalisation over MC
 *               phase-space points (State-of-the-art section), w = p q for uniform points
 *   NLL         -2 sum_e [ ln S(e) + ln(p_e q_e) - ln I ]   (unbinned ML, Introduction)
 * where p is the K pi momentum in the B frame and q the K momentum in the K pi
 * frame; the PDF of an event is S p q / I.
 *
 * Event coordinates (Eq. 1 with cos theta_K* of Eq. 4):
 *   m    = m_Kpi in [m_lo, m_hi] (GeV), cK = cos theta_K*, cpsi = cos theta_J/psi,
 *   phi  = angle between the J/psi and K pi decay planes in [-pi, pi].
 * All event arrays are FP32 structure-of-arrays, one value per event.
 *
 * Parameter vector (host, double), length amp4d_num_params():
 *   [Re c_0, Im c_0, Re c_1, Im c_1, ..., Re c_{K-1}, Im c_{K-1},
 *    M_R, Gamma_R for every resonance with float_mg = 1, in resonance order].
 * Column order: resonances in the given order; a K* with J = 0 has one column
 * (l = 0), a K* with J >= 1 three (l = -1, 0, +1); a Z has the l' = 0 column when
 * eta = -P (-1)^J = +1, then the tied l' = +-1 column.
 *
 * Streams: every call takes a cudaStream_t passed as void* (NULL = legacy
 * default stream) and is ordered on it.  Calls that return host scalars
 * synchronise that stream before returning.  A model is not thread-safe: use
 * one model per host thread.  The library owns all its device buffers.
 */
#ifndef AMP4D_H
#define AMP4D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int amp4d_status;

#define AMP4D_OK 0
#define AMP4D_ERR_ARG (-1)     /* bad argument (null pointer, size, range)          */
#define AMP4D_ERR_CUDA (-2)    /* a CUDA runtime call failed; message kept          */
#define AMP4D_ERR_OOM (-3)     /* device or pinned-host allocation failed           */
#define AMP4D_ERR_INPUT (-4)   /* an event lies outside the box or is not finite   */
#define AMP4D_ERR_DOMAIN (-5)  /* S <= 0 at a data event, or I <= 0: NLL = +inf     */
#define AMP4D_ERR_TIMEOUT (-6) /* a bounded device wait expired                     */
#define AMP4D_ERR_STATE (-7)   /* call out of order (e.g. eval before set_events)   */

#define AMP4D_CHAIN_KSTAR 0 /* resonance decays to K pi     */
#define AMP4D_CHAIN_Z 1     /* resonance decays to J/psi pi */

#define AMP4D_PATH_PLAIN 0  /* recompute every amplitude per evaluation            */
#define AMP4D_PATH_CACHED 1 /* per-event basis cache + normalisation Gram matrix   */

#define AMP4D_MAX_RES 16

#define AMP4D_EVAL_NLL 0      /* amp4d_enqueue_eval: -2 ln L only          */
#define AMP4D_EVAL_NLL_GRAD 1 /* amp4d_enqueue_eval: -2 ln L and gradient  */

typedef struct {
    double mB, mpsi, mK, mpi; /* B0, J/psi, K+, pi- masses (GeV) */
} amp4d_particle_masses;

#define AMP4D_SHAPE_BW 0   /* Breit-Wigner with barrier factors, Eq. 2-3            */
#define AMP4D_SHAPE_LASS 1 /* LASS K pi S-wave, Eq. 7-8 (a J = 0 K* only)           */

/*
 * One resonance.  Zero-initialise the record: shape 0 is the Breit-Wigner.
 *
 * shape = AMP4D_SHAPE_LASS makes a J = 0 K* the LASS S-wave of Eq. 7-9, with
 * (M, G0) the K0*(1430) pole inside it:
 *   A(m) = m / (1/a + (b/2) q^2 - i q)                   [= (m/q) sin(thB) e^{i thB}]
 *        + R e^{2 i thB} (M^2 / q0) G0 / (M^2 - m^2 - i M Gamma(m)),
 *   cot(thB) = 1/(a q) + b q / 2,  Gamma(m) = G0 (q/q0) (M/m)  (Eq. 3 at L = 0),
 * q (q0) the K momentum in the K pi frame at m (at m = M).  A is the whole mass
 * dependence of the column: LB, LR and r are not used.  lass_a > 0, lass_b >= 0
 * (GeV^-1; Eq. 8 gives 1.95 and 1.76), lass_R >= 0 (1: the elastic form; Eq. 7
 * prints 2).  Its M and G0 cannot float (float_mg must be 0).
 */
typedef struct {
    int chain;    /* AMP4D_CHAIN_KSTAR or AMP4D_CHAIN_Z                          */
    int J, P;     /* spin and intrinsic parity (+1 / -1) of the resonance        */
    int LB, LR;   /* orbital angular momenta in the B0 and resonance decays (0..4) */
    double M, G0; /* pole mass and nominal width (GeV)                           */
    double r;     /* Blatt-Weisskopf radius (GeV^-1)                             */
    int float_mg; /* 1: M and G0 are fit parameters (appended to the vector)     */
    int shape;    /* AMP4D_SHAPE_BW or AMP4D_SHAPE_LASS                          */
    double lass_a, lass_b, lass_R; /* AMP4D_SHAPE_LASS constants (see above)     */
} amp4d_resonance;

typedef struct amp4d_model amp4d_model;

/* Training and grid settings of the learned normalisation proposal. */
typedef struct {
    int nb[4];      /* grid cells per dimension of x = (m, cK, cpsi, phi) mapped to [-1, 1]^4 */
    double alpha;   /* weight of the uniform density in the defensive mixture, (0, 1]       */
    int64_t steps;  /* Adam steps                                                          */
    int batch;      /* data rows and uniform rows per step                                 */
    double lr;      /* Adam learning rate (beta1 0.9, beta2 0.999, eps 1e-8)               */
} amp4d_mlp_cfg;

/*
 * Create a model from a resonance list (Eq. 2-5, 10-12).  n_res in
 * [1, AMP4D_MAX_RES], at most 2 Z resonances, J <= 4, LB, LR <= 4.  The box is
 * m_Kpi in [m_lo, m_hi] x cK x cpsi in [-1, 1]^2 x phi in [-pi, pi].  path
 * selects AMP4D_PATH_PLAIN or AMP4D_PATH_CACHED.  *out receives the model; it
 * uses the current CUDA device.  Errors: ARG, CUDA, OOM.
 */
amp4d_status amp4d_model_create(const amp4d_particle_masses *masses, const amp4d_resonance *res,
                                int n_res, double m_lo, double m_hi, int path, amp4d_model **out);

/* Free a model and every device buffer it owns.  NULL is accepted. */
amp4d_status amp4d_model_destroy(amp4d_model *model);

/* Message for the last failure on this model (static storage owned by the model). */
const char *amp4d_last_error(const amp4d_model *model);

/* Number of basis columns K and of parameters 2K + 2 (#floated resonances). */
int amp4d_num_columns(const amp4d_model *model);
int amp4d_num_params(const amp4d_model *model);

/*
 * Data events.  m, cK, cpsi, phi: n FP32 values each, host or device memory
 * (any pointer CUDA can address); the library copies them and the caller keeps
 * ownership.  Every event must lie in the box and be finite, else
 * AMP4D_ERR_INPUT (amp4d_last_error names the first bad index).  Per-event
 * parameter-independent kinematics (p, q; the Z-chain angles of Eq. 10) are
 * computed once here in FP64 and stored as FP32.  n >= 1.
 */
amp4d_status amp4d_set_events(amp4d_model *model, const float *m, const float *cK,
                              const float *cpsi, const float *phi, int64_t n, void *stream);

/*
 * Normalisation points for the MC integral I (State-of-the-art section: the
 * PDF is normalised numerically over phase-space points).  Same layout and
 * ownership as amp4d_set_events.  w: n FP32 weights or NULL, in which case
 * w = p q (uniform points).  volume: V in I = (V / n) sum w S (the box volume for
 * uniform points, 1 for importance-sampled points whose w = p q / density).
 */
amp4d_status amp4d_set_norm_points(amp4d_model *model, const float *m, const float *cK,
                                   const float *cpsi, const float *phi, const float *w,
                                   int64_t n, double volume, void *stream);

/*
 * Binned 2D template (efficiency and background of Eq. 14).  h: nx * ny FP32
 * contents, finite and >= 0, h[iy * nx + ix] (host or device memory; copied by
 * the setters, the caller keeps ownership; ARG otherwise).  The content at (x, y) is that of the bin
 * ix = floor((x - x_lo) * nx / (x_hi - x_lo)), iy likewise, evaluated in FP64 in
 * that order; the upper edge belongs to the last bin and the template is 0
 * outside [x_lo, x_hi] x [y_lo, y_hi].
 */
typedef struct {
    const float *h;
    int nx, ny;                     /* >= 1                     */
    double x_lo, x_hi, y_lo, y_hi;  /* x_hi > x_lo, y_hi > y_lo */
} amp4d_hist2d;

/*
 * Relative signal efficiency of Eq. 14, eps = mass(m_Kpi^2, m_psipi^2) *
 * angle(cos theta_psi, phi): a template in the two mass variables (GeV^2; m_psipi
 * computed in FP64 from m_Kpi and cos theta_K*) times one in the two angles.
 * From then on the signal is normalised with efficiency-weighted points,
 * I_eps = (V / n) sum w eps S (also the Gram matrix), and the likelihood of an
 * event is p q eps S / I_eps (without a background).  Applies to the sets
 * loaded and to those loaded later.  mass = angle = NULL removes it.
 * Synchronous.  Errors: ARG, CUDA, OOM.
 */
amp4d_status amp4d_set_efficiency(amp4d_model *model, const amp4d_hist2d *mass,
                                  const amp4d_hist2d *angle, void *stream);

/*
 * Background of Eq. 14 with the fixed signal purity P in [0, 1]: the PDF of an
 * event becomes
 *   f = p q [ P eps S / I_eps + (1 - P) hb / B ],   hb = mass(m_Kpi^2, m_psipi^2) *
 *   angle(cos theta_psi, phi),   B = (V / n) sum_n w_n hb_n,
 * hb a density in the Dalitz variables and the angles (so its density in the
 * event coordinates carries p q), B over the normalisation points with their
 * weights as loaded.  With a background (P < 1) each evaluation computes I_eps
 * before the data pass (the Gram quadratic form, or the point sum first).  The
 * NLL is -2 sum ln f; in the evaluation outputs "sum ln S" becomes
 * sum ln(f / (p q)) and I is I_eps.  Shard partials are not available with a
 * background (STATE).  mass = angle = NULL removes it.
 * Synchronous.  Errors: ARG, CUDA, OOM.
 */
amp4d_status amp4d_set_background(amp4d_model *model, const amp4d_hist2d *mass,
                                  const amp4d_hist2d *angle, double purity, void *stream);

/*
 * Flavour of the data events (text after Eq. 12: the charge-conjugate decay,
 * identified by the K charge, differs only in the sign of phi, and a fraction
 * of the events may be mis-tagged).  tag: n_events FP32 values, +1 (B0) or -1
 * (B0bar), host or device memory, copied; NULL makes every event B0.  The
 * signal density of an event tagged t is
 *   (1 - w) S(m, cK, cpsi, t phi) + w S(m, cK, cpsi, -t phi),   w = mistag in [0, 0.5],
 * S at -phi being S with sin phi, sin phi~ and sin alpha negated (the mirror
 * through the K pi decay plane).  The box is symmetric in phi and p q does not
 * depend on it, so every tag shares the normalisation I (or I_eps): with tags
 * or a mistag an efficiency must be even in phi (its angular template's phi range
 * symmetric about 0 and its contents mirror-symmetric), else STATE.  Templates
 * are read at the observed phi.  amp4d_eval_density returns the tagged density.
 * amp4d_set_events resets every tag to +1; the mistag stays.  Synchronous.
 * Errors: ARG (a tag not +-1, w out of range), STATE (no events, an efficiency
 * not even in phi), CUDA, OOM.
 */
amp4d_status amp4d_set_flavour(amp4d_model *model, const float *tag, double mistag, void *stream);

/*
 * -2 ln L at params (host, amp4d_num_params doubles); *nll is host memory.
 * On AMP4D_ERR_DOMAIN *nll = +INFINITY (the minimiser treats it as a bad step).
 *
 * The synchronous evaluations (amp4d_eval_nll, amp4d_eval_nll_grad,
 * amp4d_eval_terms, amp4d_eval_partials) copy params in, enqueue the evaluation
 * on `stream`, copy the result out and synchronise the stream.  From the second
 * call of one kind at an unchanged model state the evaluation runs as a CUDA graph
 * (captured once on a private stream of the model, then launched on `stream`)
 * whose kernels read the parameters from and write the result to the model's
 * pinned host buffers directly, with the same results bit for bit.  Every other call that takes the model may
 * change what an evaluation enqueues and makes the next call capture afresh.
 * The first call may build the constant table, the basis caches or the Gram
 * matrix, and so takes longer.
 */
amp4d_status amp4d_eval_nll(amp4d_model *model, const double *params, double *nll, void *stream);

/*
 * -2 ln L and its gradient with respect to every parameter (host arrays).
 * The gradient is the adjoint of the per-event density (couplings: dS/dRe c_k =
 * 2 Re z_k, dS/dIm c_k = -2 Im z_k, z_k = sum_xi conj(a_xi) B_k,xi; masses and
 * widths: closed-form derivatives of Eq. 2-3), summed over events and points.
 */
amp4d_status amp4d_eval_nll_grad(amp4d_model *model, const double *params, double *nll,
                                 double *grad, void *stream);

/*
 * The terms of the NLL: out[0] = sum_e ln S_e, out[1] = sum_e ln(p_e q_e),
 * out[2] = I, out[3] = number of data events (host, 4 doubles).  With an
 * efficiency (Eq. 14) out[1] also holds sum_e ln eps_e and I is I_eps; with a
 * background out[0] is sum_e ln(f_e / (p_e q_e)) and NLL = -2 (out[0] + out[1]).
 */
amp4d_status amp4d_eval_terms(amp4d_model *model, const double *params, double *out,
                              void *stream);

/*
 * Per-event signal density S(e) (Eq. 5 / Eq. 12) for the data events:
 * S_out is DEVICE memory of n_events FP32 values, owned by the caller.
 * which = 0: data events; which = 1: normalisation points.
 */
amp4d_status amp4d_eval_density(amp4d_model *model, const double *params, int which,
                                float *S_out, void *stream);

/*
 * Normalised PDF of every data event, P(e) = S(e) p(e) q(e) / I (Eq. 5 with
 * the phase-space density p q; I over the current normalisation points), for
 * parity checks.  pdf_out is DEVICE memory of n_events FP32 values owned by
 * the caller.  Synchronous.  Errors: ARG, STATE (no events or points), DOMAIN
 * (I <= 0), CUDA.
 */
amp4d_status amp4d_eval_pdf(amp4d_model *model, const double *params, float *pdf_out,
                            void *stream);

/*
 * Enqueue one evaluation on the stream without synchronising (same arithmetic
 * as amp4d_eval_nll / amp4d_eval_nll_grad).  params: DEVICE memory,
 * amp4d_num_params doubles.  out: DEVICE memory of 6 + amp4d_num_params doubles
 * receiving [0] NLL (+inf on a domain error), [1] sum ln S, [2] sum ln(p q),
 * [3] I, [4] N, [5] status bits (1: S <= 0 / I <= 0, 2: invalid parameters),
 * [6 ..] the gradient (what = AMP4D_EVAL_NLL_GRAD).  With Eq. 14 templates [1]
 * to [3] change as described at amp4d_eval_terms.  Both buffers are owned by
 * the caller and must stay valid until the stream has executed the work.
 * Evaluations of one model must not overlap in time: they share the model's
 * partial-sum buffers.  Errors: ARG, STATE (no events), CUDA.
 */
amp4d_status amp4d_enqueue_eval(amp4d_model *model, int what, const double *params, double *out,
                                void *stream);

/*
 * Shard partials.  The unbinned likelihood (Introduction) is a product over
 * data events and the normalisation I of Eq. 5 is estimated as a sum over points, so
 * when the events and the points of one fit are split into shards (one model
 * per shard, e.g. one per GPU) an evaluation needs only these sums per shard:
 *   out[0] sum_e ln S_e, [1] sum_e ln(p_e q_e), [2] N (data events),
 *   [3] T = V sum_n w_n S_n (V = the volume given to amp4d_set_norm_points;
 *       on the Gram path T = V (u^T G u + v^T G v)), [4] M (points),
 *   [5] status bits (1: S <= 0 at a data event, 2: invalid parameters),
 *   [6 .. 6+P) d(sum ln S)/dtheta, [6+P .. 6+2P) dT/dtheta  (what = NLL_GRAD),
 * P = amp4d_num_params.  No logarithm of I is taken per shard.  With an
 * efficiency (Eq. 14) [1] also holds sum ln eps and T uses the efficiency-
 * weighted points; with a background the call returns STATE (the data sum needs
 * the union's I first).
 * amp4d_eval_partials: params and out are HOST memory (6 or 6 + 2P doubles),
 * synchronous.  amp4d_enqueue_partials: params and out are DEVICE memory owned
 * by the caller, enqueued on the stream without synchronising, with the same
 * rule as amp4d_enqueue_eval about overlapping evaluations of one model.
 * Errors: ARG (bad what, null or invalid parameters), STATE (no events or no
 * points in this shard), CUDA.
 */
amp4d_status amp4d_eval_partials(amp4d_model *model, int what, const double *params, double *out,
                                 void *stream);
amp4d_status amp4d_enqueue_partials(amp4d_model *model, int what, const double *params,
                                    double *out, void *stream);

/*
 * Combine n_shards partial blocks (HOST memory, contiguous, in shard order,
 * each 6 doubles, or 6 + 2 n_param for what = AMP4D_EVAL_NLL_GRAD) into the
 * evaluation of the union (host code only, no GPU call):
 *   I = sum T / sum M,  NLL = -2 [sum ln S + sum ln(pq) - N ln I],
 *   dNLL/dtheta = -2 [sum d ln S - N sum dT / sum T].
 * out (HOST) receives the amp4d_enqueue_eval layout: [0] NLL (+inf on a domain
 * error), [1] sum ln S, [2] sum ln(pq), [3] I, [4] N, [5] status bits, [6 ..]
 * the gradient.  Sums run over the shards in the order given with Neumaier
 * compensation, so the result depends on that order only through rounding and
 * is identical on every caller that passes the same blocks.
 * Errors: ARG (bad arguments, a negative count, a shard with status bit 2),
 * STATE (no points in any shard), DOMAIN (status bit 1, I <= 0); message in
 * amp4d_shard_last_error (per calling thread).
 */
amp4d_status amp4d_combine_partials(const double *parts, int n_shards, int n_param, int what,
                                    double *out);
const char *amp4d_shard_last_error(void);

/*
 * Normalisation Gram matrix G = sum_n w_n sum_xi x x^T of the real 2K-vectors
 * x = (Re B_0, Im B_0, Re B_1, ...) over the normalisation points (State-of-
 * the-art section: numerical normalisation; Eq. 5, 12 for B), so that
 * I = (V / N_mc) (u^T G u + v^T G v) with u = (Re c_0, -Im c_0, ...),
 * v = (Im c_0, Re c_0, ...).  Built in two passes: the basis of every point is
 * evaluated once into an FP32 basis matrix (with its column maxima), then the
 * tensor cores (tcgen05) accumulate exact BF16 digit slices of its fixed-point
 * columns in INT64.  The basis matrix is device scratch owned by the model:
 * 16 K bytes per normalisation point (rounded up to 512 points), allocated by
 * the first build and kept for rebuilds at new masses until the model is
 * destroyed.  amp4d_build_gram builds G for the masses and widths in params
 * (host; the couplings are not used) and synchronises; K <= 32 columns.  Models created
 * with AMP4D_PATH_CACHED and no floated masses/widths build it on their first
 * evaluation (which then synchronises) and use it for I and dI/dc thereafter;
 * amp4d_set_norm_points discards it.  amp4d_get_gram copies G (host, 2K x 2K,
 * row-major) back.  Errors: STATE (no points / no Gram), ARG (K > 32),
 * TIMEOUT (a bounded device wait expired), CUDA.
 */
amp4d_status amp4d_build_gram(amp4d_model *model, const double *params, void *stream);
amp4d_status amp4d_get_gram(amp4d_model *model, double *G, void *stream);

/*
 * Fit fractions (Eq. 13): FF_j = I_j / I, where I_j is the normalisation integral
 * of the PDF with every helicity coupling outside resonance j set to zero and I
 * the full one, both over the current normalisation points (so with the phase-
 * space density p q).  The paper writes |S|^2 in the integrands although S
 * (Eq. 12) is already a squared modulus; S is read.  The fractions need not sum
 * to one (interference).  Computed from the normalisation Gram matrix, built at
 * params when a mass or width floats or none is valid yet (which synchronises).
 * params: host, amp4d_num_params doubles; ff: host, one double per resonance in
 * the order given to amp4d_model_create.  With Eq. 14 templates the fractions
 * are still those of S: the Gram is built over the points' weights as loaded
 * (without the efficiency), and the efficiency-weighted normalisation is rebuilt
 * on the next evaluation.  Errors: ARG, STATE (no points), DOMAIN (I <= 0),
 * TIMEOUT, CUDA.
 */
amp4d_status amp4d_fit_fractions(amp4d_model *model, const double *params, double *ff, void *stream);

/*
 * Self-test of the tensor-core Gram accumulation on this GPU: X holds n points x
 * 2 rows x 64 columns of fixed-point values (int32, |X| <= 2^30, host or device
 * memory, caller-owned).  G_int (host, 64 x 64 int64) receives the kernel's
 * integer Gram: per 512-point chunk, the digit products P_ab of the base-256
 * digits d1..d4 of X (d1 = round(X / 2^24), ...) combined as
 * sum_ab 2^(8 (5 - a - b)) P_ab, the a = b = 4 term dropped and the 2^-8 and
 * 2^-16 terms rounded half up, summed over chunks.  A caller can reproduce it
 * exactly in integer arithmetic.  Uses the current device; synchronises.
 */
amp4d_status amp4d_gram_selftest(const int32_t *X, int64_t n, long long *G_int, void *stream);

/*
 * Pseudo-data from the model at params (Fit validation section: events generated
 * by MC from the fit model): accept-reject over the uniform box with density
 * S p q.  Candidate i uses Philox4x32-10 (counter (i, 0, i >> 32, 0), key seed) for
 * its coordinates and counter (i, 1, ...) for the acceptance uniform; f_max is
 * 1.5 x the largest S p q of 2^20 scan candidates (stream 2) and doubles, with a
 * restart, if a candidate exceeds it.  Accepted events keep candidate order.
 * m, cK, cpsi, phi: DEVICE outputs of n floats (caller-owned).  Synchronises.
 * With Eq. 14 templates the density is the model's PDF instead:
 * p q [P eps S / I_eps + (1 - P) hb / B] with a background (I_eps and B over the
 * normalisation points, which must be set), p q eps S with an efficiency alone.
 * Generated events are B0 (untagged).
 * Errors: ARG, STATE (a background without normalisation points), DOMAIN
 * (S p q vanishes or the candidate budget is exhausted), CUDA, OOM.
 */
amp4d_status amp4d_generate(amp4d_model *model, const double *params, uint64_t seed, int64_t n,
                            float *m, float *cK, float *cpsi, float *phi, void *stream);

/*
 * Learned importance-sampling proposal for the normalisation integral: an MLP
 * 4 -> 64 -> 64 -> 1 (tanh, softplus output g >= 0; BF16 weights with an FP32
 * master copy, FP32 accumulation) over x in [-1, 1]^4 (x0 = 2 (m - m_lo)/(m_hi -
 * m_lo) - 1, x1 = cK, x2 = cpsi, x3 = phi / pi), trained by Adam on the KL
 * objective -mean_data ln g + ln(16 mean_uniform g) with data rows drawn from
 * the given events (DEVICE SoA, n each; e.g. from amp4d_generate at the fit's
 * start point) and uniform rows, Philox-keyed by seed.  Then g at the centres of
 * the cfg->nb grid and the FP64 CDF of P_c = alpha / ncell + (1 - alpha) g_c / sum g
 * are kept in the model.  *loss (host, nullable) receives the last batch loss.
 * amp4d_proposal_sample draws n points (DEVICE outputs) cell by CDF, uniformly in
 * the cell, with weights w = p q / q(Phi), so that I = (1/n) sum w S: pass them
 * to amp4d_set_norm_points with volume 1.  Both synchronise.
 */
amp4d_status amp4d_proposal_train(amp4d_model *model, const float *m, const float *cK,
                                  const float *cpsi, const float *phi, int64_t n,
                                  const amp4d_mlp_cfg *cfg, uint64_t seed, double *loss, void *stream);
/*
 * Proposal aimed at the whole normalisation Gram matrix rather than at S: the
 * target density is sum_k |B_k|^2 p q, whose importance weights control the
 * error of every Gram element G_jk = int B_j* B_k p q and so of I(c) = c^H G c at
 * any couplings (the quantity the fit reads, Eq. 5 with the phase-space
 * density).  Builds G for the masses and widths in params (host; its couplings
 * are not used) over the current normalisation points, splits n events over
 * the columns in proportion to G_kk (at least 1 each), draws column k's share
 * from the model with the single unit coupling c_k = 1 (amp4d_generate, seed
 * gen_seed + k) and trains the proposal on their union exactly as
 * amp4d_proposal_train (cfg, seed, *loss).  Synchronises.  Errors: STATE (no
 * normalisation points), DOMAIN (a Gram diagonal element not >= 0), ARG, CUDA,
 * OOM, TIMEOUT.
 */
amp4d_status amp4d_proposal_train_gram(amp4d_model *model, const double *params, int64_t n,
                                       const amp4d_mlp_cfg *cfg, uint64_t seed, uint64_t gen_seed,
                                       double *loss, void *stream);
amp4d_status amp4d_proposal_sample(amp4d_model *model, int64_t n, uint64_t seed, float *m, float *cK,
                                   float *cpsi, float *phi, float *w, void *stream);

/*
 * The proposal pieces on explicit inputs (model-free; for validation):
 * amp4d_mlp_forward: g(x) for n rows x (DEVICE n x 4) with the FP32 weights theta
 *   (4545 floats, host or device; rounded to BF16 inside) into g (DEVICE, n).
 * amp4d_mlp_loss_grad: the KL objective on data rows xd (DEVICE nd x 4) and
 *   uniform rows xu (DEVICE nu x 4): out (host, 4546 doubles) = gradient, loss.
 * amp4d_grid_sample: the sampler on given cell values gcell (host or device,
 *   nb[0] nb[1] nb[2] nb[3] floats); outputs DEVICE, cell (DEVICE int64, nullable)
 *   receives the sampled cell index.  Philox streams as amp4d_proposal_sample.
 * All synchronise.
 */
amp4d_status amp4d_mlp_forward(const float *theta, const float *x, int64_t n, float *g, void *stream);
amp4d_status amp4d_mlp_loss_grad(const float *theta, const float *xd, int64_t nd, const float *xu,
                                 int64_t nu, double *out, void *stream);
amp4d_status amp4d_grid_sample(const float *gcell, const int *nb, double alpha, uint64_t seed,
                               int64_t n, double m_lo, double m_hi, const amp4d_particle_masses *masses,
                               float *m, float *cK, float *cpsi, float *phi, float *w, int64_t *cell,
                               void *stream);

/*
 * Allocation-free variant of amp4d_mlp_loss_grad, for callers that may not
 * call cudaMalloc: code that runs while another component's pool owns the
 * device memory budget, or code that must avoid the device-wide
 * synchronisation an allocation or free can cause.  The paper has no
 * counterpart; this is an interface of this library only.
 *
 * theta (4545 FP32 weights), xd (nd x 4 data rows) and xu (nu x 4 uniform rows)
 * are DEVICE memory; out is DEVICE memory of 4546 doubles receiving the
 * gradient of the KL objective and then its value (same arithmetic as
 * amp4d_mlp_loss_grad).  All are caller-owned.  The call is stream-ordered and
 * does not synchronise; it allocates nothing: its scratch (about 2.3 MB) is a
 * file-scope device array that every GPU which loads the library holds until
 * the process exits.  nd and nu must not exceed AMP4D_NOALLOC_MAX_ROWS, else
 * AMP4D_ERR_ARG.  Each call looks up that array's device address in the
 * current context (cudaGetSymbolAddress); the first call on a device may load
 * the library's device code there, so make it before any stream capture.  Every call uses the same array, so calls whose work
 * overlaps on the GPU (other streams, other host threads) race: order them on
 * one stream.  amp4d_noalloc_last_error describes the last failure.
 */
#define AMP4D_NOALLOC_MAX_ROWS 4096
amp4d_status amp4d_mlp_loss_grad_noalloc(const float *theta, const float *xd, int64_t nd,
                                         const float *xu, int64_t nu, double *out, void *stream);
const char *amp4d_noalloc_last_error(void);

/*
 * Device timing of evaluations (CUDA events around each phase, on the
 * evaluation's stream).  amp4d_profile_read waits for the recorded work and
 * returns, then clears, the summed milliseconds and counts of the phases
 * [0] parameter table, [1] data-event kernel, [2] normalisation kernel,
 * [3] reductions and NLL assembly (host arrays of 4).
 */
amp4d_status amp4d_profile_enable(amp4d_model *model, int on);
amp4d_status amp4d_profile_read(amp4d_model *model, double *ms, int64_t *count);

#ifdef __cplusplus
}
#endif

#endif /* AMP4D_H */
