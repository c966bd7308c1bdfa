/*
 * FP64 CPU oracle for the B0 -> J/psi K+ pi- four-dimensional amplitude fit.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed CPU
 * baseline of the benchmark load this library.  It shares no code with the GPU
 * path: it is the plain definition of what that path computes, evaluated in
 * double precision on the FP32-rounded inputs, one event at a time.
 *
 * What it follows (section / equation of Sur et al., "A GPU based
 * multidimensional amplitude analysis to search for tetraquark candidates"):
 *   - observables Phi = (m_Kpi, cos theta_K*, cos theta_J/psi, phi)      Eq. 1, Eq. 4
 *   - lineshape with barrier factors and running width                 Eq. 2, Eq. 3
 *   - K* helicity amplitude d^J_{l0}(theta_K*) e^{i l phi} d^1_{l xi}   Eq. 4
 *   - coherent sum, squared per muon helicity xi                      Eq. 5, Eq. 12
 *   - LASS K pi S-wave: effective-range term + K0*(1430) Breit-Wigner   Eq. 7, Eq. 8, Eq. 9
 *   - Z -> J/psi pi amplitude with Z-frame angles and alignment alpha  Eq. 10
 *   - efficiency x signal + background with a fixed purity             Eq. 14
 *   - B0bar events (phi -> -phi) and flavour mistag                    Eq. 12 text
 *   - parity relation of the Z helicity couplings                      Eq. 11
 *   - unbinned -2 ln L with a numerical (MC) normalisation             Introduction,
 *                                                                     State of the art
 *   - accept-reject pseudo-data generation                            Fit validation
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - Blatt-Weisskopf factors: ratio form F_L(z,z0) = sqrt(P_L(z0)/P_L(z)),
 *     P_L(x^2) = x^(2L+2) |h_L(x)|^2 (spherical Hankel), z = (r p)^2.
 *   - phase-space density p*q (K* momentum in the B frame times K momentum in
 *     the K pi frame); the PDF is S p q / I with I = int S p q dPhi.
 *   - two-body momenta use the Kallen function clamped at zero.
 *   - Wigner d by the general (factorial-sum) formula with the Condon-Shortley
 *     phase, d^1_{10} = -sin(b)/sqrt(2).
 *   - frames: the K pi system flies along +z in the B frame, the K lies in the
 *     x-z plane with p_x > 0; the J/psi helicity axis z1 is the J/psi flight
 *     direction (-z); mu+ in the J/psi frame is
 *     (sin t cos phi, -sin t sin phi, -cos t).
 *   - Z chain: cos theta_Z = cos(K, pi) in the Z frame; the J/psi axis z2 is
 *     minus the pi direction in the J/psi frame; phi~ is the azimuth of mu+
 *     about z2 from the (z2, K) half-plane; alpha is the signed angle about mu+
 *     from the (mu+, z1) plane to the (mu+, z2) plane.
 *
 *   - LASS (Eq. 7): the amplitude is the whole mass dependence of its J = 0
 *     column (no barrier factors); the resonant term carries a factor R, 1 for
 *     the elastic (unitary) form and 2 as printed; the running width is Eq. 3
 *     at L = 0.
 *
 *   - Eq. 14 templates: the efficiency and the background are each a product
 *     of a binned template in the two mass variables (m^2_Kpi, m^2_psipi) and
 *     one in the two angles (cos theta_psi, phi), read at the bin holding the
 *     point (bin i covers [lo + i d, lo + (i+1) d), the upper edge in the last
 *     bin, 0 outside the range).  The background template is a density in the
 *     Dalitz variables and the angles, so its density in (m, cK, cpsi, phi)
 *     carries the Jacobian p q like the signal's; it is normalised over the
 *     normalisation points with their weights.  S is normalised with the
 *     efficiency-weighted points.  The purity P is fixed.
 *
 *   - Flavour: the signal density of a B0bar-tagged event is S at -phi (the
 *     charge-conjugate mode differs only in the sign of phi); with a mistag
 *     fraction w an event tagged t has density (1 - w) S(t phi) + w S(-t phi).
 *     The box is symmetric in phi and p q does not depend on phi, so with a
 *     phi-even efficiency every tag has the normalisation I_eps.
 *
 * Parameters of a model: [Re c_k, Im c_k] per basis column k, then [M_R, G_R]
 * for every resonance flagged as floating, in resonance order.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define OR_MAXR 32
#define OR_MAXC (3 * OR_MAXR)
#define OR_BLOCK 2048 /* events per deterministic reduction block */

enum { CH_KSTAR = 0, CH_Z = 1 };
enum { SHAPE_BW = 0, SHAPE_LASS = 1 };

typedef struct {
    double mB, mpsi, mK, mpi, m_lo, m_hi;
    int n_res, n_col, n_float;
    int chain[OR_MAXR], J[OR_MAXR], P[OR_MAXR], LB[OR_MAXR], LR[OR_MAXR], flt[OR_MAXR];
    int float_pos[OR_MAXR]; /* index among floated resonances, or -1 */
    double M[OR_MAXR], G0[OR_MAXR], r[OR_MAXR];
    int shape[OR_MAXR];                                   /* SHAPE_BW or SHAPE_LASS */
    /* Eq. 14 templates: [0] efficiency x (m^2_Kpi, m^2_psipi), [1] efficiency x
     * (cos theta_psi, phi), [2] background x masses, [3] background x angles. */
    struct { double *h; int nx, ny; double xlo, xhi, ylo, yhi; } tpl[4];
    int has_eff, has_bkg;
    double purity;
    double mistag;   /* flavour mistag fraction w */
    double lass_a[OR_MAXR], lass_b[OR_MAXR], lass_R[OR_MAXR]; /* Eq. 7-8 constants */
    int col_res[OR_MAXC], col_lam[OR_MAXC];
    int has_z;
} or_model;

/* ------------------------------------------------------------------ */
/* Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).              */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

/* ------------------------------------------------------------------ */
/* Forward-mode dual numbers (one direction) for the mass/width         */
/* derivatives of the lineshape.                                         */
/* ------------------------------------------------------------------ */
typedef struct { double v, d; } dual;
typedef struct { cplx v, d; } cdual;

static dual dk(double v) { dual r = {v, 0.0}; return r; }
static dual dadd(dual a, dual b) { dual r = {a.v + b.v, a.d + b.d}; return r; }
static dual dsub(dual a, dual b) { dual r = {a.v - b.v, a.d - b.d}; return r; }
static dual dmul(dual a, dual b) { dual r = {a.v * b.v, a.d * b.v + a.v * b.d}; return r; }
static dual ddiv(dual a, dual b) { dual r = {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; return r; }
static dual dscale(dual a, double s) { dual r = {a.v * s, a.d * s}; return r; }
static dual dsqrt(dual a)
{
    double s = sqrt(a.v);
    dual r = {s, s > 0.0 ? a.d / (2.0 * s) : 0.0};
    return r;
}
static dual dpowi(dual a, int n)
{
    dual r = dk(1.0);
    for (int i = 0; i < n; ++i) r = dmul(r, a);
    return r;
}
static cdual cdiv(cdual a, cdual b)
{
    cdual r;
    r.v = a.v / b.v;
    r.d = (a.d * b.v - a.v * b.d) / (b.v * b.v);
    return r;
}

/* Kallen triangle function lambda(a, b, c). */
static dual kallen(dual a, dual b, dual c)
{
    dual s = dadd(dadd(dmul(a, a), dmul(b, b)), dmul(c, c));
    dual t = dadd(dadd(dmul(a, b), dmul(a, c)), dmul(b, c));
    return dsub(s, dscale(t, 2.0));
}

/* Momentum of either daughter (masses m1, m2) in the rest frame of a parent of
 * mass Mp; zero where the decay is closed. */
static dual breakup(dual Mp, dual m1, dual m2)
{
    dual l = kallen(dmul(Mp, Mp), dmul(m1, m1), dmul(m2, m2));
    if (l.v <= 0.0) return dk(0.0);
    return ddiv(dsqrt(l), dscale(Mp, 2.0));
}

double or_breakup(double Mp, double m1, double m2) { return breakup(dk(Mp), dk(m1), dk(m2)).v; }

/* Blatt-Weisskopf barrier polynomial P_L(z) = x^(2L+2) |h_L(x)|^2, z = x^2. */
static dual bw_poly(int L, dual z)
{
    dual z2 = dmul(z, z), z3 = dmul(z2, z), z4 = dmul(z3, z);
    switch (L) {
    case 0: return dk(1.0);
    case 1: return dadd(dk(1.0), z);
    case 2: return dadd(dadd(z2, dscale(z, 3.0)), dk(9.0));
    case 3: return dadd(dadd(dadd(z3, dscale(z2, 6.0)), dscale(z, 45.0)), dk(225.0));
    case 4:
        return dadd(dadd(dadd(dadd(z4, dscale(z3, 10.0)), dscale(z2, 135.0)), dscale(z, 1575.0)),
                    dk(11025.0));
    default: return dk(NAN);
    }
}

double or_bw_poly(int L, double z) { return bw_poly(L, dk(z)).v; }

/* Ratio-form barrier factor F_L = sqrt(P_L(z0) / P_L(z)). */
static dual bw_factor(int L, dual z, dual z0) { return dsqrt(ddiv(bw_poly(L, z0), bw_poly(L, z))); }

/* Masses of the resonance's daughters and of the B0's other daughter. */
static void chain_masses(const or_model *mo, int R, double *md1, double *md2, double *mspec)
{
    if (mo->chain[R] == CH_KSTAR) {
        *md1 = mo->mK; *md2 = mo->mpi; *mspec = mo->mpsi;
    } else {
        *md1 = mo->mpsi; *md2 = mo->mpi; *mspec = mo->mK;
    }
}

/*
 * Eq. 2 with the running width of Eq. 3, as a dual number in (M, G0):
 *   A(m) = F_B (p/m_B)^LB F_R (q/m)^LR / (M^2 - m^2 - i M Gamma(m)),
 *   Gamma(m) = G0 (q/q0)^(2 LR + 1) (M/m) F_R^2,
 * where p (q) is the resonance momentum in the B frame (the daughter momentum in
 * the resonance frame) at the running mass m, and p0, q0 the same at m = M.
 */
/*
 * LASS K pi S-wave of Eq. 7 with the effective-range phase of Eq. 8, as a dual
 * number in the K0*(1430) pole parameters (M, G0):
 *   A = (m/q) sin(thB) e^{i thB}
 *       + R e^{2 i thB} (M^2 / q0) G0 / (M^2 - m^2 - i M Gamma(m)),
 *   cot(thB) = 1 / (a q) + b q / 2,   Gamma(m) = G0 (q / q0) (M / m)  (Eq. 3, L = 0),
 * q (q0) the K momentum in the K pi frame at m (at m = M).  At q = 0 the first
 * term takes its limit m a (sin thB / q -> a) and e^{2 i thB} -> 1.
 */
static cdual lass_lineshape(const or_model *mo, int R, double mrun, dual M, dual G0)
{
    const double a = mo->lass_a[R], b = mo->lass_b[R];
    const double q = breakup(dk(mrun), dk(mo->mK), dk(mo->mpi)).v;
    cplx nonres, e2;
    if (q > 0.0) {
        const double cot_b = 1.0 / (a * q) + 0.5 * b * q;
        const double th = atan2(1.0, cot_b); /* sin(thB) > 0: thB in (0, pi) */
        nonres = (mrun / q) * sin(th) * cexp(I * th);
        e2 = cexp(2.0 * I * th);
    } else {
        nonres = mrun * a;
        e2 = 1.0;
    }
    dual q0 = breakup(M, dk(mo->mK), dk(mo->mpi));
    dual width = dmul(dmul(G0, ddiv(dk(q), q0)), dscale(M, 1.0 / mrun));
    dual num = dscale(ddiv(dmul(dmul(M, M), G0), q0), mo->lass_R[R]);
    dual re = dsub(dmul(M, M), dk(mrun * mrun));
    dual im = dscale(dmul(M, width), -1.0);
    cdual n = {e2 * num.v, e2 * num.d};
    cdual den = {re.v + I * im.v, re.d + I * im.d};
    cdual res = cdiv(n, den);
    res.v += nonres;
    return res;
}

static cdual lineshape(const or_model *mo, int R, double mrun, dual M, dual G0)
{
    if (mo->shape[R] == SHAPE_LASS) return lass_lineshape(mo, R, mrun, M, G0);
    double md1, md2, mspec;
    chain_masses(mo, R, &md1, &md2, &mspec);
    const int LB = mo->LB[R], LR = mo->LR[R];
    const double r2 = mo->r[R] * mo->r[R];
    dual mB = dk(mo->mB);
    dual p = breakup(mB, dk(mrun), dk(mspec));
    dual q = breakup(dk(mrun), dk(md1), dk(md2));
    dual p0 = breakup(mB, M, dk(mspec));
    dual q0 = breakup(M, dk(md1), dk(md2));
    dual FB = bw_factor(LB, dscale(dmul(p, p), r2), dscale(dmul(p0, p0), r2));
    dual FR = bw_factor(LR, dscale(dmul(q, q), r2), dscale(dmul(q0, q0), r2));
    dual num = dmul(dmul(FB, dpowi(dscale(p, 1.0 / mo->mB), LB)),
                    dmul(FR, dpowi(dscale(q, 1.0 / mrun), LR)));
    dual width = dmul(dmul(G0, dpowi(ddiv(q, q0), 2 * LR + 1)),
                      dmul(dscale(M, 1.0 / mrun), dmul(FR, FR)));
    dual re = dsub(dmul(M, M), dk(mrun * mrun));
    dual im = dscale(dmul(M, width), -1.0);
    cdual n = {num.v, num.d};
    cdual den = {re.v + I * im.v, re.d + I * im.d};
    return cdiv(n, den);
}

/* Lineshape of resonance R at running mass mrun with pole parameters (M, G0).
 * out = {Re A, Im A, Re dA/dM, Im dA/dM, Re dA/dG0, Im dA/dG0}. */
void or_lineshape(const or_model *mo, int R, double mrun, double M, double G0, double *out)
{
    dual Mv = {M, 1.0}, Gv = {G0, 0.0};
    cdual a = lineshape(mo, R, mrun, Mv, Gv);
    dual Mc = {M, 0.0}, Gd = {G0, 1.0};
    cdual b = lineshape(mo, R, mrun, Mc, Gd);
    out[0] = creal(a.v); out[1] = cimag(a.v);
    out[2] = creal(a.d); out[3] = cimag(a.d);
    out[4] = creal(b.d); out[5] = cimag(b.d);
}

/* ------------------------------------------------------------------ */
/* Wigner small-d by the general factorial sum (integer spins).         */
/* ------------------------------------------------------------------ */
static double fact(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/* d^j_{mp m}(beta) with cos(beta) given; beta in [0, pi]. */
double or_wigner_d(int j, int mp, int m, double cosb)
{
    if (abs(mp) > j || abs(m) > j) return 0.0;
    if (cosb > 1.0) cosb = 1.0;
    if (cosb < -1.0) cosb = -1.0;
    const double c = sqrt(0.5 * (1.0 + cosb)); /* cos(beta/2) */
    const double s = sqrt(0.5 * (1.0 - cosb)); /* sin(beta/2) */
    const double pre = sqrt(fact(j + mp) * fact(j - mp) * fact(j + m) * fact(j - m));
    double sum = 0.0;
    for (int k = 0; k <= 2 * j; ++k) {
        int a = j + m - k, b = j - k - mp, e = k - m + mp;
        if (a < 0 || b < 0 || e < 0) continue;
        double sign = ((k - m + mp) % 2 == 0) ? 1.0 : -1.0;
        double term = sign / (fact(a) * fact(k) * fact(b) * fact(e));
        term *= pow(c, 2 * j - 2 * k + m - mp) * pow(s, 2 * k - m + mp);
        sum += term;
    }
    return pre * sum;
}

/* ------------------------------------------------------------------ */
/* Model                                                               */
/* ------------------------------------------------------------------ */
or_model *or_model_new(const double *masses4, double m_lo, double m_hi, int n_res,
                       const int *chain, const int *J, const int *P, const int *LB,
                       const int *LR, const double *M, const double *G0, const double *r,
                       const int *flt)
{
    if (n_res <= 0 || n_res > OR_MAXR) return NULL;
    or_model *mo = (or_model *)calloc(1, sizeof(or_model));
    mo->mB = masses4[0]; mo->mpsi = masses4[1]; mo->mK = masses4[2]; mo->mpi = masses4[3];
    mo->m_lo = m_lo; mo->m_hi = m_hi;
    mo->n_res = n_res;
    int nc = 0, nf = 0;
    for (int i = 0; i < n_res; ++i) {
        mo->chain[i] = chain[i]; mo->J[i] = J[i]; mo->P[i] = P[i];
        mo->LB[i] = LB[i]; mo->LR[i] = LR[i];
        mo->M[i] = M[i]; mo->G0[i] = G0[i]; mo->r[i] = r[i];
        mo->flt[i] = flt ? flt[i] : 0;
        mo->float_pos[i] = mo->flt[i] ? nf++ : -1;
        if (chain[i] == CH_KSTAR) {
            if (J[i] == 0) {
                mo->col_res[nc] = i; mo->col_lam[nc++] = 0;
            } else {
                for (int l = -1; l <= 1; ++l) { mo->col_res[nc] = i; mo->col_lam[nc++] = l; }
            }
        } else {
            mo->has_z = 1;
            int eta = -P[i] * ((J[i] % 2) ? -1 : 1); /* Eq. 11: H_{-l} = eta H_{l} */
            if (eta == 1) { mo->col_res[nc] = i; mo->col_lam[nc++] = 0; }
            if (J[i] >= 1) { mo->col_res[nc] = i; mo->col_lam[nc++] = 1; }
        }
    }
    mo->n_col = nc;
    mo->n_float = nf;
    return mo;
}

void or_model_free(or_model *mo)
{
    if (!mo) return;
    for (int i = 0; i < 4; ++i) free(mo->tpl[i].h);
    free(mo);
}

/* Make K* resonance R (J = 0) the LASS S-wave of Eq. 7-8 with effective-range
 * constants a, b (GeV^-1) and resonant-term factor Rfac.  Returns 0, or -1 if R
 * is not a J = 0 K* or a constant is out of range. */
int or_model_set_lass(or_model *mo, int R, double a, double b, double Rfac)
{
    if (R < 0 || R >= mo->n_res || mo->chain[R] != CH_KSTAR || mo->J[R] != 0) return -1;
    if (!(a > 0.0) || !(b >= 0.0) || !(Rfac >= 0.0) || !isfinite(b) || !isfinite(Rfac)) return -1;
    mo->shape[R] = SHAPE_LASS;
    mo->lass_a[R] = a; mo->lass_b[R] = b; mo->lass_R[R] = Rfac;
    return 0;
}
int or_num_cols(const or_model *mo) { return mo->n_col; }
int or_num_params(const or_model *mo) { return 2 * mo->n_col + 2 * mo->n_float; }
void or_columns(const or_model *mo, int *res, int *lam)
{
    for (int k = 0; k < mo->n_col; ++k) { res[k] = mo->col_res[k]; lam[k] = mo->col_lam[k]; }
}

/* ------------------------------------------------------------------ */
/* Kinematics from explicit four-vectors                               */
/* ------------------------------------------------------------------ */
typedef struct { double e, x, y, z; } v4;

static v4 boost_z(v4 a, double beta)
{
    double g = 1.0 / sqrt(1.0 - beta * beta);
    v4 r = {g * (a.e + beta * a.z), a.x, a.y, g * (a.z + beta * a.e)};
    return r;
}

/* Lorentz boost of a into the rest frame of a system with four-momentum s. */
static v4 to_rest(v4 a, v4 s)
{
    double ms = sqrt(s.e * s.e - s.x * s.x - s.y * s.y - s.z * s.z);
    double bx = s.x / s.e, by = s.y / s.e, bz = s.z / s.e;
    double b2 = bx * bx + by * by + bz * bz;
    double g = s.e / ms;
    double bp = bx * a.x + by * a.y + bz * a.z;
    double k = (b2 > 0.0) ? (g - 1.0) * bp / b2 : 0.0;
    v4 r;
    r.e = g * (a.e - bp);
    r.x = a.x + (k - g * a.e) * bx;
    r.y = a.y + (k - g * a.e) * by;
    r.z = a.z + (k - g * a.e) * bz;
    return r;
}

typedef struct { double x, y, z; } v3;
static v3 v3of(v4 a) { v3 r = {a.x, a.y, a.z}; return r; }
static double dot3(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross3(v3 a, v3 b)
{
    v3 r = {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
    return r;
}
static v3 scale3(v3 a, double s) { v3 r = {a.x * s, a.y * s, a.z * s}; return r; }
static v3 sub3(v3 a, v3 b) { v3 r = {a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static v3 unit3(v3 a) { return scale3(a, 1.0 / sqrt(dot3(a, a))); }

typedef struct {
    double p, q;              /* two-body momenta of the K* chain */
    double m_psipi, cthZ;     /* Z-chain mass and helicity angle */
    double cthpsi_z;          /* J/psi helicity angle in the Z chain */
    double cphiz, sphiz;      /* (cos, sin) of phi~ */
    double calpha, salpha;    /* (cos, sin) of alpha */
    double rec_cK, rec_cpsi, rec_cphi, rec_sphi; /* K*-chain angles recovered from the vectors */
    v4 K, pi, psi;            /* B-frame four-vectors */
} or_kin;

static void kinematics(const or_model *mo, double m, double cK, double cpsi, double phi, or_kin *o)
{
    const double mB = mo->mB, mpsi = mo->mpsi, mK = mo->mK, mpi = mo->mpi;
    double p = or_breakup(mB, m, mpsi);
    double q = or_breakup(m, mK, mpi);
    o->p = p;
    o->q = q;
    double sK = sqrt(fmax(0.0, 1.0 - cK * cK));
    double spsi = sqrt(fmax(0.0, 1.0 - cpsi * cpsi));
    /* K pi frame: K at angle theta_K* from +z in the x-z plane, x > 0. */
    v4 Kr = {sqrt(mK * mK + q * q), q * sK, 0.0, q * cK};
    v4 pir = {sqrt(mpi * mpi + q * q), -q * sK, 0.0, -q * cK};
    double Ekp = sqrt(m * m + p * p);
    double beta = p / Ekp;
    v4 K = boost_z(Kr, beta), pi = boost_z(pir, beta);
    v4 psi = {sqrt(mpsi * mpsi + p * p), 0.0, 0.0, -p};
    o->K = K; o->pi = pi; o->psi = psi;

    /* J/psi rest frame. */
    v4 Kp = to_rest(K, psi), pip = to_rest(pi, psi);
    v3 nmu = {spsi * cos(phi), -spsi * sin(phi), -cpsi}; /* mu+ direction */
    /* z1: J/psi flight direction in the B frame = minus the B (= K pi) momentum here. */
    v3 z1 = unit3(scale3((v3){Kp.x + pip.x, Kp.y + pip.y, Kp.z + pip.z}, -1.0));
    v3 z2 = unit3(scale3(v3of(pip), -1.0));

    /* K* chain recovered from the vectors (round-trip check). */
    {
        v3 kd = unit3(v3of(Kp));
        v3 x1 = unit3(sub3(kd, scale3(z1, dot3(kd, z1))));
        v3 y1 = cross3(z1, x1);
        o->rec_cpsi = dot3(nmu, z1);
        double cx = dot3(nmu, x1), cy = dot3(nmu, y1), n = sqrt(cx * cx + cy * cy);
        o->rec_cphi = n > 0 ? cx / n : 1.0;
        o->rec_sphi = n > 0 ? cy / n : 0.0;
        v4 sKpi = {K.e + pi.e, K.x + pi.x, K.y + pi.y, K.z + pi.z};
        v4 Kk = to_rest(K, sKpi);
        o->rec_cK = dot3(unit3(v3of(Kk)), (v3){0.0, 0.0, 1.0});
    }

    /* Z = J/psi + pi. */
    v4 Z = {psi.e + pi.e, psi.x + pi.x, psi.y + pi.y, psi.z + pi.z};
    o->m_psipi = sqrt(Z.e * Z.e - Z.x * Z.x - Z.y * Z.y - Z.z * Z.z);
    v4 Kz = to_rest(K, Z), piz = to_rest(pi, Z);
    o->cthZ = dot3(unit3(v3of(Kz)), unit3(v3of(piz)));

    o->cthpsi_z = dot3(nmu, z2);
    {
        /* phi~ is undefined when the K flies along z2 (cos theta_K* = +-1); there
         * sin theta_Z = 0 and the l' = +-1 terms vanish, so (1, 0) is used. */
        v3 kd = unit3(v3of(Kp));
        v3 raw = sub3(kd, scale3(z2, dot3(kd, z2)));
        double nr = sqrt(dot3(raw, raw));
        o->cphiz = 1.0;
        o->sphiz = 0.0;
        if (nr > 1e-300) {
            v3 x2 = scale3(raw, 1.0 / nr);
            v3 y2 = cross3(z2, x2);
            double cx = dot3(nmu, x2), cy = dot3(nmu, y2), n = sqrt(cx * cx + cy * cy);
            if (n > 0) { o->cphiz = cx / n; o->sphiz = cy / n; }
        }
    }
    {
        v3 u1 = sub3(z1, scale3(nmu, dot3(z1, nmu)));
        v3 u2 = sub3(z2, scale3(nmu, dot3(z2, nmu)));
        double n1 = sqrt(dot3(u1, u1)), n2 = sqrt(dot3(u2, u2));
        if (n1 > 0 && n2 > 0) {
            u1 = scale3(u1, 1.0 / n1);
            u2 = scale3(u2, 1.0 / n2);
            o->calpha = dot3(u1, u2);
            o->salpha = dot3(nmu, cross3(u1, u2));
        } else {
            o->calpha = 1.0;
            o->salpha = 0.0;
        }
    }
}

/* Kinematic quantities per event, 24 doubles each:
 * [0] p, [1] q, [2] m_psipi, [3] cos theta_Z, [4] cos theta~_psi, [5] cos phi~,
 * [6] sin phi~, [7] cos alpha, [8] sin alpha, [9..12] K*-chain angles recovered
 * from the vectors (cK, cpsi, cos phi, sin phi), [13..16] K (E, px, py, pz),
 * [17..20] pi (E, px, py, pz), [21] E_psi, [22] pz_psi, [23] unused. */
void or_kinematics(const or_model *mo, const double *m, const double *cK, const double *cpsi,
                   const double *phi, int64_t n, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n; ++e) {
        or_kin k;
        kinematics(mo, m[e], cK[e], cpsi[e], phi[e], &k);
        double *o = out + 24 * e;
        o[0] = k.p; o[1] = k.q; o[2] = k.m_psipi; o[3] = k.cthZ; o[4] = k.cthpsi_z;
        o[5] = k.cphiz; o[6] = k.sphiz; o[7] = k.calpha; o[8] = k.salpha;
        o[9] = k.rec_cK; o[10] = k.rec_cpsi; o[11] = k.rec_cphi; o[12] = k.rec_sphi;
        o[13] = k.K.e; o[14] = k.K.x; o[15] = k.K.y; o[16] = k.K.z;
        o[17] = k.pi.e; o[18] = k.pi.x; o[19] = k.pi.y; o[20] = k.pi.z;
        o[21] = k.psi.e; o[22] = k.psi.z; o[23] = 0.0;
    }
}

/* ------------------------------------------------------------------ */
/* Per-event basis B[k][xi] and its mass/width derivatives             */
/* ------------------------------------------------------------------ */

/* Pole parameters in use: model values, replaced by the floated ones in params. */
static void pole_params(const or_model *mo, const double *params, double *M, double *G)
{
    for (int i = 0; i < mo->n_res; ++i) {
        M[i] = mo->M[i];
        G[i] = mo->G0[i];
        if (mo->flt[i] && params) {
            M[i] = params[2 * mo->n_col + 2 * mo->float_pos[i]];
            G[i] = params[2 * mo->n_col + 2 * mo->float_pos[i] + 1];
        }
    }
}

/*
 * Angular factor of column k for muon helicity xi = +1 (x = 0) / -1 (x = 1),
 * and the lineshape index.  K*: d^J_{l0}(theta_K*) e^{i l phi} d^1_{l xi}(theta_psi)
 * (Eq. 4).  Z: d^J_{0 l'}(theta_Z) e^{i l' phi~} d^1_{l' xi}(theta~_psi) e^{i xi alpha}
 * (Eq. 10), with l' = +-1 summed as H_{-1} = eta H_{+1} (Eq. 11).
 */
static void angular(const or_model *mo, const or_kin *k, double cK, double cpsi, double phi,
                    cplx ang[][2])
{
    for (int c = 0; c < mo->n_col; ++c) {
        int R = mo->col_res[c], l = mo->col_lam[c], J = mo->J[R];
        for (int x = 0; x < 2; ++x) {
            int xi = x == 0 ? 1 : -1;
            cplx v;
            if (mo->chain[R] == CH_KSTAR) {
                v = or_wigner_d(J, l, 0, cK) * cexp(I * l * phi) * or_wigner_d(1, l, xi, cpsi);
            } else {
                cplx eph = k->cphiz + I * k->sphiz;   /* e^{i phi~} */
                cplx eal = k->calpha + I * xi * k->salpha; /* e^{i xi alpha} */
                if (l == 0) {
                    v = or_wigner_d(J, 0, 0, k->cthZ) * or_wigner_d(1, 0, xi, k->cthpsi_z);
                } else {
                    int eta = -mo->P[R] * ((J % 2) ? -1 : 1);
                    v = or_wigner_d(J, 0, 1, k->cthZ) * eph * or_wigner_d(1, 1, xi, k->cthpsi_z) +
                        eta * or_wigner_d(J, 0, -1, k->cthZ) * conj(eph) *
                            or_wigner_d(1, -1, xi, k->cthpsi_z);
                }
                v *= eal;
            }
            ang[c][x] = v;
        }
    }
}

typedef struct {
    double pq;
    cplx B[OR_MAXC][2];
    cplx dBM[OR_MAXC][2], dBG[OR_MAXC][2]; /* derivatives wrt the column's M, G0 */
} or_event;

static void event_basis(const or_model *mo, const double *M, const double *G, double m,
                        double cK, double cpsi, double phi, int want_deriv, or_event *ev)
{
    or_kin k;
    kinematics(mo, m, cK, cpsi, phi, &k);
    ev->pq = k.p * k.q;
    cplx ang[OR_MAXC][2];
    angular(mo, &k, cK, cpsi, phi, ang);
    cplx A[OR_MAXR], dAM[OR_MAXR], dAG[OR_MAXR];
    for (int R = 0; R < mo->n_res; ++R) {
        double mrun = mo->chain[R] == CH_KSTAR ? m : k.m_psipi;
        if (want_deriv && mo->flt[R]) {
            dual Mv = {M[R], 1.0}, Gv = {G[R], 0.0}, Mc = {M[R], 0.0}, Gd = {G[R], 1.0};
            cdual a = lineshape(mo, R, mrun, Mv, Gv);
            cdual b = lineshape(mo, R, mrun, Mc, Gd);
            A[R] = a.v; dAM[R] = a.d; dAG[R] = b.d;
        } else {
            A[R] = lineshape(mo, R, mrun, dk(M[R]), dk(G[R])).v;
            dAM[R] = 0; dAG[R] = 0;
        }
    }
    for (int c = 0; c < mo->n_col; ++c) {
        int R = mo->col_res[c];
        for (int x = 0; x < 2; ++x) {
            ev->B[c][x] = A[R] * ang[c][x];
            ev->dBM[c][x] = dAM[R] * ang[c][x];
            ev->dBG[c][x] = dAG[R] * ang[c][x];
        }
    }
}

/* Basis per event, layout out[((e * K + k) * 2 + x) * 2 + {re, im}] and pq[e]. */
int or_basis(const or_model *mo, const double *params, const double *m, const double *cK,
             const double *cpsi, const double *phi, int64_t n, double *out, double *pq)
{
    double M[OR_MAXR], G[OR_MAXR];
    pole_params(mo, params, M, G);
    const int K = mo->n_col;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n; ++e) {
        or_event ev;
        event_basis(mo, M, G, m[e], cK[e], cpsi[e], phi[e], 0, &ev);
        for (int c = 0; c < K; ++c)
            for (int x = 0; x < 2; ++x) {
                out[((e * K + c) * 2 + x) * 2 + 0] = creal(ev.B[c][x]);
                out[((e * K + c) * 2 + x) * 2 + 1] = cimag(ev.B[c][x]);
            }
        if (pq) pq[e] = ev.pq;
    }
    return 0;
}

/* Signal density S = sum_xi |sum_k c_k B_k xi|^2 (Eq. 5 / Eq. 12) and p*q per event. */
int or_density(const or_model *mo, const double *params, const double *m, const double *cK,
               const double *cpsi, const double *phi, int64_t n, double *S, double *pq)
{
    double M[OR_MAXR], G[OR_MAXR];
    pole_params(mo, params, M, G);
    const int K = mo->n_col;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n; ++e) {
        or_event ev;
        event_basis(mo, M, G, m[e], cK[e], cpsi[e], phi[e], 0, &ev);
        double s = 0.0;
        for (int x = 0; x < 2; ++x) {
            cplx a = 0.0;
            for (int c = 0; c < K; ++c) a += (params[2 * c] + I * params[2 * c + 1]) * ev.B[c][x];
            s += creal(a) * creal(a) + cimag(a) * cimag(a);
        }
        S[e] = s;
        if (pq) pq[e] = ev.pq;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Compensated sums (Neumaier) in fixed-size blocks, combined in order */
/* ------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;
static void nadd(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nval(nsum a) { return a.s + a.c; }

/*
 * Sums over a point set of: [0] ln S (or w S when weights mode), and the
 * derivatives of the same quantity wrt every parameter (np of them) when grad
 * is requested.  mode 0: data (ln S and d ln S); mode 1: normalisation (w S and
 * w dS).  Returns -1 if a data event has S <= 0 (or p q <= 0).
 */
/*
 * S of one point (Eq. 5 / 12) and, when dS is non-NULL, dS/dtheta for every
 * parameter: dS/dRe c_k = 2 Re z_k, dS/dIm c_k = -2 Im z_k with
 * z_k = sum_xi conj(a_xi) B_k xi, and dS/dM_R = 2 Re sum_xi conj(a_xi)
 * sum_{k in R} c_k dB_k xi/dM_R (the same for G0).  *pq receives p q and
 * *kin (when non-NULL) the point's kinematics.
 */
static double event_S(const or_model *mo, const double *params, const double *M, const double *G,
                      double m, double cK, double cpsi, double phi, double *dS, double *pq,
                      or_kin *kin)
{
    const int K = mo->n_col;
    or_event ev;
    event_basis(mo, M, G, m, cK, cpsi, phi, dS != NULL, &ev);
    if (pq) *pq = ev.pq;
    if (kin) kinematics(mo, m, cK, cpsi, phi, kin);
    cplx a[2] = {0, 0};
    for (int x = 0; x < 2; ++x)
        for (int c = 0; c < K; ++c) a[x] += (params[2 * c] + I * params[2 * c + 1]) * ev.B[c][x];
    double S = 0.0;
    for (int x = 0; x < 2; ++x) S += creal(a[x]) * creal(a[x]) + cimag(a[x]) * cimag(a[x]);
    if (!dS) return S;
    for (int c = 0; c < K; ++c) {
        cplx z = conj(a[0]) * ev.B[c][0] + conj(a[1]) * ev.B[c][1];
        dS[2 * c] = 2.0 * creal(z);
        dS[2 * c + 1] = -2.0 * cimag(z);
    }
    for (int R = 0; R < mo->n_res; ++R) {
        if (!mo->flt[R]) continue;
        cplx yM = 0, yG = 0;
        for (int c = 0; c < K; ++c) {
            if (mo->col_res[c] != R) continue;
            cplx cc = params[2 * c] + I * params[2 * c + 1];
            for (int x = 0; x < 2; ++x) {
                yM += conj(a[x]) * cc * ev.dBM[c][x];
                yG += conj(a[x]) * cc * ev.dBG[c][x];
            }
        }
        int f = 2 * K + 2 * mo->float_pos[R];
        dS[f] = 2.0 * creal(yM);
        dS[f + 1] = 2.0 * creal(yG);
    }
    return S;
}

/*
 * Sums over a point set of: [0] ln S (or w S when weights mode), and the
 * derivatives of the same quantity wrt every parameter (np of them) when grad
 * is requested.  mode 0: data (ln S and d ln S); mode 1: normalisation (w S and
 * w dS).  Returns -1 if a data event has S <= 0 (or p q <= 0).
 */
static int accumulate(const or_model *mo, const double *params, int mode, const double *m,
                      const double *cK, const double *cpsi, const double *phi, const double *w,
                      int64_t n, int want_grad, double *sum0, double *sum_lnpq, double *grad)
{
    double M[OR_MAXR], G[OR_MAXR];
    pole_params(mo, params, M, G);
    const int NP = or_num_params(mo);
    const int64_t nblk = (n + OR_BLOCK - 1) / OR_BLOCK;
    const int stride = 2 + NP;
    double *bs = (double *)calloc((size_t)(nblk > 0 ? nblk : 1) * stride, sizeof(double));
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t b = 0; b < nblk; ++b) {
        nsum acc0 = {0, 0}, accpq = {0, 0};
        nsum accg[2 * OR_MAXC + 2 * OR_MAXR];
        memset(accg, 0, sizeof(accg));
        double dS[2 * OR_MAXC + 2 * OR_MAXR];
        int64_t e1 = (b + 1) * OR_BLOCK < n ? (b + 1) * OR_BLOCK : n;
        for (int64_t e = b * OR_BLOCK; e < e1; ++e) {
            double pq;
            const double S = event_S(mo, params, M, G, m[e], cK[e], cpsi[e], phi[e],
                                     want_grad ? dS : NULL, &pq, NULL);
            double scale;
            if (mode == 0) {
                if (!(S > 0.0) || !(pq > 0.0)) { bad = 1; continue; }
                nadd(&acc0, log(S));
                nadd(&accpq, log(pq));
                scale = 1.0 / S;
            } else {
                double we = w ? w[e] : pq;
                nadd(&acc0, we * S);
                scale = we;
            }
            if (!want_grad) continue;
            for (int i = 0; i < NP; ++i) nadd(&accg[i], scale * dS[i]);
        }
        double *o = bs + b * stride;
        o[0] = nval(acc0);
        o[1] = nval(accpq);
        for (int i = 0; i < NP; ++i) o[2 + i] = nval(accg[i]);
    }
    nsum t0 = {0, 0}, tpq = {0, 0};
    nsum tg[2 * OR_MAXC + 2 * OR_MAXR];
    memset(tg, 0, sizeof(tg));
    for (int64_t b = 0; b < nblk; ++b) {
        nadd(&t0, bs[b * stride]);
        nadd(&tpq, bs[b * stride + 1]);
        for (int i = 0; i < NP; ++i) nadd(&tg[i], bs[b * stride + 2 + i]);
    }
    free(bs);
    *sum0 = nval(t0);
    if (sum_lnpq) *sum_lnpq = nval(tpq);
    if (grad)
        for (int i = 0; i < NP; ++i) grad[i] = want_grad ? nval(tg[i]) : 0.0;
    return bad ? -1 : 0;
}

/*
 * Normalisation integral I = (V / N_mc) sum_n w_n S_n over the given points
 * (w = p q when w is NULL), and its gradient when dI is non-NULL.
 */
int or_norm(const or_model *mo, const double *params, const double *m, const double *cK,
            const double *cpsi, const double *phi, const double *w, int64_t n, double volume,
            double *Iout, double *dI)
{
    double s;
    int NP = or_num_params(mo);
    double *g = dI ? (double *)calloc(NP, sizeof(double)) : NULL;
    accumulate(mo, params, 1, m, cK, cpsi, phi, w, n, dI != NULL, &s, NULL, g);
    *Iout = volume / (double)n * s;
    if (dI) {
        for (int i = 0; i < NP; ++i) dI[i] = volume / (double)n * g[i];
        free(g);
    }
    return 0;
}

/*
 * NLL = -2 [ sum_e ln S_e + sum_e ln(p_e q_e) - N ln I ] and its gradient.
 * aux (optional, 3 doubles): sum ln S, sum ln(p q), I.
 * Returns -1 (and NLL = +inf) if a data event has S <= 0 or I <= 0.
 */
int or_nll(const or_model *mo, const double *params, const double *m, const double *cK,
           const double *cpsi, const double *phi, int64_t n, const double *nm, const double *ncK,
           const double *ncpsi, const double *nphi, const double *nw, int64_t n_mc, double volume,
           double *nll, double *grad, double *aux)
{
    const int NP = or_num_params(mo);
    double sl, slpq, Inrm;
    double *gd = grad ? (double *)calloc(NP, sizeof(double)) : NULL;
    double *gI = grad ? (double *)calloc(NP, sizeof(double)) : NULL;
    int rc = accumulate(mo, params, 0, m, cK, cpsi, phi, NULL, n, grad != NULL, &sl, &slpq, gd);
    or_norm(mo, params, nm, ncK, ncpsi, nphi, nw, n_mc, volume, &Inrm, gI);
    if (aux) { aux[0] = sl; aux[1] = slpq; aux[2] = Inrm; }
    if (rc != 0 || !(Inrm > 0.0)) {
        *nll = INFINITY;
        if (grad) { for (int i = 0; i < NP; ++i) grad[i] = 0.0; free(gd); free(gI); }
        return -1;
    }
    *nll = -2.0 * (sl + slpq - (double)n * log(Inrm));
    if (grad) {
        for (int i = 0; i < NP; ++i) grad[i] = -2.0 * (gd[i] - (double)n * gI[i] / Inrm);
        free(gd);
        free(gI);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Efficiency and background (Eq. 14)                                  */
/* ------------------------------------------------------------------ */

/* Content of a binned template at (x, y): bin ix = floor((x - xlo) * nx / (xhi - xlo)),
 * iy likewise, content h[iy * nx + ix]; the upper edge belongs to the last bin,
 * and the template is 0 outside [xlo, xhi] x [ylo, yhi]. */
static double tpl_value(const double *h, int nx, int ny, double xlo, double xhi, double ylo,
                        double yhi, double x, double y)
{
    if (!(x >= xlo && x <= xhi && y >= ylo && y <= yhi)) return 0.0;
    int ix = (int)floor((x - xlo) * nx / (xhi - xlo));
    int iy = (int)floor((y - ylo) * ny / (yhi - ylo));
    if (ix >= nx) ix = nx - 1;
    if (iy >= ny) iy = ny - 1;
    return h[(int64_t)iy * nx + ix];
}

double or_tpl_value(const double *h, int nx, int ny, const double *range, double x, double y)
{
    return tpl_value(h, nx, ny, range[0], range[1], range[2], range[3], x, y);
}

/* Set the efficiency (which = 0) or background (which = 1, with purity P in
 * [0, 1]) templates: hm over (m^2_Kpi, m^2_psipi) with range rm = {xlo, xhi, ylo,
 * yhi}, ha over (cos theta_psi, phi) with range ra.  Returns 0, or -1 on a bad
 * argument. */
int or_model_set_template(or_model *mo, int which, const double *hm, int nxm, int nym,
                          const double *rm, const double *ha, int nxa, int nya, const double *ra,
                          double purity)
{
    if (which != 0 && which != 1) return -1;
    if (nxm < 1 || nym < 1 || nxa < 1 || nya < 1 || !hm || !ha) return -1;
    if (!(rm[1] > rm[0]) || !(rm[3] > rm[2]) || !(ra[1] > ra[0]) || !(ra[3] > ra[2])) return -1;
    if (which == 1 && !(purity >= 0.0 && purity <= 1.0)) return -1;
    const double *src[2] = {hm, ha};
    const int nx[2] = {nxm, nxa}, ny[2] = {nym, nya};
    const double *rg[2] = {rm, ra};
    for (int j = 0; j < 2; ++j) {
        int t = 2 * which + j;
        free(mo->tpl[t].h);
        mo->tpl[t].h = (double *)malloc((size_t)nx[j] * ny[j] * sizeof(double));
        memcpy(mo->tpl[t].h, src[j], (size_t)nx[j] * ny[j] * sizeof(double));
        mo->tpl[t].nx = nx[j]; mo->tpl[t].ny = ny[j];
        mo->tpl[t].xlo = rg[j][0]; mo->tpl[t].xhi = rg[j][1];
        mo->tpl[t].ylo = rg[j][2]; mo->tpl[t].yhi = rg[j][3];
    }
    if (which == 0) mo->has_eff = 1;
    else { mo->has_bkg = 1; mo->purity = purity; }
    return 0;
}

/* Flavour mistag fraction w in [0, 0.5] (Eq. 12 text).  Returns 0, or -1. */
int or_model_set_mistag(or_model *mo, double w)
{
    if (!(w >= 0.0 && w <= 0.5)) return -1;
    mo->mistag = w;
    return 0;
}

static double tpl_at(const or_model *mo, int t, double x, double y)
{
    return tpl_value(mo->tpl[t].h, mo->tpl[t].nx, mo->tpl[t].ny, mo->tpl[t].xlo, mo->tpl[t].xhi,
                     mo->tpl[t].ylo, mo->tpl[t].yhi, x, y);
}

/* eps and the background template value hb at one point (1 and 0 when unset),
 * with m^2_psipi from the point's four-vectors. */
static void point_templates(const or_model *mo, double m, double cK, double cpsi, double phi,
                            double *eps, double *hb)
{
    or_kin k;
    kinematics(mo, m, cK, cpsi, phi, &k);
    const double x = m * m, y = k.m_psipi * k.m_psipi;
    *eps = mo->has_eff ? tpl_at(mo, 0, x, y) * tpl_at(mo, 1, cpsi, phi) : 1.0;
    *hb = mo->has_bkg ? tpl_at(mo, 2, x, y) * tpl_at(mo, 3, cpsi, phi) : 0.0;
}

/* Per point: out[3 e] = eps, out[3 e + 1] = hb, out[3 e + 2] = m^2_psipi. */
void or_templates(const or_model *mo, const double *m, const double *cK, const double *cpsi,
                  const double *phi, int64_t n, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n; ++e) {
        or_kin k;
        kinematics(mo, m[e], cK[e], cpsi[e], phi[e], &k);
        point_templates(mo, m[e], cK[e], cpsi[e], phi[e], &out[3 * e], &out[3 * e + 1]);
        out[3 * e + 2] = k.m_psipi * k.m_psipi;
    }
}

/*
 * -2 ln L of Eq. 14.  Per event the PDF in (m, cK, cpsi, phi) is
 *   f = p q [ P eps S / I_eps + (1 - P) hb / B ],
 * with S the flavour-tagged density (1 - w) S(t phi) + w S(-t phi) for tag t
 * (tag NULL: every event B0),
 *   I_eps = (V / N_mc) sum_n w_n eps_n S_n,   B = (V / N_mc) sum_n w_n hb_n,
 * over the normalisation points (w = p q when nw is NULL); without a background
 * P = 1.  NLL = -2 sum_e ln f_e and
 *   d ln f_e / dtheta = (P eps_e p_e q_e / (I_eps f_e)) (dS_e - S_e dI_eps / I_eps).
 * aux (5 doubles): sum ln(f / (p q)), sum ln(p q), I_eps, B, sum_e r_e with
 * r_e = P eps_e S_e p_e q_e / (I_eps f_e) the signal probability of event e.
 * Returns -1 (NLL = +inf) if some f_e <= 0, p q <= 0 or I_eps <= 0.
 */
int or_nll_eq14(const or_model *mo, const double *params, const double *m, const double *cK,
                const double *cpsi, const double *phi, const double *tag, int64_t n,
                const double *nm, const double *ncK, const double *ncpsi, const double *nphi,
                const double *nw, int64_t n_mc, double volume, double *nll, double *grad,
                double *aux)
{
    const int NP = or_num_params(mo);
    const double P = mo->has_bkg ? mo->purity : 1.0;
    /* normalisation points: efficiency-weighted weights and the background sum */
    double *weps = (double *)malloc((size_t)(n_mc > 0 ? n_mc : 1) * sizeof(double));
    double *whb = (double *)malloc((size_t)(n_mc > 0 ? n_mc : 1) * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_mc; ++i) {
        double eps, hb, w = nw ? nw[i] : 0.0;
        point_templates(mo, nm[i], ncK[i], ncpsi[i], nphi[i], &eps, &hb);
        if (!nw) {
            or_kin k;
            kinematics(mo, nm[i], ncK[i], ncpsi[i], nphi[i], &k);
            w = k.p * k.q;
        }
        weps[i] = w * eps;
        whb[i] = w * hb;
    }
    double sI, Bs = 0.0;
    double *gI = (double *)calloc(NP > 0 ? NP : 1, sizeof(double));
    accumulate(mo, params, 1, nm, ncK, ncpsi, nphi, weps, n_mc, grad != NULL, &sI, NULL, gI);
    const double Ie = volume / (double)n_mc * sI;
    {
        nsum b = {0, 0};
        for (int64_t i = 0; i < n_mc; ++i) nadd(&b, whb[i]);
        Bs = volume / (double)n_mc * nval(b);
    }
    free(weps);
    free(whb);
    for (int i = 0; i < NP; ++i) gI[i] *= volume / (double)n_mc;
    /* data events, in blocks of fixed size summed in block order */
    double Mp[OR_MAXR], Gp[OR_MAXR];
    pole_params(mo, params, Mp, Gp);
    const int64_t nblk = (n + OR_BLOCK - 1) / OR_BLOCK;
    const int stride = 3 + NP;
    double *bs = (double *)calloc((size_t)(nblk > 0 ? nblk : 1) * stride, sizeof(double));
    int bad = !(Ie > 0.0) || (P < 1.0 && !(Bs > 0.0));
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t b = 0; b < nblk; ++b) {
        nsum sl = {0, 0}, spq = {0, 0}, sr = {0, 0};
        nsum sg[2 * OR_MAXC + 2 * OR_MAXR];
        memset(sg, 0, sizeof(sg));
        double dS[2 * OR_MAXC + 2 * OR_MAXR], dSb[2 * OR_MAXC + 2 * OR_MAXR];
        int64_t e1 = (b + 1) * OR_BLOCK < n ? (b + 1) * OR_BLOCK : n;
        for (int64_t e = b * OR_BLOCK; e < e1; ++e) {
            double pq, pqb, eps, hb;
            /* flavour: density (1 - w) S(t phi) + w S(-t phi), templates at the observed phi */
            const double t = tag ? tag[e] : 1.0, w = mo->mistag;
            double S = event_S(mo, params, Mp, Gp, m[e], cK[e], cpsi[e], t * phi[e],
                               grad ? dS : NULL, &pq, NULL);
            if (w > 0.0) {
                const double Sb = event_S(mo, params, Mp, Gp, m[e], cK[e], cpsi[e], -t * phi[e],
                                          grad ? dSb : NULL, &pqb, NULL);
                S = (1.0 - w) * S + w * Sb;
                if (grad)
                    for (int i = 0; i < NP; ++i) dS[i] = (1.0 - w) * dS[i] + w * dSb[i];
            }
            point_templates(mo, m[e], cK[e], cpsi[e], phi[e], &eps, &hb);
            const double sig = P * eps * S / Ie;
            const double g = sig + (P < 1.0 ? (1.0 - P) * hb / Bs : 0.0);   /* f / (p q) */
            if (!(g > 0.0) || !(pq > 0.0)) { bad = 1; continue; }
            nadd(&sl, log(g));
            nadd(&spq, log(pq));
            nadd(&sr, sig / g);
            if (!grad) continue;
            const double c = P * eps / (Ie * g);
            for (int i = 0; i < NP; ++i) nadd(&sg[i], c * (dS[i] - S * gI[i] / Ie));
        }
        double *o = bs + b * stride;
        o[0] = nval(sl);
        o[1] = nval(spq);
        o[2] = nval(sr);
        for (int i = 0; i < NP; ++i) o[3 + i] = nval(sg[i]);
    }
    nsum tl = {0, 0}, tpq = {0, 0}, tr = {0, 0};
    nsum tg[2 * OR_MAXC + 2 * OR_MAXR];
    memset(tg, 0, sizeof(tg));
    for (int64_t b = 0; b < nblk; ++b) {
        nadd(&tl, bs[b * stride]);
        nadd(&tpq, bs[b * stride + 1]);
        nadd(&tr, bs[b * stride + 2]);
        for (int i = 0; i < NP; ++i) nadd(&tg[i], bs[b * stride + 3 + i]);
    }
    free(bs);
    free(gI);
    if (aux) { aux[0] = nval(tl); aux[1] = nval(tpq); aux[2] = Ie; aux[3] = Bs; aux[4] = nval(tr); }
    if (bad) {
        *nll = INFINITY;
        if (grad) for (int i = 0; i < NP; ++i) grad[i] = 0.0;
        return -1;
    }
    *nll = -2.0 * (nval(tl) + nval(tpq));
    if (grad) for (int i = 0; i < NP; ++i) grad[i] = -2.0 * nval(tg[i]);
    return 0;
}

/*
 * The sums of one shard of a fit whose data events and normalisation points are
 * split into shards: -2 ln L of the unbinned fit needs, over the union,
 * sum ln S, sum ln(p q), N, and I = V sum w S / M, so per shard
 *   out[0] sum ln S, [1] sum ln(p q), [2] N, [3] T = V sum_n w_n S_n, [4] M,
 *   [5] 1 if a data event has S <= 0 or p q <= 0, else 0,
 *   [6 .. 6+NP) d(sum ln S)/dtheta, [6+NP .. 6+2NP) dT/dtheta  (grad != 0).
 * Either set may be empty (n = 0 or n_mc = 0 gives zero sums).
 */
int or_partials(const or_model *mo, const double *params, const double *m, const double *cK,
                const double *cpsi, const double *phi, int64_t n, const double *nm,
                const double *ncK, const double *ncpsi, const double *nphi, const double *nw,
                int64_t n_mc, double volume, int grad, double *out)
{
    const int NP = or_num_params(mo);
    double sl = 0.0, slpq = 0.0, s = 0.0;
    double *gd = (double *)calloc(NP > 0 ? NP : 1, sizeof(double));
    double *gs = (double *)calloc(NP > 0 ? NP : 1, sizeof(double));
    int rc = 0;
    if (n > 0) rc = accumulate(mo, params, 0, m, cK, cpsi, phi, NULL, n, grad, &sl, &slpq, gd);
    if (n_mc > 0) accumulate(mo, params, 1, nm, ncK, ncpsi, nphi, nw, n_mc, grad, &s, NULL, gs);
    out[0] = sl;
    out[1] = slpq;
    out[2] = (double)n;
    out[3] = volume * s;
    out[4] = (double)n_mc;
    out[5] = rc != 0 ? 1.0 : 0.0;
    if (grad)
        for (int i = 0; i < NP; ++i) {
            out[6 + i] = gd[i];
            out[6 + NP + i] = volume * gs[i];
        }
    free(gd);
    free(gs);
    return rc;
}

/* Gram matrix G = sum_n w_n sum_xi x x^T of the real 2K-vectors
 * x = (Re B_0, Im B_0, Re B_1, ...), G stored row-major 2K x 2K. */
int or_gram(const or_model *mo, const double *params, const double *m, const double *cK,
            const double *cpsi, const double *phi, const double *w, int64_t n, double *G)
{
    double M[OR_MAXR], Gm[OR_MAXR];
    pole_params(mo, params, M, Gm);
    const int K = mo->n_col, D = 2 * K;
    const int64_t nblk = (n + OR_BLOCK - 1) / OR_BLOCK;
    double *bs = (double *)calloc((size_t)(nblk > 0 ? nblk : 1) * D * D, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nblk; ++b) {
        double *o = bs + b * D * D;
        int64_t e1 = (b + 1) * OR_BLOCK < n ? (b + 1) * OR_BLOCK : n;
        double xv[2 * OR_MAXC];
        for (int64_t e = b * OR_BLOCK; e < e1; ++e) {
            or_event ev;
            event_basis(mo, M, Gm, m[e], cK[e], cpsi[e], phi[e], 0, &ev);
            double we = w ? w[e] : ev.pq;
            for (int x = 0; x < 2; ++x) {
                for (int c = 0; c < K; ++c) {
                    xv[2 * c] = creal(ev.B[c][x]);
                    xv[2 * c + 1] = cimag(ev.B[c][x]);
                }
                for (int i = 0; i < D; ++i)
                    for (int j = 0; j < D; ++j) o[i * D + j] += we * xv[i] * xv[j];
            }
        }
    }
    for (int i = 0; i < D * D; ++i) {
        nsum t = {0, 0};
        for (int64_t b = 0; b < nblk; ++b) nadd(&t, bs[b * D * D + i]);
        G[i] = nval(t);
    }
    free(bs);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Accept-reject generator (Fit validation: pseudo-data from the model) */
/* ------------------------------------------------------------------ */

/* Candidate i: Philox(counter = (i, stream, 0, 0), key = seed) gives the four
 * coordinates; counter (i, stream + 1, 0, 0) gives the acceptance uniform. */
static void candidate(const or_model *mo, uint64_t seed, uint64_t i, uint32_t stream, float *x4,
                      double *u)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)i, stream, (uint32_t)(i >> 32), 0u}, out[4];
    or_philox4x32_10(ctr, key, out);
    x4[0] = (float)(mo->m_lo + (mo->m_hi - mo->m_lo) * u01(out[0]));
    x4[1] = (float)(2.0 * u01(out[1]) - 1.0);
    x4[2] = (float)(2.0 * u01(out[2]) - 1.0);
    x4[3] = (float)(M_PI * (2.0 * u01(out[3]) - 1.0));
    uint32_t ctr2[4] = {(uint32_t)i, stream + 1u, (uint32_t)(i >> 32), 0u};
    or_philox4x32_10(ctr2, key, out);
    *u = u01(out[0]);
}

static double f_of(const or_model *mo, const double *params, const double *M, const double *G,
                   const float *x4)
{
    or_event ev;
    event_basis(mo, M, G, x4[0], x4[1], x4[2], x4[3], 0, &ev);
    double S = 0.0;
    for (int x = 0; x < 2; ++x) {
        cplx a = 0.0;
        for (int c = 0; c < mo->n_col; ++c) a += (params[2 * c] + I * params[2 * c + 1]) * ev.B[c][x];
        S += creal(a) * creal(a) + cimag(a) * cimag(a);
    }
    return S * ev.pq;
}

/*
 * Draw n_want events distributed as S p q over the box.  f_max is a scan of
 * n_scan candidates (stream 2) times 1.5; if an accepted-stage candidate ever
 * exceeds f_max the whole draw restarts with 2 f_max.  Output: FP32 SoA.
 * Returns the number of candidates used (or -1 if max_cand was reached).
 */
int64_t or_generate(const or_model *mo, const double *params, uint64_t seed, int64_t n_want,
                    int64_t n_scan, int64_t max_cand, float *om, float *ocK, float *ocpsi,
                    float *ophi, double *fmax_used)
{
    double M[OR_MAXR], G[OR_MAXR];
    pole_params(mo, params, M, G);
    double fmax = 0.0;
#pragma omp parallel for schedule(static) reduction(max : fmax)
    for (int64_t i = 0; i < n_scan; ++i) {
        float x4[4];
        double u;
        candidate(mo, seed, (uint64_t)i, 2u, x4, &u);
        double f = f_of(mo, params, M, G, x4);
        if (f > fmax) fmax = f;
    }
    fmax *= 1.5;
    const int64_t chunk = 1 << 16;
    double *f = (double *)malloc(chunk * sizeof(double));
    double *uu = (double *)malloc(chunk * sizeof(double));
    float *xs = (float *)malloc(chunk * 4 * sizeof(float));
restart:;
    int64_t got = 0, used = 0;
    while (got < n_want) {
        if (used >= max_cand) { free(f); free(uu); free(xs); return -1; }
        int over = 0;
#pragma omp parallel for schedule(static) reduction(| : over)
        for (int64_t j = 0; j < chunk; ++j) {
            candidate(mo, seed, (uint64_t)(used + j), 0u, xs + 4 * j, &uu[j]);
            f[j] = f_of(mo, params, M, G, xs + 4 * j);
            if (f[j] > fmax) over = 1;
        }
        if (over) {
            fmax *= 2.0;
            goto restart;
        }
        int64_t j = 0;
        for (; j < chunk && got < n_want; ++j) {
            if (uu[j] * fmax < f[j]) {
                om[got] = xs[4 * j]; ocK[got] = xs[4 * j + 1];
                ocpsi[got] = xs[4 * j + 2]; ophi[got] = xs[4 * j + 3];
                ++got;
            }
        }
        used += j;
    }
    free(f); free(uu); free(xs);
    if (fmax_used) *fmax_used = fmax;
    return used;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* Learned importance-sampling proposal (normalisation integral):      */
/* MLP 4 -> 64 -> 64 -> 1 with tanh hidden units and softplus output,  */
/* a density g over x in [-1, 1]^4 trained on events drawn from the    */
/* model; then a piecewise-constant proposal on a cell grid mixed with */
/* the uniform density.                                                 */
/* Parameter layout: W1[64][4], b1[64], W2[64][64], b2[64], W3[64], b3. */
/* ------------------------------------------------------------------ */
#define MLP_H 64
#define MLP_NP (MLP_H * 4 + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1)

int or_mlp_num_params(void) { return MLP_NP; }

static double softplus_d(double o) { return o > 30.0 ? o : log1p(exp(o)); }
static double sigmoid_d(double o) { return 1.0 / (1.0 + exp(-o)); }

typedef struct {
    double h1[MLP_H], h2[MLP_H], o, g;
} mlp_act;

static void mlp_fwd(const double *th, const double *x, mlp_act *a)
{
    const double *W1 = th, *b1 = W1 + MLP_H * 4, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const double *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
    for (int i = 0; i < MLP_H; ++i) {
        double z = b1[i];
        for (int j = 0; j < 4; ++j) z += W1[i * 4 + j] * x[j];
        a->h1[i] = tanh(z);
    }
    for (int i = 0; i < MLP_H; ++i) {
        double z = b2[i];
        for (int j = 0; j < MLP_H; ++j) z += W2[i * MLP_H + j] * a->h1[j];
        a->h2[i] = tanh(z);
    }
    double o = b3[0];
    for (int j = 0; j < MLP_H; ++j) o += W3[j] * a->h2[j];
    a->o = o;
    a->g = softplus_d(o);
}

/* g(x) for n points (x: n x 4, row-major). */
void or_mlp_forward(const double *th, const double *x, int64_t n, double *g)
{
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n; ++e) {
        mlp_act a;
        mlp_fwd(th, x + 4 * e, &a);
        g[e] = a.g;
    }
}

/* Accumulate coef * dg/dtheta of one point into grad. */
static void mlp_bwd_add(const double *th, const double *x, const mlp_act *a, double coef, double *grad)
{
    const double *W2 = th + MLP_H * 4 + MLP_H, *W3 = W2 + MLP_H * MLP_H + MLP_H;
    double *gW1 = grad, *gb1 = gW1 + MLP_H * 4, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H;
    double *gW3 = gb2 + MLP_H, *gb3 = gW3 + MLP_H;
    const double dO = coef * sigmoid_d(a->o);
    double d2[MLP_H], d1[MLP_H];
    for (int j = 0; j < MLP_H; ++j) {
        gW3[j] += dO * a->h2[j];
        d2[j] = dO * W3[j] * (1.0 - a->h2[j] * a->h2[j]);
    }
    gb3[0] += dO;
    for (int j = 0; j < MLP_H; ++j) d1[j] = 0.0;
    for (int i = 0; i < MLP_H; ++i) {
        gb2[i] += d2[i];
        for (int j = 0; j < MLP_H; ++j) {
            gW2[i * MLP_H + j] += d2[i] * a->h1[j];
            d1[j] += W2[i * MLP_H + j] * d2[i];
        }
    }
    for (int j = 0; j < MLP_H; ++j) {
        d1[j] *= 1.0 - a->h1[j] * a->h1[j];
        gb1[j] += d1[j];
        for (int k = 0; k < 4; ++k) gW1[j * 4 + k] += d1[j] * x[k];
    }
}

/*
 * KL objective of a density model g over the box X = [-1, 1]^4 (volume 16):
 *   L = -(1/nd) sum_d ln g(x_d) + ln( 16 (1/nu) sum_u g(x_u) ),
 * x_d drawn from the target, x_u uniform.  grad = dL/dtheta.  Serial (order fixed).
 */
int or_mlp_loss_grad(const double *th, const double *xd, int64_t nd, const double *xu, int64_t nu,
                     double *loss, double *grad)
{
    memset(grad, 0, MLP_NP * sizeof(double));
    double *gu = (double *)calloc(MLP_NP, sizeof(double));
    double sl = 0.0, su = 0.0;
    for (int64_t e = 0; e < nd; ++e) {
        mlp_act a;
        mlp_fwd(th, xd + 4 * e, &a);
        sl += log(a.g);
        mlp_bwd_add(th, xd + 4 * e, &a, -1.0 / ((double)nd * a.g), grad);
    }
    for (int64_t e = 0; e < nu; ++e) {
        mlp_act a;
        mlp_fwd(th, xu + 4 * e, &a);
        su += a.g;
        mlp_bwd_add(th, xu + 4 * e, &a, 1.0, gu);
    }
    for (int i = 0; i < MLP_NP; ++i) grad[i] += gu[i] / su;
    free(gu);
    *loss = -sl / (double)nd + log(16.0 * su / (double)nu);
    return 0;
}

/* One Adam step (Kingma & Ba, 2015) at step number t >= 1. */
void or_adam_step(double *th, double *m, double *v, const double *grad, int64_t n, double lr,
                  double beta1, double beta2, double eps, int64_t t)
{
    const double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        th[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/*
 * Grid proposal: cells nb[0] x nb[1] x nb[2] x nb[3] over x in [-1, 1]^4 (cell index
 * ((i0 nb1 + i1) nb2 + i2) nb3 + i3), cell values gc >= 0.  Cell probabilities
 * P_c = alpha / ncell + (1 - alpha) gc_c / sum gc, CDF in double (serial sums).
 * Sample i: Philox(counter (i, 0, i >> 32, 0), key seed) gives u0 (cell by CDF
 * search: first c with cdf_c > u0) and u1..u3, a second call (counter (i, 1, ...))
 * gives u4; x_d = lo_d + width_d u_{d+1}.  Map to (m, cK, cpsi, phi):
 * m = m_lo + (m_hi - m_lo)(x0 + 1)/2, cK = x1, cpsi = x2, phi = pi x3, rounded to FP32.
 * Density in the observables q = P_c ncell / 16 * 2 / ((m_hi - m_lo) pi); weight
 * w = p q_ps / q with p q_ps the phase-space density at the FP32 point.
 */
void or_grid_sample(const double *gc, const int *nb, double alpha, uint64_t seed, int64_t n,
                    double m_lo, double m_hi, double mB, double mpsi, double mK, double mpi,
                    float *om, float *ocK, float *ocpsi, float *ophi, double *w, int64_t *cell)
{
    const int64_t nc = (int64_t)nb[0] * nb[1] * nb[2] * nb[3];
    double sg = 0.0;
    for (int64_t c = 0; c < nc; ++c) sg += gc[c];
    double *cdf = (double *)malloc(nc * sizeof(double));
    double acc = 0.0;
    for (int64_t c = 0; c < nc; ++c) {
        acc += alpha / (double)nc + (1.0 - alpha) * gc[c] / sg;
        cdf[c] = acc;
    }
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint32_t c0[4] = {(uint32_t)i, 0u, (uint32_t)((uint64_t)i >> 32), 0u}, r0[4];
        uint32_t c1[4] = {(uint32_t)i, 1u, (uint32_t)((uint64_t)i >> 32), 0u}, r1[4];
        or_philox4x32_10(c0, key, r0);
        or_philox4x32_10(c1, key, r1);
        /* stratified in the CDF: point i takes its cell at u in [i/n, (i+1)/n) of the
           total, so every point is marginally distributed as the proposal while the
           points of one call cover the CDF evenly */
        const double u0 = ((double)i + u01(r0[0])) / (double)n * cdf[nc - 1];
        int64_t lo = 0, hi = nc - 1;
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (cdf[mid] > u0) hi = mid;
            else lo = mid + 1;
        }
        const int64_t c = lo;
        int64_t rem = c;
        int idx[4];
        for (int d = 3; d >= 0; --d) { idx[d] = (int)(rem % nb[d]); rem /= nb[d]; }
        const double us[4] = {u01(r0[1]), u01(r0[2]), u01(r0[3]), u01(r1[0])};
        double x[4];
        for (int d = 0; d < 4; ++d) x[d] = -1.0 + 2.0 * (idx[d] + us[d]) / nb[d];
        float fm = (float)(m_lo + (m_hi - m_lo) * 0.5 * (x[0] + 1.0));
        /* keep the FP32 mass inside the box (the cell density is constant) */
        if ((double)fm > m_hi) fm = nextafterf(fm, 0.0f);
        if ((double)fm < m_lo) fm = nextafterf(fm, 3.0e38f);
        const float fcK = (float)x[1], fcpsi = (float)x[2], fphi = (float)(M_PI * x[3]);
        const double Pc = cdf[c] - (c > 0 ? cdf[c - 1] : 0.0);
        const double q = Pc / cdf[nc - 1] * (double)nc / 16.0 * 2.0 / ((m_hi - m_lo) * M_PI);
        const double p = or_breakup(mB, fm, mpsi), qq = or_breakup(fm, mK, mpi);
        om[i] = fm; ocK[i] = fcK; ocpsi[i] = fcpsi; ophi[i] = fphi;
        w[i] = p * qq / q;
        cell[i] = c;
    }
    free(cdf);
}
