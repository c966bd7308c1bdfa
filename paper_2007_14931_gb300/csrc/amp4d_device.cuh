// Device-side data structures and per-event amplitude arithmetic (FP32).
//
// Event records are structure-of-arrays FP32, one record of npad values per
// quantity; npad is a multiple of 4 so every record is read with float4 loads.
// Parameter-independent kinematics are produced once per event set in FP64
// (kernels in amp4d_prepare.cu) and stored here as FP32.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/amp4d.h"

namespace amp4d {

// Record indices.
enum : int {
    REC_M = 0,     // m_Kpi
    REC_CK = 1,    // cos theta_K*
    REC_CPSI = 2,  // cos theta_J/psi
    REC_PHI = 3,   // phi
    REC_P = 4,     // K pi momentum in the B frame
    REC_Q = 5,     // K momentum in the K pi frame
    REC_CPHI = 6,  // cos phi (FP64 once, stored FP32)
    REC_SPHI = 7,  // sin phi
    REC_NK = 8,    // records of a K*-only model
    REC_MZ = 8,    // m_J/psi pi
    REC_PZ = 9,    // Z momentum in the B frame
    REC_QZ = 10,   // pi momentum in the Z frame
    REC_CZ = 11,   // cos theta_Z
    REC_CTZ = 12,  // cos theta~_J/psi
    REC_CPZ = 13,  // cos phi~
    REC_SPZ = 14,  // sin phi~
    REC_CA = 15,   // cos alpha
    REC_SA = 16,   // sin alpha
    REC_NZ = 17,   // records of a model with a Z
};

// Per-resonance constants of Eq. 2-3 at the current (M, G0), built by
// k_build_table in FP64 at the start of every evaluation.  Every constant that
// scales a whole basis column (the pole barrier factors sqrt(KB KR), m_B^-LB and
// the irrational Wigner-d normalisations) is folded into the column's coupling
// in FP64; the couplings and the constants left inside the per-event FP32
// arithmetic are stored as unevaluated sums hi + lo, so no per-evaluation
// constant carries a systematic FP32 rounding into S.
struct ResDev {
    float Mhi, Mlo;   // pole mass M
    float M2lo;       // M^2 - Mhi^2 = Mlo (2 Mhi + Mlo)
    float r2hi, r2lo; // Blatt-Weisskopf radius squared
    float Ghi, Glo;   // G0 M^2 KR / q0^(2 LR + 1): M Gamma(m) = G q^(2LR+1) / (P_LR(r^2 q^2) m)
    float dNhi, dNlo; // d ln(sqrt(KB KR))/dM, KB = P_LB(r^2 p0^2), KR = P_LR(r^2 q0^2)
    float dGhi, dGlo; // d ln(M Gamma)/dM at fixed m
    float iGhi, iGlo; // 1 / G0
    // Horner pairs for P_J(c) = sum_i a_i c^i (d^J_00) and P_J'(c) = sum_i b_i c^i
    // (d1 = -sin P_J'): hp[0] = (a_4, 0), hp[j] = (a_{4-j}, b_{4-j}) for j = 1..4.
    float2 hp[5];
    // LASS S-wave (Eq. 7-8; shape == AMP4D_SHAPE_LASS): a, a b / 2 and the
    // resonant-term constant R M^2 G0 / q0, each as hi + lo.
    float ahi, alo, chi, clo, RKhi, RKlo;
    int shape;
    int chain, J, LB, LR;
    int col;          // first basis column
    int fpos;         // index among floated resonances, -1 if fixed
    int eta;          // Z: H_{-l} = eta H_{l} (Eq. 11)
    int zcol0;        // Z: column of l' = 0 or -1 when absent
    int zcol1;        // Z: column of l' = +-1 or -1 when absent
};

// Static description of a resonance (internal order: K* first, then Z).
struct ResStatic {
    double M, G0, r;          // model values (replaced by floated parameters)
    double lass_a, lass_b, lass_R;  // AMP4D_SHAPE_LASS constants (Eq. 7-8)
    int chain, J, LB, LR;     // LB = LR = 0 for the LASS S-wave
    int col, fpos, eta, zcol0, zcol1, shape;
};

struct ModelStatic {
    double mB, mpsi, mK, mpi;
    double mix_beta;   // Eq. 14: (1 - P) / B with a background, else 0
    double mistag;     // flavour mistag fraction w
    int n_res, n_col, n_float, n_param;
    ResStatic res[AMP4D_MAX_RES];
};

struct ModelDev {
    int n_res, n_col, n_float, n_param;
    ResDev res[AMP4D_MAX_RES];
    float2 c[3 * AMP4D_MAX_RES];   // folded couplings by column, high part
    float2 cl[3 * AMP4D_MAX_RES];  // folded couplings by column, low part
    // The same couplings by internal resonance, so that a loop unrolled over
    // resonances addresses them at fixed offsets: K* k at kc[k][l + 1] for
    // l = -1, 0, +1 (J = 0: kc[k][1] only); Z z at zc[z][0] (l' = 0) and
    // zc[z][1] (l' = +-1).  Absent columns hold 0.
    ResDev zr[2];                  // the Z resonances, res[n_res - NZ + z]
    float2 kc[AMP4D_MAX_RES][3], kcl[AMP4D_MAX_RES][3];
    float2 zc[2][2], zcl[2][2];
    // The same couplings as pre-broadcast pairs for packed FP32x2 products (see
    // cfma2p): {(h.x, h.x), (-h.y, h.y), (l.x, l.x), (-l.y, l.y)} for h + l = c';
    // the K* l = -1 entry holds -c' (its basis factor is -A d1).
    float2 kp[AMP4D_MAX_RES][3][4];
    float2 zp[2][2][4];
    // Where column k's coupling is copied: K* (t << 2 | slot) or Z (0x100 | z << 2 | slot).
    int col_dst[3 * AMP4D_MAX_RES];
    int static_bad;                // a fixed resonance has no valid pole constants
    // Eq. 14 with a background: alpha = P / I_eps (written each evaluation once
    // I_eps is known) and beta = (1 - P) / B, each hi + lo.
    float mahi, malo, mbhi, mblo;
    // Flavour mistag fraction w (hi + lo) and 1 - w.
    float mwhi, mwlo, m1w;
};

// ----------------------------------------------------------------------------
// Exact, order-independent sums across CTAs: a 128-bit two's-complement
// fixed-point integer per quantity, a[0] = high word (units of 1), a[1] = low
// word (units of 2^-64).  Adding a double x (|x| < 2^62) converts it exactly
// (its fraction has at most 52 significant bits below the binary point that
// matter; smaller contributions than 2^-64 are dropped) and adds it with two
// 64-bit atomics, carrying out of the low word.  Integer addition is
// associative, so the total is the same bits whatever order the CTAs finish in.
// ----------------------------------------------------------------------------
// A value that is not finite or not below 2^62 in magnitude cannot be added; it
// sets status bit 1 (the same domain flag as S <= 0), so it is never dropped
// silently.
__device__ __forceinline__ void acc128_add(unsigned long long *a, double x, unsigned *status)
{
    if (!(fabs(x) < 0x1p62)) {
        atomicOr(status, 1u);
        return;
    }
    const double fl = floor(x);
    const unsigned long long hi = (unsigned long long)(long long)fl;
    const unsigned long long lo = (unsigned long long)((x - fl) * 0x1p64);
    const unsigned long long old = atomicAdd(a + 1, lo);
    const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    atomicAdd(a, hi + carry);
}
// Read with ld.global.cg (L2): the words were written by other CTAs' atomics,
// and a finishing CTA of the same launch must not see a stale L1 line.
__device__ __forceinline__ double acc128_value(const unsigned long long *a)
{
    return (double)(long long)__ldcg(a) + (double)__ldcg(a + 1) * 0x1p-64;
}

// ----------------------------------------------------------------------------
// Complex helpers
// ----------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a += b * c
__device__ __forceinline__ void cfma(float2 &a, float2 b, float2 c)
{
    a.x = fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x));
    a.y = fmaf(b.x, c.y, fmaf(b.y, c.x, a.y));
}
// a += conj(b) * c
__device__ __forceinline__ void cfma_conj(float2 &a, float2 b, float2 c)
{
    a.x = fmaf(b.x, c.x, fmaf(b.y, c.y, a.x));
    a.y = fmaf(b.x, c.y, fmaf(-b.y, c.x, a.y));
}
// a += conj(b c)
__device__ __forceinline__ void cfma_conjp(float2 &a, float2 b, float2 c)
{
    a.x = fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x));
    a.y = fmaf(-b.x, c.y, fmaf(-b.y, c.x, a.y));
}
// a += (hi + lo) * c, with the low part inside the FMA chain of the high-part
// product, so the constant hi + lo is applied before each term is rounded (an
// addition after the rounding would drop it whenever it is below half an ulp):
//   tx = fma(hi.x, c.x, fma(-hi.y, c.y, fma(lo.x, c.x, -lo.y c.y))),
//   ty = fma(hi.x, c.y, fma(hi.y, c.x, fma(lo.x, c.y, lo.y c.x))),  a += t.
// Evaluated with packed FP32x2 operations on pre-broadcast pairs
// q = {(hi.x, hi.x), (-hi.y, hi.y), (lo.x, lo.x), (-lo.y, lo.y)} and the swapped
// factor cs = (c.y, c.x): each component follows the scalar chain above in the
// same order, in half the instructions.
__device__ __forceinline__ void cfma2p(float2 &a, const float2 *q, float2 c, float2 cs)
{
    float2 t = __fmul2_rn(q[3], cs);
    t = __ffma2_rn(q[2], c, t);
    t = __ffma2_rn(q[1], cs, t);
    t = __ffma2_rn(q[0], c, t);
    a = __fadd2_rn(a, t);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// ----------------------------------------------------------------------------
// Barrier polynomial P_L(z) = x^(2L+2) |h_L(x)|^2, z = x^2, by Horner.
// ----------------------------------------------------------------------------
__device__ __forceinline__ float bw_poly(int L, float z)
{
    switch (L) {
    case 0: return 1.0f;
    case 1: return z + 1.0f;
    case 2: return fmaf(z + 3.0f, z, 9.0f);
    case 3: return fmaf(fmaf(z + 6.0f, z, 45.0f), z, 225.0f);
    default: return fmaf(fmaf(fmaf(z + 10.0f, z, 135.0f), z, 1575.0f), z, 11025.0f);
    }
}

__device__ __forceinline__ float ipow(float x, int n)
{
    float r = 1.0f;
    for (int i = 0; i < n; ++i) r *= x;
    return r;
}

// ----------------------------------------------------------------------------
// Wigner d for J <= 4 from the Legendre polynomials, without irrational factors:
//   d0 = d^J_{00}(c) = P_J(c),
//   d1 = -s P_J'(c) = sqrt(J (J+1)) d^J_{10}(c),  d^J_{-1,0} = -d^J_{10}.
// The 1/sqrt(J (J+1)) is folded into the l = +-1 couplings.  Both polynomials
// are evaluated by Horner from the resonance's coefficients, so the same
// instructions serve every J (no branch on the spin).
// ----------------------------------------------------------------------------
// Both polynomials run as one packed Horner chain over cc = (c, c); the P_J'
// lane starts at 0, so its first step returns b_3 exactly.
__device__ __forceinline__ void wigner_l0(const ResDev &r, float2 cc, float s, float &d0, float &d1)
{
    float2 h = r.hp[0];
    h = __ffma2_rn(h, cc, r.hp[1]);
    h = __ffma2_rn(h, cc, r.hp[2]);
    h = __ffma2_rn(h, cc, r.hp[3]);
    h = __ffma2_rn(h, cc, r.hp[4]);
    d0 = h.x;
    d1 = -s * h.y;
}

// d^1_{l xi}(theta) for l in {-1, 0, 1}, xi in {+1 (x=0), -1 (x=1)}; the l = 0
// row is given without its 1/sqrt(2), which is folded into the l = 0 couplings.
__device__ __forceinline__ void wigner_1(float c, float s, float d[3][2])
{
    const float h = 0.5f;
    d[0][0] = h * (1.0f - c); d[0][1] = h * (1.0f + c);   // l = -1
    d[1][0] = s;              d[1][1] = -s;               // l = 0 (times 1/sqrt 2)
    d[2][0] = h * (1.0f + c); d[2][1] = h * (1.0f - c);   // l = +1
}

// ----------------------------------------------------------------------------
// Lineshape of Eq. 2 with Eq. 3 at running mass mrun (momenta p, q), without
// the column constant sqrt(KB KR) m_B^-LB (folded into the couplings):
//   A' = p^LB (q/m)^LR / sqrt(P_LB(z_B) P_LR(z_R)) / (M^2 - m^2 - i M Gamma(m)),
//   M Gamma(m) = G q^(2LR+1) / (P_LR(z_R) m),  z_B = r^2 p^2,  z_R = r^2 q^2.
// Also returns 1/D and M Gamma for the adjoint.
// ----------------------------------------------------------------------------
struct LineOut {
    float2 A;
    float2 invD;   // 1 / D
    float MG;      // M Gamma(m)
};

__device__ __forceinline__ LineOut lineshape(const ResDev &r, float mrun, float invm, float p,
                                             float q)
{
    const float p2 = p * p, q2 = q * q;
    const float PB = bw_poly(r.LB, fmaf(r.r2hi, p2, r.r2lo * p2));
    const float PR = bw_poly(r.LR, fmaf(r.r2hi, q2, r.r2lo * q2));
    const float rs = __frcp_rn(sqrtf(PB * PR));
    const float num = rs * ipow(p, r.LB) * ipow(q * invm, r.LR);
    const float X = ipow(q, 2 * r.LR + 1) * invm * __frcp_rn(PR);
    const float MG = fmaf(r.Ghi, X, r.Glo * X);
    // M^2 - m^2 = (hi - m)(hi + m) + lo (2 hi + lo) for M = hi + lo: (hi - m) is
    // exact near the pole, and the constant lo (2 hi + lo) enters the FMA before
    // its one rounding.  (Adding lo to hi - m first would round at the same
    // offset from the FP32 grid that m and hi share for every event: a
    // systematic error in every lineshape.)
    const float Dr = fmaf(r.Mhi - mrun, r.Mhi + mrun, r.M2lo);
    const float den = __frcp_rn(fmaf(Dr, Dr, MG * MG));
    LineOut o;
    o.invD = make_float2(Dr * den, MG * den);          // 1/(Dr - i MG) = (Dr + i MG)/|D|^2
    o.A = make_float2(num * o.invD.x, num * o.invD.y);
    o.MG = MG;
    return o;
}

// LASS S-wave of Eq. 7-8 from the K0*(1430) Breit-Wigner denominator 1/D of
// lineshape() (built with LB = LR = 0, so M Gamma(m) = (M^2 G0/q0) q/m, Eq. 3 at
// L = 0).  Eq. 8 is taken as a q cot(thB) = v = 1 + (a b/2) q^2 with s = a q:
//   (m/q) sin(thB) e^{i thB} = m a / (v - i s) = (m a)(v + i s) / (v^2 + s^2),
//   e^{2 i thB} = (v + i s) / (v - i s) = ((v^2 - s^2) + 2 i v s) / (v^2 + s^2),
//   A = (m a) w + R (M^2 G0 / q0) e^{2 i thB} / D,   w = 1 / (v - i s).
// Every constant (a, a b/2, R M^2 G0/q0) multiplies inside an FMA with its low
// part as the addend, and the one added constant (1) is exact, so no constant
// leaves a systematic FP32 rounding in A.  Finite at q = 0 (A = m a + R K/D).
__device__ __forceinline__ float2 lass_shape(const ResDev &r, float m, float q, float2 invD)
{
    const float q2 = q * q;
    const float sq = fmaf(r.ahi, q, r.alo * q);
    const float v = 1.0f + fmaf(r.chi, q2, r.clo * q2);
    const float n = __frcp_rn(fmaf(v, v, sq * sq));
    const float ma = fmaf(r.ahi, m, r.alo * m);
    const float2 w = make_float2(v * n, sq * n);
    const float2 e2 = make_float2((v - sq) * (v + sq) * n, 2.0f * v * sq * n);
    const float2 t = make_float2(e2.x * invD.x - e2.y * invD.y, e2.x * invD.y + e2.y * invD.x);
    return make_float2(fmaf(ma, w.x, fmaf(r.RKhi, t.x, r.RKlo * t.x)),
                       fmaf(ma, w.y, fmaf(r.RKhi, t.y, r.RKlo * t.y)));
}

// Lineshape of a K* chain resonance: Eq. 2-3, or the LASS S-wave of Eq. 7-8.
__device__ __forceinline__ float2 kstar_lineshape(const ResDev &r, float mrun, float invm, float p,
                                                  float q)
{
    const LineOut L = lineshape(r, mrun, invm, p, q);
    if (r.shape != AMP4D_SHAPE_LASS) return L.A;
    return lass_shape(r, mrun, q, L.invD);
}

}  // namespace amp4d
