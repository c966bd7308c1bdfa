// Reductions, the final NLL/gradient assembly, the per-evaluation resonance
// table, and the dispatch of the per-event kernels to their instantiations.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "amp4d_device.cuh"
#include "amp4d_launch.h"
#include "amp4d_finish.cuh"

namespace amp4d {

int grad_num_slots(int nk_max, int nz, int n_float) { return 1 + 6 * nk_max + 4 * nz + 2 * n_float; }

// ---------------------------------------------------------------------------
// Deterministic column sums of per-block partials: block j sums column j over
// nblk rows in a fixed order with Neumaier compensation.
// ---------------------------------------------------------------------------
__global__ void k_reduce_cols(const double *__restrict__ part, int nblk, int ncol,
                              double *__restrict__ out)
{
    __shared__ double ss[256], sc[256];
    const int col = blockIdx.x;
    double s = 0.0, c = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 256) {
        const double x = part[(int64_t)b * ncol + col];
        const double t = s + x;
        c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            const double a = ss[threadIdx.x], b = ss[threadIdx.x + h];
            const double t = a + b;
            const double e = (fabs(a) >= fabs(b)) ? (a - t) + b : (b - t) + a;
            ss[threadIdx.x] = t;
            sc[threadIdx.x] += sc[threadIdx.x + h] + e;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[col] = ss[0] + sc[0];
}

// ---------------------------------------------------------------------------
// NLL = -2 [ sum ln S + sum ln(pq) - N ln I ],  I = vol_over_n * sum w S, and
// dNLL = -2 [ sum dS/S - N (vol_over_n sum w dS) / I ] mapped to parameters.
// out: [0] nll, [1] sum ln S, [2] sum ln pq, [3] I, [4] N, [5] status bits
// (1: domain, 2: invalid parameters), [6..] grad.
// ---------------------------------------------------------------------------
// With the Eq. 14 background (ar non-null) the data sum is already sum ln(f / (p q))
// and the signal probabilities' sum R = acc(ar) replaces N:
// NLL = -2 [ sum ln g + sum ln(pq) ], dNLL = -2 [ sum d(ln g) - R dI / I ].
__global__ void k_finish(const unsigned long long *__restrict__ ad, const unsigned long long *__restrict__ an,
                         const int *__restrict__ slot_param, const double *__restrict__ pscale,
                         int nslot, int nparam,
                         double n_events, double lnpq, double vol_over_n,
                         const unsigned *__restrict__ status, double *__restrict__ out,
                         const unsigned long long *__restrict__ ar)
{
    const double rd0 = acc128_value(ad), rn0 = acc128_value(an);
    const double I = vol_over_n * rn0;
    unsigned st = *status;
    const double nll = ar ? -2.0 * (rd0 + lnpq) : -2.0 * (rd0 + lnpq - n_events * log(I));
    const double nI = ar ? acc128_value(ar) : n_events;   // coefficient of dI / I
    if (!(I > 0.0) || !isfinite(nll)) st |= 1u;
    const bool bad = st != 0u;
    if (threadIdx.x == 0) {
        out[0] = bad ? INFINITY : nll;
        out[1] = rd0;
        out[2] = lnpq;
        out[3] = I;
        out[4] = n_events;
        out[5] = (double)st;
    }
    if (slot_param == nullptr) return;
    for (int p = threadIdx.x; p < nparam; p += blockDim.x) out[6 + p] = 0.0;
    __syncthreads();
    for (int s = 1 + threadIdx.x; s < nslot; s += blockDim.x) {
        const int p = slot_param[s];
        if (p >= 0)
            out[6 + p] = bad ? 0.0
                             : -2.0 * pscale[p] *
                                   (acc128_value(ad + 2 * s) - nI * vol_over_n * acc128_value(an + 2 * s) / I);
    }
}

// Eq. 14 with a background: alpha = P / I_eps from the point sum of the pass that
// ran first, into the device table (its hi + lo pair).
__global__ void k_mix_alpha(const unsigned long long *__restrict__ an, double vol_over_n,
                            double purity, ModelDev *__restrict__ md, unsigned *__restrict__ status)
{
    if (threadIdx.x == 0) store_alpha(md, vol_over_n * acc128_value(an), purity, status);
}

// ---------------------------------------------------------------------------
// Shard partials (ln L of the unbinned fit is a sum over events and I a sum over
// points, so a split of both sets is exactly recombined from these sums):
// out: [0] sum ln S, [1] sum ln pq, [2] N, [3] T = V sum w S (I = T / M over the
// union of the shards), [4] M, [5] status bits, [6 .. 6+P) d(sum ln S)/dtheta,
// [6+P .. 6+2P) dT/dtheta.  No logarithm of I is taken here.
// ---------------------------------------------------------------------------
__global__ void k_partials(const unsigned long long *__restrict__ ad, const unsigned long long *__restrict__ an,
                           const int *__restrict__ slot_param, const double *__restrict__ pscale,
                           int nslot, int nparam, double n_events, double lnpq, double n_points,
                           double volume, const unsigned *__restrict__ status,
                           double *__restrict__ out)
{
    if (threadIdx.x == 0) {
        out[0] = acc128_value(ad);
        out[1] = lnpq;
        out[2] = n_events;
        out[3] = volume * acc128_value(an);
        out[4] = n_points;
        out[5] = (double)*status;
    }
    if (slot_param == nullptr) return;
    for (int p = threadIdx.x; p < 2 * nparam; p += blockDim.x) out[6 + p] = 0.0;
    __syncthreads();
    for (int s = 1 + threadIdx.x; s < nslot; s += blockDim.x) {
        const int p = slot_param[s];
        if (p >= 0) {
            out[6 + p] = pscale[p] * acc128_value(ad + 2 * s);
            out[6 + nparam + p] = volume * pscale[p] * acc128_value(an + 2 * s);
        }
    }
}

// ---------------------------------------------------------------------------
// NLL and gradient with the normalisation from the Gram matrix G (cached path):
// with the folded couplings c'_k = kappa_k c_k, u = (Re c', -Im c'), v = (Im c',
// Re c') interleaved, I = vol_over_n (u^T G u + v^T G v) and
// dI/dRe c'_k = 2 vol_over_n ((Gu)_2k + (Gv)_2k+1),
// dI/dIm c'_k = 2 vol_over_n ((Gv)_2k - (Gu)_2k+1).  One block; fixed order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_finish_gram(
    const unsigned long long *__restrict__ ad, const int *__restrict__ slot_param,
    const double *__restrict__ pscale, int nslot, int ncol, int nparam, double n_events,
    double lnpq, double vol_over_n, const double *__restrict__ params, const double *__restrict__ G,
    const unsigned *__restrict__ status, double *__restrict__ out, int with_grad, double n_points,
    int partials, const unsigned long long *__restrict__ ar, ModelDev *__restrict__ alpha_md,
    double purity)
{
    extern __shared__ double sG[];   // dim x dim, then u, v, Gu, Gv (96 each)
    FinishArgs f;
    f.ad = ad; f.slot_param = slot_param; f.pscale = pscale; f.nslot = nslot; f.ncol = ncol;
    f.nparam = nparam; f.n_events = n_events; f.lnpq = lnpq; f.vol_over_n = vol_over_n;
    f.params = params; f.G = G; f.status = status; f.out = out; f.with_grad = with_grad;
    f.n_points = n_points; f.partials = partials; f.ar = ar; f.alpha_md = alpha_md; f.purity = purity;
    finish_gram_body(f, sG);
}

// ---------------------------------------------------------------------------
// Per-evaluation resonance table (Eq. 2-3 constants at the current M, G0), one
// thread per resonance in FP64:
//   p0 = p(M), q0 = q(M) two-body momenta at the pole, KB = P_LB(r^2 p0^2),
//   KR = P_LR(r^2 q0^2), G = G0 M^2 KR / q0^(2LR+1), and the mass derivatives
//   of ln KB, ln KR and ln(M Gamma) for the adjoint.
// Each thread also folds its columns' constants into their couplings (pscale
// keeps them for the gradient) and validates the parameters (status bit 2).
// ---------------------------------------------------------------------------
__device__ double two_body_d(double M, double m1, double m2)
{
    const double a = (M - m1 - m2) * (M + m1 + m2);
    const double b = (M - m1 + m2) * (M + m1 - m2);
    const double l = a * b;
    return l > 0.0 ? sqrt(l) / (2.0 * M) : 0.0;
}

__device__ double bw_poly_d(int L, double z)
{
    switch (L) {
    case 0: return 1.0;
    case 1: return z + 1.0;
    case 2: return (z + 3.0) * z + 9.0;
    case 3: return ((z + 6.0) * z + 45.0) * z + 225.0;
    default: return (((z + 10.0) * z + 135.0) * z + 1575.0) * z + 11025.0;
    }
}

__device__ double bw_poly_deriv_d(int L, double z)
{
    switch (L) {
    case 0: return 0.0;
    case 1: return 1.0;
    case 2: return 2.0 * z + 3.0;
    case 3: return (3.0 * z + 12.0) * z + 45.0;
    default: return ((4.0 * z + 30.0) * z + 270.0) * z + 1575.0;
    }
}

__device__ double powi_d(double x, int n)
{
    double r = 1.0;
    for (int i = 0; i < n; ++i) r *= x;
    return r;
}

__device__ __forceinline__ void split_store(double re, double im, float2 &hi, float2 &lo)
{
    hi = make_float2((float)re, (float)im);
    lo = make_float2((float)(re - (double)hi.x), (float)(im - (double)hi.y));
}

// Pre-broadcast pairs of sg (hi + lo) for cfma2p (sg = +-1, exact).
__device__ __forceinline__ void pack_pairs(float2 hi, float2 lo, float sg, float2 *q)
{
    q[0] = make_float2(sg * hi.x, sg * hi.x);
    q[1] = make_float2(-sg * hi.y, sg * hi.y);
    q[2] = make_float2(sg * lo.x, sg * lo.x);
    q[3] = make_float2(-sg * lo.y, sg * lo.y);
}

__global__ void k_build_table(const ModelStatic *__restrict__ st, const double *__restrict__ params,
                              ModelDev *__restrict__ md, double *__restrict__ pscale,
                              unsigned *__restrict__ status, unsigned long long *__restrict__ acc,
                              int nacc)
{
    const int t = threadIdx.x;
    for (int i = t; i < nacc; i += blockDim.x) acc[i] = 0ull;   // this evaluation's sums
    __shared__ int bad, sbad;   // any invalid input; invalid pole constants of a fixed resonance
    if (t == 0) bad = sbad = 0;
    __syncthreads();
    const int nres = st->n_res, ncol = st->n_col, npar = st->n_param;
    for (int i = t; i < npar; i += blockDim.x) {
        if (!isfinite(params[i])) atomicOr(&bad, 1);
        if (i >= 2 * ncol) pscale[i] = 1.0;
    }
    if (t < nres) {
        const ResStatic &r = st->res[t];
        double M = r.M, G0 = r.G0;
        if (r.fpos >= 0) {
            M = params[2 * ncol + 2 * r.fpos];
            G0 = params[2 * ncol + 2 * r.fpos + 1];
        }
        if (!(M > 0.0) || !(G0 > 0.0)) {
            atomicOr(&bad, 1);
            if (r.fpos < 0) atomicOr(&sbad, 1);
            M = r.M;
            G0 = r.G0;
        }
        const double mB = st->mB;
        double d1, d2, sp;
        if (r.chain == AMP4D_CHAIN_KSTAR) { d1 = st->mK; d2 = st->mpi; sp = st->mpsi; }
        else { d1 = st->mpsi; d2 = st->mpi; sp = st->mK; }
        const double p0 = two_body_d(mB, M, sp), q0 = two_body_d(M, d1, d2);
        if (!(q0 > 0.0)) {
            atomicOr(&bad, 1);
            if (r.fpos < 0) atomicOr(&sbad, 1);
        }
        const double r2 = r.r * r.r;
        const double z0B = r2 * p0 * p0, z0R = r2 * q0 * q0;
        const double KB = bw_poly_d(r.LB, z0B), KR = bw_poly_d(r.LR, z0R);
        const double dp02 = M * (M * M - mB * mB - sp * sp) / (mB * mB);   // d(p0^2)/dM
        const double dd = d1 * d1 - d2 * d2;
        const double dq02 = (M * M * M * M - dd * dd) / (2.0 * M * M * M); // d(q0^2)/dM
        const double dlnKB = bw_poly_deriv_d(r.LB, z0B) / KB * r2 * dp02;
        const double dlnKR = bw_poly_deriv_d(r.LR, z0R) / KR * r2 * dq02;
        const double dlnq0 = 0.5 * dq02 / (q0 * q0);
        const double G = G0 * M * M * KR / powi_d(q0, 2 * r.LR + 1);
        ResDev d;
        d.Mhi = (float)M;
        d.Mlo = (float)(M - (double)d.Mhi);
        d.M2lo = (float)((M - (double)d.Mhi) * ((double)d.Mhi + M));
        d.r2hi = (float)r2;
        d.r2lo = (float)(r2 - (double)d.r2hi);
        d.Ghi = (float)G;
        d.Glo = (float)(G - (double)d.Ghi);
        const double dN = 0.5 * (dlnKB + dlnKR);
        const double dG = 2.0 / M - (2 * r.LR + 1) * dlnq0 + dlnKR;
        const double iG = 1.0 / G0;
        d.dNhi = (float)dN; d.dNlo = (float)(dN - (double)d.dNhi);
        d.dGhi = (float)dG; d.dGlo = (float)(dG - (double)d.dGhi);
        d.iGhi = (float)iG; d.iGlo = (float)(iG - (double)d.iGhi);
        // LASS S-wave (Eq. 7-8): built with LB = LR = 0, so G = M^2 G0 / q0.
        d.shape = r.shape;
        d.ahi = d.alo = d.chi = d.clo = d.RKhi = d.RKlo = 0.f;
        if (r.shape == AMP4D_SHAPE_LASS) {
            const double a = r.lass_a, c = 0.5 * r.lass_a * r.lass_b, RK = r.lass_R * G;
            d.ahi = (float)a; d.alo = (float)(a - (double)d.ahi);
            d.chi = (float)c; d.clo = (float)(c - (double)d.chi);
            d.RKhi = (float)RK; d.RKlo = (float)(RK - (double)d.RKhi);
        }
        // Legendre coefficients of P_J and P_J' (exact in FP32), lowest power first.
        {
            const float P[5][5] = {{1.f, 0.f, 0.f, 0.f, 0.f},
                                   {0.f, 1.f, 0.f, 0.f, 0.f},
                                   {-0.5f, 0.f, 1.5f, 0.f, 0.f},
                                   {0.f, -1.5f, 0.f, 2.5f, 0.f},
                                   {0.375f, 0.f, -3.75f, 0.f, 4.375f}};
            const int J = r.J < 0 ? 0 : (r.J > 4 ? 4 : r.J);
            d.hp[0] = make_float2(P[J][4], 0.f);
            for (int j = 1; j < 5; ++j)
                d.hp[j] = make_float2(P[J][4 - j], (float)(5 - j) * P[J][5 - j]);
        }
        d.chain = r.chain;
        d.J = r.J;
        d.LB = r.LB;
        d.LR = r.LR;
        d.col = r.col;
        d.fpos = r.fpos;
        d.eta = r.eta;
        d.zcol0 = r.zcol0;
        d.zcol1 = r.zcol1;
        md->res[t] = d;
        int zi = -1;   // index among the Z resonances (internal order: K* first)
        if (r.chain == AMP4D_CHAIN_Z) {
            zi = 0;
            for (int i = 0; i < t; ++i) zi += st->res[i].chain == AMP4D_CHAIN_Z ? 1 : 0;
            md->zr[zi] = d;
            for (int j = 0; j < 2; ++j) {
                md->zc[zi][j] = md->zcl[zi][j] = make_float2(0.f, 0.f);
                for (int i = 0; i < 4; ++i) md->zp[zi][j][i] = make_float2(0.f, 0.f);
            }
        } else {
            for (int j = 0; j < 3; ++j) {
                md->kc[t][j] = md->kcl[t][j] = make_float2(0.f, 0.f);
                for (int i = 0; i < 4; ++i) md->kp[t][j][i] = make_float2(0.f, 0.f);
            }
        }
        // Column constants: sqrt(KB KR) m_B^-LB times 1/sqrt(2) for the l = 0 J/psi
        // factor d^1_{0 xi}, or 1/sqrt(J (J+1)) for the l = +-1 factor d^J_{+-1 0}.
        const double base = sqrt(KB * KR) / powi_d(mB, r.LB);
        const double k0 = base * 0.70710678118654752440;
        const double k1 = r.J > 0 ? base / sqrt((double)(r.J * (r.J + 1))) : 0.0;
        int cols[3], ncols = 0;
        double kap[3];
        if (r.chain == AMP4D_CHAIN_KSTAR) {
            if (r.J == 0) { cols[0] = r.col; kap[0] = k0; ncols = 1; }
            else {
                cols[0] = r.col; kap[0] = k1;
                cols[1] = r.col + 1; kap[1] = k0;
                cols[2] = r.col + 2; kap[2] = k1;
                ncols = 3;
            }
        } else {
            if (r.zcol0 >= 0) { cols[ncols] = r.zcol0; kap[ncols++] = k0; }
            if (r.zcol1 >= 0) { cols[ncols] = r.zcol1; kap[ncols++] = k1; }
        }
        for (int j = 0; j < ncols; ++j) {
            const int k = cols[j];
            split_store(params[2 * k] * kap[j], params[2 * k + 1] * kap[j], md->c[k], md->cl[k]);
            if (zi < 0) {
                const int sl = r.J == 0 ? 1 : j;
                md->kc[t][sl] = md->c[k];
                md->kcl[t][sl] = md->cl[k];
                pack_pairs(md->c[k], md->cl[k], sl == 0 ? -1.f : 1.f, md->kp[t][sl]);
                md->col_dst[k] = (t << 2) | sl;
            } else {
                const int sl = k == r.zcol0 ? 0 : 1;
                md->zc[zi][sl] = md->c[k];
                md->zcl[zi][sl] = md->cl[k];
                pack_pairs(md->c[k], md->cl[k], 1.f, md->zp[zi][sl]);
                md->col_dst[k] = 0x100 | (zi << 2) | sl;
            }
            pscale[2 * k] = kap[j];
            pscale[2 * k + 1] = kap[j];
        }
    }
    if (t == 0) {
        md->n_res = nres;
        md->n_col = ncol;
        md->n_float = st->n_float;
        md->n_param = npar;
        md->mahi = md->malo = 0.f;   // alpha: written once I_eps is known
        md->mbhi = (float)st->mix_beta;
        md->mblo = (float)(st->mix_beta - (double)md->mbhi);
        md->mwhi = (float)st->mistag;
        md->mwlo = (float)(st->mistag - (double)md->mwhi);
        md->m1w = (float)(1.0 - st->mistag);
    }
    __syncthreads();
    if (t == 0) {
        md->static_bad = sbad;
        *status = bad ? 2u : 0u;
    }
}

// Per-evaluation update when no mass or width floats: every pole constant and
// column constant kappa_k (kept in pscale) is unchanged since the last full
// build, so only the folded couplings c'_k = kappa_k c_k are rewritten, in the
// same FP64 arithmetic as k_build_table (identical bits).
__global__ void k_update_couplings(const ModelStatic *__restrict__ st, const double *__restrict__ params,
                                   ModelDev *__restrict__ md, const double *__restrict__ pscale,
                                   unsigned *__restrict__ status, unsigned long long *__restrict__ acc,
                                   int nacc)
{
    const int t = threadIdx.x;
    for (int i = t; i < nacc; i += blockDim.x) acc[i] = 0ull;   // this evaluation's sums
    __shared__ int bad;
    if (t == 0) bad = 0;
    __syncthreads();
    const int ncol = st->n_col, npar = st->n_param;
    for (int i = t; i < npar; i += blockDim.x)
        if (!isfinite(params[i])) atomicOr(&bad, 1);
    for (int k = t; k < ncol; k += blockDim.x) {
        const double kap = pscale[2 * k];
        float2 hi, lo;
        split_store(params[2 * k] * kap, params[2 * k + 1] * kap, hi, lo);
        md->c[k] = hi;
        md->cl[k] = lo;
        const int dst = md->col_dst[k], sl = dst & 3;
        if (dst & 0x100) {
            md->zc[(dst >> 2) & 3][sl] = hi;
            md->zcl[(dst >> 2) & 3][sl] = lo;
            pack_pairs(hi, lo, 1.f, md->zp[(dst >> 2) & 3][sl]);
        } else {
            md->kc[dst >> 2][sl] = hi;
            md->kcl[dst >> 2][sl] = lo;
            pack_pairs(hi, lo, sl == 0 ? -1.f : 1.f, md->kp[dst >> 2][sl]);
        }
    }
    __syncthreads();
    if (t == 0) *status = (bad || md->static_bad) ? 2u : 0u;
}

// ---------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------
template <int NK> cudaError_t launch_eval_nk(const LaunchArgs &a, int mode);
template <int NK> cudaError_t launch_grad_nk(const LaunchArgs &a, bool norm);
template <int NK> cudaError_t launch_lcache_nk(const LaunchArgs &a, float2 *lc);
extern template cudaError_t launch_lcache_nk<2>(const LaunchArgs &, float2 *);
extern template cudaError_t launch_lcache_nk<10>(const LaunchArgs &, float2 *);
extern template cudaError_t launch_lcache_nk<16>(const LaunchArgs &, float2 *);
extern template cudaError_t launch_eval_nk<2>(const LaunchArgs &, int);
extern template cudaError_t launch_eval_nk<10>(const LaunchArgs &, int);
extern template cudaError_t launch_eval_nk<16>(const LaunchArgs &, int);
extern template cudaError_t launch_grad_nk<2>(const LaunchArgs &, bool);
extern template cudaError_t launch_grad_nk<10>(const LaunchArgs &, bool);
extern template cudaError_t launch_grad_nk<16>(const LaunchArgs &, bool);

int nk_bucket(int nk)
{
    if (nk <= 2) return 2;
    if (nk <= 10) return 10;
    return 16;
}

cudaError_t launch_eval(const LaunchArgs &a, int mode)
{
    switch (a.nk_max) {
    case 2: return launch_eval_nk<2>(a, mode);
    case 10: return launch_eval_nk<10>(a, mode);
    case 16: return launch_eval_nk<16>(a, mode);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_grad(const LaunchArgs &a, bool norm)
{
    switch (a.nk_max) {
    case 2: return launch_grad_nk<2>(a, norm);
    case 10: return launch_grad_nk<10>(a, norm);
    case 16: return launch_grad_nk<16>(a, norm);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_lcache(const LaunchArgs &a, float2 *lc)
{
    switch (a.nk_max) {
    case 2: return launch_lcache_nk<2>(a, lc);
    case 10: return launch_lcache_nk<10>(a, lc);
    case 16: return launch_lcache_nk<16>(a, lc);
    default: return cudaErrorInvalidValue;
    }
}

// PDF of Eq. 5 with the phase-space density: P(e) = S(e) p(e) q(e) / I, in
// place over S (FP32, n events).
// PDF per data event from S: p q [alpha eps S + beta hb] (Eq. 14; alpha = P / I,
// eps = 1 and beta = 0 without templates), in FP64 and rounded once.
__global__ void k_pdf_scale(const float *__restrict__ rec, int64_t npad, int64_t n, double alpha,
                            double beta, const float *__restrict__ eps, const float *__restrict__ hb,
                            float *__restrict__ S)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        double g = alpha * (eps ? (double)eps[e] : 1.0) * (double)S[e];
        if (hb) g += beta * (double)hb[e];
        S[e] = (float)((double)rec[REC_P * npad + e] * (double)rec[REC_Q * npad + e] * g);
    }
}

// Eq. 14 density without the phase-space factor, for the generator: S <- alpha eps S
// + beta hb (hb null: beta = 0), in FP64 and rounded once.
__global__ void k_eq14_density(float *__restrict__ S, const float *__restrict__ eps,
                               const float *__restrict__ hb, int64_t n, double alpha, double beta)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        double g = alpha * (double)eps[e] * (double)S[e];
        if (hb) g += beta * (double)hb[e];
        S[e] = (float)g;
    }
}

cudaError_t launch_eq14_density(float *S, const float *eps, const float *hb, int64_t n, double alpha,
                                double beta, cudaStream_t s)
{
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_eq14_density<<<(int)std::max<int64_t>(1, blocks), 256, 0, s>>>(S, eps, hb, n, alpha, beta);
    return cudaGetLastError();
}

cudaError_t launch_pdf_scale(const float *rec, int64_t npad, int64_t n, double alpha, double beta,
                             const float *eps, const float *hb, float *S, cudaStream_t s)
{
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_pdf_scale<<<(int)std::max<int64_t>(1, blocks), 256, 0, s>>>(rec, npad, n, alpha, beta, eps,
                                                                    hb, S);
    return cudaGetLastError();
}

cudaError_t launch_reduce_cols(const double *part, int nblk, int ncol, double *out,
                               cudaStream_t s)
{
    k_reduce_cols<<<ncol, 256, 0, s>>>(part, nblk, ncol, out);
    return cudaGetLastError();
}

cudaError_t launch_finish(const unsigned long long *ad, const unsigned long long *an, const int *slot_param,
                          const double *pscale, int nslot, int nparam, double n_events,
                          double lnpq, double vol_over_n, const unsigned *status, double *out,
                          cudaStream_t s, const unsigned long long *ar)
{
    k_finish<<<1, 128, 0, s>>>(ad, an, slot_param, pscale, nslot, nparam, n_events, lnpq,
                               vol_over_n, status, out, ar);
    return cudaGetLastError();
}

cudaError_t launch_mix_alpha(const unsigned long long *an, double vol_over_n, double purity,
                             ModelDev *md, unsigned *status, cudaStream_t s)
{
    k_mix_alpha<<<1, 32, 0, s>>>(an, vol_over_n, purity, md, status);
    return cudaGetLastError();
}

cudaError_t launch_finish_gram(const unsigned long long *ad, const int *slot_param, const double *pscale,
                               int nslot, int ncol, int nparam, double n_events, double lnpq,
                               double vol_over_n, const double *params, const double *G,
                               const unsigned *status, double *out, int with_grad, cudaStream_t s,
                               double n_points, int partials, const unsigned long long *ar,
                               ModelDev *alpha_md, double purity)
{
    const size_t smem = finish_gram_smem(ncol);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_finish_gram, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_finish_gram<<<1, 256, smem, s>>>(ad, slot_param, pscale, nslot, ncol, nparam, n_events, lnpq,
                                       vol_over_n, params, G, status, out, with_grad, n_points,
                                       partials, ar, alpha_md, purity);
    return cudaGetLastError();
}

cudaError_t launch_partials(const unsigned long long *ad, const unsigned long long *an, const int *slot_param,
                            const double *pscale, int nslot, int nparam, double n_events,
                            double lnpq, double n_points, double volume, const unsigned *status,
                            double *out, cudaStream_t s)
{
    k_partials<<<1, 128, 0, s>>>(ad, an, slot_param, pscale, nslot, nparam, n_events, lnpq,
                                 n_points, volume, status, out);
    return cudaGetLastError();
}

cudaError_t launch_build_table(const ModelStatic *st, const double *params, ModelDev *md,
                               double *pscale, unsigned *status, cudaStream_t s,
                               bool couplings_only, unsigned long long *acc, int nacc)
{
    if (couplings_only)
        k_update_couplings<<<1, 64, 0, s>>>(st, params, md, pscale, status, acc, nacc);
    else
        k_build_table<<<1, 64, 0, s>>>(st, params, md, pscale, status, acc, nacc);
    return cudaGetLastError();
}

int eval_block() { return 256; }
int grad_block() { return 128; }

}  // namespace amp4d
