// The evaluation's closing step on the Gram path (one CTA, any block size):
// I = (V/N)(u^T G u + v^T G v) from the Gram matrix G and the folded couplings,
// -2 ln L and its gradient from the 128-bit sums of the data pass.  Used by the
// standalone finishing kernel and by the last CTA of the data kernel.
#pragma once

#include "amp4d_device.cuh"
#include "amp4d_launch.h"

namespace amp4d {

__device__ __forceinline__ void store_alpha(ModelDev *md, double I, double purity, unsigned *status)
{
    double a = 0.0;
    if (I > 0.0 && isfinite(I)) a = purity / I;
    else atomicOr(status, 1u);
    md->mahi = (float)a;
    md->malo = (float)(a - (double)md->mahi);
}

// Shared memory the body needs: (4 ncol^2 + 4 x 96 + 2) doubles.
__host__ __device__ constexpr size_t finish_gram_smem(int ncol) { return ((size_t)4 * ncol * ncol + 4 * 96 + 2) * sizeof(double); }

// (G x)_i by a group of 8 lanes (lane8 = 0..7): lane-strided FMA chains in a
// fixed order, then xor shuffles within the group.  Every lane of the warp
// calls it (active = false contributes 0).  The standalone finish and the rows
// that the data kernel's CTAs compute for the fused finish use this same order,
// so both give the same bits.
__device__ __forceinline__ double gram_row8(const double *G, int dim, const double *x, int i, int lane8,
                                            bool active)
{
    double a = 0.0;
    if (active)
        for (int j = lane8; j < dim; j += 8) a = fma(G[i * dim + j], x[j], a);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

// Component j of u = (Re c', -Im c') (which = 0) or v = (Im c', Re c') (which = 1)
// for the folded couplings c'_k = pscale_k c_k.
__device__ __forceinline__ double coupling_vec(const double *pscale, const double *params, int j, int which)
{
    const int k = j >> 1;
    const double re = pscale[2 * k] * params[2 * k], im = pscale[2 * k] * params[2 * k + 1];
    return which == 0 ? ((j & 1) ? -im : re) : ((j & 1) ? re : im);
}

// Rows 4 b .. 4 b + 3 of the stacked [G u; G v] (2 dim rows) into guv, by warp 0 of
// CTA b (b < dim / 2): the fused finish reads them instead of recomputing G u.
__device__ __forceinline__ void gram_rows_for_finish(const FinishArgs &f, int b)
{
    const int dim = 2 * f.ncol, lane = threadIdx.x & 31, g = lane >> 3, lane8 = lane & 7;
    const int r = 4 * b + g;
    const bool active = r < 2 * dim;
    const int which = active ? r / dim : 0, i = active ? r % dim : 0;
    double x[8];   // the lane's components j = lane8 + 8 t (dim <= 64)
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int j = lane8 + 8 * t;
        x[t] = (active && j < dim) ? coupling_vec(f.pscale, f.params, j, which) : 0.0;
    }
    double a = 0.0;
    if (active) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int j = lane8 + 8 * t;
            if (j < dim) a = fma(f.G[i * dim + j], x[t], a);
        }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (active && lane8 == 0) f.guv[r] = a;
}

__device__ __forceinline__ void finish_gram_body(const FinishArgs &f, double *sG)
{
    const unsigned long long *__restrict__ ad = f.ad;
    const int *__restrict__ slot_param = f.slot_param;
    const double *__restrict__ pscale = f.pscale;
    const int nslot = f.nslot, ncol = f.ncol, nparam = f.nparam, with_grad = f.with_grad,
              partials = f.partials;
    const double n_events = f.n_events, lnpq = f.lnpq, vol_over_n = f.vol_over_n,
                 n_points = f.n_points, purity = f.purity;
    const double *__restrict__ params = f.params;
    const double *__restrict__ G = f.G;
    const unsigned *__restrict__ status = f.status;
    double *__restrict__ out = f.out;
    const unsigned long long *__restrict__ ar = f.ar;
    ModelDev *__restrict__ alpha_md = f.alpha_md;
    // shared: G (dim x dim), then u, v, Gu, Gv and two scalars
    double *u = sG + 4 * ncol * ncol, *v = u + 96, *Gu = v + 96, *Gv = Gu + 96;
    double &qsh = Gv[96], &Ish = Gv[97];
    const int dim = 2 * ncol, t = threadIdx.x;
    for (int j = t; j < dim; j += blockDim.x) {
        u[j] = coupling_vec(pscale, params, j, 0);
        v[j] = coupling_vec(pscale, params, j, 1);
    }
    if (f.guv) {
        // fused into the data kernel: its CTAs computed the rows of G u and G v
        for (int i = t; i < dim; i += blockDim.x) {
            Gu[i] = __ldcg(f.guv + i);
            Gv[i] = __ldcg(f.guv + dim + i);
        }
        __syncthreads();
    } else {
        for (int i = t; i < dim * dim; i += blockDim.x) sG[i] = G[i];
        __syncthreads();
        // (Gu)_i and (Gv)_i: 8 lanes per row (gram_row8); the loop count is uniform
        // across the block.
        const int lane8 = t & 7, rows_per_pass = blockDim.x >> 3;
        for (int base = 0; base < dim; base += rows_per_pass) {
            const int i = base + (t >> 3);
            const double a = gram_row8(sG, dim, u, i, lane8, i < dim);
            const double b = gram_row8(sG, dim, v, i, lane8, i < dim);
            if (i < dim && lane8 == 0) { Gu[i] = a; Gv[i] = b; }
        }
        __syncthreads();
    }
    if (t < 32) {
        double q = 0.0;
        for (int i = t; i < dim; i += 32) q = fma(u[i], Gu[i], fma(v[i], Gv[i], q));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if (t == 0) qsh = q;
    }
    __syncthreads();
    const double q = qsh;
    if (alpha_md) {   // Eq. 14 with a background: only alpha = P / I_eps, before the data pass
        if (t == 0) store_alpha(alpha_md, vol_over_n * q, purity, const_cast<unsigned *>(status));
        return;
    }
    if (partials) {
        // Shard partials (layout of k_partials) with T = V (u^T G u + v^T G v).
        const double volume = vol_over_n * n_points;
        if (t == 0) {
            out[0] = acc128_value(ad);
            out[1] = lnpq;
            out[2] = n_events;
            out[3] = volume * q;
            out[4] = n_points;
            out[5] = (double)*status;
        }
        if (!with_grad) return;
        for (int p = t; p < 2 * nparam; p += blockDim.x) out[6 + p] = 0.0;
        __syncthreads();
        for (int s = 1 + t; s < nslot; s += blockDim.x) {
            const int p = slot_param[s];
            if (p < 0) continue;
            out[6 + p] = pscale[p] * acc128_value(ad + 2 * s);
            if (p < dim) {
                const int k = p >> 1;
                const double dq = (p & 1) ? 2.0 * (Gv[2 * k] - Gu[2 * k + 1])
                                          : 2.0 * (Gu[2 * k] + Gv[2 * k + 1]);
                out[6 + nparam + p] = volume * pscale[p] * dq;
            }
        }
        return;
    }
    if (t == 0) {
        const double I = vol_over_n * q;
        unsigned st = *status;
        const double rd0 = acc128_value(ad);
        const double nll = ar ? -2.0 * (rd0 + lnpq) : -2.0 * (rd0 + lnpq - n_events * log(I));
        if (!(I > 0.0) || !isfinite(nll)) st |= 1u;
        out[0] = st ? INFINITY : nll;
        out[1] = rd0;
        out[2] = lnpq;
        out[3] = I;
        out[4] = n_events;
        out[5] = (double)st;
        Ish = st ? 0.0 : I;
    }
    if (!with_grad) return;
    __syncthreads();
    const double Iv = Ish;
    const double nI = ar ? acc128_value(ar) : n_events;   // coefficient of dI / I
    for (int p = t; p < nparam; p += blockDim.x) out[6 + p] = 0.0;
    __syncthreads();
    for (int s = 1 + t; s < nslot; s += blockDim.x) {
        const int p = slot_param[s];
        if (p < 0 || p >= dim || Iv == 0.0) continue;
        const int k = p >> 1;
        const double dq = (p & 1) ? 2.0 * (Gv[2 * k] - Gu[2 * k + 1]) : 2.0 * (Gu[2 * k] + Gv[2 * k + 1]);
        out[6 + p] = -2.0 * pscale[p] * (acc128_value(ad + 2 * s) - nI * vol_over_n * dq / Iv);
    }
}

}  // namespace amp4d
