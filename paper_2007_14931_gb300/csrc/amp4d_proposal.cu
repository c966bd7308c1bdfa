// Pseudo-data generation and the learned importance-sampling proposal.
//
// Generator (Fit validation section: events generated from the model by MC):
// accept-reject over the uniform box.  Candidate i takes its coordinates from
// Philox4x32-10 (Salmon et al., SC'11) with counter (i, 0, i >> 32, 0) and key =
// seed, its acceptance uniform from counter (i, 1, ...); f_max is 1.5 x the
// largest S p q over 2^20 scan candidates (counter stream 2), doubled and the
// draw restarted if any candidate exceeds it.  Accepted events keep candidate
// order (per-block counts, an exclusive scan, in-order scatter): deterministic.
//
// Proposal: an MLP 4 -> 64 -> 64 -> 1 (tanh hidden units, softplus output g >= 0)
// over x in [-1, 1]^4 (x0 = 2 (m - m_lo)/(m_hi - m_lo) - 1, x1 = cos theta_K*,
// x2 = cos theta_psi, x3 = phi / pi) is trained by Adam on the KL objective
//     L = -mean_data ln g(x) + ln(16 mean_uniform g(x)),
// with BF16 weights (an FP32 master copy) and FP32 accumulation.  It is then
// evaluated at the centres of a cell grid; the defensive mixture
//     P_c = alpha / ncell + (1 - alpha) g_c / sum g
// is cumulated in FP64, and points are drawn cell-by-CDF, uniformly inside the
// cell, with exact weights w = p q / q(Phi) so that I = (1/N) sum w S.
#include <cmath>
#include <cstdint>
#include <cuda_bf16.h>

#include "amp4d_device.cuh"
#include "amp4d_launch.h"
#include "amp4d_mlp.cuh"

namespace amp4d {

// ---------------------------------------------------------------------------
// Philox4x32-10
// ---------------------------------------------------------------------------
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[1] = (uint32_t)p1;
        c[3] = (uint32_t)p0;
        c[0] = n0;
        c[2] = n2;
    }
}

__device__ __forceinline__ double u01d(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

__device__ __forceinline__ void philox_stream(uint64_t i, uint32_t stream, uint64_t seed, uint32_t out[4])
{
    out[0] = (uint32_t)i;
    out[1] = stream;
    out[2] = (uint32_t)(i >> 32);
    out[3] = 0u;
    philox4x32_10(out, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// ---------------------------------------------------------------------------
// Generator
// ---------------------------------------------------------------------------
__global__ void k_gen_candidates(float *__restrict__ rec, int64_t npad, int64_t n, uint64_t first,
                                 uint32_t stream, uint64_t seed, double m_lo, double m_hi,
                                 float *__restrict__ uacc)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t r[4];
        philox_stream(first + e, stream, seed, r);
        rec[REC_M * npad + e] = (float)(m_lo + (m_hi - m_lo) * u01d(r[0]));
        rec[REC_CK * npad + e] = (float)(2.0 * u01d(r[1]) - 1.0);
        rec[REC_CPSI * npad + e] = (float)(2.0 * u01d(r[2]) - 1.0);
        rec[REC_PHI * npad + e] = (float)(M_PI * (2.0 * u01d(r[3]) - 1.0));
        if (uacc) {
            uint32_t r2[4];
            philox_stream(first + e, stream + 1u, seed, r2);
            uacc[e] = (float)u01d(r2[0]);
        }
    }
}

// f = S p q per candidate; flags = u f_max < f; block counts; over = any f > f_max.
constexpr int GEN_BLOCK = 256;
constexpr int GEN_PER_THREAD = 4;
constexpr int GEN_TILE = GEN_BLOCK * GEN_PER_THREAD;

__global__ void k_gen_accept(const float *__restrict__ rec, int64_t npad, int64_t n,
                             const float *__restrict__ S, const float *__restrict__ uacc, double fmax,
                             unsigned *__restrict__ blk_count, unsigned *__restrict__ over,
                             unsigned *__restrict__ fmax_bits)
{
    __shared__ unsigned cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    unsigned local = 0;
    for (int j = 0; j < GEN_PER_THREAD; ++j) {
        const int64_t e = (int64_t)blockIdx.x * GEN_TILE + j * GEN_BLOCK + threadIdx.x;
        if (e >= n) break;
        const float f = S[e] * rec[REC_P * npad + e] * rec[REC_Q * npad + e];
        if (fmax_bits) atomicMax(fmax_bits, __float_as_uint(fmaxf(f, 0.0f)));
        if (uacc) {
            if ((double)f > fmax) atomicOr(over, 1u);
            if ((double)uacc[e] * fmax < (double)f) ++local;
        }
    }
    if (local) atomicAdd(&cnt, local);
    __syncthreads();
    if (threadIdx.x == 0) blk_count[blockIdx.x] = cnt;
}

// Exclusive scan of block counts (single block, sequential chunks per thread).
__global__ void k_scan_counts(const unsigned *__restrict__ cnt, int nb, unsigned long long *__restrict__ off)
{
    __shared__ unsigned long long part[1024];
    const int t = threadIdx.x, per = (nb + 1023) / 1024;
    unsigned long long s = 0;
    for (int i = t * per; i < min(nb, (t + 1) * per); ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        unsigned long long acc = 0;
        for (int i = 0; i < 1024; ++i) {
            const unsigned long long v = part[i];
            part[i] = acc;
            acc += v;
        }
        off[nb] = acc;
    }
    __syncthreads();
    unsigned long long acc = part[t];
    for (int i = t * per; i < min(nb, (t + 1) * per); ++i) {
        off[i] = acc;
        acc += cnt[i];
    }
}

// In-order scatter of accepted candidates (block-local order by candidate index).
__global__ void k_gen_scatter(const float *__restrict__ rec, int64_t npad, int64_t n,
                              const float *__restrict__ S, const float *__restrict__ uacc, double fmax,
                              const unsigned long long *__restrict__ off, int64_t base, int64_t n_want,
                              float *__restrict__ om, float *__restrict__ ocK,
                              float *__restrict__ ocpsi, float *__restrict__ ophi)
{
    __shared__ unsigned flags[GEN_TILE];
    __shared__ unsigned pos[GEN_TILE];
    for (int j = 0; j < GEN_PER_THREAD; ++j) {
        const int l = j * GEN_BLOCK + threadIdx.x;
        const int64_t e = (int64_t)blockIdx.x * GEN_TILE + l;
        unsigned a = 0;
        if (e < n) {
            const float f = S[e] * rec[REC_P * npad + e] * rec[REC_Q * npad + e];
            a = ((double)uacc[e] * fmax < (double)f) ? 1u : 0u;
        }
        flags[l] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int l = 0; l < GEN_TILE; ++l) {
            pos[l] = acc;
            acc += flags[l];
        }
    }
    __syncthreads();
    for (int j = 0; j < GEN_PER_THREAD; ++j) {
        const int l = j * GEN_BLOCK + threadIdx.x;
        if (!flags[l]) continue;
        const int64_t e = (int64_t)blockIdx.x * GEN_TILE + l;
        const int64_t o = base + (int64_t)off[blockIdx.x] + pos[l];
        if (o >= n_want) continue;
        om[o] = rec[REC_M * npad + e];
        ocK[o] = rec[REC_CK * npad + e];
        ocpsi[o] = rec[REC_CPSI * npad + e];
        ophi[o] = rec[REC_PHI * npad + e];
    }
}

cudaError_t launch_gen_candidates(float *rec, int64_t npad, int64_t n, uint64_t first,
                                  uint32_t stream_id, uint64_t seed, double m_lo, double m_hi,
                                  float *uacc, cudaStream_t st)
{
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_gen_candidates<<<grid, 256, 0, st>>>(rec, npad, n, first, stream_id, seed, m_lo, m_hi, uacc);
    return cudaGetLastError();
}

int gen_tile() { return GEN_TILE; }

cudaError_t launch_gen_accept(const float *rec, int64_t npad, int64_t n, const float *S,
                              const float *uacc, double fmax, unsigned *blk_count, unsigned *over,
                              unsigned *fmax_bits, cudaStream_t st)
{
    const int nb = (int)((n + GEN_TILE - 1) / GEN_TILE);
    k_gen_accept<<<nb, GEN_BLOCK, 0, st>>>(rec, npad, n, S, uacc, fmax, blk_count, over, fmax_bits);
    return cudaGetLastError();
}

cudaError_t launch_gen_scatter(const float *rec, int64_t npad, int64_t n, const float *S,
                               const float *uacc, double fmax, const unsigned *blk_count,
                               unsigned long long *off, int64_t base, int64_t n_want, float *om,
                               float *ocK, float *ocpsi, float *ophi, cudaStream_t st)
{
    const int nb = (int)((n + GEN_TILE - 1) / GEN_TILE);
    k_scan_counts<<<1, 1024, 0, st>>>(blk_count, nb, off);
    k_gen_scatter<<<nb, GEN_BLOCK, 0, st>>>(rec, npad, n, S, uacc, fmax, off, base, n_want, om, ocK,
                                           ocpsi, ophi);
    return cudaGetLastError();
}

// The MLP kernels (forward, grid, KL gradient) are in amp4d_mlp.cu.

// One Adam step on the FP32 master weights, refreshing the BF16 copy.
__global__ void k_adam(float *__restrict__ th, float *__restrict__ m, float *__restrict__ v,
                       const double *__restrict__ grad, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2, __nv_bfloat16 *__restrict__ wb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = (float)grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float t = th[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    th[i] = t;
    wb[i] = __float2bfloat16_rn(t);
}

__global__ void k_to_bf16(const float *__restrict__ th, int n, __nv_bfloat16 *__restrict__ wb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16_rn(th[i]);
}

// Training batch: data rows picked by Philox (stream 3) from the event set,
// uniform rows from stream 4; both mapped to [-1, 1]^4.
__global__ void k_mlp_batch(const float *__restrict__ em, const float *__restrict__ ecK,
                            const float *__restrict__ ecpsi, const float *__restrict__ ephi, int64_t n,
                            int64_t nd, int64_t nu, uint64_t seed, uint64_t step, double m_lo,
                            double m_hi, float *__restrict__ xd, float *__restrict__ xu)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nd) {
        uint32_t r[4];
        philox_stream(step * (uint64_t)(nd + nu) + i, 3u, seed, r);
        const int64_t e = (int64_t)(((uint64_t)r[0] | ((uint64_t)r[1] << 32)) % (uint64_t)n);
        xd[4 * i] = (float)(2.0 * ((double)em[e] - m_lo) / (m_hi - m_lo) - 1.0);
        xd[4 * i + 1] = ecK[e];
        xd[4 * i + 2] = ecpsi[e];
        xd[4 * i + 3] = (float)((double)ephi[e] / M_PI);
    } else if (i < nd + nu) {
        uint32_t r[4];
        philox_stream(step * (uint64_t)(nd + nu) + i, 4u, seed, r);
        const int64_t j = i - nd;
        for (int k = 0; k < 4; ++k) xu[4 * j + k] = (float)(2.0 * u01d(r[k]) - 1.0);
    }
}

// ---------------------------------------------------------------------------
// Grid proposal: FP64 CDF of the mixture and sampling.
// ---------------------------------------------------------------------------
constexpr int CDF_BLOCK = 1024;

// Per-block sums of g (FP64) for the normalisation of the grid density.
__global__ void k_block_sum(const float *__restrict__ g, int64_t n, double *__restrict__ bs)
{
    __shared__ double s[CDF_BLOCK];
    const int64_t i = blockIdx.x * (int64_t)CDF_BLOCK + threadIdx.x;
    s[threadIdx.x] = i < n ? (double)g[i] : 0.0;
    __syncthreads();
    for (int h = CDF_BLOCK / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) bs[blockIdx.x] = s[0];
}

// Exclusive prefix of the block sums and the total (single thread; nb is small).
__global__ void k_prefix_small(const double *__restrict__ bs, int nb, double *__restrict__ pre)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double acc = 0.0;
    for (int i = 0; i < nb; ++i) {
        pre[i] = acc;
        acc += bs[i];
    }
    pre[nb] = acc;
}

// cdf[c] = sum_{c' <= c} P_c', P_c = alpha / ncell + (1 - alpha) g_c / sum g.
__global__ void k_cdf(const float *__restrict__ g, int64_t n, const double *__restrict__ gpre,
                      double alpha, double *__restrict__ cdf)
{
    __shared__ double s[CDF_BLOCK];
    const int64_t i = blockIdx.x * (int64_t)CDF_BLOCK + threadIdx.x;
    const double sg = gpre[gridDim.x];
    s[threadIdx.x] = i < n ? (double)g[i] : 0.0;
    __syncthreads();
    for (int off = 1; off < CDF_BLOCK; off <<= 1) {  // inclusive Hillis-Steele scan
        const double v = threadIdx.x >= off ? s[threadIdx.x - off] : 0.0;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    if (i < n) cdf[i] = alpha * (double)(i + 1) / (double)n + (1.0 - alpha) * (gpre[blockIdx.x] + s[threadIdx.x]) / sg;
}

__global__ void k_grid_sample(const double *__restrict__ cdf, int nb0, int nb1, int nb2, int nb3,
                              uint64_t seed, int64_t n, double m_lo, double m_hi, double mB,
                              double mpsi, double mK, double mpi, float *__restrict__ om,
                              float *__restrict__ ocK, float *__restrict__ ocpsi,
                              float *__restrict__ ophi, float *__restrict__ w,
                              int64_t *__restrict__ cell)
{
    const int64_t nc = (int64_t)nb0 * nb1 * nb2 * nb3;
    const double total = cdf[nc - 1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t r0[4], r1[4];
        philox_stream((uint64_t)i, 0u, seed, r0);
        philox_stream((uint64_t)i, 1u, seed, r1);
        // Stratified in the CDF: point i takes u in [i/n, (i + 1)/n) of the total.
        // Each point is marginally drawn from the proposal (the weights stay exact),
        // and a call's points cover the CDF evenly: the estimate of I keeps only the
        // variation of S p q / q inside each stratum (about one cell), not the
        // fluctuation of how many points land in each region.
        const double u0 = ((double)i + u01d(r0[0])) / (double)n * total;
        int64_t lo = 0, hi = nc - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cdf[mid] > u0) hi = mid;
            else lo = mid + 1;
        }
        const int64_t c = lo;
        int64_t rem = c;
        const int i3 = (int)(rem % nb3); rem /= nb3;
        const int i2 = (int)(rem % nb2); rem /= nb2;
        const int i1 = (int)(rem % nb1); rem /= nb1;
        const int i0 = (int)rem;
        const double x0 = -1.0 + 2.0 * (i0 + u01d(r0[1])) / nb0;
        const double x1 = -1.0 + 2.0 * (i1 + u01d(r0[2])) / nb1;
        const double x2 = -1.0 + 2.0 * (i2 + u01d(r0[3])) / nb2;
        const double x3 = -1.0 + 2.0 * (i3 + u01d(r1[0])) / nb3;
        float fm = (float)(m_lo + (m_hi - m_lo) * 0.5 * (x0 + 1.0));
        // the FP32 rounding may step just outside the box: take the nearest FP32
        // value inside (q is constant over the cell, so the weight is unchanged)
        if ((double)fm > m_hi) fm = nextafterf(fm, 0.0f);
        if ((double)fm < m_lo) fm = nextafterf(fm, 3.0e38f);
        const double Pc = cdf[c] - (c > 0 ? cdf[c - 1] : 0.0);
        const double q = Pc / total * (double)nc / 16.0 * 2.0 / ((m_hi - m_lo) * M_PI);
        const double mm = (double)fm;
        auto two_body = [](double M, double m1, double m2) {
            const double a = (M - m1 - m2) * (M + m1 + m2), b = (M - m1 + m2) * (M + m1 - m2);
            const double l = a * b;
            return l > 0.0 ? sqrt(l) / (2.0 * M) : 0.0;
        };
        const double pq = two_body(mB, mm, mpsi) * two_body(mm, mK, mpi);
        om[i] = fm;
        ocK[i] = (float)x1;
        ocpsi[i] = (float)x2;
        ophi[i] = (float)(M_PI * x3);
        w[i] = (float)(pq / q);
        if (cell) cell[i] = c;
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_adam(float *th, float *m, float *v, const double *grad, float lr, float b1,
                        float b2, float eps, int64_t t, __nv_bfloat16 *wb, cudaStream_t st)
{
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)t));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)t));
    k_adam<<<(MLP_P + 255) / 256, 256, 0, st>>>(th, m, v, grad, MLP_P, lr, b1, b2, eps, c1, c2, wb);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float *th, __nv_bfloat16 *wb, cudaStream_t st)
{
    k_to_bf16<<<(MLP_P + 255) / 256, 256, 0, st>>>(th, MLP_P, wb);
    return cudaGetLastError();
}

cudaError_t launch_mlp_batch(const float *em, const float *ecK, const float *ecpsi, const float *ephi,
                             int64_t n, int64_t nd, int64_t nu, uint64_t seed, uint64_t step,
                             double m_lo, double m_hi, float *xd, float *xu, cudaStream_t st)
{
    k_mlp_batch<<<(int)((nd + nu + 255) / 256), 256, 0, st>>>(em, ecK, ecpsi, ephi, n, nd, nu, seed,
                                                             step, m_lo, m_hi, xd, xu);
    return cudaGetLastError();
}

int64_t cdf_scratch(int64_t ncell) { return (ncell + CDF_BLOCK - 1) / CDF_BLOCK + 1; }

cudaError_t launch_grid_cdf(const float *g, int64_t ncell, double alpha, double *scratch,
                            double *cdf, cudaStream_t st)
{
    const int nb = (int)((ncell + CDF_BLOCK - 1) / CDF_BLOCK);
    double *bs = scratch, *pre = scratch + nb + 1;
    k_block_sum<<<nb, CDF_BLOCK, 0, st>>>(g, ncell, bs);
    k_prefix_small<<<1, 32, 0, st>>>(bs, nb, pre);
    k_cdf<<<nb, CDF_BLOCK, 0, st>>>(g, ncell, pre, alpha, cdf);
    return cudaGetLastError();
}

cudaError_t launch_grid_sample(const double *cdf, const int nb[4], uint64_t seed, int64_t n,
                               double m_lo, double m_hi, double mB, double mpsi, double mK,
                               double mpi, float *om, float *ocK, float *ocpsi, float *ophi, float *w,
                               int64_t *cell, cudaStream_t st)
{
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
    k_grid_sample<<<grid, 256, 0, st>>>(cdf, nb[0], nb[1], nb[2], nb[3], seed, n, m_lo, m_hi, mB, mpsi,
                                        mK, mpi, om, ocK, ocpsi, ophi, w, cell);
    return cudaGetLastError();
}

}  // namespace amp4d

namespace amp4d {

// Glorot-uniform initial weights from a host Philox stream (stream 5); biases 0,
// b3 = ln(e - 1) so that g starts near 1.
void mlp_init_params(float *th, uint64_t seed)
{
    auto uni = [&](uint64_t i) {
        uint32_t c[4] = {(uint32_t)i, 5u, (uint32_t)(i >> 32), 0u};
        philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        return ((double)c[0] + 0.5) * (1.0 / 4294967296.0) * 2.0 - 1.0;
    };
    for (int i = 0; i < MLP_P; ++i) th[i] = 0.0f;
    const double a1 = std::sqrt(6.0 / (4 + MH)), a2 = std::sqrt(6.0 / (2 * MH)), a3 = std::sqrt(6.0 / (MH + 1));
    for (int i = 0; i < MH * 4; ++i) th[i] = (float)(a1 * uni(i));
    for (int i = 0; i < MH * MH; ++i) th[OFF_W2 + i] = (float)(a2 * uni(1000 + i));
    for (int i = 0; i < MH; ++i) th[OFF_W3 + i] = (float)(a3 * uni(10000 + i));
    th[OFF_B3] = (float)std::log(std::exp(1.0) - 1.0);
}

}  // namespace amp4d
