// The learned-proposal MLP on the tensor cores: forward (points and grid cell
// centres) and the gradient of the KL training objective, with warp-level
// mma.sync.m16n8k16 BF16 x BF16 -> FP32.
//
// Network: x in [-1, 1]^4 -> h1 = tanh(W1 x + b1) (64) -> h2 = tanh(W2 h1 + b2)
// (64) -> o = W3 . h2 + b3 -> g = softplus(o).  The 64 x 64 layer is the dense
// contraction: per tile of points it is a [points x 64] x [64 x 64] product
// forward, and two more of that shape backward (delta2 W2 and the weight
// gradient delta2^T h1).  Layer 1 (K = 4) and layer 3 (N = 1) stay on the FP32
// pipe.
//
// Precision.  The network is defined by its BF16 weights, which enter the MMAs
// exactly.  Activations and deltas are FP32 and enter as sums of BF16 terms:
// x = x_hi + x_mid + x_lo (three terms: the residual is below 2^-24 |x|) for the
// forward contraction, two terms (residual below 2^-17 |x|) for the backward
// ones.  Every BF16 x BF16 product is exact in the FP32 accumulator, so the
// forward result is the FP32 network on the BF16 weights up to the order of the
// FP32 sums.
//
// Fragment layout (PTX ISA, mma.m16n8k16 with .bf16 operands): lane = 4 g + t.
//   A (16 x 16, row = point): a0 = (g, 2t..2t+1), a1 = (g+8, 2t..2t+1),
//                             a2 = (g, 2t+8..2t+9), a3 = (g+8, 2t+8..2t+9);
//   B (16 x 8, k x n):        b0 = (2t..2t+1, g), b1 = (2t+8..2t+9, g);
//   C/D (16 x 8, FP32):       d0, d1 = (g, 2t..2t+1), d2, d3 = (g+8, 2t..2t+1);
// the lower 16 bits of a register hold the element with the smaller k.  A warp
// takes 16 points; lane (g, t) holds points g and g + 8.  The accumulator of
// n-tiles 2c and 2c + 1 of one layer is, element for element, the A fragment of
// k-chunk c of the next contraction, so activations stay in registers between
// layers; layer 1 computes its outputs directly in that layout.
#include <algorithm>
#include <cstdint>
#include <cuda_bf16.h>

#include "amp4d_launch.h"
#include "amp4d_mlp.cuh"

namespace amp4d {

namespace {

constexpr int WP = 72;          // staged row pitch in BF16 (144 B): ldmatrix rows and
constexpr int WPW = WP / 2;     // the 32-bit fragment loads are bank-conflict free
constexpr int MLP_WARPS = 4;
constexpr int MLP_THREADS = 32 * MLP_WARPS;
constexpr int MLP_TILE = 16 * MLP_WARPS;         // points per CTA tile (gradient kernel)
static_assert(MLP_TILE == MLP_GRAD_TILE, "tile of the gradient kernel");
constexpr int MLP_SETS_CTAS = 2 * 152;           // at most this many CTAs per point set

// Weights in shared memory: FP32 vectors (layer 1, biases, layer 3), then W2
// (row = output unit) and, for the gradient kernel, W2 transposed, both BF16
// with pitch WP.
struct WOff {
    static constexpr int W1 = 0, B1 = W1 + MH * 4, B2 = B1 + MH, W3 = B2 + MH, B3 = W3 + MH;
    static constexpr int NF = 452;                       // floats, 16-byte multiple
    static constexpr int W2_BYTES = NF * 4;
    static constexpr int W2T_BYTES = W2_BYTES + MH * WP * 2;
    static constexpr int FWD_BYTES = W2T_BYTES;          // forward kernels stop here
    static constexpr int GRAD_W_BYTES = W2T_BYTES + MH * WP * 2;
};

__device__ __forceinline__ float softplus_f(float o) { return o > 20.0f ? o : log1pf(expf(o)); }
__device__ __forceinline__ float sigmoid_f(float o) { return 1.0f / (1.0f + expf(-o)); }

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v)
{
    return *reinterpret_cast<uint32_t *>(&v);
}

// (x0, x1) as NT BF16 pair terms, largest first; x0 in the low half.  Each
// residual x - bf16(x) is exact in FP32.
template <int NT>
__device__ __forceinline__ void split2(float x0, float x1, uint32_t (&o)[NT])
{
#pragma unroll
    for (int s = 0; s < NT; ++s) {
        const __nv_bfloat162 v = __floats2bfloat162_rn(x0, x1);
        o[s] = bf2_bits(v);
        const float2 f = __bfloat1622float2(v);
        x0 -= f.x;
        x1 -= f.y;
    }
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
        "{%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}

__device__ __forceinline__ void ldsm_x2_t(uint32_t &r0, uint32_t &r1, const void *p)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];\n"
                 : "=r"(r0), "=r"(r1)
                 : "r"(s));
}

// Weights from the BF16 parameter vector into shared memory (block-wide).
__device__ __forceinline__ void load_mlp_weights(const __nv_bfloat16 *__restrict__ wb, unsigned char *sm,
                                                 bool transposed)
{
    float *wf = reinterpret_cast<float *>(sm);
    __nv_bfloat16 *w2 = reinterpret_cast<__nv_bfloat16 *>(sm + WOff::W2_BYTES);
    __nv_bfloat16 *w2t = reinterpret_cast<__nv_bfloat16 *>(sm + WOff::W2T_BYTES);
    for (int i = threadIdx.x; i < MH * 4 + MH; i += blockDim.x) wf[WOff::W1 + i] = __bfloat162float(wb[i]);
    for (int i = threadIdx.x; i < MH; i += blockDim.x) {
        wf[WOff::B2 + i] = __bfloat162float(wb[OFF_B2 + i]);
        wf[WOff::W3 + i] = __bfloat162float(wb[OFF_W3 + i]);
    }
    if (threadIdx.x == 0) wf[WOff::B3] = __bfloat162float(wb[OFF_B3]);
    for (int e = threadIdx.x; e < MH * MH; e += blockDim.x) {
        const int i = e / MH, j = e % MH;
        const __nv_bfloat16 v = wb[OFF_W2 + e];
        w2[i * WP + j] = v;
        if (transposed) w2t[j * WP + i] = v;
    }
    __syncthreads();
}

// Warp forward of 16 points.  x[r][k]: the lane's points g (r = 0) and g + 8
// (r = 1).  Outputs: h1 in the A-fragment layout, h1[c][h][r][e] = unit
// 16 c + 8 h + 2 t + e of point r; z2 accumulators / h2 in the D layout,
// h2[u][2 r + e] = unit 8 u + 2 t + e of point r; o[r] on every lane of the group.
struct FwdState {
    float h1[4][2][2][2];
    float h2[8][4];
    float o[2];
};

__device__ __forceinline__ void mlp_forward_warp(const unsigned char *sm, const float (&x)[2][4], FwdState &s)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float *wf = reinterpret_cast<const float *>(sm);
    const uint32_t *w2 = reinterpret_cast<const uint32_t *>(sm + WOff::W2_BYTES);
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int j = 16 * c + 8 * h + 2 * t + e;
                const float4 w = *reinterpret_cast<const float4 *>(wf + WOff::W1 + 4 * j);
                const float b = wf[WOff::B1 + j];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    float z = fmaf(w.x, x[r][0], b);
                    z = fmaf(w.y, x[r][1], z);
                    z = fmaf(w.z, x[r][2], z);
                    z = fmaf(w.w, x[r][3], z);
                    s.h1[c][h][r][e] = tanhf(z);
                }
            }
    float acc[8][4];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[u][q] = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t a0[3], a1[3], a2[3], a3[3];
        split2<3>(s.h1[c][0][0][0], s.h1[c][0][0][1], a0);
        split2<3>(s.h1[c][0][1][0], s.h1[c][0][1][1], a1);
        split2<3>(s.h1[c][1][0][0], s.h1[c][1][0][1], a2);
        split2<3>(s.h1[c][1][1][0], s.h1[c][1][1][1], a3);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t b0 = w2[(8 * u + g) * WPW + 8 * c + t], b1 = w2[(8 * u + g) * WPW + 8 * c + t + 4];
#pragma unroll
            for (int q = 2; q >= 0; --q) {     // smallest term first
                const uint32_t a[4] = {a0[q], a1[q], a2[q], a3[q]};
                mma_bf16(acc[u], a, b0, b1);
            }
        }
    }
    float o0 = 0.0f, o1 = 0.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int i = 8 * u + 2 * t + e;
            const float b = wf[WOff::B2 + i], w3 = wf[WOff::W3 + i];
            s.h2[u][e] = tanhf(acc[u][e] + b);
            s.h2[u][2 + e] = tanhf(acc[u][2 + e] + b);
            o0 = fmaf(w3, s.h2[u][e], o0);
            o1 = fmaf(w3, s.h2[u][2 + e], o1);
        }
    o0 += __shfl_xor_sync(0xffffffffu, o0, 1);
    o0 += __shfl_xor_sync(0xffffffffu, o0, 2);
    o1 += __shfl_xor_sync(0xffffffffu, o1, 1);
    o1 += __shfl_xor_sync(0xffffffffu, o1, 2);
    s.o[0] = o0 + wf[WOff::B3];
    s.o[1] = o1 + wf[WOff::B3];
}

// g(x) for n points x (n x 4, row-major in [-1, 1]^4), 16 points per warp.
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_forward(const __nv_bfloat16 *__restrict__ wb,
                                                             const float *__restrict__ x, int64_t n,
                                                             float *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char sm[];
    load_mlp_weights(wb, sm, false);
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t nt = (n + 15) / 16;
    for (int64_t tile = blockIdx.x * (int64_t)MLP_WARPS + (threadIdx.x >> 5); tile < nt;
         tile += (int64_t)gridDim.x * MLP_WARPS) {
        float xv[2][4];
        int64_t p[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            p[r] = tile * 16 + g + 8 * r;
#pragma unroll
            for (int k = 0; k < 4; ++k) xv[r][k] = p[r] < n ? x[4 * p[r] + k] : 0.0f;
        }
        FwdState s;
        mlp_forward_warp(sm, xv, s);
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (t == 0 && p[r] < n) out[p[r]] = softplus_f(s.o[r]);
    }
}

// Cell-centre values of the grid: cell c = ((i0 nb1 + i1) nb2 + i2) nb3 + i3.
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_grid(const __nv_bfloat16 *__restrict__ wb, int nb0,
                                                          int nb1, int nb2, int nb3, float *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char sm[];
    load_mlp_weights(wb, sm, false);
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t nc = (int64_t)nb0 * nb1 * nb2 * nb3;
    const int64_t nt = (nc + 15) / 16;
    for (int64_t tile = blockIdx.x * (int64_t)MLP_WARPS + (threadIdx.x >> 5); tile < nt;
         tile += (int64_t)gridDim.x * MLP_WARPS) {
        float xv[2][4];
        int64_t c[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            c[r] = tile * 16 + g + 8 * r;
            int64_t rem = c[r] < nc ? c[r] : 0;
            const int i3 = (int)(rem % nb3); rem /= nb3;
            const int i2 = (int)(rem % nb2); rem /= nb2;
            const int i1 = (int)(rem % nb1); rem /= nb1;
            const int i0 = (int)rem;
            xv[r][0] = -1.0f + (2.0f * i0 + 1.0f) / nb0;
            xv[r][1] = -1.0f + (2.0f * i1 + 1.0f) / nb1;
            xv[r][2] = -1.0f + (2.0f * i2 + 1.0f) / nb2;
            xv[r][3] = -1.0f + (2.0f * i3 + 1.0f) / nb3;
        }
        FwdState s;
        mlp_forward_warp(sm, xv, s);
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (t == 0 && c[r] < nc) out[c[r]] = softplus_f(s.o[r]);
    }
}

// Shared memory of the gradient kernel after the weights: the tile's staged
// operands of the weight-gradient contractions, each as BF16 hi and lo parts
// with pitch WP: h1 (and a ones column at 64: the b2 gradient), delta2,
// delta1, and x with a ones column at 4 (the b1 gradient, pitch 8); then the
// per-warp sums of the W3 and b3 gradients and of the loss terms.
struct GOff {
    static constexpr int MAT = MLP_TILE * WP * 2;
    static constexpr int H1H = WOff::GRAD_W_BYTES, H1L = H1H + MAT;
    static constexpr int D2H = H1L + MAT, D2L = D2H + MAT;
    static constexpr int D1H = D2L + MAT, D1L = D1H + MAT;
    static constexpr int XH = D1L + MAT, XL = XH + MLP_TILE * 16;
    static constexpr int RED = XL + MLP_TILE * 16;
    static constexpr int RW = 68;                       // floats per warp: W3 (64), b3, loss
    static constexpr int BYTES = RED + MLP_WARPS * RW * 4;
};

// Gradient of the KL objective.  CTAs [0, nbd) take the data rows, the rest the
// uniform rows, in tiles of MLP_TILE points (16 per warp).  Per point: forward,
// dO = coef sigmoid(o) (coef = -1/(nd g) for data, 1 for uniform points), delta2
// = dO W3 (1 - h2^2), delta1 = (delta2 W2) (1 - h1^2); per tile the weight
// gradients delta2^T [h1 | 1] and delta1^T [x | 1] on the tensor cores, in FP32
// accumulators that persist over the CTA's tiles.  part[b][0..4544] = the CTA's
// gradient contribution, part[b][4545] = its sum of ln g (data) or of g.
__global__ void __launch_bounds__(MLP_THREADS, 1) k_mlp_grad(const __nv_bfloat16 *__restrict__ wb,
                                                             const float *__restrict__ xd, int64_t nd,
                                                             const float *__restrict__ xu, int64_t nu,
                                                             int nbd, float *__restrict__ part)
{
    extern __shared__ __align__(16) unsigned char sm[];
    load_mlp_weights(wb, sm, true);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const bool data = (int)blockIdx.x < nbd;
    const int64_t np = data ? nd : nu;
    const float *__restrict__ xs = data ? xd : xu;
    const int cta = data ? (int)blockIdx.x : (int)blockIdx.x - nbd;
    const int ncta = data ? nbd : (int)gridDim.x - nbd;
    const float *wf = reinterpret_cast<const float *>(sm);
    const uint32_t *w2t = reinterpret_cast<const uint32_t *>(sm + WOff::W2T_BYTES);
    uint32_t *h1h = reinterpret_cast<uint32_t *>(sm + GOff::H1H), *h1l = reinterpret_cast<uint32_t *>(sm + GOff::H1L);
    uint32_t *d2h = reinterpret_cast<uint32_t *>(sm + GOff::D2H), *d2l = reinterpret_cast<uint32_t *>(sm + GOff::D2L);
    uint32_t *d1h = reinterpret_cast<uint32_t *>(sm + GOff::D1H), *d1l = reinterpret_cast<uint32_t *>(sm + GOff::D1L);
    uint32_t *xh = reinterpret_cast<uint32_t *>(sm + GOff::XH), *xl = reinterpret_cast<uint32_t *>(sm + GOff::XL);
    float gw2[9][4], gw1[4], w3a[8][2];
#pragma unroll
    for (int v = 0; v < 9; ++v)
#pragma unroll
        for (int q = 0; q < 4; ++q) gw2[v][q] = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) gw1[q] = 0.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u) w3a[u][0] = w3a[u][1] = 0.0f;
    float b3a = 0.0f, lsum = 0.0f;
    const float inv_nd = 1.0f / (float)nd;
    const int row0 = 16 * warp + g;            // staged row of the lane's point r: row0 + 8 r
    const int64_t ntile = (np + MLP_TILE - 1) / MLP_TILE;
    for (int64_t tile = cta; tile < ntile; tile += ncta) {
        float xv[2][4];
        bool valid[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int64_t p = tile * MLP_TILE + row0 + 8 * r;
            valid[r] = p < np;
#pragma unroll
            for (int k = 0; k < 4; ++k) xv[r][k] = valid[r] ? xs[4 * p + k] : 0.0f;
            // x and its ones column (word t of the row: (x0, x1), (x2, x3), (1, 0), (0, 0)),
            // and the ones column of h1 (words 32..35: (1, 0), 0, 0, 0)
            const int row = row0 + 8 * r;
            const float e0 = t == 0 ? xv[r][0] : t == 1 ? xv[r][2] : t == 2 ? 1.0f : 0.0f;
            const float e1 = t == 0 ? xv[r][1] : t == 1 ? xv[r][3] : 0.0f;
            uint32_t sx[2];
            split2<2>(e0, e1, sx);
            xh[row * 4 + t] = sx[0];
            xl[row * 4 + t] = sx[1];
            h1h[row * WPW + 32 + t] = t == 0 ? bf2_bits(__floats2bfloat162_rn(1.0f, 0.0f)) : 0u;
            h1l[row * WPW + 32 + t] = 0u;
        }
        FwdState s;
        mlp_forward_warp(sm, xv, s);
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    uint32_t sh[2];
                    split2<2>(s.h1[c][h][r][0], s.h1[c][h][r][1], sh);
                    const int w = (row0 + 8 * r) * WPW + 8 * c + 4 * h + t;
                    h1h[w] = sh[0];
                    h1l[w] = sh[1];
                }
        float dO[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            dO[r] = 0.0f;
            if (valid[r]) {
                const float gv = softplus_f(s.o[r]);
                if (t == 0) lsum += data ? logf(gv) : gv;
                dO[r] = (data ? -inv_nd / gv : 1.0f) * sigmoid_f(s.o[r]);
            }
        }
        if (t == 0) b3a += dO[0] + dO[1];
        float d2[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float w3 = wf[WOff::W3 + 8 * u + 2 * t + e];
                const float ha = s.h2[u][e], hb = s.h2[u][2 + e];
                w3a[u][e] = fmaf(dO[0], ha, fmaf(dO[1], hb, w3a[u][e]));
                d2[u][e] = dO[0] * w3 * fmaf(-ha, ha, 1.0f);
                d2[u][2 + e] = dO[1] * w3 * fmaf(-hb, hb, 1.0f);
            }
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                uint32_t sd[2];
                split2<2>(d2[u][2 * r], d2[u][2 * r + 1], sd);
                const int w = (row0 + 8 * r) * WPW + 4 * u + t;
                d2h[w] = sd[0];
                d2l[w] = sd[1];
            }
        // delta1' = delta2 W2: K = output unit i, N = input unit j, B[i][j] = W2T[j][i]
        float a1[8][4];
#pragma unroll
        for (int v = 0; v < 8; ++v)
#pragma unroll
            for (int q = 0; q < 4; ++q) a1[v][q] = 0.0f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint32_t A0[2], A1[2], A2[2], A3[2];
            split2<2>(d2[2 * c][0], d2[2 * c][1], A0);
            split2<2>(d2[2 * c][2], d2[2 * c][3], A1);
            split2<2>(d2[2 * c + 1][0], d2[2 * c + 1][1], A2);
            split2<2>(d2[2 * c + 1][2], d2[2 * c + 1][3], A3);
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const uint32_t b0 = w2t[(8 * v + g) * WPW + 8 * c + t];
                const uint32_t b1 = w2t[(8 * v + g) * WPW + 8 * c + t + 4];
#pragma unroll
                for (int q = 1; q >= 0; --q) {
                    const uint32_t a[4] = {A0[q], A1[q], A2[q], A3[q]};
                    mma_bf16(a1[v], a, b0, b1);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < 8; ++v)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float ha = s.h1[v >> 1][v & 1][r][0], hb = s.h1[v >> 1][v & 1][r][1];
                uint32_t sd[2];
                split2<2>(a1[v][2 * r] * fmaf(-ha, ha, 1.0f), a1[v][2 * r + 1] * fmaf(-hb, hb, 1.0f), sd);
                const int w = (row0 + 8 * r) * WPW + 4 * v + t;
                d1h[w] = sd[0];
                d1l[w] = sd[1];
            }
        __syncthreads();
        // Weight gradients of the tile; warp w takes output rows 16 w .. 16 w + 15.
        // A = delta^T from the [point][unit] staging (ldmatrix .trans); B = [h1 | 1]
        // or [x | 1] from their [point][column] staging (.trans).  hi x hi + hi x lo +
        // lo x hi per product.
        const int q = lane >> 3, rr = lane & 7;
        const unsigned char *bh1h = sm + GOff::H1H, *bh1l = sm + GOff::H1L;
        const unsigned char *bd2h = sm + GOff::D2H, *bd2l = sm + GOff::D2L;
        const unsigned char *bd1h = sm + GOff::D1H, *bd1l = sm + GOff::D1L;
        const unsigned char *bxh = sm + GOff::XH, *bxl = sm + GOff::XL;
#pragma unroll
        for (int ks = 0; ks < MLP_TILE / 16; ++ks) {
            const int arow = 16 * ks + (q >> 1) * 8 + rr, acol = 16 * warp + (q & 1) * 8;
            const int brow = 16 * ks + (q & 1) * 8 + rr;
            uint32_t Ah[4], Al[4];
            ldsm_x4_t(Ah, bd2h + (arow * WP + acol) * 2);
            ldsm_x4_t(Al, bd2l + (arow * WP + acol) * 2);
#pragma unroll
            for (int vp = 0; vp < 4; ++vp) {
                const int bcol = 8 * (2 * vp + (q >> 1));
                uint32_t Bh[4], Bl[4];
                ldsm_x4_t(Bh, bh1h + (brow * WP + bcol) * 2);
                ldsm_x4_t(Bl, bh1l + (brow * WP + bcol) * 2);
                mma_bf16(gw2[2 * vp], Al, Bh[0], Bh[1]);
                mma_bf16(gw2[2 * vp], Ah, Bl[0], Bl[1]);
                mma_bf16(gw2[2 * vp], Ah, Bh[0], Bh[1]);
                mma_bf16(gw2[2 * vp + 1], Al, Bh[2], Bh[3]);
                mma_bf16(gw2[2 * vp + 1], Ah, Bl[2], Bl[3]);
                mma_bf16(gw2[2 * vp + 1], Ah, Bh[2], Bh[3]);
            }
            {   // columns 64..71: the ones column (exact in the hi part, lo = 0)
                uint32_t b0, b1;
                ldsm_x2_t(b0, b1, bh1h + (brow * WP + 64) * 2);
                mma_bf16(gw2[8], Al, b0, b1);
                mma_bf16(gw2[8], Ah, b0, b1);
            }
            ldsm_x4_t(Ah, bd1h + (arow * WP + acol) * 2);
            ldsm_x4_t(Al, bd1l + (arow * WP + acol) * 2);
            uint32_t xb0, xb1, xl0, xl1;
            ldsm_x2_t(xb0, xb1, bxh + brow * 16);
            ldsm_x2_t(xl0, xl1, bxl + brow * 16);
            mma_bf16(gw1, Al, xb0, xb1);
            mma_bf16(gw1, Ah, xl0, xl1);
            mma_bf16(gw1, Ah, xb0, xb1);
        }
        __syncthreads();
    }
    // W3, b3 and the loss terms: over the lanes of equal t, then over the warps.
    float *red = reinterpret_cast<float *>(sm + GOff::RED);
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float v = w3a[u][e];
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            if (g == 0) red[warp * GOff::RW + 8 * u + 2 * t + e] = v;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        b3a += __shfl_xor_sync(0xffffffffu, b3a, o);
        lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    }
    if (lane == 0) {
        red[warp * GOff::RW + 64] = b3a;
        red[warp * GOff::RW + 65] = lsum;
    }
    __syncthreads();
    float *out = part + (int64_t)blockIdx.x * (MLP_P + 1);
    for (int i = threadIdx.x; i < 66; i += MLP_THREADS) {
        float sum = 0.0f;
        for (int w = 0; w < MLP_WARPS; ++w) sum += red[w * GOff::RW + i];
        out[i < 64 ? OFF_W3 + i : (i == 64 ? OFF_B3 : MLP_P)] = sum;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int i = 16 * warp + g + 8 * (e >> 1), n = 2 * t + (e & 1);
#pragma unroll
        for (int v = 0; v < 8; ++v) out[OFF_W2 + i * MH + 8 * v + n] = gw2[v][e];
        if (n == 0) out[OFF_B2 + i] = gw2[8][e];
        if (n < 4) out[i * 4 + n] = gw1[e];
        else if (n == 4) out[OFF_B1 + i] = gw1[e];
    }
}

// grad = sum over data blocks + (sum over uniform blocks) / S_u; loss terms.
// out: grad[MLP_P] (FP64), then [MLP_P] = loss.  CTA b takes the 32 parameters
// 32 b .. 32 b + 31 (lane = parameter, coalesced rows); its 8 warps sum every
// 8th partial row in FP64 and the warps' sums are added in a fixed order, so
// the result does not depend on timing.  Every CTA forms S_u itself from the
// uniform blocks' last column (one warp, shuffle reduction); CTA 0 writes the loss.
constexpr int FIN_WARPS = 8;
__global__ void __launch_bounds__(32 * FIN_WARPS) k_mlp_grad_finish(const float *__restrict__ part, int nblk_d,
                                                                   int nblk_u, int64_t nd, int64_t nu,
                                                                   double *__restrict__ out)
{
    __shared__ double sa[FIN_WARPS][32], sb[FIN_WARPS][32];
    __shared__ double su_sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.x * 32 + lane;
    if (warp == 0) {
        double su = 0.0, sl = 0.0;
        for (int b = lane; b < nblk_u; b += 32) su += part[(int64_t)(nblk_d + b) * (MLP_P + 1) + MLP_P];
        for (int b = lane; b < nblk_d; b += 32) sl += part[(int64_t)b * (MLP_P + 1) + MLP_P];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            su += __shfl_xor_sync(0xffffffffu, su, o);
            sl += __shfl_xor_sync(0xffffffffu, sl, o);
        }
        if (lane == 0) {
            su_sh = su;
            if (blockIdx.x == 0) out[MLP_P] = -sl / (double)nd + log(16.0 * su / (double)nu);
        }
    }
    double a = 0.0, b = 0.0;
    if (q < MLP_P) {
        for (int k = warp; k < nblk_d; k += FIN_WARPS) a += part[(int64_t)k * (MLP_P + 1) + q];
        for (int k = warp; k < nblk_u; k += FIN_WARPS) b += part[(int64_t)(nblk_d + k) * (MLP_P + 1) + q];
    }
    sa[warp][lane] = a;
    sb[warp][lane] = b;
    __syncthreads();
    if (warp == 0 && q < MLP_P) {
        double ta = 0.0, tb = 0.0;
#pragma unroll
        for (int w = 0; w < FIN_WARPS; ++w) {
            ta += sa[w][lane];
            tb += sb[w][lane];
        }
        out[q] = ta + tb / su_sh;
    }
}

int sets_ctas(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + MLP_TILE - 1) / MLP_TILE, MLP_SETS_CTAS)); }

}  // namespace

int mlp_num_params() { return MLP_P; }

cudaError_t launch_mlp_forward(const __nv_bfloat16 *wb, const float *x, int64_t n, float *g,
                               cudaStream_t st)
{
    const int64_t tiles = (n + 15) / 16;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + MLP_WARPS - 1) / MLP_WARPS, 152 * 8));
    k_mlp_forward<<<grid, MLP_THREADS, WOff::FWD_BYTES, st>>>(wb, x, n, g);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grid(const __nv_bfloat16 *wb, const int nb[4], float *g, cudaStream_t st)
{
    const int64_t nc = (int64_t)nb[0] * nb[1] * nb[2] * nb[3];
    const int64_t tiles = (nc + 15) / 16;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + MLP_WARPS - 1) / MLP_WARPS, 152 * 8));
    k_mlp_grid<<<grid, MLP_THREADS, WOff::FWD_BYTES, st>>>(wb, nb[0], nb[1], nb[2], nb[3], g);
    return cudaGetLastError();
}

size_t mlp_grad_smem() { return GOff::BYTES; }

int mlp_grad_blocks(int64_t nd, int64_t nu) { return sets_ctas(nd) + sets_ctas(nu); }

cudaError_t launch_mlp_grad(const __nv_bfloat16 *wb, const float *xd, int64_t nd, const float *xu,
                            int64_t nu, float *part, double *out, cudaStream_t st)
{
    const int nbd = sets_ctas(nd), nbu = sets_ctas(nu);
    const size_t smem = mlp_grad_smem();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_mlp_grad<<<nbd + nbu, MLP_THREADS, smem, st>>>(wb, xd, nd, xu, nu, nbd, part);
    k_mlp_grad_finish<<<(MLP_P + 31) / 32, 32 * FIN_WARPS, 0, st>>>(part, nbd, nbu, nd, nu, out);
    return cudaGetLastError();
}

}  // namespace amp4d
