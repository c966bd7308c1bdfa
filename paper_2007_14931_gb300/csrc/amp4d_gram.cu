// Normalisation Gram matrix on the tensor cores (tcgen05, sm_103a).
//
// With the couplings fixed by the fit, the MC normalisation of the State-of-
// the-art section, I = (V/N) sum_n w_n S(x_n) with S = sum_xi |sum_k c_k B_k,xi|^2
// (Eq. 5, 12), is a quadratic form I = (V/N) (u^T G u + v^T G v) in the real
// 2K-vectors u = (Re c, -Im c), v = (Im c, Re c) of
//     G = sum_n w_n sum_xi x x^T,   x = (Re B_0, Im B_0, Re B_1, ...)(n, xi),
// so while masses and widths stay fixed every evaluation needs only G (2K x 2K).
//
// G is a dense contraction over 2 N_mc rows and is built here exactly enough
// for |dI/I| ~ 1e-11 with BF16 tensor-core products:
//  * k_gram_basis (every warp of the GPU) evaluates the basis of each point once
//    (Eq. 2-5, 10-12), writes x = sqrt(w) B' in FP32 to the basis matrix Xb and
//    finds max_n |x_i| per column; column i gets the power-of-two scale s_i with
//    |x_i s_i| < 2^30;
//  * in k_gram_tc, eleven converter warps read Xb, round X_i = rint(x_i s_i 2^30)
//    and split it exactly into four signed base-256 digits d1..d4 (|d1| <= 64,
//    |d2..4| <= 128), each exact in BF16;
//  * tcgen05.mma (kind::f16, BF16 x BF16 -> FP32 in tensor memory) forms the
//    digit products P_ab = sum d_a d_b over chunks of 1024 rows: every partial
//    sum is an integer below 2^24, so the FP32 accumulation is exact;
//  * after each chunk the epilogue warps read the accumulators (tcgen05.ld),
//    combine sum_ab 2^(8(5-a-b)) P_ab into INT64 fixed point (the a = b = 4
//    term, ~2^-48 relative, is dropped; 2^-8 and 2^-16 terms are rounded) and
//    add them into a per-CTA INT64 G in shared memory;
//  * k_gram_reduce sums the per-CTA INT64 partials (exact, order-free) and
//    converts once to FP64.
// Xb layout: k-step t (8 points) holds R = 2K rows of 16 FP32 values, value k =
// 2 q + xi of row i being x_i of point 8 t + q and helicity xi (row-major, 64 B
// per row): a converter lane reads 16 B (4 k of one row) and writes 8 B per
// digit slice.  Operand tiles: each K-step covers 16 rows (8 points x 2 xi); the
// four digit slices of the 64 padded columns form a 256 x 16 BF16 tile in the
// canonical K-major no-swizzle layout (8-row x 16-byte core matrices,
// K-direction core stride 144 B, row-group stride 288 B, stages 9248 B apart).
// Per K-step two MMAs, M = 128:
//   MMA1: A = slices {1,2} (rows 0..127) x B = slices {1..4} (N = 256)
//   MMA2: A = slices {3,4} (rows 128..255) x B = slice 3     (N = 64)
// Warp roles in k_gram_tc (16 warps, so 128 registers a thread): warps 0-10
// convert (one K-step per warp at a time), warps 11-14 are the epilogue (warp w
// reads TMEM lanes 32 (w % 4) ..), warp 15 allocates tensor memory and issues
// the MMAs.  Every mbarrier wait is bounded; on expiry the CTA
// raises an error flag, drains and frees its tensor memory.
#include <cstdint>
#include <cuda_bf16.h>

#include "amp4d_eval.cuh"

namespace amp4d {

constexpr int GT_PROD_WARPS = 11;          // converter warps 0-10
constexpr int GT_EPI_WARP0 = GT_PROD_WARPS;  // epilogue warps 11-14 (TMEM lane quarter warp % 4)
constexpr int GT_MMA_WARP = GT_PROD_WARPS + 4;
constexpr int GT_THREADS = (GT_PROD_WARPS + 5) * 32;
constexpr int GT_NSTAGE = 16;
constexpr int GT_LBO = 144;                // K-direction core-matrix stride (128 B + 16 B pad)
constexpr int GT_SBO = 288;                // 8-row group stride
constexpr int GT_STAGE_BYTES = 32 * GT_SBO + 32;   // 9248: stage starts 8 banks apart
constexpr int GT_CHUNK_KSTEPS = 64;        // 1024 rows = 512 points per chunk
constexpr int GT_CHUNK_POINTS = GT_CHUNK_KSTEPS * 8;
constexpr int GT_TMEM_COLS = 512;
constexpr long long GT_WAIT_CYCLES = 4000000000ll;  // ~2 s at 2 GHz
constexpr int GT_GS = 65;                  // row stride of the INT64 accumulators (bank spread)

struct GramSmem {
    alignas(1024) uint8_t stage[GT_NSTAGE][GT_STAGE_BYTES];
    // M[h] (h = 0: slice-1 rows, 1: slice-2 rows): row i is added to only by
    // epilogue thread 64 h + i, without atomics; G = (M + M^T) / 2 (below)
    unsigned long long M[2][64 * GT_GS];
    unsigned long long full[GT_NSTAGE], empty[GT_NSTAGE], acc_full, acc_empty, drain;
    float scale[64];
    uint32_t tmem_base;
    int abort_flag;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b))
                 : "memory");
}

// Bounded wait for the phase of the given parity; false on expiry or abort
// (abort_flag may be null: then only the time limit ends the wait).
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, uint32_t parity, volatile int *abort_flag)
{
    const long long t0 = clock64();
    uint32_t ok = 0;
    while (true) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(b)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (abort_flag && *abort_flag) return false;
        if (clock64() - t0 > GT_WAIT_CYCLES) {
            if (abort_flag) *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(GT_LBO >> 4) << 16) |
           ((uint64_t)(GT_SBO >> 4) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long *b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(b))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Byte offset of element (row r in 0..255, k in 0..15) inside a stage tile.
__device__ __forceinline__ int tile_off(int r, int k)
{
    return (r >> 3) * GT_SBO + (k >> 3) * GT_LBO + (r & 7) * 16 + (k & 7) * 2;
}

// The basis values of one point with both muon helicities of a column together:
// fn(column, B'_c,+1, B'_c,-1), scaled as the folded couplings expect.
template <int NK, int NZ, typename F>
__device__ __forceinline__ void for_each_basis_pair(const ModelDev &md, const float *r, F &&fn)
{
    EvState<NK, NZ> ev;
    eval_event<NK, NZ>(md, r, ev);
    const int nK = md.n_res - NZ;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        if (k >= nK) continue;
        const ResDev &rs = md.res[k];
        const float2 Bl[3] = {make_float2(-ev.B1[k].x, -ev.B1[k].y), ev.B0[k], ev.B1[k]};
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            if (rs.J == 0 && l != 1) continue;
            const int col = rs.J == 0 ? rs.col : rs.col + l;
            fn(col, cmul(Bl[l], ev.Psi[l][0]), cmul(Bl[l], ev.Psi[l][1]));
        }
    }
    if constexpr (NZ > 0) {
#pragma unroll
        for (int z = 0; z < NZ; ++z) {
            const ResDev &rs = md.zr[z];
            if (rs.zcol0 >= 0) fn(rs.zcol0, cmul(ev.AZ[z], ev.Om0[z][0]), cmul(ev.AZ[z], ev.Om0[z][1]));
            if (rs.zcol1 >= 0) fn(rs.zcol1, cmul(ev.AZ[z], ev.Om1[z][0]), cmul(ev.AZ[z], ev.Om1[z][1]));
        }
    }
}

// Pass 1: the basis matrix Xb (layout above) and max_n |x_i(n)| per row i (as
// float bits, non-negative).  Points n .. nalloc - 1 (nalloc a multiple of 32)
// are written as zeros.  Every lane of a warp runs the same iterations (the
// column maxima are warp reductions); lanes past n evaluate point n - 1 and
// store zeros.
template <int NK, int NZ>
__global__ void __launch_bounds__(256) k_gram_basis(const float *__restrict__ rec, int64_t npad,
                                                    int64_t n, int64_t nalloc, int wrec,
                                                    const ModelDev *__restrict__ gmd, int R,
                                                    float *__restrict__ Xb, unsigned *__restrict__ colmax)
{
    constexpr int NREC = NZ > 0 ? REC_NZ : REC_NK;
    __shared__ ModelDev md;
    __shared__ unsigned smax[64];
    load_model(gmd, &md);
    if (threadIdx.x < 64) smax[threadIdx.x] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < nalloc;
         base += stride) {
        const int64_t p = base + lane;
        const bool valid = p < n;
        const int64_t pe = valid ? p : n - 1;
        float v[NREC];
#pragma unroll
        for (int k = 0; k < NREC; ++k) v[k] = __ldcs(rec + k * npad + pe);
        const float sw = valid ? sqrtf(__ldcs(rec + wrec * npad + pe)) : 0.0f;
        float *xp = Xb + (p >> 3) * (int64_t)R * 16 + 2 * (p & 7);
        for_each_basis_pair<NK, NZ>(md, v, [&](int col, float2 b0, float2 b1) {
            const float2 re = make_float2(b0.x * sw, b1.x * sw), im = make_float2(b0.y * sw, b1.y * sw);
            __stcs(reinterpret_cast<float2 *>(xp + (2 * col) * 16), re);
            __stcs(reinterpret_cast<float2 *>(xp + (2 * col + 1) * 16), im);
            const unsigned mr = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(fabsf(re.x), fabsf(re.y))));
            const unsigned mi = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(fabsf(im.x), fabsf(im.y))));
            if (lane == 0) {
                atomicMax(&smax[2 * col], mr);
                atomicMax(&smax[2 * col + 1], mi);
            }
        });
    }
    __syncthreads();
    if (threadIdx.x < R && smax[threadIdx.x]) atomicMax(&colmax[threadIdx.x], smax[threadIdx.x]);
}

// Base-256 digits of the fixed-point value X (|X| <= 2^30), each rounded half up
// (the self-test's split): X = d1 2^24 + d2 2^16 + d3 2^8 + d4.
__device__ __forceinline__ void digits_int(int X, float d[4])
{
    const int d1 = (X + (1 << 23)) >> 24;
    const int r1 = X - (d1 << 24);
    const int d2 = (r1 + (1 << 15)) >> 16;
    const int r2 = r1 - (d2 << 16);
    const int d3 = (r2 + 128) >> 8;
    d[0] = (float)d1;
    d[1] = (float)d2;
    d[2] = (float)d3;
    d[3] = (float)(r2 - (d3 << 8));
}

// The same split of an integer-valued FP32 y (|y| <= 2^30) in FP32 arithmetic,
// ties to even: adding and subtracting 1.5 x 2^(p + 23) rounds to a multiple of
// 2^p (p = 24, 16, 8), and every remainder is an integer below 2^24 in
// magnitude, so each step is exact.
__device__ __forceinline__ void digits_fp(float y, float d[4])
{
    const float t1 = __fsub_rn(__fadd_rn(y, 0x1.8p47f), 0x1.8p47f);
    const float r1 = __fsub_rn(y, t1);
    const float t2 = __fsub_rn(__fadd_rn(r1, 0x1.8p39f), 0x1.8p39f);
    const float r2 = __fsub_rn(r1, t2);
    const float t3 = __fsub_rn(__fadd_rn(r2, 0x1.8p31f), 0x1.8p31f);
    d[0] = __fmul_rn(t1, 0x1p-24f);
    d[1] = __fmul_rn(t2, 0x1p-16f);
    d[2] = __fmul_rn(t3, 0x1p-8f);
    d[3] = __fsub_rn(r2, t3);
}

// Store the digits d[j][a] of the values at k0 + j (j = 0..3, k0 a multiple of 4)
// of one row: one 8-byte store per digit slice a.  A digit is an integer of at
// most 8 significant bits, so its BF16 is the upper half of its FP32 bits.
__device__ __forceinline__ void store_digits4(uint8_t *tile, int row, int k0, const float d[4][4])
{
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const uint32_t lo = __byte_perm(__float_as_uint(d[0][a]), __float_as_uint(d[1][a]), 0x7632);
        const uint32_t hi = __byte_perm(__float_as_uint(d[2][a]), __float_as_uint(d[3][a]), 0x7632);
        *reinterpret_cast<uint2 *>(tile + tile_off(a * 64 + row, k0)) = make_uint2(lo, hi);
    }
}

__device__ __forceinline__ long long rshift_round(long long v, int s)
{
    return (v + (1ll << (s - 1))) >> s;
}

// Pass 2: the digit products.  Xb holds the basis matrix of n points (zeros up
// to the end of the last chunk), R rows per K-step.  SYNTH: the converters take
// the fixed-point values X directly from synth ([point][xi][64] int32, all 64
// rows) instead of rounding Xb -- the self-test of the exact integer
// accumulation.
template <bool SYNTH>
__global__ void __launch_bounds__(GT_THREADS, 1)
    k_gram_tc(const float *__restrict__ Xb, int R, int64_t n, const float *__restrict__ gscale,
              long long *__restrict__ part, int *__restrict__ err, const int *__restrict__ synth)
{
    extern __shared__ uint8_t smem_raw[];
    GramSmem &S = *reinterpret_cast<GramSmem *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // Set-up: zero tiles and G, scales, barriers, tensor memory.
    for (int i = tid; i < GT_NSTAGE * GT_STAGE_BYTES / 16; i += GT_THREADS)
        reinterpret_cast<uint4 *>(&S.stage[0][0])[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < 2 * 64 * GT_GS; i += GT_THREADS) (&S.M[0][0])[i] = 0ull;
    if (tid < 64) S.scale[tid] = gscale ? gscale[tid] : 1.0f;
    if (tid == 0) {
        S.abort_flag = 0;
        for (int s = 0; s < GT_NSTAGE; ++s) {
            mbar_init(&S.full[s], 32);   // the lanes of one converter warp
            mbar_init(&S.empty[s], 1);
        }
        mbar_init(&S.acc_full, 1);
        mbar_init(&S.acc_empty, 128);
        mbar_init(&S.drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == GT_MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem_base)),
                     "r"(GT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    volatile int *abort_flag = &S.abort_flag;
    const int64_t nchunks = (n + GT_CHUNK_POINTS - 1) / GT_CHUNK_POINTS;

    if (warp < GT_PROD_WARPS) {
        // ----------------------------------------------------------- converters
        // The CTA's K-steps ks = warp, warp + 11, ... in order (K-step kk = ks % 64
        // of its chunk ks / 64).  Lane (h, rsub, kq & 1), h = lane >> 4, handles
        // values 4 kq .. 4 kq + 3 (kq = 2 h + (lane & 1)) of rows 8 i + rsub, so
        // each half-warp stores 128 contiguous bytes per digit slice (one
        // wavefront, no bank conflict).  The next K-step's values are loaded while
        // this one is converted, and the one after is prefetched into L2.
        const int rows = SYNTH ? 64 : R;
        const int ni = (rows + 7) >> 3;
        const int rsub = (lane >> 1) & 7, kq = ((lane >> 4) << 1) | (lane & 1);
        const int64_t kblk = (int64_t)R * 16;   // floats per K-step of Xb
        auto gstep = [&](int64_t ks) {          // global K-step of the CTA's ks, or -1
            const int64_t c = blockIdx.x + (ks / GT_CHUNK_KSTEPS) * (int64_t)gridDim.x;
            return c < nchunks ? c * GT_CHUNK_KSTEPS + ks % GT_CHUNK_KSTEPS : (int64_t)-1;
        };
        float4 cur[8], nxt[8];
        auto load = [&](int64_t g, float4(&buf)[8]) {
            const float4 *src = reinterpret_cast<const float4 *>(Xb + g * kblk);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int row = 8 * i + rsub;
                buf[i] = (i < ni && row < R) ? __ldcs(src + row * 4 + kq) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        auto prefetch_l2 = [&](int64_t g) {
            if (!SYNTH && g >= 0 && lane == 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(Xb + g * kblk),
                             "r"((unsigned)(kblk * sizeof(float)))
                             : "memory");
        };
        int64_t ks = warp, g = gstep(ks);
        if (!SYNTH && g >= 0) load(g, cur);
        prefetch_l2(gstep(ks + GT_PROD_WARPS));
        while (g >= 0 && !*abort_flag) {
            const int64_t gn = gstep(ks + GT_PROD_WARPS);
            if (!SYNTH && gn >= 0) load(gn, nxt);
            prefetch_l2(gstep(ks + 2 * GT_PROD_WARPS));
            const int s = (int)(ks % GT_NSTAGE);
            const int64_t use = ks / GT_NSTAGE;
            if (use > 0 && !mbar_wait(&S.empty[s], (uint32_t)((use - 1) & 1), abort_flag)) break;
            uint8_t *tile = S.stage[s];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int row = 8 * i + rsub;
                if (i >= ni || row >= rows) continue;
                float d[4][4];
                if constexpr (SYNTH) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int k = 4 * kq + j;
                        const int64_t e = g * 8 + (k >> 1);
                        digits_int(e < n ? __ldg(synth + (e * 2 + (k & 1)) * 64 + row) : 0, d[j]);
                    }
                } else {
                    const float sc = S.scale[row];
                    const float x[4] = {cur[i].x, cur[i].y, cur[i].z, cur[i].w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) digits_fp(rintf(x[j] * sc), d[j]);
                }
                store_digits4(tile, row, 4 * kq, d);
            }
            fence_async_smem();
            mbar_arrive(&S.full[s]);
#pragma unroll
            for (int i = 0; i < 8; ++i) cur[i] = nxt[i];
            ks += GT_PROD_WARPS;
            g = gn;
        }
    } else if (warp < GT_MMA_WARP) {
        // ------------------------------------------------------------ epilogue
        // a warp reaches the TMEM lanes of its quarter warp % 4 (TMEM lane ==
        // accumulator row)
        const int row = ((warp & 3) << 5) | lane;
        const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        int64_t it = 0;
        for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x, ++it) {
            // warp-collective: tcgen05.ld below is .sync.aligned
            const bool got = mbar_wait(&S.acc_full, (uint32_t)(it & 1), abort_flag);
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            const int i = row & 63;
            const bool lo = row < 64;        // slice-1 rows (lo) or slice-2 rows (hi)
            unsigned long long *Mrow = S.M[lo ? 0 : 1] + i * GT_GS;
            for (int jb = 0; jb < 64; jb += 16) {
                float q1[16], q2[16], q3[16], q4[16], q5[16];
                tmem_ld16(lane_addr + jb, q1);        // P_a1
                tmem_ld16(lane_addr + 64 + jb, q2);   // P_a2
                tmem_ld16(lane_addr + 128 + jb, q3);  // P_a3
                tmem_ld16(lane_addr + 192 + jb, q4);  // P_a4
                tmem_ld16(lane_addr + 256 + jb, q5);  // lo: P_33, hi: P_43
                tmem_wait_ld();
                if (jb == 48) {
                    // the accumulators are all in registers: release them to the MMAs
                    tc_fence_before();
                    mbar_arrive(&S.acc_empty);
                }
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const long long p1 = __float2ll_rn(q1[t]), p2 = __float2ll_rn(q2[t]);
                    const long long p3 = __float2ll_rn(q3[t]), p4 = __float2ll_rn(q4[t]);
                    const long long p5 = __float2ll_rn(q5[t]);
                    long long D, T;
                    if (lo) {   // a = 1: (1,1) 2^24, (1,2) 2^16, (1,3) 2^8, (1,4) 1, (3,3) 2^-8
                        D = (p1 << 24) + (p2 << 16) + (p3 << 8) + p4 + rshift_round(p5, 8);
                        T = (p3 << 8) + p4;                         // (3,1), (4,1)
                    } else {    // a = 2: (2,1) 2^16, (2,2) 2^8, (2,3) 1, (2,4) 2^-8, (4,3) 2^-16
                        const long long r24 = rshift_round(p4, 8), r43 = rshift_round(p5, 16);
                        D = (p1 << 16) + (p2 << 8) + p3 + r24 + r43;
                        T = p3 + r24 + r43;                         // (3,2), (4,2), (3,4)
                    }
                    // D belongs to G_ij and T to G_ji: M_ij gets both
                    Mrow[jb + t] += (unsigned long long)(D + T);
                }
            }
        }
    } else if (lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        const uint32_t id1 = mma_idesc(128, 256), id2 = mma_idesc(128, 64);
        int64_t it = 0;
        bool issued = false;
        for (int64_t c = blockIdx.x; c < nchunks && !*abort_flag; c += gridDim.x, ++it) {
            if (it > 0 && !mbar_wait(&S.acc_empty, (uint32_t)((it - 1) & 1), abort_flag)) break;
            tc_fence_after();
            bool ok = true;
            for (int kk = 0; kk < GT_CHUNK_KSTEPS; ++kk) {
                const int64_t ks = it * GT_CHUNK_KSTEPS + kk;
                const int s = (int)(ks % GT_NSTAGE);
                if (!mbar_wait(&S.full[s], (uint32_t)((ks / GT_NSTAGE) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t base = smem_u32(S.stage[s]);
                const uint64_t dA1 = smem_desc(base), dB1 = smem_desc(base);
                const uint64_t dA2 = smem_desc(base + 16 * GT_SBO), dB2 = smem_desc(base + 16 * GT_SBO);  // rows 128..
                mma_bf16(tmem, dA1, dB1, id1, kk > 0);
                mma_bf16(tmem + 256, dA2, dB2, id2, kk > 0);
                mma_commit(&S.empty[s]);
                issued = true;
            }
            if (!ok) break;
            mma_commit(&S.acc_full);
        }
        // Drain: every MMA issued by this thread has completed before teardown.
        if (issued) {
            mma_commit(&S.drain);
            if (!mbar_wait(&S.drain, 0u, nullptr)) S.abort_flag = 1;
        }
    }

    // Teardown: wait for the last accumulator hand-off, free tensor memory.
    tc_fence_before();
    __syncthreads();
    if (warp == GT_MMA_WARP) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(GT_TMEM_COLS)
                     : "memory");
    }
    if (S.abort_flag && tid == 0) atomicExch(err, 1);
    for (int i = tid; i < 64 * 64; i += GT_THREADS)
    {
        // G = D + T^T is exactly symmetric (every digit-product term is, rounded
        // ones included), and M = D + T, so M + M^T = 2 G exactly.
        const int r = i >> 6, c = i & 63;
        const unsigned long long a = S.M[0][r * GT_GS + c] + S.M[1][r * GT_GS + c];
        const unsigned long long b = S.M[0][c * GT_GS + r] + S.M[1][c * GT_GS + r];
        part[(int64_t)blockIdx.x * 4096 + i] = (long long)(a + b) >> 1;
    }
}

// Sum the per-CTA INT64 partials and convert: with X_i = x_i g_i (g = gscale) and
// sum_n X_i X_j = 2^24 G_int, G_ij = sum_n x_i x_j = 2^24 G_int / (g_i g_j).
__global__ void k_gram_reduce(const long long *__restrict__ part, int nblk,
                              const float *__restrict__ gscale, int dim, double *__restrict__ G)
{
    const int i = blockIdx.x, j = threadIdx.x;
    if (i >= dim || j >= dim) return;
    long long s = 0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * 4096 + i * 64 + j];
    G[i * dim + j] = (double)s * 0x1p24 / ((double)gscale[i] * (double)gscale[j]);
}

__global__ void k_gram_scales(const unsigned *__restrict__ colmax, float *__restrict__ gscale)
{
    const int i = threadIdx.x;
    if (i >= 64) return;
    const float m = __uint_as_float(colmax[i]);
    int ex = 0;
    if (m > 0.0f) frexpf(m, &ex);
    gscale[i] = ldexpf(1.0f, 30 - ex);   // |x| < 2^ex, so |x s| < 2^30
}

static cudaError_t launch_tc(bool synth_mode, const float *Xb, int R, int64_t n, const float *gscale,
                             long long *part, int *err, const int *synth, int grid, cudaStream_t st)
{
    const size_t smem = sizeof(GramSmem) + 1024;
    auto kern = synth_mode ? k_gram_tc<true> : k_gram_tc<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, GT_THREADS, smem, st>>>(Xb, R, n, gscale, part, err, synth);
    return cudaGetLastError();
}

template <int NK, int NZ>
static cudaError_t gram_t(const GramArgs &a)
{
    cudaError_t e = cudaMemsetAsync(a.colmax, 0, 64 * sizeof(unsigned), a.stream);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gram_basis<NK, NZ>, 256, 0);
    if (e != cudaSuccess) return e;
    k_gram_basis<NK, NZ><<<a.nsm * (nb > 0 ? nb : 1), 256, 0, a.stream>>>(
        a.rec, a.npad, a.n, gram_basis_points(a.n), a.wrec, a.md, a.dim, a.xb, a.colmax);
    k_gram_scales<<<1, 64, 0, a.stream>>>(a.colmax, a.gscale);
    e = launch_tc(false, a.xb, a.dim, a.n, a.gscale, a.part, a.err, nullptr, a.grid_tc, a.stream);
    if (e != cudaSuccess) return e;
    k_gram_reduce<<<a.dim, 64, 0, a.stream>>>(a.part, a.grid_tc, a.gscale, a.dim, a.G);
    return cudaGetLastError();
}

cudaError_t launch_gram(const GramArgs &a)
{
#define AMP4D_GRAM_CASE(NKV, NZV) \
    if (a.nk_max == NKV && a.nz == NZV) return gram_t<NKV, NZV>(a);
    AMP4D_GRAM_CASE(2, 0)
    AMP4D_GRAM_CASE(2, 1)
    AMP4D_GRAM_CASE(2, 2)
    AMP4D_GRAM_CASE(10, 0)
    AMP4D_GRAM_CASE(10, 1)
    AMP4D_GRAM_CASE(10, 2)
    AMP4D_GRAM_CASE(16, 0)
    AMP4D_GRAM_CASE(16, 1)
    AMP4D_GRAM_CASE(16, 2)
#undef AMP4D_GRAM_CASE
    return cudaErrorInvalidValue;
}

int gram_chunk_points() { return GT_CHUNK_POINTS; }

int64_t gram_basis_points(int64_t n) { return (n + GT_CHUNK_POINTS - 1) / GT_CHUNK_POINTS * GT_CHUNK_POINTS; }

// Sum of the per-CTA INT64 partials, no scaling (self-test).
__global__ void k_gram_reduce_int(const long long *__restrict__ part, int nblk,
                                  long long *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4096) return;
    long long s = 0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * 4096 + i];
    out[i] = s;
}

cudaError_t launch_gram_selftest(const int *synth, int64_t n, long long *part, int grid, int *err,
                                 long long *out, cudaStream_t st)
{
    cudaError_t e = launch_tc(true, nullptr, 64, n, nullptr, part, err, synth, grid, st);
    if (e != cudaSuccess) return e;
    k_gram_reduce_int<<<16, 256, 0, st>>>(part, grid, out);
    return cudaGetLastError();
}

}  // namespace amp4d
