// Per-event amplitude, likelihood and adjoint-gradient kernel templates.
//
// One thread handles one event per iteration (coalesced scalar loads of every
// record), grid-stride over the event set.  Per event, in FP32 registers:
//   lineshapes A_R (Eq. 2-3), from the basis cache for fixed resonances,
//   d^J_{l0}(theta_K*), e^{i l phi} d^1_{l xi}(theta_psi) (Eq. 4),
//   the Z-chain factors (Eq. 10-11) from precomputed Z-frame angles,
//   a_xi = sum_k c_k B_k,xi and S = |a_+|^2 + |a_-|^2 (Eq. 5, 12).
// Data kernels sum ln S, normalisation kernels sum w S; each thread keeps a
// compensated FP32 sum (ln S split as ln(mantissa) + exponent ln 2), blocks
// reduce in FP64 and add their sums to exact 128-bit accumulators (acc128_add).
// Instantiated per resonance-count bucket in amp4d_eval_nk*.cu.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "amp4d_device.cuh"
#include "amp4d_finish.cuh"
#include "amp4d_launch.h"

namespace amp4d {

// The per-evaluation table as the per-event kernels read it: in the constant
// bank, so that every field of a resonance of a loop unrolled over resonances
// is an operand at a fixed address (no shared-memory load per use).  Each
// translation unit has its own copy; with_const_table fills it on the stream
// right before a launch.
static __constant__ ModelDev c_md;

struct ConstTableSync {
    std::mutex mu;
    cudaEvent_t done[64] = {};
};
static ConstTableSync &const_table_sync()
{
    static ConstTableSync s;
    return s;
}

// Copies the device table gmd (written by k_build_table on the same stream)
// into c_md and enqueues launch().  There is one c_md per device, so launches
// from different streams are serialised: each waits for the previous user's
// kernels before overwriting the table.  Under stream capture (a CUDA graph of
// an evaluation) the wait and the record become external event nodes, so every
// replay of the graph takes part in the same serialisation.
template <typename Launch>
static cudaError_t with_const_table(const ModelDev *gmd, cudaStream_t st, Launch &&launch)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return e;
    const bool capturing = cap == cudaStreamCaptureStatusActive;
    ConstTableSync &sy = const_table_sync();
    std::lock_guard<std::mutex> lock(sy.mu);
    if (!sy.done[dev]) e = cudaEventCreateWithFlags(&sy.done[dev], cudaEventDisableTiming);
    else e = cudaStreamWaitEvent(st, sy.done[dev], capturing ? cudaEventWaitExternal : 0);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbolAsync(c_md, gmd, sizeof(ModelDev), 0, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    e = launch();
    if (e != cudaSuccess) return e;
    return capturing ? cudaEventRecordWithFlags(sy.done[dev], st, cudaEventRecordExternal)
                     : cudaEventRecord(sy.done[dev], st);
}


// Resonances internal order: K* first (at most NK), then Z (exactly NZ).
template <int NK, int NZ>
struct EvState {
    float2 a[2];
    float S;
    float2 ab[2];                 // flavour mistag: the amplitudes at -phi (every angular phase conjugated)
    float Sb;                     // and S there
    float2 B0[NK], B1[NK];        // K* k: A_k d0 and A_k d1 (l = 0 and l = +1; l = -1 is -B1)
    float2 Psi[3][2];
    float2 AZ[NZ > 0 ? NZ : 1];
    float2 Om0[NZ > 0 ? NZ : 1][2], Om1[NZ > 0 ? NZ : 1][2];
    float m, invm, p, q;          // kept to recompute lineshapes for mass/width derivatives
    float cK, sK;                 // and the K* helicity angle, for d^J of floated states
    float mZ, invmZ, pZ, qZ;
};

// Lineshape of a resonance for this event: the basis-cache value (loaded up
// front) when a cache is given and the resonance's mass and width are fixed,
// else computed.
template <bool KSTAR>
__device__ __forceinline__ float2 cached_or_computed(const ResDev &rs, bool have_lc, float2 cached,
                                                     float m, float invm, float p, float q)
{
    if (have_lc && rs.fpos < 0) return cached;
    if constexpr (KSTAR) return kstar_lineshape(rs, m, invm, p, q);
    return lineshape(rs, m, invm, p, q).A;
}

// lc (nullable): basis cache [resonance][lcn] of lineshapes A'_R per event e.
// FX: every resonance is fixed and lc is given, so every lineshape comes from
// the cache and the masses and momenta (records M, P, Q, MZ, PZ, QZ) are unused.
// MT (flavour mistag): also the amplitudes and S at -phi.  The mirror phi -> -phi
// flips sin phi, sin phi~ and sin alpha and leaves every cosine, mass and
// momentum unchanged, so the mirrored amplitude is the same coupling sums with
// every angular phase factor (e^{i l phi}, e^{i l' phi~}, e^{i xi alpha}) conjugated.
template <int NK, int NZ, bool FX = false, bool MT = false>
__device__ __forceinline__ void eval_event(const ModelDev &md, const float *r,
                                           EvState<NK, NZ> &ev,
                                           const float2 *__restrict__ lc = nullptr,
                                           int64_t lcn = 0, int64_t e = 0)
{
    const float cK = r[REC_CK], cpsi = r[REC_CPSI];
    float m = 0.f, p = 0.f, q = 0.f, invm = 0.f;
    if constexpr (!FX) {
        m = r[REC_M]; p = r[REC_P]; q = r[REC_Q];
        invm = __frcp_rn(m);
    }
    ev.m = m; ev.invm = invm; ev.p = p; ev.q = q;
    const float sK = sqrtf(fmaxf(0.0f, fmaf(-cK, cK, 1.0f)));
    const float2 cc = make_float2(cK, cK);
    ev.cK = cK; ev.sK = sK;
    const float spsi = sqrtf(fmaxf(0.0f, fmaf(-cpsi, cpsi, 1.0f)));
    const float cph = r[REC_CPHI], sph = r[REC_SPHI];   // e^{i phi}, FP64 at ingest
    float d1p[3][2];
    wigner_1(cpsi, spsi, d1p);
#pragma unroll
    for (int x = 0; x < 2; ++x) {
        ev.Psi[0][x] = make_float2(cph * d1p[0][x], -sph * d1p[0][x]);  // e^{-i phi}
        ev.Psi[1][x] = make_float2(d1p[1][x], 0.0f);
        ev.Psi[2][x] = make_float2(cph * d1p[2][x], sph * d1p[2][x]);   // e^{+i phi}
    }
    float2 u[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    const int nK = md.n_res - NZ;
    // Every cached lineshape of the event is requested before any is used, so
    // the loads overlap instead of waiting one after another behind the
    // per-resonance branches.
    const bool have_lc = FX || lc != nullptr;
    float2 LK[NK], LZ[NZ > 0 ? NZ : 1];
    if (have_lc) {
#pragma unroll
        for (int k = 0; k < NK; ++k)
            LK[k] = k < nK ? __ldg(lc + k * lcn + e) : make_float2(0.f, 0.f);
#pragma unroll
        for (int z = 0; z < NZ; ++z) LZ[z] = __ldg(lc + (nK + z) * lcn + e);
    }
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        if (k < nK) {
            const ResDev &rs = md.res[k];
            const float2 LA = FX ? LK[k] : cached_or_computed<true>(rs, have_lc, LK[k], m, invm, p, q);
            float d0, d1;
            wigner_l0(rs, cc, sK, d0, d1);
            const float2 b0 = cscale(LA, d0), b1 = cscale(LA, d1);
            ev.B0[k] = b0;
            ev.B1[k] = b1;
            // J = 0: the l = +-1 couplings are 0 and d1 = 0, so no branch on J.
            // kp[k][0] holds -c'_{k,-1}: the l = -1 factor is -A d1.
            const float2 b0s = make_float2(b0.y, b0.x), b1s = make_float2(b1.y, b1.x);
            cfma2p(u[0], md.kp[k][0], b1, b1s);
            cfma2p(u[1], md.kp[k][1], b0, b0s);
            cfma2p(u[2], md.kp[k][2], b1, b1s);
        } else {
            ev.B0[k] = ev.B1[k] = make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int x = 0; x < 2; ++x) {
        float2 a = make_float2(0.f, 0.f);
        cfma(a, ev.Psi[0][x], u[0]);
        cfma(a, ev.Psi[1][x], u[1]);
        cfma(a, ev.Psi[2][x], u[2]);
        ev.a[x] = a;
        if constexpr (MT) {
            float2 b = make_float2(0.f, 0.f);
            cfma_conj(b, ev.Psi[0][x], u[0]);
            cfma_conj(b, ev.Psi[1][x], u[1]);
            cfma_conj(b, ev.Psi[2][x], u[2]);
            ev.ab[x] = b;
        }
    }
    if constexpr (NZ > 0) {
        float mZ = 0.f, pZ = 0.f, qZ = 0.f, invmZ = 0.f;
        if constexpr (!FX) {
            mZ = r[REC_MZ]; pZ = r[REC_PZ]; qZ = r[REC_QZ];
            invmZ = __frcp_rn(mZ);
        }
        const float cZ = r[REC_CZ], ctz = r[REC_CTZ];
        const float2 ephz = make_float2(r[REC_CPZ], r[REC_SPZ]);
        const float ca = r[REC_CA], sa = r[REC_SA];
        ev.mZ = mZ; ev.invmZ = invmZ; ev.pZ = pZ; ev.qZ = qZ;
        const float sZ = sqrtf(fmaxf(0.0f, fmaf(-cZ, cZ, 1.0f)));
        const float stz = sqrtf(fmaxf(0.0f, fmaf(-ctz, ctz, 1.0f)));
        float d1t[3][2];
        wigner_1(ctz, stz, d1t);
#pragma unroll
        for (int z = 0; z < NZ; ++z) {
            const ResDev &rs = md.zr[z];
            const float2 LA = FX ? LZ[z] : cached_or_computed<false>(rs, have_lc, LZ[z], mZ, invmZ, pZ, qZ);
            float dz0, dz1;
            wigner_l0(rs, make_float2(cZ, cZ), sZ, dz0, dz1);  // d^J_{00}, d^J_{0,+-1} ~ -+ dz1
            ev.AZ[z] = LA;
#pragma unroll
            for (int x = 0; x < 2; ++x) {
                const float2 eal = make_float2(ca, x == 0 ? sa : -sa);  // e^{i xi alpha}
                float2 o0 = cscale(eal, dz0 * d1t[1][x]);
                float2 t = cscale(ephz, -dz1 * d1t[2][x]);
                float2 ephm = make_float2(ephz.x, -ephz.y);
                t = cadd(t, cscale(ephm, (float)rs.eta * dz1 * d1t[0][x]));
                float2 o1 = cmul(t, eal);
                ev.Om0[z][x] = o0;
                ev.Om1[z][x] = o1;
                float2 s = make_float2(0.f, 0.f);
                if (rs.zcol0 >= 0) cfma2p(s, md.zp[z][0], o0, make_float2(o0.y, o0.x));
                if (rs.zcol1 >= 0) cfma2p(s, md.zp[z][1], o1, make_float2(o1.y, o1.x));
                cfma(ev.a[x], LA, s);
                if constexpr (MT) {
                    const float2 c0 = make_float2(o0.x, -o0.y), c1 = make_float2(o1.x, -o1.y);
                    float2 sb = make_float2(0.f, 0.f);
                    if (rs.zcol0 >= 0) cfma2p(sb, md.zp[z][0], c0, make_float2(c0.y, c0.x));
                    if (rs.zcol1 >= 0) cfma2p(sb, md.zp[z][1], c1, make_float2(c1.y, c1.x));
                    cfma(ev.ab[x], LA, sb);
                }
            }
        }
    }
    ev.S = cabs2(ev.a[0]) + cabs2(ev.a[1]);
    if constexpr (MT) ev.Sb = cabs2(ev.ab[0]) + cabs2(ev.ab[1]);
}

// The flavour-tagged density (1 - w) S + w S(-phi) = S + w (S(-phi) - S).
template <bool MT, int NK, int NZ>
__device__ __forceinline__ float observed_S(const ModelDev &md, const EvState<NK, NZ> &ev)
{
    if constexpr (!MT) return ev.S;
    const float d = ev.Sb - ev.S;
    return fmaf(md.mwhi, d, fmaf(md.mwlo, d, ev.S));
}

// w_0 for the real Psi_{0 xi} (p = Psi_{0 xi}.x): the bits of adj_w, whose zero
// products leave the FMA chain unchanged, in half the FMAs.
template <bool MT>
__device__ __forceinline__ float2 adj_w_real(const float2 (&as)[2], const float2 (&asb)[2],
                                             const float2 (&psi)[2])
{
    float2 t = make_float2(0.f, 0.f);
#pragma unroll
    for (int x = 0; x < 2; ++x) {
        t.x = fmaf(as[x].x, psi[x].x, t.x);
        t.y = fmaf(-as[x].y, psi[x].x, t.y);
    }
    if constexpr (MT) {
#pragma unroll
        for (int x = 0; x < 2; ++x) {
            t.x = fmaf(asb[x].x, psi[x].x, t.x);
            t.y = fmaf(-asb[x].y, psi[x].x, t.y);
        }
    }
    return t;
}

// Adjoint vectors w_l = sum_xi conj(as_xi) Psi_{l xi} of the scaled amplitudes,
// with the mistag term conj(asb_xi Psi_{l xi}) for the mirrored amplitudes.
template <bool MT>
__device__ __forceinline__ float2 adj_w(const float2 (&as)[2], const float2 (&asb)[2],
                                        const float2 (&psi)[2])
{
    float2 t = make_float2(0.f, 0.f);
    cfma_conj(t, as[0], psi[0]);
    cfma_conj(t, as[1], psi[1]);
    if constexpr (MT) {
        cfma_conjp(t, asb[0], psi[0]);
        cfma_conjp(t, asb[1], psi[1]);
    }
    return t;
}

// Adjoint factors of a floated resonance's lineshape, with the double-float
// couplings (each low part inside its product, as in the coherent sum): for a
// K* k, y = sum_l c'_{k,l} d_l w_l, where the l = -1 basis factor is -A d1 and
// kp[k][0] holds -c'_{k,-1}; for a Z z, y = sum_l' c'_{z,l'} w_l'.  A coupling
// rounded to FP32 would leave a relative error of up to 2^-24 in y that differs
// between the data events and the normalisation points (their angular
// distributions differ), so it would not cancel in the mass and width gradient.
__device__ __forceinline__ float2 kstar_adj_y(const ModelDev &md, int k, float d0, float d1,
                                              const float2 (&wl)[3])
{
    const float2 t0 = cscale(wl[0], d1), t1 = cscale(wl[1], d0), t2 = cscale(wl[2], d1);
    float2 y = make_float2(0.f, 0.f);
    cfma2p(y, md.kp[k][0], t0, make_float2(t0.y, t0.x));
    cfma2p(y, md.kp[k][1], t1, make_float2(t1.y, t1.x));
    cfma2p(y, md.kp[k][2], t2, make_float2(t2.y, t2.x));
    return y;
}
__device__ __forceinline__ float2 z_adj_y(const ModelDev &md, const ResDev &rs, int z, float2 w0, float2 w1)
{
    float2 y = make_float2(0.f, 0.f);
    if (rs.zcol0 >= 0) cfma2p(y, md.zp[z][0], w0, make_float2(w0.y, w0.x));
    if (rs.zcol1 >= 0) cfma2p(y, md.zp[z][1], w1, make_float2(w1.y, w1.x));
    return y;
}

// Shared-memory staging of the all-cached kernel's inputs (k_grad_fx, STG): each
// thread copies the records and cache rows of its next event pair into its own
// shared-memory slots with cp.async while it evaluates the current pair, then
// reads them with ld.shared.  Only the copying thread reads a slot, so a
// cp.async.wait_group of that thread is the only synchronisation.
__device__ __forceinline__ uint32_t shared_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async_8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(shared_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(shared_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ float4 lds4(const void *p)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(shared_u32(p)));
    return v;
}
__device__ __forceinline__ float2 lds2(const void *p)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(shared_u32(p)));
    return v;
}
// The cached values of an adjacent event pair: from global memory (evict-first)
// or, SM, from the thread's staging slots.
template <bool SM>
__device__ __forceinline__ float4 ld_pair(const float2 *p)
{
    if constexpr (SM) return lds4(p);
    else return __ldcs(reinterpret_cast<const float4 *>(p));
}

// Evaluation of NE events at once with the lineshapes of fixed resonances from
// the basis cache: the per-resonance constants are read once for all NE events.
// SM (NE = 2 only): lc points to the staging slots (row stride lcn, e[0] the
// thread's slot) instead of the cache.
// r[j] holds the records of event e[j]; lc is the basis cache [resonance][lcn].
// LFM: which floated resonances have their lineshape computed per event (Eq.
// 2-3) from the mass and momentum records instead of the cache: 0 none, 1 the
// floated Z, 2 every floated resonance (K* and Z).
template <int NK, int NZ, int NE, int LFM = 0, bool MT = false, bool SM = false, bool FULL = false,
          int NJ0 = -1>
__device__ __forceinline__ void eval_events_fx(const ModelDev &md, const float (&r)[NE][NZ > 0 ? REC_NZ : REC_NK],
                                               EvState<NK, NZ> (&ev)[NE],
                                               const float2 *__restrict__ lc, int64_t lcn,
                                               const int64_t (&e)[NE])
{
    const int nK = FULL ? NK : md.n_res - NZ;   // FULL: the model fills the K* bucket
    float2 cc[NE];
    float sK[NE];
    float2 u[NE][3];
    float2 LK[NE][NK], LZ[NE][NZ > 0 ? NZ : 1];
    if constexpr (NE == 2) {
        // events e[0] and e[0] + 1 (even e[0]): one 16-byte load per resonance
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const float4 t = k < nK ? ld_pair<SM>(lc + k * lcn + e[0]) : make_float4(0.f, 0.f, 0.f, 0.f);
            LK[0][k] = make_float2(t.x, t.y);
            LK[1][k] = make_float2(t.z, t.w);
        }
#pragma unroll
        for (int z = 0; z < NZ; ++z) {
            const float4 t = ld_pair<SM>(lc + (nK + z) * lcn + e[0]);
            LZ[0][z] = make_float2(t.x, t.y);
            LZ[1][z] = make_float2(t.z, t.w);
        }
    } else {
#pragma unroll
        for (int j = 0; j < NE; ++j) {
#pragma unroll
            for (int k = 0; k < NK; ++k)
                LK[j][k] = k < nK ? __ldg(lc + k * lcn + e[j]) : make_float2(0.f, 0.f);
#pragma unroll
            for (int z = 0; z < NZ; ++z) LZ[j][z] = __ldg(lc + (nK + z) * lcn + e[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < NE; ++j) {
        const float cK = r[j][REC_CK], cpsi = r[j][REC_CPSI];
        sK[j] = sqrtf(fmaxf(0.0f, fmaf(-cK, cK, 1.0f)));
        cc[j] = make_float2(cK, cK);
        ev[j].cK = cK; ev[j].sK = sK[j];
        const float spsi = sqrtf(fmaxf(0.0f, fmaf(-cpsi, cpsi, 1.0f)));
        const float cph = r[j][REC_CPHI], sph = r[j][REC_SPHI];
        float d1p[3][2];
        wigner_1(cpsi, spsi, d1p);
#pragma unroll
        for (int x = 0; x < 2; ++x) {
            ev[j].Psi[0][x] = make_float2(cph * d1p[0][x], -sph * d1p[0][x]);
            ev[j].Psi[1][x] = make_float2(d1p[1][x], 0.0f);
            ev[j].Psi[2][x] = make_float2(cph * d1p[2][x], sph * d1p[2][x]);
        }
#pragma unroll
        for (int l = 0; l < 3; ++l) u[j][l] = make_float2(0.f, 0.f);
        if constexpr (LFM == 2) {
            ev[j].m = r[j][REC_M];
            ev[j].p = r[j][REC_P];
            ev[j].q = r[j][REC_Q];
            ev[j].invm = __frcp_rn(ev[j].m);
        }
    }
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        if (k < nK) {
            const ResDev &rs = md.res[k];
#pragma unroll
            for (int j = 0; j < NE; ++j) {
                if constexpr (LFM == 2) {
                    if (rs.fpos >= 0) LK[j][k] = lineshape(rs, ev[j].m, ev[j].invm, ev[j].p, ev[j].q).A;
                }
                if (NE == 2 && (NJ0 >= 0 ? k >= NK - NJ0 : rs.J == 0)) {
                    // d^0_00 = 1, no l = +-1 terms: the same bits as the general form
                    // (with one event per thread the branch costs more than it saves)
                    const float2 b0 = LK[j][k];
                    ev[j].B0[k] = b0;
                    ev[j].B1[k] = make_float2(0.f, 0.f);
                    cfma2p(u[j][1], md.kp[k][1], b0, make_float2(b0.y, b0.x));
                    continue;
                }
                float d0, d1;
                wigner_l0(rs, cc[j], sK[j], d0, d1);
                const float2 b0 = cscale(LK[j][k], d0), b1 = cscale(LK[j][k], d1);
                ev[j].B0[k] = b0;
                ev[j].B1[k] = b1;
                const float2 b0s = make_float2(b0.y, b0.x), b1s = make_float2(b1.y, b1.x);
                cfma2p(u[j][0], md.kp[k][0], b1, b1s);
                cfma2p(u[j][1], md.kp[k][1], b0, b0s);
                cfma2p(u[j][2], md.kp[k][2], b1, b1s);
            }
        } else {
#pragma unroll
            for (int j = 0; j < NE; ++j) ev[j].B0[k] = ev[j].B1[k] = make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int j = 0; j < NE; ++j)
#pragma unroll
        for (int x = 0; x < 2; ++x) {
            float2 a = make_float2(0.f, 0.f);
            cfma(a, ev[j].Psi[0][x], u[j][0]);
            // Psi_{0 xi} is real: the same bits as the complex form (whose zero term
            // enters its FMA chain first) in half the FMAs
            const float p1 = ev[j].Psi[1][x].x;
            a.x = fmaf(p1, u[j][1].x, a.x);
            a.y = fmaf(p1, u[j][1].y, a.y);
            cfma(a, ev[j].Psi[2][x], u[j][2]);
            ev[j].a[x] = a;
            if constexpr (MT) {
                float2 b = make_float2(0.f, 0.f);
                cfma_conj(b, ev[j].Psi[0][x], u[j][0]);
                b.x = fmaf(p1, u[j][1].x, b.x);
                b.y = fmaf(p1, u[j][1].y, b.y);
                cfma_conj(b, ev[j].Psi[2][x], u[j][2]);
                ev[j].ab[x] = b;
            }
        }
    if constexpr (NZ > 0) {
        if constexpr (LFM >= 1) {
#pragma unroll
            for (int j = 0; j < NE; ++j) {
                ev[j].mZ = r[j][REC_MZ];
                ev[j].pZ = r[j][REC_PZ];
                ev[j].qZ = r[j][REC_QZ];
                ev[j].invmZ = __frcp_rn(ev[j].mZ);
            }
        }
#pragma unroll
        for (int z = 0; z < NZ; ++z) {
            const ResDev &rs = md.zr[z];
            // the angular factors from the basis cache: rows n_res + 4 z + (Om0 x=0, Om0 x=1,
            // Om1 x=0, Om1 x=1)
            const float2 *zr = lc + (int64_t)(md.n_res + 4 * z) * lcn;
            if constexpr (NE == 2) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 t = ld_pair<SM>(zr + q * lcn + e[0]);
                    float2 *dst0 = q < 2 ? &ev[0].Om0[z][q] : &ev[0].Om1[z][q - 2];
                    float2 *dst1 = q < 2 ? &ev[1].Om0[z][q] : &ev[1].Om1[z][q - 2];
                    *dst0 = make_float2(t.x, t.y);
                    *dst1 = make_float2(t.z, t.w);
                }
            } else {
#pragma unroll
                for (int j = 0; j < NE; ++j)
#pragma unroll
                    for (int x = 0; x < 2; ++x) {
                        ev[j].Om0[z][x] = __ldg(zr + x * lcn + e[j]);
                        ev[j].Om1[z][x] = __ldg(zr + (2 + x) * lcn + e[j]);
                    }
            }
#pragma unroll
            for (int j = 0; j < NE; ++j) {
                float2 LA = LZ[j][z];
                if constexpr (LFM >= 1) {
                    if (rs.fpos >= 0) LA = lineshape(rs, ev[j].mZ, ev[j].invmZ, ev[j].pZ, ev[j].qZ).A;
                }
                ev[j].AZ[z] = LA;
#pragma unroll
                for (int x = 0; x < 2; ++x) {
                    const float2 o0 = ev[j].Om0[z][x], o1 = ev[j].Om1[z][x];
                    float2 s = make_float2(0.f, 0.f);
                    // NJ0 >= 0: every Z has both columns (the host checks)
                    if (NJ0 >= 0 || rs.zcol0 >= 0) cfma2p(s, md.zp[z][0], o0, make_float2(o0.y, o0.x));
                    if (NJ0 >= 0 || rs.zcol1 >= 0) cfma2p(s, md.zp[z][1], o1, make_float2(o1.y, o1.x));
                    cfma(ev[j].a[x], LA, s);
                    if constexpr (MT) {
                        const float2 c0 = make_float2(o0.x, -o0.y), c1 = make_float2(o1.x, -o1.y);
                        float2 sb = make_float2(0.f, 0.f);
                        if (NJ0 >= 0 || rs.zcol0 >= 0) cfma2p(sb, md.zp[z][0], c0, make_float2(c0.y, c0.x));
                        if (NJ0 >= 0 || rs.zcol1 >= 0) cfma2p(sb, md.zp[z][1], c1, make_float2(c1.y, c1.x));
                        cfma(ev[j].ab[x], LA, sb);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NE; ++j) {
        ev[j].S = cabs2(ev[j].a[0]) + cabs2(ev[j].a[1]);
        if constexpr (MT) ev[j].Sb = cabs2(ev[j].ab[0]) + cabs2(ev[j].ab[1]);
    }
}

// Compensated FP32 accumulator.
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum in FP64 (fixed order), added to the 128-bit accumulator acc.
template <int BLOCK>
__device__ __forceinline__ void block_accumulate(double v, double *smem, unsigned long long *acc,
                                                 unsigned *status)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) smem[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < BLOCK / 32; ++i) t += smem[i];
        acc128_add(acc, t, status);
    }
}

__device__ __forceinline__ void load_model(const ModelDev *g, ModelDev *s)
{
    const int n = sizeof(ModelDev) / 4;
    const int *src = reinterpret_cast<const int *>(g);
    int *dst = reinterpret_cast<int *>(s);
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

// The per-event data term of -2 ln L.  Without a background: ln S, and the
// adjoint scale 2/S.  With the Eq. 14 background (MIX): g = alpha eps S + beta hb
// = f / (p q) with alpha = P / I_eps, ln g, the scale 2 alpha eps / g, and the
// signal probability r = alpha eps S / g (its sum replaces N in dI/I).  ln is
// taken as ln(mantissa) + exponent ln 2.  Returns false when the logged value is
// not > 0 (a domain error).
template <bool MIX>
__device__ __forceinline__ bool data_term(const ModelDev &md, float S, const float *__restrict__ meps,
                                          const float *__restrict__ mhb, int64_t e, Kahan &lsum,
                                          int &esum, float &scale, float &r)
{
    float v = S, ae = 1.0f;
    if constexpr (MIX) {
        const float ep = __ldg(meps + e), hv = __ldg(mhb + e);
        ae = fmaf(md.mahi, ep, md.malo * ep);
        v = fmaf(ae, S, fmaf(md.mbhi, hv, md.mblo * hv));
    }
    if (!(v > 0.0f)) return false;
    int ex;
    float mant = frexpf(v, &ex);
    if (mant < 0.70710678f) { mant *= 2.0f; ex -= 1; }
    lsum.add(logf(mant));
    esum += ex;
    const float iv = __frcp_rn(v);
    scale = 2.0f * ae * iv;
    if constexpr (MIX) r = ae * S * iv;
    return true;
}

// MODE_SUM_LNS: data sum of ln S; MODE_SUM_WS: normalisation sum of w S;
// MODE_WRITE: S per event to out.
enum { MODE_SUM_LNS = 0, MODE_SUM_WS = 1, MODE_WRITE = 2 };

// Records read by the all-cached kernels (FX): all but phi (its cosine and sine
// are records); the K* (Z) masses and momenta only when floated K* (Z)
// lineshapes are computed per event (LFM 2, LFM >= 1); the Z-chain angles only
// when their angular factors are not read from the basis cache (ZC).
template <bool FX, int LFM = 0, bool ZC = false>
__host__ __device__ __forceinline__ constexpr bool record_used(int k)
{
    return !FX || !(k == REC_PHI || (LFM < 2 && (k == REC_M || k == REC_P || k == REC_Q)) ||
                    (LFM < 1 && (k == REC_MZ || k == REC_PZ || k == REC_QZ)) ||
                    (ZC && k >= REC_CZ && k <= REC_SA));
}

// Number of records the all-cached kernels read (record_used<true, LFM, true>).
template <int NREC, int LFM>
__host__ __device__ constexpr int records_used_fx()
{
    int c = 0;
    for (int k = 0; k < NREC; ++k) c += record_used<true, LFM, true>(k) ? 1 : 0;
    return c;
}

// Z-chain angular factors of one event (Eq. 10-11) for each muon helicity xi
// (x = 0: +1, x = 1: -1): with the Z's own d^J and its parity factor eta,
//   Om0 = e^{i xi alpha} d^J_00(theta_Z) d^1_{0 xi}(theta~_psi)            (l' = 0),
//   Om1 = e^{i xi alpha} [-d^J_{01} e^{i phi~} d^1_{1 xi} + eta d^J_{01} e^{-i phi~} d^1_{-1 xi}]
// in the kernels' normalisation (d1 = -sin P_J' stands for sqrt(J (J+1)) d^J_{10}).
// They do not depend on any parameter: the all-cached kernels read them from the
// basis cache, built with this same arithmetic.
__device__ __forceinline__ void z_angular(const ResDev &rs, float cZ, float ctz, float2 ephz, float ca,
                                          float sa, float2 (&o0)[2], float2 (&o1)[2])
{
    const float sZ = sqrtf(fmaxf(0.0f, fmaf(-cZ, cZ, 1.0f)));
    const float stz = sqrtf(fmaxf(0.0f, fmaf(-ctz, ctz, 1.0f)));
    float d1t[3][2];
    wigner_1(ctz, stz, d1t);
    float dz0, dz1;
    wigner_l0(rs, make_float2(cZ, cZ), sZ, dz0, dz1);
#pragma unroll
    for (int x = 0; x < 2; ++x) {
        const float2 eal = make_float2(ca, x == 0 ? sa : -sa);
        o0[x] = cscale(eal, dz0 * d1t[1][x]);
        float2 t = cscale(ephz, -dz1 * d1t[2][x]);
        const float2 ephm = make_float2(ephz.x, -ephz.y);
        t = cadd(t, cscale(ephm, (float)rs.eta * dz1 * d1t[0][x]));
        o1[x] = cmul(t, eal);
    }
}

template <int NK, int NZ, int MODE, int BLOCK, bool FX, bool MIX = false, bool MT = false>
__global__ void __launch_bounds__(BLOCK) k_eval(const float *__restrict__ rec, int64_t npad,
                                                int64_t n, int wrec, const ModelDev *__restrict__ gmd,
                                                unsigned long long *__restrict__ acc, float *__restrict__ S_out,
                                                unsigned *__restrict__ status,
                                                const float2 *__restrict__ lc,
                                                const float *__restrict__ meps = nullptr,
                                                const float *__restrict__ mhb = nullptr)
{
    constexpr int NREC = NZ > 0 ? REC_NZ : REC_NK;
    const ModelDev &md = c_md;   // gmd is its source (copied by with_const_table)
    __shared__ double red[BLOCK / 32];
    Kahan ksum;
    int esum = 0;
    bool bad = false;
    // One event per thread and iteration, coalesced scalar loads of every record.
    for (int64_t e = blockIdx.x * (int64_t)BLOCK + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * BLOCK) {
        float v[NREC];
#pragma unroll
        for (int k = 0; k < NREC; ++k) v[k] = record_used<FX>(k) ? __ldg(rec + k * npad + e) : 0.f;
        EvState<NK, NZ> ev;
        eval_event<NK, NZ, FX, MT>(md, v, ev, lc, npad, e);
        if (MODE == MODE_SUM_LNS) {
            float scale, r;
            if (!data_term<MIX>(md, observed_S<MT>(md, ev), meps, mhb, e, ksum, esum, scale, r)) {
                bad = true;
                continue;
            }
        } else if (MODE == MODE_SUM_WS) {
            ksum.add(__ldg(rec + wrec * npad + e) * ev.S);
        } else {
            S_out[e] = observed_S<MT>(md, ev);
        }
    }
    if (MODE == MODE_WRITE) return;
    if (bad) atomicOr(status, 1u);
    double tot = ksum.value();
    if (MODE == MODE_SUM_LNS) tot += (double)esum * 0.69314718055994530942;
    block_accumulate<BLOCK>(tot, red, acc, status);
}

// ---------------------------------------------------------------------------
// Adjoint gradient.  Slots (internal order), after slot 0 = ln S or w S sum:
//   K* k:  1 + 6k + {0..5}   dS/d(Re, Im) c for l = -1, 0, +1
//   Z z:   1 + 6NK + 4z + {0..3}  dS/d(Re, Im) c for the l' = 0 and l' = +-1 columns
//   R:     1 + 6NK + 4NZ + 2 fpos + {0, 1}  dS/dM, dS/dG0 of the floated resonance
//          with index fpos among the floated ones (no slots for fixed resonances)
// Every slot is scaled by 1/S (data) or w (normalisation).  In slot pairs
// (below): K* k, l at pair 3k + l; Z z at pairs 3NK + 2z + {0, 1}; a floated
// resonance at pair 3NK + 2NZ + fpos.
// ---------------------------------------------------------------------------

// dA/dM and dA/dG0 from Eq. 2-3: A = N / D, D = M^2 - m^2 - i M Gamma(m).  The
// per-resonance derivative constants are double-float: a systematic FP32
// rounding of them would not cancel between the data and normalisation terms.
__device__ __forceinline__ void lineshape_derivs(const ResDev &rs, float2 A, float2 invD,
                                                 float MG, float2 &dAdM, float2 &dAdG)
{
    // dD/dM = 2M - i MG dln(MG)/dM, and f = dln A/dM = dN - (dD/dM)/D with the
    // 2 M_lo part of dD/dM inside the FMAs.  The constant dN enters the chain
    // before the final rounding of Re f: subtracting the rounded Re((dD/dM)/D)
    // from dN would round dN onto that value's FP32 grid at the same offset for
    // every event of a binade, a coherent error in the mass gradient (measured
    // 2e-7 of the cancelling sum over the K*(892) peak; 5e-9 in this order).
    const float2 dD = make_float2(2.0f * rs.Mhi, -fmaf(MG, rs.dGhi, MG * rs.dGlo));
    const float c0 = fmaf(-2.0f * rs.Mlo, invD.x, rs.dNlo) + rs.dNhi;
    const float2 f = make_float2(fmaf(-dD.x, invD.x, fmaf(dD.y, invD.y, c0)),
                                 -fmaf(dD.x, invD.y, fmaf(dD.y, invD.x, 2.0f * rs.Mlo * invD.y)));
    dAdM = cmul(A, f);
    // dA/dG0 = -A (dD/dG0)/D = i A (MG / G0) / D
    const float2 g = cmul(A, invD);
    const float s = fmaf(MG, rs.iGhi, MG * rs.iGlo);
    dAdG = make_float2(-g.y * s, g.x * s);
}

// End of an adjoint CTA: FP64 block sum of ln S (or w S), compensated FP32 block
// sums of every gradient slot in thread order, each added to its 128-bit
// accumulator (acc + 2 s for slot s).
template <bool NORM, int BLOCK>
__device__ __forceinline__ void grad_block_tail(const Kahan &acc0, int esum, bool bad,
                                                unsigned *__restrict__ status, double *red,
                                                const float2 *gsl, unsigned long long *__restrict__ acc,
                                                int nslot)
{
    const int tid = threadIdx.x;
    if (bad) atomicOr(status, 1u);
    double t0 = acc0.value();
    if (!NORM) t0 += (double)esum * 0.69314718055994530942;
    t0 = warp_sum(t0);
    if ((tid & 31) == 0) red[tid >> 5] = t0;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int ww = 0; ww < BLOCK / 32; ++ww) t += red[ww];
        acc128_add(acc, t, status);
    }
    // Block sums of every gradient slot as compensated FP32 (Neumaier) sums
    // written once in FP64: the FP32 slot values are summed to about 2^-48 of
    // sum |x| without the FP64 pipe, which on this GPU runs at a small fraction of
    // the FP32 rate.  Thread s sums slot s over the threads j in the rotated
    // order (j + pair index) mod BLOCK: the 16 pairs and 2 components a warp reads
    // at once then sit in 32 different banks (in thread order every read of a
    // warp fell into 2 banks, 16-way conflicts).  The order is fixed per slot.
    static_assert((BLOCK & (BLOCK - 1)) == 0, "BLOCK is a power of two");
    for (int s2 = 1 + tid; s2 < nslot; s2 += BLOCK) {
        const float *col = reinterpret_cast<const float *>(gsl + ((s2 - 1) >> 1) * BLOCK) + ((s2 - 1) & 1);
        const int rot = (s2 - 1) >> 1;
        float sm = 0.f, cm = 0.f;
        for (int j = 0; j < BLOCK; ++j) {
            const float x = col[2 * ((j + rot) & (BLOCK - 1))];
            const float t = sm + x;
            cm += (fabsf(sm) >= fabsf(x)) ? (sm - t) + x : (x - t) + sm;
            sm = t;
        }
        acc128_add(acc + 2 * s2, (double)sm + (double)cm, status);
    }
}

// All-cached adjoint kernel with NE events per thread and iteration (NE = 2: an
// adjacent pair 2t, 2t + 1; NE = 1: one event), every warp load coalesced.  The
// constants of a resonance and each gradient slot pair are read once for the NE
// events.  An event index at or beyond n holds a padding or repeated event that
// gets zero weight.  LFM selects which floated lineshapes are computed per event
// (eval_events_fx), MIX the Eq. 14 background, MT the flavour mistag.
// FULL: the model's K* count equals the bucket NK.  NJ0 >= 0 (with FULL): the last
// NJ0 K* of the internal order are the scalars (J = 0), the others have J > 0, and
// every Z has both columns (l' = 0 and l' = +-1).
template <int NK, int NZ, bool NORM, int BLOCK, int NE, int CTAS, int LFM, bool MIX = false,
          bool MT = false, bool STG = false, bool FULL = false, int NJ0 = -1>
__global__ void __launch_bounds__(BLOCK, CTAS) k_grad_fx(const float *__restrict__ rec, int64_t npad,
                                                         int64_t n, int wrec,
                                                         unsigned long long *__restrict__ acc,
                                                         unsigned *__restrict__ status,
                                                         const float2 *__restrict__ lc, int nslot,
                                                         const float *__restrict__ meps,
                                                         const float *__restrict__ mhb,
                                                         unsigned long long *__restrict__ acc_r,
                                                         FinishArgs fin)
{
    constexpr int NREC = NZ > 0 ? REC_NZ : REC_NK;
    const ModelDev &md = c_md;
    __shared__ double red[BLOCK / 32];
    extern __shared__ float2 gsl[];  // [(nslot - 1) / 2][BLOCK]
    const int tid = threadIdx.x;
    const int npair = (nslot - 1) >> 1;
    for (int i = 0; i < npair; ++i) gsl[i * BLOCK + tid] = make_float2(0.f, 0.f);
    if constexpr (!NORM) {
        // fused finish: rows of G u and G v, 4 per CTA, by warp 0 of the first CTAs
        if (fin.ticket && tid < 32 && (int)blockIdx.x < fin.ncol) gram_rows_for_finish(fin, blockIdx.x);
    }
    float2 *g = gsl + tid;
    Kahan acc0, rsum;
    int esum = 0;
    bool bad = false;
    const int nK = FULL ? NK : md.n_res - NZ;   // FULL: the model fills the K* bucket
    // NE = 2: thread t takes the adjacent events 2t and 2t + 1 of its stride
    // (8-byte record loads; e0 is even and npad a multiple of 4, so e0 + 1 < npad
    // holds a real or a padding event); otherwise events e0 + j * stride.  The
    // records and cached lineshapes are read once per launch: evict-first loads
    // (ld.global.cs) keep them from displacing the small per-evaluation data in L2.
    const int64_t estride = (int64_t)gridDim.x * BLOCK;
    const int64_t first = NE == 2 ? 2 * (blockIdx.x * (int64_t)BLOCK + tid) : blockIdx.x * (int64_t)BLOCK + tid;
    // STG (NE = 2): after the slot pairs, the staging slots of the records read
    // ([NRU][BLOCK] pairs) and of the cache rows ([nrow][BLOCK] pairs of float2)
    static_assert(!STG || NE == 2, "staging takes adjacent event pairs");
    constexpr int NRU = records_used_fx<NREC, LFM>();
    float2 *stg_rec = gsl + npair * BLOCK;
    float4 *stg_lc = reinterpret_cast<float4 *>(stg_rec + NRU * BLOCK);
    // cache rows: the nK K* lineshapes, then NZ Z lineshapes and 4 NZ Z factors
    float4 *stg_z = stg_lc + nK * BLOCK + tid;
    auto stage = [&](int64_t es) {
        int ru = 0;
#pragma unroll
        for (int k = 0; k < NREC; ++k) {
            if (!record_used<true, LFM, true>(k)) continue;
            cp_async_8(stg_rec + ru * BLOCK + tid, rec + k * npad + es);
            ++ru;
        }
        const float2 *src = lc + es;
#pragma unroll
        for (int k = 0; k < NK; ++k)
            if (k < nK) cp_async_16(stg_lc + k * BLOCK + tid, src + (int64_t)k * npad);
        src += (int64_t)nK * npad;
#pragma unroll
        for (int r = 0; r < 5 * NZ; ++r) cp_async_16(stg_z + r * BLOCK, src + (int64_t)r * npad);
        cp_async_commit();
    };
    if constexpr (STG) {
        if (first < n) stage(first);
    }
    for (int64_t e0 = first; e0 < n; e0 += NE * estride) {
        int64_t e[NE];
        bool valid[NE];
        float v[NE][NREC];
        if constexpr (NE == 2) {
            e[0] = e0;
            e[1] = e0 + 1;
            valid[0] = true;
            valid[1] = e0 + 1 < n;
            if constexpr (STG) cp_async_wait_all();   // this pair's slots have landed
            int ru = 0;
#pragma unroll
            for (int k = 0; k < NREC; ++k) {
                float2 t = make_float2(0.f, 0.f);
                if (record_used<true, LFM, true>(k)) {
                    if constexpr (STG) t = lds2(stg_rec + ru * BLOCK + tid);
                    else t = __ldcs(reinterpret_cast<const float2 *>(rec + k * npad + e0));
                    ++ru;
                }
                v[0][k] = t.x;
                v[1][k] = t.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < NE; ++j) {
                const int64_t ej = e0 + j * estride;
                valid[j] = ej < n;
                e[j] = valid[j] ? ej : e0;
#pragma unroll
                for (int k = 0; k < NREC; ++k)
                    v[j][k] = record_used<true, LFM, true>(k) ? __ldg(rec + k * npad + e[j]) : 0.f;
            }
        }
        EvState<NK, NZ> ev[NE];
        if constexpr (STG) {
            const int64_t es[NE] = {2 * tid, 2 * tid + 1};   // the thread's slot (in float2)
            eval_events_fx<NK, NZ, NE, LFM, MT, true, FULL, NJ0>(
                md, v, ev, reinterpret_cast<const float2 *>(stg_lc), 2 * BLOCK, es);
            // S depends on every staged value, so once both are computed every
            // ld.shared of the slots has completed: restage them for the next pair
            asm volatile("" ::"f"(ev[0].S), "f"(ev[1].S));
            if (e0 + NE * estride < n) stage(e0 + NE * estride);
        } else {
            eval_events_fx<NK, NZ, NE, LFM, MT, false, FULL, NJ0>(md, v, ev, lc, npad, e);
        }
        float2 as[NE][2], asb[NE][2];
#pragma unroll
        for (int j = 0; j < NE; ++j) {
            float scale = 0.f;
            if (valid[j]) {
                if (!NORM) {
                    float r = 0.f;
                    if (!data_term<MIX>(md, observed_S<MT>(md, ev[j]), meps, mhb, e[j], acc0, esum,
                                        scale, r)) {
                        bad = true;
                        scale = 0.f;
                    } else if constexpr (MIX) {
                        rsum.add(r);
                    }
                } else {
                    const float w = __ldg(rec + wrec * npad + e[j]);
                    acc0.add(w * ev[j].S);
                    scale = 2.0f * w;
                }
            }
            // mistag: (1 - w) on the amplitudes, w on the mirrored ones
            const float sa = MT ? scale * md.m1w : scale, sb = scale * md.mwhi;
#pragma unroll
            for (int x = 0; x < 2; ++x) {
                as[j][x] = cscale(ev[j].a[x], sa);
                asb[j][x] = MT ? cscale(ev[j].ab[x], sb) : make_float2(0.f, 0.f);
            }
        }
        float2 wl[NE][3];
#pragma unroll
        for (int j = 0; j < NE; ++j)
#pragma unroll
            for (int l = 0; l < 3; ++l)
                wl[j][l] = l == 1 ? adj_w_real<MT>(as[j], asb[j], ev[j].Psi[l]) : adj_w<MT>(as[j], asb[j], ev[j].Psi[l]);
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            if (k >= nK) continue;
            // a scalar: only the l = 0 slot moves (B1 = 0)
            const bool j0 = NE == 2 && (NJ0 >= 0 ? k >= NK - NJ0 : md.res[k].J == 0);
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                if (j0 && l != 1) continue;
                float2 gp = g[(3 * k + l) * BLOCK];
#pragma unroll
                for (int j = 0; j < NE; ++j) {
                    const float2 B = l == 0 ? make_float2(-ev[j].B1[k].x, -ev[j].B1[k].y)
                                            : (l == 1 ? ev[j].B0[k] : ev[j].B1[k]);
                    gp.x = fmaf(B.x, wl[j][l].x, fmaf(-B.y, wl[j][l].y, gp.x));
                    gp.y = fmaf(-B.x, wl[j][l].y, fmaf(-B.y, wl[j][l].x, gp.y));
                }
                g[(3 * k + l) * BLOCK] = gp;
            }
            if constexpr (LFM == 2) {
                const ResDev &rs = md.res[k];
                if (rs.fpos >= 0) {
                    // floated K*: y = sum_l c_{k,l} d_l w_l, then scale dS/dM = Re(dA/dM y)
                    float2 gmk = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < NE; ++j) {
                        float d0, d1;
                        wigner_l0(rs, make_float2(ev[j].cK, ev[j].cK), ev[j].sK, d0, d1);
                        const float2 y = kstar_adj_y(md, k, d0, d1, wl[j]);
                        const LineOut L = lineshape(rs, ev[j].m, ev[j].invm, ev[j].p, ev[j].q);
                        float2 dM, dG;
                        lineshape_derivs(rs, L.A, L.invD, L.MG, dM, dG);
                        gmk.x += cmul(dM, y).x;
                        gmk.y += cmul(dG, y).x;
                    }
                    float2 &gm = g[(3 * NK + 2 * NZ + rs.fpos) * BLOCK];
                    gm.x += gmk.x;
                    gm.y += gmk.y;
                }
            }
        }
        if constexpr (NZ > 0) {
#pragma unroll
            for (int z = 0; z < NZ; ++z) {
                const ResDev &rs = md.zr[z];
                float2 g0 = g[(3 * NK + 2 * z) * BLOCK], g1 = g[(3 * NK + 2 * z + 1) * BLOCK];
                float2 gmg = make_float2(0.f, 0.f);   // scale dS/dM, dS/dG0 of a floated Z
#pragma unroll
                for (int j = 0; j < NE; ++j) {
                    float2 w0 = make_float2(0.f, 0.f), w1 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int x = 0; x < 2; ++x) {
                        cfma_conj(w0, as[j][x], ev[j].Om0[z][x]);
                        cfma_conj(w1, as[j][x], ev[j].Om1[z][x]);
                        if constexpr (MT) {
                            cfma_conjp(w0, asb[j][x], ev[j].Om0[z][x]);
                            cfma_conjp(w1, asb[j][x], ev[j].Om1[z][x]);
                        }
                    }
                    const float2 A = ev[j].AZ[z];
                    g0.x = fmaf(A.x, w0.x, fmaf(-A.y, w0.y, g0.x));
                    g0.y = fmaf(-A.x, w0.y, fmaf(-A.y, w0.x, g0.y));
                    g1.x = fmaf(A.x, w1.x, fmaf(-A.y, w1.y, g1.x));
                    g1.y = fmaf(-A.x, w1.y, fmaf(-A.y, w1.x, g1.y));
                    if constexpr (LFM >= 1) {
                        if (rs.fpos >= 0) {
                            // y = sum_l' c_l' w_l', then scale dS/dM = Re(dA/dM y)
                            const float2 y = z_adj_y(md, rs, z, w0, w1);
                            const LineOut L = lineshape(rs, ev[j].mZ, ev[j].invmZ, ev[j].pZ, ev[j].qZ);
                            float2 dM, dG;
                            lineshape_derivs(rs, L.A, L.invD, L.MG, dM, dG);
                            gmg.x += cmul(dM, y).x;
                            gmg.y += cmul(dG, y).x;
                        }
                    }
                }
                g[(3 * NK + 2 * z) * BLOCK] = g0;
                g[(3 * NK + 2 * z + 1) * BLOCK] = g1;
                if constexpr (LFM >= 1) {
                    if (rs.fpos >= 0) {
                        float2 &gm = g[(3 * NK + 2 * NZ + rs.fpos) * BLOCK];
                        gm.x += gmg.x;
                        gm.y += gmg.y;
                    }
                }
            }
        }
    }
    grad_block_tail<NORM, BLOCK>(acc0, esum, bad, status, red, gsl, acc, nslot);
    if constexpr (MIX) {
        __syncthreads();
        block_accumulate<BLOCK>(rsum.value(), red, acc_r, status);
    }
    if constexpr (!NORM) {
        // Gram path: the CTA that draws the last ticket finishes the evaluation,
        // once every CTA's sums are in the accumulators (each thread fences its
        // atomics before its CTA takes a ticket), in the slot memory, which the
        // block tail no longer reads.
        if (fin.ticket) {
            __shared__ int last;
            __threadfence();
            __syncthreads();
            if (tid == 0) last = atomicAdd(fin.ticket, 1u) == gridDim.x - 1;
            __syncthreads();
            if (last) {
                __threadfence();
                finish_gram_body(fin, reinterpret_cast<double *>(gsl));
            }
        }
    }
}

// Per-thread gradient accumulators live in shared memory, which keeps the
// register count low enough for 4 blocks/SM.  Slots come in (Re, Im) or
// (M, Gamma0) pairs, slots 1 + 2p and 2 + 2p forming pair p; pair p of thread t
// is one float2 at p * BLOCK + t, so each update is one 64-bit load and store
// and a warp's accesses cover every bank twice (two wavefronts, no conflict).
// Events are read one per iteration with coalesced scalar loads.
template <int NK, int NZ, bool NORM, int BLOCK, bool MIX = false, bool MT = false>
__global__ void __launch_bounds__(BLOCK, GRAD_CTAS_PER_SM) k_grad(const float *__restrict__ rec, int64_t npad,
                                                   int64_t n, int wrec, const ModelDev *__restrict__ gmd,
                                                   unsigned long long *__restrict__ acc,
                                                   unsigned *__restrict__ status,
                                                   const float2 *__restrict__ lc, int nslot,
                                                   const float *__restrict__ meps,
                                                   const float *__restrict__ mhb,
                                                   unsigned long long *__restrict__ acc_r)
{
    constexpr int NREC = NZ > 0 ? REC_NZ : REC_NK;
    const ModelDev &md = c_md;   // gmd is its source (copied by with_const_table)
    __shared__ double red[BLOCK / 32];
    extern __shared__ float2 gsl[];  // [(nslot - 1) / 2][BLOCK]
    const int tid = threadIdx.x;
    const int npair = (nslot - 1) >> 1;
    for (int i = 0; i < npair; ++i) gsl[i * BLOCK + tid] = make_float2(0.f, 0.f);
    float2 *g = gsl + tid;           // g[p * BLOCK] = slot pair p of this thread
    Kahan acc0, rsum;
    int esum = 0;
    bool bad = false;
    const int nK = md.n_res - NZ;
    for (int64_t e = blockIdx.x * (int64_t)BLOCK + tid; e < n; e += (int64_t)gridDim.x * BLOCK) {
        float v[NREC];
#pragma unroll
        for (int k = 0; k < NREC; ++k) v[k] = __ldg(rec + k * npad + e);
        EvState<NK, NZ> ev;
        eval_event<NK, NZ, false, MT>(md, v, ev, lc, npad, e);
        float scale;
        if (!NORM) {
            float r = 0.f;
            if (!data_term<MIX>(md, observed_S<MT>(md, ev), meps, mhb, e, acc0, esum, scale, r)) {
                bad = true;
                continue;
            }
            if constexpr (MIX) rsum.add(r);
        } else {
            const float w = __ldg(rec + wrec * npad + e);
            acc0.add(w * ev.S);
            scale = 2.0f * w;
        }
        // The scaled amplitudes as_xi = scale a_xi carry the 1/S (data) or w
        // (normalisation) factor, so every slot update below is two FMAs.
        float2 as[2];
#pragma unroll
        for (int x = 0; x < 2; ++x) as[x] = cscale(ev.a[x], MT ? scale * md.m1w : scale);
        float2 asb[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if constexpr (MT) {
#pragma unroll
            for (int x = 0; x < 2; ++x) asb[x] = cscale(ev.ab[x], scale * md.mwhi);
        }
        // w_l = sum_xi conj(as_xi) Psi_{l xi}
        float2 wl[3];
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            float2 t = make_float2(0.f, 0.f);
            cfma_conj(t, as[0], ev.Psi[l][0]);
            cfma_conj(t, as[1], ev.Psi[l][1]);
            if constexpr (MT) {
                cfma_conjp(t, asb[0], ev.Psi[l][0]);
                cfma_conjp(t, asb[1], ev.Psi[l][1]);
            }
            wl[l] = t;
        }
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            if (k >= nK) continue;
            const ResDev &rs = md.res[k];
            // scale dS/d(Re, Im) c_{k,l} = (Re, -Im) of B_l w_l, with B_{-1} = -B1,
            // B_0 = B0, B_{+1} = B1 (unused slots of a J = 0 state receive 0).
            const float2 Bl[3] = {make_float2(-ev.B1[k].x, -ev.B1[k].y), ev.B0[k], ev.B1[k]};
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                float2 gp = g[(3 * k + l) * BLOCK];
                gp.x = fmaf(Bl[l].x, wl[l].x, fmaf(-Bl[l].y, wl[l].y, gp.x));
                gp.y = fmaf(-Bl[l].x, wl[l].y, fmaf(-Bl[l].y, wl[l].x, gp.y));
                g[(3 * k + l) * BLOCK] = gp;
            }
            if (rs.fpos >= 0) {
                // y = sum_l c_{k,l} d_l w_l, then scale dS/dM = Re(dA/dM y)
                float d0, d1;
                wigner_l0(rs, make_float2(ev.cK, ev.cK), ev.sK, d0, d1);
                const float2 y = kstar_adj_y(md, k, d0, d1, wl);
                const LineOut L = lineshape(rs, ev.m, ev.invm, ev.p, ev.q);
                float2 dM, dG;
                lineshape_derivs(rs, L.A, L.invD, L.MG, dM, dG);
                const float2 a = cmul(dM, y), b = cmul(dG, y);
                float2 &gm = g[(3 * NK + 2 * NZ + rs.fpos) * BLOCK];
                gm.x += a.x;
                gm.y += b.x;
            }
        }
        if constexpr (NZ > 0) {
#pragma unroll
            for (int z = 0; z < NZ; ++z) {
                const ResDev &rs = md.zr[z];
                float2 w0 = make_float2(0.f, 0.f), w1 = make_float2(0.f, 0.f);
#pragma unroll
                for (int x = 0; x < 2; ++x) {
                    cfma_conj(w0, as[x], ev.Om0[z][x]);
                    cfma_conj(w1, as[x], ev.Om1[z][x]);
                    if constexpr (MT) {
                        cfma_conjp(w0, asb[x], ev.Om0[z][x]);
                        cfma_conjp(w1, asb[x], ev.Om1[z][x]);
                    }
                }
                const float2 A = ev.AZ[z];
                float2 g0 = g[(3 * NK + 2 * z) * BLOCK], g1 = g[(3 * NK + 2 * z + 1) * BLOCK];
                g0.x = fmaf(A.x, w0.x, fmaf(-A.y, w0.y, g0.x));
                g0.y = fmaf(-A.x, w0.y, fmaf(-A.y, w0.x, g0.y));
                g1.x = fmaf(A.x, w1.x, fmaf(-A.y, w1.y, g1.x));
                g1.y = fmaf(-A.x, w1.y, fmaf(-A.y, w1.x, g1.y));
                g[(3 * NK + 2 * z) * BLOCK] = g0;
                g[(3 * NK + 2 * z + 1) * BLOCK] = g1;
                if (rs.fpos >= 0) {
                    const float2 y = z_adj_y(md, rs, z, w0, w1);
                    const LineOut L = lineshape(rs, ev.mZ, ev.invmZ, ev.pZ, ev.qZ);
                    float2 dM, dG;
                    lineshape_derivs(rs, L.A, L.invD, L.MG, dM, dG);
                    const float2 a = cmul(dM, y), b = cmul(dG, y);
                    float2 &gm = g[(3 * NK + 2 * NZ + rs.fpos) * BLOCK];
                    gm.x += a.x;
                    gm.y += b.x;
                }
            }
        }
    }
    grad_block_tail<NORM, BLOCK>(acc0, esum, bad, status, red, gsl, acc, nslot);
    if constexpr (MIX) {
        __syncthreads();
        block_accumulate<BLOCK>(rsum.value(), red, acc_r, status);
    }
}

constexpr int EVAL_BLOCK = 256;
constexpr int GRAD_BLOCK = 128;

template <int NK, int NZ, bool FX>
cudaError_t launch_eval_fx(const LaunchArgs &a, int mode)
{
    return with_const_table(a.md, a.stream, [&]() {
        switch (mode) {
        case MODE_SUM_LNS: {
            auto kern = k_eval<NK, NZ, MODE_SUM_LNS, EVAL_BLOCK, FX, false, false>;
            if (a.mix_eps && a.mt) kern = k_eval<NK, NZ, MODE_SUM_LNS, EVAL_BLOCK, FX, true, true>;
            else if (a.mix_eps) kern = k_eval<NK, NZ, MODE_SUM_LNS, EVAL_BLOCK, FX, true, false>;
            else if (a.mt) kern = k_eval<NK, NZ, MODE_SUM_LNS, EVAL_BLOCK, FX, false, true>;
            kern<<<a.grid, EVAL_BLOCK, 0, a.stream>>>(a.rec, a.npad, a.n, a.wrec, a.md, a.acc, a.out,
                                                     a.status, a.lcache, a.mix_eps, a.mix_hb);
            break;
        }
        case MODE_SUM_WS:
            k_eval<NK, NZ, MODE_SUM_WS, EVAL_BLOCK, FX><<<a.grid, EVAL_BLOCK, 0, a.stream>>>(
                a.rec, a.npad, a.n, a.wrec, a.md, a.acc, a.out, a.status, a.lcache);
            break;
        default:
            if (a.mt)
                k_eval<NK, NZ, MODE_WRITE, EVAL_BLOCK, FX, false, true><<<a.grid, EVAL_BLOCK, 0, a.stream>>>(
                    a.rec, a.npad, a.n, a.wrec, a.md, a.acc, a.out, a.status, a.lcache);
            else
                k_eval<NK, NZ, MODE_WRITE, EVAL_BLOCK, FX><<<a.grid, EVAL_BLOCK, 0, a.stream>>>(
                    a.rec, a.npad, a.n, a.wrec, a.md, a.acc, a.out, a.status, a.lcache);
            break;
        }
        return cudaGetLastError();
    });
}

template <int NK, int NZ>
cudaError_t launch_eval_t(const LaunchArgs &a, int mode)
{
    return (a.lcache && a.all_fixed) ? launch_eval_fx<NK, NZ, true>(a, mode)
                                     : launch_eval_fx<NK, NZ, false>(a, mode);
}

template <int NK, int NZ, bool NORM, bool FX>
cudaError_t launch_grad_k(const LaunchArgs &a)
{
    size_t smem = (size_t)a.nslot * GRAD_BLOCK * sizeof(float);
    if (FX && !NORM && a.fin.ticket) smem = std::max(smem, finish_gram_smem(a.fin.ncol));
    constexpr int EPT = GRAD_EVENTS_PER_THREAD_CACHED, CPS = GRAD_CTAS_PER_SM_CACHED;
    constexpr int CPS1 = GRAD_CTAS_PER_SM_KFLOAT;
    const bool mix = !NORM && a.mix_eps != nullptr;
    if constexpr (FX) {
        // lfm: 0 all lineshapes cached; 1 the floated Z computed per event (two events
        // per thread); 2 floated K* too (one event per thread, for registers)
        const int lfm = a.all_fixed ? 0 : (a.kstar_fixed ? 1 : 2);
        using KernT = decltype(&k_grad_fx<NK, NZ, NORM, GRAD_BLOCK, EPT, CPS, 0>);
        KernT kern = lfm == 0 ? k_grad_fx<NK, NZ, NORM, GRAD_BLOCK, EPT, CPS, 0>
                   : lfm == 1 ? k_grad_fx<NK, NZ, NORM, GRAD_BLOCK, EPT, CPS, 1>
                              : k_grad_fx<NK, NZ, NORM, GRAD_BLOCK, 1, CPS1, 2>;
        // Staging of the next event pair in shared memory (STG) for the all-cached
        // mode, where the slots and the staging still leave room for CPS CTAs per SM
        // (with the floated Z computed per event, 168 registers, it measured 4 %
        // slower).
        constexpr int NREC = NZ > 0 ? REC_NZ : REC_NK;
        const size_t stg = (size_t)((a.nslot - 1) / 2) * GRAD_BLOCK * sizeof(float2) +
                           (size_t)records_used_fx<NREC, 0>() * GRAD_BLOCK * sizeof(float2) +
                           (size_t)a.nrow * GRAD_BLOCK * sizeof(float4);
        const bool use_stg = lfm == 0 && !mix && !a.mt && EPT == 2 &&
                             (size_t)CPS * (std::max(stg, smem) + 1024) <= 228 * 1024;
        // FULL: the model fills its K* bucket, so no run-time test of the K* count
        const bool full = a.nk == NK;
        bool structured = false;   // a structure variant of an unstaged data kernel
        if (use_stg) {
            smem = std::max(smem, stg);
            kern = full ? k_grad_fx<NK, NZ, NORM, GRAD_BLOCK, EPT, CPS, 0, false, false, true, true>
                        : k_grad_fx<NK, NZ, NORM, GRAD_BLOCK, EPT, CPS, 0, false, false, true>;
            if constexpr (!NORM) {
                // the data kernel also with the scalars' positions fixed (up to three)
                // when every Z has both columns
                if (full && a.zboth) switch (a.nj0) {
                    case 0: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, false, false, true, true, 0>; break;
                    case 1: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, false, false, true, true, 1>; break;
                    case 2: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, false, false, true, true, 2>; break;
                    case 3: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, false, false, true, true, 3>; break;
                    default: break;
                    }
            }
        } else if (!NORM && lfm == 0 && full && a.zboth && a.nj0 <= 3 && !a.mt) {
            // unstaged data kernel (the slots and staging of two Z exceed 3 CTAs/SM, or the
            // Eq. 14 background) with the model's structure fixed
            if constexpr (!NORM) {
            if (mix) switch (a.nj0) {
                case 0: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, true, false, false, true, 0>; break;
                case 1: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, true, false, false, true, 1>; break;
                case 2: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, true, false, false, true, 2>; break;
                default: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, true, false, false, true, 3>; break;
                }
            else switch (a.nj0) {
                case 0: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, false, false, false, true, 0>; break;
                case 1: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, false, false, false, true, 1>; break;
                case 2: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, false, false, false, true, 2>; break;
                default: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, false, false, false, true, 3>; break;
                }
            structured = true;
            }
        } else if (lfm == 1 && full && !mix && !a.mt) {
            kern = k_grad_fx<NK, NZ, NORM, GRAD_BLOCK, EPT, CPS, 1, false, false, false, true>;
            // and with the scalars' positions and the Z columns fixed
            if (a.zboth) switch (a.nj0) {
                case 0: kern = k_grad_fx<NK, NZ, NORM, GRAD_BLOCK, EPT, CPS, 1, false, false, false, true, 0>; break;
                case 1: kern = k_grad_fx<NK, NZ, NORM, GRAD_BLOCK, EPT, CPS, 1, false, false, false, true, 1>; break;
                case 2: kern = k_grad_fx<NK, NZ, NORM, GRAD_BLOCK, EPT, CPS, 1, false, false, false, true, 2>; break;
                case 3: kern = k_grad_fx<NK, NZ, NORM, GRAD_BLOCK, EPT, CPS, 1, false, false, false, true, 3>; break;
                default: break;
                }
        }
        if constexpr (!NORM) {
            switch (use_stg || structured ? -1 : lfm * 4 + (mix ? 2 : 0) + (a.mt ? 1 : 0)) {
            case 1: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, false, true>; break;
            case 2: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, true, false>; break;
            case 3: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 0, true, true>; break;
            case 5: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 1, false, true>; break;
            case 6: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 1, true, false>; break;
            case 7: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, EPT, CPS, 1, true, true>; break;
            case 9: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, 1, CPS1, 2, false, true>; break;
            case 10: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, 1, CPS1, 2, true, false>; break;
            case 11: kern = k_grad_fx<NK, NZ, false, GRAD_BLOCK, 1, CPS1, 2, true, true>; break;
            default: break;
            }
        }
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        return with_const_table(a.md, a.stream, [&]() {
            kern<<<a.grid, GRAD_BLOCK, smem, a.stream>>>(a.rec, a.npad, a.n, a.wrec, a.acc, a.status,
                                                         a.lcache, a.nslot, a.mix_eps, a.mix_hb,
                                                         a.acc_r, a.fin);
            return cudaGetLastError();
        });
    } else {
        auto kern = k_grad<NK, NZ, NORM, GRAD_BLOCK>;
        if constexpr (!NORM) {
            if (mix && a.mt) kern = k_grad<NK, NZ, false, GRAD_BLOCK, true, true>;
            else if (mix) kern = k_grad<NK, NZ, false, GRAD_BLOCK, true, false>;
            else if (a.mt) kern = k_grad<NK, NZ, false, GRAD_BLOCK, false, true>;
        }
        if (smem > 48 * 1024) {   // above the default dynamic shared-memory limit
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        return with_const_table(a.md, a.stream, [&]() {
            kern<<<a.grid, GRAD_BLOCK, smem, a.stream>>>(a.rec, a.npad, a.n, a.wrec, a.md, a.acc,
                                                         a.status, a.lcache, a.nslot, a.mix_eps,
                                                         a.mix_hb, a.acc_r);
            return cudaGetLastError();
        });
    }
}

template <int NK, int NZ>
cudaError_t launch_grad_t(const LaunchArgs &a, bool norm)
{
    const bool fx = a.lcache != nullptr;
    if (norm) return fx ? launch_grad_k<NK, NZ, true, true>(a) : launch_grad_k<NK, NZ, true, false>(a);
    return fx ? launch_grad_k<NK, NZ, false, true>(a) : launch_grad_k<NK, NZ, false, false>(a);
}

// Basis cache: A'_R (Eq. 2-3 without its column constant) of every resonance for
// every event of a set, [internal resonance][npad] complex FP32, then for each Z
// its four angular factors (z_angular: Om0 and Om1 for xi = +1, -1), rows
// n_res + 4 z .. n_res + 4 z + 3.  The K* angular factors (Eq. 4) stay per
// evaluation: they are cheap polynomials, while the lineshapes carry the square
// roots and reciprocals and the Z-chain factors about 45 instructions per event.
template <int NK, int NZ>
__global__ void __launch_bounds__(256) k_build_lcache(const float *__restrict__ rec, int64_t npad,
                                                      const ModelDev *__restrict__ gmd,
                                                      float2 *__restrict__ lc)
{
    __shared__ ModelDev md;
    load_model(gmd, &md);
    const int nK = md.n_res - NZ;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npad;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float m = rec[REC_M * npad + e], p = rec[REC_P * npad + e], q = rec[REC_Q * npad + e];
        const float invm = __frcp_rn(m);
#pragma unroll
        for (int k = 0; k < NK; ++k)
            if (k < nK) lc[k * npad + e] = kstar_lineshape(md.res[k], m, invm, p, q);
        if constexpr (NZ > 0) {
            const float mZ = rec[REC_MZ * npad + e], pZ = rec[REC_PZ * npad + e];
            const float qZ = rec[REC_QZ * npad + e], invmZ = __frcp_rn(mZ);
            const float cZ = rec[REC_CZ * npad + e], ctz = rec[REC_CTZ * npad + e];
            const float2 ephz = make_float2(rec[REC_CPZ * npad + e], rec[REC_SPZ * npad + e]);
            const float ca = rec[REC_CA * npad + e], sa = rec[REC_SA * npad + e];
#pragma unroll
            for (int z = 0; z < NZ; ++z) {
                lc[(nK + z) * npad + e] = lineshape(md.res[nK + z], mZ, invmZ, pZ, qZ).A;
                float2 o0[2], o1[2];
                z_angular(md.zr[z], cZ, ctz, ephz, ca, sa, o0, o1);
                float2 *zr = lc + (int64_t)(md.n_res + 4 * z) * npad;
                zr[e] = o0[0];
                zr[npad + e] = o0[1];
                zr[2 * npad + e] = o1[0];
                zr[3 * npad + e] = o1[1];
            }
        }
    }
}

template <int NK, int NZ>
cudaError_t launch_lcache_t(const LaunchArgs &a, float2 *lc)
{
    k_build_lcache<NK, NZ><<<a.grid, 256, 0, a.stream>>>(a.rec, a.npad, a.md, lc);
    return cudaGetLastError();
}

template <int NK>
cudaError_t launch_lcache_nk(const LaunchArgs &a, float2 *lc)
{
    switch (a.nz) {
    case 0: return launch_lcache_t<NK, 0>(a, lc);
    case 1: return launch_lcache_t<NK, 1>(a, lc);
    case 2: return launch_lcache_t<NK, 2>(a, lc);
    default: return cudaErrorInvalidValue;
    }
}

// Entry for one resonance-count bucket NK, dispatching on the number of Z.
template <int NK>
cudaError_t launch_eval_nk(const LaunchArgs &a, int mode)
{
    switch (a.nz) {
    case 0: return launch_eval_t<NK, 0>(a, mode);
    case 1: return launch_eval_t<NK, 1>(a, mode);
    case 2: return launch_eval_t<NK, 2>(a, mode);
    default: return cudaErrorInvalidValue;
    }
}

template <int NK>
cudaError_t launch_grad_nk(const LaunchArgs &a, bool norm)
{
    switch (a.nz) {
    case 0: return launch_grad_t<NK, 0>(a, norm);
    case 1: return launch_grad_t<NK, 1>(a, norm);
    case 2: return launch_grad_t<NK, 2>(a, norm);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace amp4d
