// One-time preparation of an event (or normalisation-point) set, in FP64.
//
// Per event: validates the coordinates against the box, computes the two-body
// momenta p (K pi in the B frame) and q (K in the K pi frame), cos phi and
// sin phi, and for models
// with a Z the J/psi pi chain quantities of Eq. 10: m_psipi, the Z momentum in
// the B frame, the pi momentum in the Z frame, cos theta_Z, cos theta~_psi,
// (cos, sin) phi~ and (cos, sin) alpha.  Results are stored as FP32 records;
// padding events (n <= e < npad) repeat the last event.  Each block also writes
// its FP64 partial of sum ln(p q) over real events.
//
// Frame conventions (Fig. 1 and the angle definitions under Eq. 4 and Eq. 10):
// the K pi system moves along +z in the B frame with the K in the x-z plane at
// p_x > 0; the J/psi axis z1 is the J/psi flight direction (-z); in the J/psi
// frame the mu+ direction is (sin cos phi, -sin sin phi, -cos); the Z-chain
// J/psi axis z2 is opposite to the pi momentum in the J/psi frame.
#include <cmath>
#include <cstdint>

#include "amp4d_device.cuh"
#include "amp4d_launch.h"

namespace amp4d {

constexpr int PREP_BLOCK = 256;

__device__ __forceinline__ double two_body(double M, double m1, double m2)
{
    // lambda(M^2, m1^2, m2^2) = (M^2 - (m1+m2)^2)(M^2 - (m1-m2)^2), clamped at 0
    const double a = (M - m1 - m2) * (M + m1 + m2);
    const double b = (M - m1 + m2) * (M + m1 - m2);
    const double l = a * b;
    return l > 0.0 ? sqrt(l) / (2.0 * M) : 0.0;
}

struct d3 {
    double x, y, z;
};
__device__ __forceinline__ double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3 cross(d3 a, d3 b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ d3 axpy(double s, d3 a, d3 b) { return {s * a.x + b.x, s * a.y + b.y, s * a.z + b.z}; }
__device__ __forceinline__ double norm(d3 a) { return sqrt(dot(a, a)); }
__device__ __forceinline__ d3 scaled(d3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }

template <bool HZ>
__global__ void __launch_bounds__(PREP_BLOCK) k_prepare(PrepArgs a)
{
    __shared__ double red[PREP_BLOCK / 32];
    double lnpq = 0.0;
    float *rec = a.rec;
    const int64_t np = a.npad;
    for (int64_t e = blockIdx.x * (int64_t)PREP_BLOCK + threadIdx.x; e < np;
         e += (int64_t)gridDim.x * PREP_BLOCK) {
        const int64_t es = e < a.n ? e : a.n - 1;
        const float fm = rec[REC_M * np + es], fcK = rec[REC_CK * np + es];
        const float fcpsi = rec[REC_CPSI * np + es], fphi = rec[REC_PHI * np + es];
        if (e >= a.n) {
            rec[REC_M * np + e] = fm;
            rec[REC_CK * np + e] = fcK;
            rec[REC_CPSI * np + e] = fcpsi;
            rec[REC_PHI * np + e] = fphi;
            if (a.wrec >= 0 && a.have_w) rec[a.wrec * np + e] = 0.0f;
        }
        const bool ok = isfinite(fm) && isfinite(fcK) && isfinite(fcpsi) && isfinite(fphi) &&
                        (double)fm >= a.m_lo && (double)fm <= a.m_hi && fabsf(fcK) <= 1.0f &&
                        fabsf(fcpsi) <= 1.0f && fabsf(fphi) <= 3.14159274f;
        if (!ok && e < a.n) atomicMin(a.bad, (unsigned long long)e);
        const double m = ok ? (double)fm : 0.5 * (a.m_lo + a.m_hi);
        const double cK = ok ? (double)fcK : 0.0, cpsi = ok ? (double)fcpsi : 0.0;
        const double phi = ok ? (double)fphi : 0.0;
        const double p = two_body(a.mB, m, a.mpsi);
        const double q = two_body(m, a.mK, a.mpi);
        rec[REC_P * np + e] = (float)p;
        rec[REC_Q * np + e] = (float)q;
        {
            double sphi0, cphi0;
            sincos(phi, &sphi0, &cphi0);
            rec[REC_CPHI * np + e] = (float)cphi0;
            rec[REC_SPHI * np + e] = (float)sphi0;
        }
        if (e < a.n) lnpq += log(p * q);
        if (a.wrec >= 0 && !a.have_w) rec[a.wrec * np + e] = e < a.n ? (float)(p * q) : 0.0f;
        if (HZ) {
            const double mK = a.mK, mpi = a.mpi, mpsi = a.mpsi, mB = a.mB;
            const double sK = sqrt(fmax(0.0, 1.0 - cK * cK));
            const double spsi = sqrt(fmax(0.0, 1.0 - cpsi * cpsi));
            // K pi frame -> B frame: boost along +z, gamma = E/m, beta gamma = p/m.
            const double g = sqrt(m * m + p * p) / m, bg = p / m;
            const double EKs = sqrt(mK * mK + q * q), Epis = sqrt(mpi * mpi + q * q);
            const double EK = g * EKs + bg * q * cK, pzK = g * q * cK + bg * EKs;
            const double Epi = g * Epis - bg * q * cK, pzpi = -g * q * cK + bg * Epis;
            const double px = q * sK;  // K: +px, pi: -px
            const double Epsi = sqrt(mpsi * mpsi + p * p);
            // B frame -> J/psi frame (J/psi moves along -z with momentum p).
            const double pzK1 = (Epsi * pzK + p * EK) / mpsi;
            const double pzpi1 = (Epsi * pzpi + p * Epi) / mpsi;
            // Z = J/psi + pi invariant mass.
            const double mZ2 = mpsi * mpsi + mpi * mpi + 2.0 * (Epsi * Epi + p * pzpi);
            const double mZ = sqrt(mZ2);
            const double pZ = two_body(mB, mZ, mK);
            const double qZ = two_body(mZ, mpsi, mpi);
            // cos theta_Z from invariants: K and pi energies and momenta in the Z frame.
            const double EKz = (mB * mB - mZ2 - mK * mK) / (2.0 * mZ);
            const double Epiz = (mZ2 + mpi * mpi - mpsi * mpsi) / (2.0 * mZ);
            const double pKz = sqrt(fmax(0.0, EKz * EKz - mK * mK));
            const double kpi = 0.5 * (m * m - mK * mK - mpi * mpi);  // p_K . p_pi
            double cZ = (pKz * qZ > 0.0) ? (EKz * Epiz - kpi) / (pKz * qZ) : 1.0;
            cZ = fmin(1.0, fmax(-1.0, cZ));
            // J/psi frame directions.
            double sph, cph;
            sincos(phi, &sph, &cph);
            const d3 n = {spsi * cph, -spsi * sph, -cpsi};          // mu+
            const d3 z1 = {0.0, 0.0, -1.0};
            const d3 vpi = {-px, 0.0, pzpi1}, vK = {px, 0.0, pzK1};
            const d3 z2 = scaled(vpi, -1.0 / norm(vpi));
            const double ctz = dot(n, z2);
            const d3 kh = scaled(vK, 1.0 / norm(vK));
            d3 x2 = axpy(-dot(kh, z2), z2, kh);
            double cpz = 1.0, spz = 0.0;
            const double nx2 = norm(x2);
            if (nx2 > 1e-300) {
                x2 = scaled(x2, 1.0 / nx2);
                const d3 y2 = cross(z2, x2);
                const double cx = dot(n, x2), cy = dot(n, y2), r = sqrt(cx * cx + cy * cy);
                if (r > 0.0) { cpz = cx / r; spz = cy / r; }
            }
            double ca = 1.0, sa = 0.0;
            d3 u1 = axpy(-dot(z1, n), n, z1), u2 = axpy(-dot(z2, n), n, z2);
            const double n1 = norm(u1), n2 = norm(u2);
            if (n1 > 0.0 && n2 > 0.0) {
                u1 = scaled(u1, 1.0 / n1);
                u2 = scaled(u2, 1.0 / n2);
                ca = dot(u1, u2);
                sa = dot(n, cross(u1, u2));
            }
            rec[REC_MZ * np + e] = (float)mZ;
            rec[REC_PZ * np + e] = (float)pZ;
            rec[REC_QZ * np + e] = (float)qZ;
            rec[REC_CZ * np + e] = (float)cZ;
            rec[REC_CTZ * np + e] = (float)ctz;
            rec[REC_CPZ * np + e] = (float)cpz;
            rec[REC_SPZ * np + e] = (float)spz;
            rec[REC_CA * np + e] = (float)ca;
            rec[REC_SA * np + e] = (float)sa;
        }
    }
    if (a.part_lnpq == nullptr) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lnpq += __shfl_xor_sync(0xffffffffu, lnpq, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lnpq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < PREP_BLOCK / 32; ++i) t += red[i];
        a.part_lnpq[blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// Eq. 14 templates.  Per point, in FP64: x = m^2 and y = m^2_psipi, the latter in
// the K pi frame, where the J/psi has momentum p* = p m_B / m along the K pi
// flight axis and the pi momentum q at angle theta_K* to it:
//   m^2_psipi = m_psi^2 + m_pi^2 + 2 (E_psi E_pi - p* q cos theta_K*).
// eps = effM(x, y) effA(cos theta_psi, phi) (1 without an efficiency) and
// hb = bkgM(x, y) bkgA(cos theta_psi, phi) (0 without a background), each
// template read at the bin holding the point.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double tpl_read(const TplDev &t, double x, double y)
{
    if (!(x >= t.xlo && x <= t.xhi && y >= t.ylo && y <= t.yhi)) return 0.0;
    int ix = (int)floor((x - t.xlo) * t.nx / (t.xhi - t.xlo));
    int iy = (int)floor((y - t.ylo) * t.ny / (t.yhi - t.ylo));
    ix = ix < t.nx ? ix : t.nx - 1;
    iy = iy < t.ny ? iy : t.ny - 1;
    return (double)t.h[(int64_t)iy * t.nx + ix];
}

__global__ void __launch_bounds__(PREP_BLOCK) k_templates(TplArgs a)
{
    __shared__ double red[PREP_BLOCK / 32];
    double part = 0.0;
    const int64_t np = a.npad;
    for (int64_t e = blockIdx.x * (int64_t)PREP_BLOCK + threadIdx.x; e < np;
         e += (int64_t)gridDim.x * PREP_BLOCK) {
        const double m = a.rec[REC_M * np + e], cK = a.rec[REC_CK * np + e];
        const double cpsi = a.rec[REC_CPSI * np + e];
        // the stored phi is flavour-aligned (t phi); the templates take the observed phi
        const double phi = a.rec[REC_PHI * np + e] * (a.tag ? (double)a.tag[e] : 1.0);
        const double p = two_body(a.mB, m, a.mpsi), q = two_body(m, a.mK, a.mpi);
        const double ps = p * a.mB / m;
        const double Epsi = sqrt(a.mpsi * a.mpsi + ps * ps), Epi = sqrt(a.mpi * a.mpi + q * q);
        const double x = m * m;
        const double y = a.mpsi * a.mpsi + a.mpi * a.mpi + 2.0 * (Epsi * Epi - ps * q * cK);
        const double eps = a.t[0].h ? tpl_read(a.t[0], x, y) * tpl_read(a.t[1], cpsi, phi) : 1.0;
        const double hb = a.t[2].h ? tpl_read(a.t[2], x, y) * tpl_read(a.t[3], cpsi, phi) : 0.0;
        const bool real = e < a.n;
        if (a.wout) {
            const double w0 = a.w0[e];
            a.wout[e] = (float)(w0 * eps);
            if (real) part += w0 * hb;
        } else {
            a.eps[e] = (float)eps;
            a.hb[e] = (float)hb;
            if (real) part += log(eps);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < PREP_BLOCK / 32; ++i) t += red[i];
        a.part[blockIdx.x] = t;
    }
}

// Flavour: multiply the phi-odd records (phi, sin phi and, with a Z, sin phi~ and
// sin alpha) of each event by f = old tag x new tag (+1 or -1), so that the stored
// event is the flavour-aligned one.  Padding events follow the last event.
__global__ void __launch_bounds__(PREP_BLOCK) k_flavour(float *rec, int64_t npad, int64_t n,
                                                        const float *old_tag, const float *new_tag,
                                                        int has_z)
{
    for (int64_t e = blockIdx.x * (int64_t)PREP_BLOCK + threadIdx.x; e < npad;
         e += (int64_t)gridDim.x * PREP_BLOCK) {
        const int64_t es = e < n ? e : n - 1;
        const float f = (old_tag ? old_tag[es] : 1.0f) * (new_tag ? new_tag[es] : 1.0f);
        if (f > 0.0f) continue;
        rec[REC_PHI * npad + e] = -rec[REC_PHI * npad + e];
        rec[REC_SPHI * npad + e] = -rec[REC_SPHI * npad + e];
        if (has_z) {
            rec[REC_SPZ * npad + e] = -rec[REC_SPZ * npad + e];
            rec[REC_SA * npad + e] = -rec[REC_SA * npad + e];
        }
    }
}

cudaError_t launch_flavour(float *rec, int64_t npad, int64_t n, const float *old_tag,
                           const float *new_tag, int has_z, int grid, cudaStream_t st)
{
    k_flavour<<<grid, PREP_BLOCK, 0, st>>>(rec, npad, n, old_tag, new_tag, has_z);
    return cudaGetLastError();
}

cudaError_t launch_templates(const TplArgs &a)
{
    k_templates<<<a.grid, PREP_BLOCK, 0, a.stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const PrepArgs &a)
{
    if (a.has_z)
        k_prepare<true><<<a.grid, PREP_BLOCK, 0, a.stream>>>(a);
    else
        k_prepare<false><<<a.grid, PREP_BLOCK, 0, a.stream>>>(a);
    return cudaGetLastError();
}

int prepare_block() { return PREP_BLOCK; }

}  // namespace amp4d
