"""Deterministic 4D product quadrature of the normalisation integral
I = int S(Phi) p q dPhi over the box (m_Kpi, cos theta_K*, cos theta_J/psi, phi).

TEST INFRASTRUCTURE ONLY (part of the oracle): it judges Monte Carlo and
importance-sampled estimates of I; the product path never imports it.

I is the normalisation of the signal PDF S p q / I (the phase-space reading of
Eq. 1-5: dm^2_Kpi dm^2_J/psi pi is proportional to p q dm dcos theta_K*).  The
rule is a tensor product built from what the integrand is made of:

* J/psi angles (cos theta_psi, phi): for each muon helicity the amplitude is a
  linear combination of the spin-1 rotation functions of the mu+ direction (Eq. 4
  in the K* chain, Eq. 10-12 in the Z chain, the alignment angle included), so S
  is a polynomial of degree 2 in that direction's components.  A 6-point
  Gauss-Legendre rule in cos theta_psi and a 9-point trapezoid rule in phi
  integrate every such term exactly.
* cos theta_K*: integrated in theta_K* (cos theta_K* = cos t, weight sin t), which
  makes the sin theta_K* factors of d^J_{l0} analytic, with composite
  Gauss-Legendre panels whose breakpoints sit where m_J/psi pi crosses M_Z + k G_Z
  for each Z (m^2_J/psi pi is linear in cos theta_K* at fixed m_Kpi).
* m_Kpi: composite Gauss-Legendre panels with breakpoints at M_R + k G_R for each
  K* and where each Z band meets cos theta_K* = +-1, and the substitutions s = sqrt(m - m_K - m_pi) on the first panel and
  t = sqrt(m_B - m_psi - m) on the last, which make the square-root edges of the
  momenta q and p smooth.  The integrand is 0 above m_B - m_psi (p = 0).
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg

# Multiples of a resonance width at which panels break.
_BAND = (0.25, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0)


def psi_rule(n_gl=6, n_phi=9):
    """(cos theta_psi, phi, weight) of the exact rule for the J/psi angles."""
    x, w = npleg.leggauss(n_gl)
    ph = -math.pi + 2.0 * math.pi * np.arange(n_phi) / n_phi
    cpsi, phi = np.meshgrid(x, ph, indexing="ij")
    wt = np.einsum("i,j->ij", w, np.full(n_phi, 2.0 * math.pi / n_phi))
    return cpsi.ravel(), phi.ravel(), wt.ravel()


def _panels(bps, n):
    x, w = npleg.leggauss(n)
    nodes, wts = [], []
    for a, b in zip(bps[:-1], bps[1:]):
        nodes.append(0.5 * (b - a) * x + 0.5 * (b + a))
        wts.append(0.5 * (b - a) * w)
    return np.concatenate(nodes), np.concatenate(wts)


def _z_band_edges(mo, m_lo, m_end):
    """m_Kpi values where the band m_J/psi pi = M_Z + k G_Z of each Z meets the
    edge cos theta_K* = +-1 of the box (the cos theta_K* integral has a kink in
    m_Kpi there).  m_J/psi pi at the edges is tabulated on a fine m grid and
    each crossing refined by bisection."""
    import workloads as W
    zs = [r for r in mo.res_list if r.chain == W.CHAIN_Z]
    if not zs:
        return []
    def edge_mz(m, ck):
        k = mo.kinematics((np.array([m]), np.array([ck]), np.zeros(1), np.zeros(1)))
        return k[0, 2]
    grid = np.linspace(m_lo, m_end, 400)
    out = []
    for ck in (-1.0, 1.0):
        k = mo.kinematics((grid, np.full(len(grid), ck), np.zeros(len(grid)), np.zeros(len(grid))))
        mz = k[:, 2]
        for r in zs:
            for kk in (0.0,) + _BAND:
                for sgn in (-1.0, 1.0):
                    v = r.M + sgn * kk * r.G0
                    d = mz - v
                    for i in np.nonzero(d[:-1] * d[1:] < 0)[0]:
                        a, b = grid[i], grid[i + 1]
                        fa = edge_mz(a, ck) - v
                        for _ in range(60):
                            mid = 0.5 * (a + b)
                            fm = edge_mz(mid, ck) - v
                            if (fm < 0) == (fa < 0):
                                a, fa = mid, fm
                            else:
                                b = mid
                        out.append(0.5 * (a + b))
    return out


def m_rule(res_list, masses, m_lo, n=24, extra=()):
    """Nodes and weights in m_Kpi over [m_lo, m_B - m_psi]; extra: more breakpoints."""
    mB, mpsi, mK, mpi = masses
    m_end, m_th = mB - mpsi, mK + mpi
    import workloads as W
    bps = {m_lo, m_end, m_lo + 0.02, m_end - 0.02}
    cand = list(extra)
    for r in res_list:
        if r.chain != W.CHAIN_KSTAR:   # a Z is a band in (m_Kpi, cos theta_K*)
            continue
        for k in _BAND:
            for sgn in (-1.0, 1.0):
                cand.append(r.M + sgn * k * r.G0)
    for v in cand:
        if m_lo + 0.02 < v < m_end - 0.02:
            bps.add(v)
    bps = sorted(bps)
    # merge breakpoints closer than 1e-6 GeV (a panel of zero width adds nothing)
    merged = [bps[0]]
    for v in bps[1:]:
        if v - merged[-1] > 1e-6:
            merged.append(v)
    bps = merged
    x, w = npleg.leggauss(n)
    nodes, wts = [], []
    for a, b in zip(bps[:-1], bps[1:]):
        if a == m_lo:
            s0, s1 = math.sqrt(a - m_th), math.sqrt(b - m_th)
            s = 0.5 * (s1 - s0) * x + 0.5 * (s1 + s0)
            nodes.append(m_th + s * s)
            wts.append(0.5 * (s1 - s0) * w * 2.0 * s)
        elif b == m_end:
            t1 = math.sqrt(b - a)
            t = 0.5 * t1 * x + 0.5 * t1
            nodes.append(m_end - t * t)
            wts.append(0.5 * t1 * w * 2.0 * t)
        else:
            nodes.append(0.5 * (b - a) * x + 0.5 * (b + a))
            wts.append(0.5 * (b - a) * w)
    return np.concatenate(nodes), np.concatenate(wts)


def theta_rule(mo, m, n=16):
    """Nodes in cos theta_K* and weights (sin t dt) at fixed m_Kpi, with panel
    breaks in theta_K* where m_J/psi pi = M_Z + k G_Z for each Z of the model."""
    import workloads as W
    zs = [r for r in mo.res_list if r.chain == W.CHAIN_Z]
    bps = {0.0, math.pi}
    if zs:
        # m^2_J/psi pi at cos theta_K* = -1 and +1 (linear in between)
        k = mo.kinematics((np.array([m, m]), np.array([-1.0, 1.0]), np.zeros(2), np.zeros(2)))
        lo2, hi2 = k[0, 2] ** 2, k[1, 2] ** 2
        a, b = 0.5 * (hi2 + lo2), 0.5 * (hi2 - lo2)
        for r in zs:
            for kk in (0.0,) + _BAND:
                for sgn in (-1.0, 1.0):
                    v = r.M + sgn * kk * r.G0
                    if v <= 0.0 or b == 0.0:
                        continue
                    c = (v * v - a) / b
                    if -1.0 < c < 1.0:
                        bps.add(math.acos(c))
    t, wt = _panels(sorted(bps), n)
    return np.cos(t), wt * np.sin(t)


def normalisation_quadrature(mo, params, n_m=24, n_theta=16, n_gl=6, n_phi=9):
    """I = int S p q dPhi of the oracle model mo at params by the product rule."""
    m_end = mo.masses[0] - mo.masses[1]
    mn, mw = m_rule(mo.res_list, mo.masses, mo.box[0], n_m, _z_band_edges(mo, mo.box[0], m_end))
    cpsi, phi, wpsi = psi_rule(n_gl, n_phi)
    tot = 0.0
    for m, w in zip(mn, mw):
        cK, wK = theta_rule(mo, m, n_theta)
        CK = np.repeat(cK, len(cpsi))
        S, pq = mo.density(params, (np.full(len(CK), m), CK, np.tile(cpsi, len(cK)),
                                    np.tile(phi, len(cK))))
        f = (S * pq).reshape(len(cK), len(cpsi))
        tot += w * float(wK @ (f @ wpsi))
    return tot
