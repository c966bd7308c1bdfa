"""Pins of the oracle's 4D product quadrature of the normalisation integral
I = int S p q dPhi (oracle/quadrature.py), which judges the Monte Carlo and
importance-sampled estimates of I:

* K*-only models: the exact angular closure (different spins and helicities do
  not interfere after the angular integrals) reduces I to a 1D integral in m,
  done here by adaptive QUADPACK quadrature;
* a Z alone: its J/psi-angle integral is rotation invariant, so I is a 2D
  integral of |A_Z|^2 d^1(theta_Z)^2 p q over (m_Kpi, cos theta_K*), done here by
  nested adaptive quadrature with the kinematics of the oracle;
* K* + Z: the rule is converged (two orders agree) and a uniform Monte Carlo
  estimate lies within its statistical error.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
import workloads as W
from oracle import quadrature as Q
from test_oracle_pins import _norm_1d


def test_quadrature_reproduces_the_kstar_angular_closure():
    res = W.KSTAR_TABLE
    mo = O.Model(res)
    c = W.draw_couplings(res, 4242)
    p = W.couplings_to_params(c)
    assert Q.normalisation_quadrature(mo, p, 16, 12) / _norm_1d(mo, c) == pytest.approx(1.0, abs=1e-10)


def test_quadrature_of_a_z_alone_matches_its_rotation_invariant_form():
    res = [W.Z4430]
    mo = O.Model(res)
    c = np.array([0.7 - 0.2j, -0.3 + 0.5j])   # lambda' = 0 and lambda' = +-1 columns
    p = W.couplings_to_params(c)
    m_end = W.M_B - W.M_PSI

    def angular(m, cK):
        k = mo.kinematics((np.array([m]), np.array([cK]), np.zeros(1), np.zeros(1)))
        mz, cz = k[0, 2], k[0, 3]
        A = mo.lineshape(0, mz)[0]
        return 2 * math.pi * 4 / 3 * abs(A) ** 2 * (
            abs(c[0]) ** 2 * O.wigner_d(1, 0, 0, cz) ** 2 +
            abs(c[1]) ** 2 * (O.wigner_d(1, 0, 1, cz) ** 2 + O.wigner_d(1, 0, -1, cz) ** 2))

    def band(m):
        # cos theta_K* where m_J/psi pi = M_Z + k G_Z (m^2_J/psi pi is linear in it)
        k = mo.kinematics((np.array([m, m]), np.array([-1.0, 1.0]), np.zeros(2), np.zeros(2)))
        lo2, hi2 = k[0, 2] ** 2, k[1, 2] ** 2
        pts = []
        for kk in (-4, -2, -1, -0.5, 0, 0.5, 1, 2, 4):
            v = W.Z4430.M + kk * W.Z4430.G0
            ck = (v * v - 0.5 * (hi2 + lo2)) / (0.5 * (hi2 - lo2))
            if -1 < ck < 1:
                pts.append(ck)
        return sorted(pts)

    def inner(m):
        v, _ = integrate.quad(lambda ck: angular(m, ck), -1.0, 1.0, points=band(m) or None,
                              epsabs=0, epsrel=1e-13, limit=400)
        return O.breakup(W.M_B, m, W.M_PSI) * O.breakup(m, W.M_K, W.M_PI) * v

    # the outer integrand varies fastest where the Z band meets the box edge
    edges = sorted(set(Q._z_band_edges(mo, W.M_LO, m_end)))
    ref, _ = integrate.quad(inner, W.M_LO, m_end, points=edges, epsabs=0, epsrel=1e-12, limit=400)
    # as the reference for a 1e-4 target the rule needs 1e-6; it reaches about 1e-8 here
    assert Q.normalisation_quadrature(mo, p, 24, 16) / ref == pytest.approx(1.0, abs=1e-7)


def test_quadrature_of_kstar_plus_z_is_converged():
    res = [W.RESONANCES["K*(892)"], W.RESONANCES["K2*(1430)"], W.Z4430]
    mo = O.Model(res)
    p = W.couplings_to_params(W.draw_couplings(res, 77))
    a = Q.normalisation_quadrature(mo, p, 16, 12)
    b = Q.normalisation_quadrature(mo, p, 24, 16)
    assert a / b == pytest.approx(1.0, abs=1e-7)


def test_uniform_monte_carlo_lies_within_its_error_of_the_quadrature():
    cfg = W.CONFIGS["learned"]
    res = cfg.resonances
    mo = O.Model(res)
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed))
    I_q = Q.normalisation_quadrature(mo, p, 16, 12)
    pts = W.uniform_points(1 << 21, 9001)
    S, pq = mo.density(p, pts)
    f = W.BOX_VOLUME * S * pq
    assert abs(f.mean() - I_q) < 4 * f.std() / math.sqrt(len(f))
