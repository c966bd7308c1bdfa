"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, textbook closed forms, library special functions,
conservation laws, exact angular integrals, brute-force quadrature, symmetry
invariances of the likelihood and finite differences.
"""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from scipy import integrate, special

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


# ---------------------------------------------------------------- Wigner d (Eq. 4, Eq. 10)
def _legendre(J, x):
    return npleg.legval(x, [0] * J + [1])


def _legendre_deriv(J, x):
    return npleg.legval(x, npleg.legder([0] * J + [1]))


ANGLES = np.linspace(-0.999, 0.999, 37)


@pytest.mark.parametrize("J", [0, 1, 2, 3, 4])
def test_wigner_d_l0_is_legendre(J):
    """d^J_{00} = P_J(cos), d^J_{+-1,0} = -+ sin P_J'(cos) / sqrt(J(J+1))."""
    for c in ANGLES:
        s = math.sqrt(1 - c * c)
        assert O.wigner_d(J, 0, 0, c) == pytest.approx(_legendre(J, c), abs=1e-13)
        if J >= 1:
            ref = -s * _legendre_deriv(J, c) / math.sqrt(J * (J + 1))
            assert O.wigner_d(J, 1, 0, c) == pytest.approx(ref, abs=1e-13)
            assert O.wigner_d(J, -1, 0, c) == pytest.approx(-ref, abs=1e-13)
            # d^J_{0 l} = (-1)^l d^J_{l 0}
            assert O.wigner_d(J, 0, 1, c) == pytest.approx(-ref, abs=1e-13)
            assert O.wigner_d(J, 0, -1, c) == pytest.approx(ref, abs=1e-13)


def test_wigner_d1_closed_forms():
    for c in ANGLES:
        s = math.sqrt(1 - c * c)
        ref = {(1, 1): (1 + c) / 2, (1, -1): (1 - c) / 2, (-1, 1): (1 - c) / 2,
               (-1, -1): (1 + c) / 2, (0, 1): s / math.sqrt(2), (0, -1): -s / math.sqrt(2),
               (1, 0): -s / math.sqrt(2), (-1, 0): s / math.sqrt(2), (0, 0): c}
        for (mp, m), v in ref.items():
            assert O.wigner_d(1, mp, m, c) == pytest.approx(v, abs=1e-14)


@pytest.mark.parametrize("j", [1, 2, 3, 4])
def test_wigner_d_unitarity(j):
    rng = np.random.default_rng(j)
    for c in rng.uniform(-1, 1, 7):
        d = np.array([[O.wigner_d(j, mp, m, c) for m in range(-j, j + 1)]
                      for mp in range(-j, j + 1)])
        assert np.allclose(d.T @ d, np.eye(2 * j + 1), atol=1e-13)


@pytest.mark.parametrize("j", [1, 2, 3, 4])
def test_wigner_d_special_angles(j):
    for mp in range(-j, j + 1):
        for m in range(-j, j + 1):
            assert O.wigner_d(j, mp, m, 1.0) == pytest.approx(1.0 if mp == m else 0.0, abs=1e-14)
            ref = (-1) ** (j - m) if mp == -m else 0.0
            assert O.wigner_d(j, mp, m, -1.0) == pytest.approx(ref, abs=1e-14)


def test_wigner_d_orthogonality():
    x, w = npleg.leggauss(12)
    for lam in (0, 1):
        for J in range(lam, 5):
            for Jp in range(lam, 5):
                v = sum(wi * O.wigner_d(J, lam, 0, xi) * O.wigner_d(Jp, lam, 0, xi)
                        for xi, wi in zip(x, w))
                assert v == pytest.approx(2 / (2 * J + 1) if J == Jp else 0.0, abs=1e-13)


# ---------------------------------------------------------------- barrier factors, momenta
@pytest.mark.parametrize("L", [0, 1, 2, 3, 4])
def test_bw_poly_is_spherical_hankel(L):
    """P_L(x^2) = x^(2L+2) (j_L(x)^2 + y_L(x)^2)."""
    for x in (0.05, 0.3, 0.9, 1.7, 3.2):
        ref = x ** (2 * L + 2) * (special.spherical_jn(L, x) ** 2 + special.spherical_yn(L, x) ** 2)
        assert O.bw_poly(L, x * x) == pytest.approx(ref, rel=1e-12)


def test_breakup_energy_conservation():
    for Mp, m1, m2 in [(0.8955, W.M_K, W.M_PI), (2.1, W.M_K, W.M_PI), (W.M_B, 1.4, W.M_PSI),
                       (4.43, W.M_PSI, W.M_PI), (W.M_B, 4.43, W.M_K)]:
        q = O.breakup(Mp, m1, m2)
        assert math.hypot(m1, q) + math.hypot(m2, q) == pytest.approx(Mp, rel=1e-14)
    assert O.breakup(0.6, W.M_K, W.M_PI) == 0.0  # closed channel


# ---------------------------------------------------------------- lineshape (Eq. 2, Eq. 3)
def _all_model():
    return O.Model(W.KSTAR_TABLE + [W.Z4430])


def test_lineshape_at_pole():
    """At m = M: p = p0, q = q0, F = 1, Gamma(M) = G0, so
    A(M) = i (p0/m_B)^LB (q0/M)^LR / (M G0): peak phase +pi/2, height 1/(M G0)."""
    mo = _all_model()
    for R, r in enumerate(mo.res_list):
        if r.chain == W.CHAIN_KSTAR:
            p0 = O.breakup(W.M_B, r.M, W.M_PSI)
            q0 = O.breakup(r.M, W.M_K, W.M_PI)
        else:
            p0 = O.breakup(W.M_B, r.M, W.M_K)
            q0 = O.breakup(r.M, W.M_PSI, W.M_PI)
        A, _, _ = mo.lineshape(R, r.M)
        ref = 1j * (p0 / W.M_B) ** r.LB * (q0 / r.M) ** r.LR / (r.M * r.G0)
        assert abs(A - ref) <= 1e-12 * abs(ref)


def test_lineshape_vanishes_at_threshold():
    """Near the K pi threshold A ~ q^L_R: A -> 0 as q -> 0 for L_R >= 1."""
    mo = _all_model()
    mth = W.M_K + W.M_PI
    for R, r in enumerate(mo.res_list):
        if r.chain != W.CHAIN_KSTAR:
            continue
        m1, m2 = mth + 1e-7, mth + 1e-11
        q1, q2 = O.breakup(m1, W.M_K, W.M_PI), O.breakup(m2, W.M_K, W.M_PI)
        a1 = abs(mo.lineshape(R, m1)[0])
        a2 = abs(mo.lineshape(R, m2)[0])
        assert a2 / a1 == pytest.approx((q2 / q1) ** r.LR, rel=1e-3)


def test_lineshape_derivatives_match_finite_differences():
    mo = _all_model()
    for R, r in enumerate(mo.res_list):
        mrun = r.M + 0.37 * r.G0 if r.chain == W.CHAIN_KSTAR else 4.3
        A, dM, dG = mo.lineshape(R, mrun)
        h = 1e-6
        fdM = (mo.lineshape(R, mrun, M=r.M + h)[0] - mo.lineshape(R, mrun, M=r.M - h)[0]) / (2 * h)
        fdG = (mo.lineshape(R, mrun, G0=r.G0 + h)[0] - mo.lineshape(R, mrun, G0=r.G0 - h)[0]) / (2 * h)
        assert abs(dM - fdM) <= 1e-7 * max(abs(dM), 1e-12) + 1e-12
        assert abs(dG - fdG) <= 1e-7 * max(abs(dG), 1e-12) + 1e-12


# ---------------------------------------------------------------- LASS S-wave (Eq. 7, Eq. 8)
def _lass_model(R=W.LASS_R, a=W.LASS_A, b=W.LASS_B):
    import dataclasses
    return O.Model([dataclasses.replace(W.LASS, lass_R=R, lass_a=a, lass_b=b)])


_LASS_M = np.linspace(W.M_K + W.M_PI + 1e-4, 2.18, 61)


def test_lass_background_is_the_effective_range_amplitude():
    """Resonant term off (R = 0): the first term of Eq. 7 with the phase of Eq. 8
    is m times the textbook effective-range partial wave
    f = 1 / (q cot d - i q), q cot d = 1/a + r_e q^2 / 2, with r_e = b."""
    for a, b in ((W.LASS_A, W.LASS_B), (3.1, 0.0), (0.7, 5.0)):
        mo = _lass_model(R=0.0, a=a, b=b)
        for m in _LASS_M:
            q = O.breakup(m, W.M_K, W.M_PI)
            ref = m / (1.0 / a + 0.5 * b * q * q - 1j * q)
            A, dM, dG = mo.lineshape(0, m)
            assert abs(A - ref) <= 1e-13 * abs(ref)
            assert dM == 0 and dG == 0


def test_lass_elastic_unitarity():
    """With R = 1 and the running width of Eq. 3 at L = 0, T = A q / m is an
    elastic partial wave: sin(d) e^{i d} with d = thB + dR, so T lies on the
    unitarity circle |T - i/2| = 1/2, and its phase is the background phase of
    Eq. 8 plus the Breit-Wigner phase cot dR = (M^2 - m^2) / (M Gamma(m)).  The
    printed factor 2 (R = 2) leaves the circle away from the background."""
    mo1, mo2 = _lass_model(R=1.0), _lass_model(R=2.0)
    M, G0 = W.LASS.M, W.LASS.G0
    q0 = O.breakup(M, W.M_K, W.M_PI)
    off = 0
    for m in _LASS_M:
        q = O.breakup(m, W.M_K, W.M_PI)
        T = mo1.lineshape(0, m)[0] * q / m
        assert abs(abs(T - 0.5j) - 0.5) < 1e-13
        thB = math.atan2(1.0, 1.0 / (W.LASS_A * q) + 0.5 * W.LASS_B * q)
        dR = math.atan2(M * G0 * (q / q0) * (M / m), M * M - m * m)
        d = thB + dR
        assert abs(T - math.sin(d) * complex(math.cos(d), math.sin(d))) < 1e-13
        T2 = mo2.lineshape(0, m)[0] * q / m
        off += abs(abs(T2 - 0.5j) - 0.5) > 1e-3
    assert off > len(_LASS_M) // 2


def test_lass_at_the_pole():
    """At m = M the resonant term of Eq. 7 is R e^{2i thB} i M / q0 (Gamma(M) = G0)."""
    M = W.LASS.M
    q0 = O.breakup(M, W.M_K, W.M_PI)
    e2 = (1 / W.LASS_A + 0.5 * W.LASS_B * q0 ** 2 + 1j * q0) / \
         (1 / W.LASS_A + 0.5 * W.LASS_B * q0 ** 2 - 1j * q0)
    bg = _lass_model(R=0.0).lineshape(0, M)[0]
    for R in (1.0, 2.0, 0.37):
        A = _lass_model(R=R).lineshape(0, M)[0]
        ref = R * e2 * 1j * M / q0
        assert abs((A - bg) - ref) <= 1e-13 * abs(ref)


def test_lass_threshold_limit():
    """At q = 0 the background tends to m a (the scattering length) and
    e^{2i thB} to 1: the amplitude is continuous at the K pi threshold."""
    mo = _lass_model()
    mth = W.M_K + W.M_PI
    M, G0 = W.LASS.M, W.LASS.G0
    q0 = O.breakup(M, W.M_K, W.M_PI)
    a0 = mo.lineshape(0, mth)[0]
    ref = mth * W.LASS_A + W.LASS_R * (M * M * G0 / q0) / (M * M - mth * mth)
    assert abs(a0 - ref) <= 1e-13 * abs(ref)
    # above threshold A - A(threshold) = O(q), q ~ sqrt(m - m_th)
    for dm in (1e-8, 1e-10, 1e-12):
        q = O.breakup(mth + dm, W.M_K, W.M_PI)
        assert abs(mo.lineshape(0, mth + dm)[0] - a0) < 10.0 * q


def test_lass_derivatives_match_finite_differences():
    mo = _lass_model()
    M, G0 = W.LASS.M, W.LASS.G0
    for mrun in (0.7, 1.2, M + 0.1 * G0, 2.0):
        _, dM, dG = mo.lineshape(0, mrun)
        h = 1e-6
        fdM = (mo.lineshape(0, mrun, M=M + h)[0] - mo.lineshape(0, mrun, M=M - h)[0]) / (2 * h)
        fdG = (mo.lineshape(0, mrun, G0=G0 + h)[0] - mo.lineshape(0, mrun, G0=G0 - h)[0]) / (2 * h)
        assert abs(dM - fdM) <= 1e-7 * abs(dM)
        assert abs(dG - fdG) <= 1e-7 * abs(dG)


def test_lass_density_is_the_scalar_wave():
    """Eq. 9 with the LASS term alone: one J = 0 column, d^0_00 = 1 and
    sum_xi |d^1_{0 xi}(theta_psi)|^2 = sin^2 theta_psi, so
    S = |H|^2 |A_LASS(m)|^2 sin^2 theta_psi, flat in cos theta_K* and phi."""
    mo = _lass_model()
    assert mo.n_cols == 1
    H = 0.6 - 0.3j
    pts = W.uniform_points(500, 17)
    S, _ = mo.density([H.real, H.imag], pts)
    for i in range(0, 500, 7):
        m, cpsi = float(pts[0][i]), float(pts[2][i])
        A = mo.lineshape(0, m)[0]
        ref = abs(H) ** 2 * abs(A) ** 2 * (1.0 - cpsi * cpsi)
        assert S[i] == pytest.approx(ref, rel=1e-12, abs=1e-300)


def test_lass_model_gradient_matches_central_differences():
    """Eq. 9 model (LASS + the other K* states + Z(4430)) with every other mass
    and width floating: the oracle's analytic NLL gradient against central
    differences."""
    cfg = W.CONFIGS["lass_z"]
    res = cfg.resonances
    mo = O.Model(res, float_names=cfg.float_mg)
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed),
                              W.float_mg_values(res, cfg.float_mg))
    ev = W.peaked_points(400, 3, res)
    nm = W.uniform_points(800, 4)
    _, g, _, rc = mo.nll(p, ev, nm, grad=True)
    assert rc == 0
    rng = np.random.default_rng(5)
    for i in sorted(rng.choice(len(p), 12, replace=False)) + [0, 1, len(p) - 1]:
        h = 1e-6 * max(1.0, abs(p[i]))
        up, dn = p.copy(), p.copy()
        up[i] += h
        dn[i] -= h
        fd = (mo.nll(up, ev, nm)[0] - mo.nll(dn, ev, nm)[0]) / (2 * h)
        assert abs(g[i] - fd) <= 1e-5 * max(1.0, abs(g[i]))


def test_lass_rejected_where_it_does_not_apply():
    import dataclasses
    with pytest.raises(ValueError):
        O.Model([dataclasses.replace(W.RESONANCES["K*(892)"], shape=W.SHAPE_LASS)])
    with pytest.raises(ValueError):
        _lass_model(a=0.0)


# ---------------------------------------------------------------- efficiency and background (Eq. 14)
def _hist(h, rng):
    return W.Hist2D(np.asarray(h, dtype=np.float32), rng)


def test_template_bin_rule():
    """Bin i covers [lo + i d, lo + (i+1) d); the upper edge is in the last bin;
    0 outside the range."""
    h = _hist([[1, 2, 3, 4], [11, 12, 13, 14]], (0.0, 1.0, 0.0, 2.0))
    cases = [((0.0, 0.0), 1), ((0.2499, 0.0), 1), ((0.25, 0.0), 2), ((0.9, 1.0), 14),
             ((1.0, 2.0), 14), ((0.5, 0.999), 3), ((0.74, 1.5), 13), ((-1e-9, 0.5), 0),
             ((0.5, 2.0 + 1e-9), 0), ((1.0 + 1e-9, 1.0), 0)]
    for (x, y), ref in cases:
        assert O.tpl_value(h, x, y) == ref, (x, y)


def test_templates_read_the_dalitz_variables():
    """The mass template is read at (m^2_Kpi, m^2_psipi); m^2_psipi from the
    oracle's four-vectors equals the closed form in the K pi frame,
    m_psi^2 + m_pi^2 + 2 (E_psi E_pi - p* q cos theta_K*), p* = p m_B / m."""
    mo = O.Model([W.RESONANCES["K*(892)"]])
    ym = _hist(np.arange(1, 401, dtype=float).reshape(400, 1), (0.0, 1e3, 8.0, 24.0))
    ones_a = _hist(np.ones((1, 1)), W.ANGLE_RANGE)
    mo.set_template(0, ym, ones_a)
    pts = W.uniform_points(300, 21, box=(W.M_LO, W.M_END - 1e-6))
    eps, hb, m2z = mo.templates(pts)
    for i in range(300):
        m, cK = float(pts[0][i]), float(pts[1][i])
        p = O.breakup(W.M_B, m, W.M_PSI)
        q = O.breakup(m, W.M_K, W.M_PI)
        ps = p * W.M_B / m
        ref = W.M_PSI ** 2 + W.M_PI ** 2 + 2 * (math.hypot(W.M_PSI, ps) * math.hypot(W.M_PI, q) - ps * q * cK)
        assert m2z[i] == pytest.approx(ref, rel=1e-12)
        assert eps[i] == O.tpl_value(ym, m * m, m2z[i]) and hb[i] == 0.0


def _eq14_case(name="tiny", n_ev=3000, n_mc=6000):
    cfg = W.CONFIGS[name]
    res = cfg.resonances
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed))
    ev = W.peaked_points(n_ev, 31, res)
    nm = W.uniform_points(n_mc, 32)
    return res, p, ev, nm


def test_eq14_reduces_to_the_signal_fit():
    """P = 1 with a constant efficiency c: f = p q c S / (c I) = p q S / I, the
    signal-only likelihood, for any c."""
    res, p, ev, nm = _eq14_case()
    plain = O.Model(res)
    nll0, g0, aux0, rc0 = plain.nll(p, ev, nm, grad=True)
    for c in (1.0, float(np.float32(0.37))):   # templates hold FP32 contents
        mo = O.Model(res)
        mo.set_template(0, _hist(np.full((3, 2), c), W.MASS2_RANGE), _hist(np.ones((2, 5)), W.ANGLE_RANGE))
        nll, g, aux, rc = mo.nll_eq14(p, ev, nm, grad=True)
        assert rc == 0 and rc0 == 0
        assert nll == pytest.approx(nll0, rel=1e-12)
        assert np.allclose(g, g0, rtol=1e-9, atol=1e-9 * np.max(np.abs(g0)))
        assert aux[2] == pytest.approx(c * aux0[2], rel=1e-12)
        assert aux[4] == pytest.approx(len(ev[0]), rel=1e-12)


def test_eq14_pure_background():
    """P = 0: f = p q hb / B does not depend on the couplings; with a flat
    background B = int p q dPhi = 8 pi int p(m) q(m) dm (quadrature) within the
    Monte Carlo error of the points."""
    res, p, ev, nm = _eq14_case(n_mc=200_000)
    mo = O.Model(res)
    one_m, one_a = _hist(np.ones((4, 4)), W.MASS2_RANGE), _hist(np.ones((2, 2)), W.ANGLE_RANGE)
    mo.set_template(1, one_m, one_a, purity=0.0)
    nll, g, aux, rc = mo.nll_eq14(p, ev, nm, grad=True)
    nll2, _, _, _ = mo.nll_eq14(p * 1.7 + 0.1, ev, nm)
    assert rc == 0 and nll2 == pytest.approx(nll, rel=1e-13)
    assert np.all(g == 0.0)
    quad = 8 * math.pi * integrate.quad(
        lambda m: O.breakup(W.M_B, m, W.M_PSI) * O.breakup(m, W.M_K, W.M_PI), W.M_LO, W.M_HI,
        limit=200, epsabs=0, epsrel=1e-12)[0]
    pq = O.Model(res).density(p, nm)[1]
    sem = W.BOX_VOLUME * np.std(pq) / math.sqrt(len(pq))
    assert abs(aux[3] - quad) < 4 * sem
    assert nll == pytest.approx(-2 * (aux[1] - len(ev[0]) * math.log(aux[3])), rel=1e-12)


def test_eq14_pdf_integrates_to_one():
    """With efficiency and background templates and P = 0.85 the PDF
    p q [P eps S / I_eps + (1 - P) hb / B] integrates to 1: its mean over an
    independent uniform sample times the box volume, within the Monte Carlo error."""
    res, p, ev, nm = _eq14_case(n_mc=100_000)
    em, ea, bm, ba, P = W.eq14_templates(3)
    mo = O.Model(res)
    mo.set_template(0, em, ea)
    mo.set_template(1, bm, ba, purity=P)
    _, _, aux, rc = mo.nll_eq14(p, ev, nm)
    assert rc == 0
    fresh = W.uniform_points(100_000, 33)
    S, pq = mo.density(p, fresh)
    eps, hb, _ = mo.templates(fresh)
    f = pq * (P * eps * S / aux[2] + (1 - P) * hb / aux[3])
    est = W.BOX_VOLUME * f.mean()
    sem = W.BOX_VOLUME * f.std() / math.sqrt(len(f))
    assert abs(est - 1.0) < 4 * sem + 0.0


def test_eq14_mean_signal_probability_is_the_purity():
    """For events drawn from f, the signal probability r = P eps S p q / (I_eps f)
    has mean P: signal events thinned by the efficiency and background events
    drawn from p q hb, mixed P : 1 - P, give sum r / N = P within its binomial-like
    spread (a wrong mixing weight or normalisation moves it)."""
    cfg = W.CONFIGS["kstar10"]
    res = cfg.resonances
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed))
    mo = O.Model(res)
    em, ea, bm, ba, P = W.eq14_templates(7)
    mo.set_template(0, em, ea)
    mo.set_template(1, bm, ba, purity=P)
    rng = np.random.default_rng(8)
    n = 8000
    n_sig = int(round(P * n))
    sig, _, _ = mo.generate(p, 3 * n_sig, 9)
    eps, _, _ = mo.templates(sig)
    keep = rng.uniform(size=len(eps)) < eps
    sig = [np.asarray(a)[keep][:n_sig] for a in sig]
    u = W.uniform_points(60 * (n - n_sig), 10, box=(W.M_LO, W.M_END - 1e-6))
    _, pq = mo.density(p, u)
    _, hb, _ = mo.templates(u)
    w = pq * hb
    keep = rng.uniform(size=len(w)) * w.max() < w
    bkg = [np.asarray(a)[keep][:n - n_sig] for a in u]
    ev = [np.concatenate([a, b]) for a, b in zip(sig, bkg)]
    assert len(ev[0]) == n
    _, _, aux, rc = mo.nll_eq14(p, ev, W.uniform_points(200_000, 11))
    assert rc == 0
    # r lies in [0, 1]: its spread is at most 1/2 per event
    assert abs(aux[4] / n - P) < 4 * 0.5 / math.sqrt(n)


def test_eq14_gradient_matches_central_differences():
    res, p, ev, nm = _eq14_case("kstar10_z", 400, 800)
    cfg = W.CONFIGS["kstar10_z"]
    mo = O.Model(res, float_names=["K*(892)", "Z(4430)"])
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed),
                              W.float_mg_values(res, ["K*(892)", "Z(4430)"]))
    em, ea, bm, ba, P = W.eq14_templates(4)
    mo.set_template(0, em, ea)
    mo.set_template(1, bm, ba, purity=P)
    _, g, _, rc = mo.nll_eq14(p, ev, nm, grad=True)
    assert rc == 0
    rng = np.random.default_rng(6)
    for i in sorted(rng.choice(len(p), 14, replace=False)) + [len(p) - 1, len(p) - 3]:
        h = 1e-6 * max(1.0, abs(p[i]))
        up, dn = p.copy(), p.copy()
        up[i] += h
        dn[i] -= h
        fd = (mo.nll_eq14(up, ev, nm)[0] - mo.nll_eq14(dn, ev, nm)[0]) / (2 * h)
        assert abs(g[i] - fd) <= 1e-5 * max(1.0, abs(g[i]))


# ---------------------------------------------------------------- flavour (B0bar: phi -> -phi; mistag)
def _phi_even(hist):
    """The angular template made even in phi (its y axis, range symmetric about 0)."""
    return W.Hist2D(((hist.h + hist.h[::-1, :]) / 2).astype(np.float32), hist.range)


def _flavour_case(name="kstar10_z", n_ev=1500, n_mc=4000, seed=41):
    cfg = W.CONFIGS[name]
    res = cfg.resonances
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed))
    ev = W.peaked_points(n_ev, seed, res)
    nm = W.uniform_points(n_mc, seed + 1)
    tag = np.where(np.random.default_rng(seed + 2).uniform(size=n_ev) < 0.5, 1.0, -1.0)
    return res, p, ev, nm, tag


def test_flavour_tag_is_the_mirrored_event():
    """No mistag: a B0bar-tagged event has the density of the B0 event at -phi
    (with a phi-even efficiency the template values agree too)."""
    res, p, ev, nm, tag = _flavour_case()
    mirrored = (ev[0], ev[1], ev[2], (tag * ev[3]).astype(np.float32))
    em, ea, bm, ba, P = W.eq14_templates(12)
    for templates in (False, True):
        a, b = O.Model(res), O.Model(res)
        if templates:
            for mo in (a, b):
                mo.set_template(0, em, _phi_even(ea))
                mo.set_template(1, bm, _phi_even(ba), purity=P)
        nll_t, g_t, _, rc = a.nll_eq14(p, ev, nm, grad=True, tag=tag)
        nll_m, g_m, _, rc2 = b.nll_eq14(p, mirrored, nm, grad=True)
        assert rc == 0 and rc2 == 0
        assert nll_t == pytest.approx(nll_m, rel=1e-13)
        assert np.allclose(g_t, g_m, rtol=1e-11, atol=1e-11 * np.max(np.abs(g_m)))


def test_half_mistag_makes_the_tag_uninformative():
    """w = 1/2: the density (S(phi) + S(-phi)) / 2 of an event does not depend
    on its tag."""
    res, p, ev, nm, tag = _flavour_case()
    mo = O.Model(res)
    mo.set_mistag(0.5)
    n1, g1, _, _ = mo.nll_eq14(p, ev, nm, grad=True, tag=tag)
    n2, g2, _, _ = mo.nll_eq14(p, ev, nm, grad=True, tag=-tag)
    n3, _, _, _ = mo.nll_eq14(p, ev, nm)
    assert n1 == pytest.approx(n2, rel=1e-14) and n1 == pytest.approx(n3, rel=1e-14)
    assert np.allclose(g1, g2, rtol=1e-12, atol=1e-12 * np.max(np.abs(g1)))
    with pytest.raises(ValueError):
        mo.set_mistag(0.6)


def test_one_normalisation_serves_both_flavours():
    """The box is symmetric in phi and p q even in it, so int S(-phi) p q = int
    S(phi) p q: over a phi-mirrored point sample the two sums are equal, and an
    independent sample's sum agrees within its Monte Carlo error."""
    res, p, _, _, _ = _flavour_case()
    mo = O.Model(res)
    u = W.uniform_points(100_000, 45)
    um = (u[0], u[1], u[2], -u[3])
    both = tuple(np.concatenate([a, b]) for a, b in zip(u, um))
    I_u, I_m = mo.norm(p, u), mo.norm(p, um)
    I_b = mo.norm(p, both)
    assert I_b == pytest.approx(0.5 * (I_u + I_m), rel=1e-13)
    S, pq = mo.density(p, u)
    sem = W.BOX_VOLUME * np.std(S * pq) / math.sqrt(len(S))
    assert abs(I_u - I_m) < 4 * math.sqrt(2) * sem


def test_phi_even_efficiency_keeps_one_normalisation():
    """With an efficiency even in phi, int eps S(-phi) p q = int eps S(phi) p q:
    over a phi-mirrored point sample the efficiency-weighted sums of the two
    flavours' densities are equal; with an efficiency odd-skewed in phi they
    differ.  This is why tags and a mistag share I_eps only for a phi-even
    efficiency."""
    res, p, _, _, _ = _flavour_case()
    em, ea, _, _, _ = W.eq14_templates(15)
    u = W.uniform_points(50_000, 46)
    both = tuple(np.concatenate([a, b]) for a, b in zip(u, (u[0], u[1], u[2], -u[3])))
    mirrored = (both[0], both[1], both[2], -both[3])
    for ang, even in ((_phi_even(ea), True), (ea, False)):
        mo = O.Model(res)
        mo.set_template(0, em, ang)
        eps, _, _ = mo.templates(both)
        S, pq = mo.density(p, both)
        Sm, _ = mo.density(p, mirrored)
        a, b = np.sum(eps * S * pq), np.sum(eps * Sm * pq)
        if even:
            assert a == pytest.approx(b, rel=1e-12)
        else:
            assert abs(a / b - 1) > 1e-4


def test_flavour_gradient_matches_central_differences():
    res, p, ev, nm, tag = _flavour_case("kstar10_z", 400, 800)
    fl = ["K*(892)", "Z(4430)"]
    mo = O.Model(res, float_names=fl)
    p = W.couplings_to_params(W.draw_couplings(res, W.CONFIGS["kstar10_z"].coupling_seed),
                              W.float_mg_values(res, fl))
    em, ea, bm, ba, P = W.eq14_templates(13)
    mo.set_template(0, em, _phi_even(ea))
    mo.set_template(1, bm, ba, purity=P)
    mo.set_mistag(0.07)
    _, g, _, rc = mo.nll_eq14(p, ev, nm, grad=True, tag=tag)
    assert rc == 0
    rng = np.random.default_rng(14)
    for i in sorted(rng.choice(len(p), 12, replace=False)) + [len(p) - 1, len(p) - 4]:
        h = 1e-6 * max(1.0, abs(p[i]))
        up, dn = p.copy(), p.copy()
        up[i] += h
        dn[i] -= h
        fd = (mo.nll_eq14(up, ev, nm, tag=tag)[0] - mo.nll_eq14(dn, ev, nm, tag=tag)[0]) / (2 * h)
        assert abs(g[i] - fd) <= 1e-5 * max(1.0, abs(g[i]))


# ---------------------------------------------------------------- kinematics
def test_kstar_angles_round_trip():
    mo = _all_model()
    pts = W.uniform_points(2000, 11)
    k = mo.kinematics(pts)
    ok = k[:, 0] > 1e-6
    assert np.allclose(k[ok, 9], pts[1][ok], atol=1e-11)
    assert np.allclose(k[ok, 10], pts[2][ok], atol=1e-12)
    assert np.allclose(k[ok, 11], np.cos(pts[3][ok].astype(np.float64)), atol=1e-11)
    assert np.allclose(k[ok, 12], np.sin(pts[3][ok].astype(np.float64)), atol=1e-11)


def test_dalitz_slope():
    """At fixed m_Kpi, m^2_psi pi is linear in cos theta_K* with slope -2 p q m_B / m."""
    mo = _all_model()
    for m in (0.7, 0.9, 1.4, 2.0, 2.15):
        c = np.linspace(-0.9, 0.9, 7)
        pts = (np.full(7, m), c, np.zeros(7), np.zeros(7))
        k = mo.kinematics(pts)
        m2 = k[:, 2] ** 2
        p, q = k[0, 0], k[0, 1]
        slope = np.polyfit(c, m2, 1)[0]
        assert slope == pytest.approx(-2 * p * q * W.M_B / m, rel=1e-10)
        assert np.max(np.abs(np.polyfit(c, m2, 2)[0])) < 1e-9


def test_cos_theta_z_invariant_mass_identity():
    """In the Z frame: m_Kpi^2 = mK^2 + mpi^2 + 2 (E_K E_pi - |p_K||p_pi| cos theta_Z),
    with E_K, E_pi, |p| fixed by m_psi pi (two-body relations in the Z frame)."""
    mo = _all_model()
    pts = W.uniform_points(500, 12)
    k = mo.kinematics(pts)
    mz = k[:, 2]
    EK = (W.M_B ** 2 - mz ** 2 - W.M_K ** 2) / (2 * mz)
    Epi = (mz ** 2 + W.M_PI ** 2 - W.M_PSI ** 2) / (2 * mz)
    pK = np.sqrt(np.maximum(EK ** 2 - W.M_K ** 2, 0))
    ppi = np.sqrt(np.maximum(Epi ** 2 - W.M_PI ** 2, 0))
    m2 = W.M_K ** 2 + W.M_PI ** 2 + 2 * (EK * Epi - pK * ppi * k[:, 3])
    ok = k[:, 0] > 1e-3
    assert np.allclose(m2[ok], pts[0][ok].astype(np.float64) ** 2, rtol=1e-10)


def test_z_frame_angles_are_unit():
    mo = _all_model()
    k = mo.kinematics(W.uniform_points(500, 13))
    assert np.allclose(k[:, 5] ** 2 + k[:, 6] ** 2, 1, atol=1e-12)
    assert np.allclose(k[:, 7] ** 2 + k[:, 8] ** 2, 1, atol=1e-12)
    assert np.all(np.abs(k[:, 3]) <= 1 + 1e-12) and np.all(np.abs(k[:, 4]) <= 1 + 1e-12)


# ---------------------------------------------------------------- exact angular integrals
def _angular_rule(n_gl=6, n_phi=9):
    x, w = npleg.leggauss(n_gl)
    ph = -math.pi + 2 * math.pi * np.arange(n_phi) / n_phi
    wp = np.full(n_phi, 2 * math.pi / n_phi)
    cK, cpsi, phi = np.meshgrid(x, x, ph, indexing="ij")
    wt = np.einsum("i,j,k->ijk", w, w, wp)
    return cK.ravel(), cpsi.ravel(), phi.ravel(), wt.ravel()


def _kstar_angular_closed_form(mo, c, m):
    """int S dcK dcpsi dphi for a K*-only model: the phi integral removes
    lambda != lambda', the cos theta_K* integral removes J != J'
    (int d^J_{l0} d^J'_{l0} = 2/(2J+1) delta), and sum_xi int d^1_{l xi}^2 = 4/3."""
    tot = 0.0
    for lam in (-1, 0, 1):
        byJ = {}
        for k, (R, l) in enumerate(zip(mo.col_res, mo.col_lam)):
            if l != lam:
                continue
            r = mo.res_list[R]
            byJ.setdefault(r.J, 0j)
            byJ[r.J] += c[k] * mo.lineshape(R, m)[0]
        tot += sum(2 / (2 * J + 1) * abs(v) ** 2 for J, v in byJ.items())
    return 2 * math.pi * 4 / 3 * tot


def test_angular_closure_kstar_all_spins():
    res = W.KSTAR_TABLE
    mo = O.Model(res)
    c = W.draw_couplings(res, 99)
    p = W.couplings_to_params(c)
    cK, cpsi, phi, wt = _angular_rule()
    for m in (0.7, 0.9, 1.2, 1.43, 1.78, 2.05, 2.17):
        S, _ = mo.density(p, (np.full(len(cK), m), cK, cpsi, phi))
        assert np.dot(wt, S) == pytest.approx(_kstar_angular_closed_form(mo, c, m), rel=1e-12)


def test_z_only_angular_integral_is_rotation_invariant():
    """For a Z-only model at fixed (m, cK) the J/psi angles enter through a rotation of
    the mu+ direction, so int S dcpsi dphi = 2 pi (4/3) sum_l' |H_l'|^2 |A_Z d^1_{0 l'}(theta_Z)|^2."""
    res = [W.Z4430]
    mo = O.Model(res)
    c = np.array([0.7 - 0.2j, -0.3 + 0.5j])  # columns: lambda' = 0, lambda' = +-1
    p = W.couplings_to_params(c)
    x, w = npleg.leggauss(6)
    ph = -math.pi + 2 * math.pi * np.arange(9) / 9
    cpsi, phi = np.meshgrid(x, ph, indexing="ij")
    wt = np.einsum("i,j->ij", w, np.full(9, 2 * math.pi / 9)).ravel()
    cpsi, phi = cpsi.ravel(), phi.ravel()
    for m, cK in [(0.9, 0.3), (1.4, -0.7), (1.9, 0.95), (2.1, -0.1)]:
        n = len(cpsi)
        pts = (np.full(n, m), np.full(n, cK), cpsi, phi)
        S, _ = mo.density(p, pts)
        kin = mo.kinematics(pts)
        mz, cz = kin[0, 2], kin[0, 3]
        A = mo.lineshape(0, mz)[0]
        ref = 2 * math.pi * 4 / 3 * abs(A) ** 2 * (
            abs(c[0]) ** 2 * O.wigner_d(1, 0, 0, cz) ** 2 +
            abs(c[1]) ** 2 * (O.wigner_d(1, 0, 1, cz) ** 2 + O.wigner_d(1, 0, -1, cz) ** 2))
        assert np.dot(wt, S) == pytest.approx(ref, rel=1e-12)


# ---------------------------------------------------------------- normalisation
M_END = W.M_B - W.M_PSI           # p = 0 beyond this
M_TH = W.M_K + W.M_PI             # q = 0 below this


def _m_rule(res, n=24):
    """Composite Gauss-Legendre rule on [M_LO, M_END] with panels refined around each
    pole, s = sqrt(m - M_TH) on the first panel and t = sqrt(M_END - m) on the last,
    which make the square-root edges of p and q smooth."""
    bps = {W.M_LO, M_END}
    for r in res:
        for k in (0.25, 0.5, 1, 2, 4, 8, 16):
            for sgn in (-1, 1):
                v = r.M + sgn * k * r.G0
                if W.M_LO + 0.02 < v < M_END - 0.02:
                    bps.add(v)
    bps.add(W.M_LO + 0.02)
    bps.add(M_END - 0.02)
    bps = sorted(bps)
    x, w = npleg.leggauss(n)
    nodes, wts = [], []
    for a, b in zip(bps[:-1], bps[1:]):
        if a == W.M_LO:
            s0, s1 = math.sqrt(a - M_TH), math.sqrt(b - M_TH)
            s = 0.5 * (s1 - s0) * x + 0.5 * (s1 + s0)
            nodes.append(M_TH + s * s)
            wts.append(0.5 * (s1 - s0) * w * 2 * s)
        elif b == M_END:
            t0, t1 = 0.0, math.sqrt(b - a)
            t = 0.5 * (t1 - t0) * x + 0.5 * (t1 + t0)
            nodes.append(M_END - t * t)
            wts.append(0.5 * (t1 - t0) * w * 2 * t)
        else:
            nodes.append(0.5 * (b - a) * x + 0.5 * (b + a))
            wts.append(0.5 * (b - a) * w)
    return np.concatenate(nodes), np.concatenate(wts)


def _norm_1d(mo, c):
    def f(m):
        return O.breakup(W.M_B, m, W.M_PSI) * O.breakup(m, W.M_K, W.M_PI) * \
            _kstar_angular_closed_form(mo, c, m)
    pts = sorted({r.M for r in mo.res_list})
    v, err = integrate.quad(f, W.M_LO, M_END, points=pts, epsabs=0, epsrel=1e-13, limit=800)
    return v


def test_pdf_integrates_to_one_tiny_model():
    """Brute-force 4D tensor quadrature of P = S p q / I on the two-K* model, with I
    from the exact angular integral and an adaptive 1D quadrature in m."""
    res = W.CONFIGS["tiny"].resonances
    mo = O.Model(res)
    c = W.draw_couplings(res, W.CONFIGS["tiny"].coupling_seed)
    p = W.couplings_to_params(c)
    I1 = _norm_1d(mo, c)
    mn, mw = _m_rule(res)
    cK, cpsi, phi, wt = _angular_rule()
    tot = 0.0
    for m, w in zip(mn, mw):
        S, pq = mo.density(p, (np.full(len(cK), m), cK, cpsi, phi))
        tot += w * np.dot(wt, S * pq)
    assert tot / I1 == pytest.approx(1.0, abs=1e-10)


# ---------------------------------------------------------------- fit fractions (Eq. 13)
def test_fit_fraction_of_a_single_resonance_is_one():
    res = [r for r in W.CONFIGS["tiny"].resonances if r.name == "K*(892)"]
    mo = O.Model(res)
    c = W.draw_couplings(res, 5)
    pts = W.uniform_points(20000, 3)
    assert mo.fit_fractions(W.couplings_to_params(c), pts)[0] == pytest.approx(1.0, abs=1e-14)


def test_fit_fractions_of_different_spins_sum_to_one():
    """K*(892) (J = 1) and K2*(1430) (J = 2): integrated over the full angular range
    their interference vanishes (the phi integral removes lambda != lambda', and
    int d^1_{l0} d^2_{l0} dcos = 0), so with an exact angular rule the two
    fractions add up to one."""
    res = W.CONFIGS["tiny"].resonances
    mo = O.Model(res)
    c = W.draw_couplings(res, W.CONFIGS["tiny"].coupling_seed)
    p = W.couplings_to_params(c)
    mn, mw = _m_rule(res)
    cK, cpsi, phi, wt = _angular_rule()
    M = np.repeat(mn, len(cK))
    pts = (M, np.tile(cK, len(mn)), np.tile(cpsi, len(mn)), np.tile(phi, len(mn)))
    wq = np.repeat(mw, len(cK)) * np.tile(wt, len(mn)) * \
        np.array([O.breakup(W.M_B, m, W.M_PSI) * O.breakup(m, W.M_K, W.M_PI) for m in M])
    ff = mo.fit_fractions(p, pts, w=wq, volume=1.0)
    assert ff.sum() == pytest.approx(1.0, abs=1e-12)
    assert np.all(ff > 0)


def test_fit_fractions_invariant_under_global_phase_and_scale():
    res = W.CONFIGS["kstar10_z"].resonances
    mo = O.Model(res)
    c = W.draw_couplings(res, 3)
    pts = W.uniform_points(30000, 4)
    f0 = mo.fit_fractions(W.couplings_to_params(c), pts)
    f1 = mo.fit_fractions(W.couplings_to_params(c * 2.5 * np.exp(0.7j)), pts)
    assert np.allclose(f0, f1, rtol=1e-12, atol=1e-15)


def test_mc_normalisation_within_statistical_error():
    res = W.CONFIGS["tiny"].resonances
    mo = O.Model(res)
    c = W.draw_couplings(res, W.CONFIGS["tiny"].coupling_seed)
    p = W.couplings_to_params(c)
    I1 = _norm_1d(mo, c)
    pts = W.uniform_points(200_000, 5)
    S, pq = mo.density(p, pts)
    f = W.BOX_VOLUME * S * pq
    Imc = mo.norm(p, pts)
    assert Imc == pytest.approx(f.mean(), rel=1e-12)
    sigma = f.std() / math.sqrt(len(f))
    assert abs(Imc - I1) < 4 * sigma


def test_gram_reproduces_normalisation():
    """I = (V/N) (u^T G u + u'^T G u') with u = (Re c, -Im c), u' = (Im c, Re c) interleaved."""
    res = W.KSTAR_TABLE + [W.Z4430]
    mo = O.Model(res)
    c = W.draw_couplings(res, 3)
    p = W.couplings_to_params(c)
    pts = W.uniform_points(3000, 6)
    G = mo.gram(p, pts)
    u = np.empty(2 * len(c)); u[0::2] = c.real; u[1::2] = -c.imag
    v = np.empty(2 * len(c)); v[0::2] = c.imag; v[1::2] = c.real
    I_g = W.BOX_VOLUME / 3000 * (u @ G @ u + v @ G @ v)
    assert I_g == pytest.approx(mo.norm(p, pts), rel=1e-12)
    assert np.allclose(G, G.T, rtol=0, atol=1e-12 * np.abs(G).max())


# ---------------------------------------------------------------- likelihood
def _setup(name="kstar10_z", n=3000, n_mc=6000, float_names=None):
    cfg = W.CONFIGS[name]
    res = cfg.resonances
    fl = cfg.float_mg if float_names is None else float_names
    mo = O.Model(res, float_names=fl)
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c, W.float_mg_values(res, fl))
    ev = W.peaked_points(n, cfg.data_seed, res)
    nm = W.uniform_points(n_mc, cfg.norm_seed)
    return mo, c, p, ev, nm


def test_nll_invariant_under_global_phase_and_scale():
    mo, c, p, ev, nm = _setup()
    nll0 = mo.nll(p, ev, nm)[0]
    K = len(c)
    for beta in (0.3, -2.0):
        c2 = c * np.exp(1j * beta)
        p2 = p.copy(); p2[0:2 * K:2] = c2.real; p2[1:2 * K:2] = c2.imag
        assert mo.nll(p2, ev, nm)[0] == pytest.approx(nll0, abs=1e-12 * abs(nll0))
    p3 = p.copy(); p3[:2 * K] *= 3.7
    assert mo.nll(p3, ev, nm)[0] == pytest.approx(nll0, abs=1e-12 * abs(nll0))


def test_nll_gradient_matches_central_differences():
    mo, c, p, ev, nm = _setup(n=1500, n_mc=3000)
    _, g, _, rc = mo.nll(p, ev, nm, grad=True)
    assert rc == 0
    h = 1e-5
    scale = np.abs(g).max()
    for i in range(len(p)):
        pp = p.copy(); pp[i] += h
        a = mo.nll(pp, ev, nm)[0]
        pp[i] -= 2 * h
        b = mo.nll(pp, ev, nm)[0]
        fd = (a - b) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3 * scale), (i, fd, g[i])


def test_gradient_phase_and_scale_identities():
    """NLL is homogeneous of degree 0 in c and invariant under c -> e^{i b} c, so
    sum_k (Re c dIm - Im c dRe) = 0 and sum_k (Re c dRe + Im c dIm) = 0."""
    mo, c, p, ev, nm = _setup(n=2000, n_mc=4000)
    _, g, _, _ = mo.nll(p, ev, nm, grad=True)
    K = len(c)
    gr, gi = g[0:2 * K:2], g[1:2 * K:2]
    scale = np.sum(np.abs(c.real * gr) + np.abs(c.imag * gi))
    assert abs(np.sum(c.real * gi - c.imag * gr)) < 1e-10 * scale
    assert abs(np.sum(c.real * gr + c.imag * gi)) < 1e-10 * scale


def test_nll_sums_match_exact_serial_sums():
    """The compensated, blocked OpenMP reduction of sum ln S, sum ln(p q) and
    sum p q S against correctly rounded serial sums (math.fsum) of the per-event
    values, and -2 ln L written from those sums (the unbinned likelihood of the
    Introduction with I = V/N sum w S)."""
    mo, c, p, ev, nm = _setup(n=9001, n_mc=12007)
    nll, _, aux, rc = mo.nll(p, ev, nm)
    assert rc == 0
    S, pq = mo.density(p, ev)
    Sn, pqn = mo.density(p, nm)
    l_exact = math.fsum(np.log(S))
    lpq_exact = math.fsum(np.log(pq))
    I_exact = W.BOX_VOLUME / len(nm[0]) * math.fsum(pqn * Sn)
    assert aux[0] == pytest.approx(l_exact, rel=1e-14, abs=1e-9)
    assert aux[1] == pytest.approx(lpq_exact, rel=1e-14, abs=1e-9)
    assert aux[2] == pytest.approx(I_exact, rel=1e-14)
    nll_exact = -2.0 * (l_exact + lpq_exact - len(ev[0]) * math.log(I_exact))
    assert nll == pytest.approx(nll_exact, rel=1e-13)


def test_nll_domain_error_on_zero_density():
    mo, c, p, ev, nm = _setup("tiny", n=50, n_mc=100, float_names=())
    p0 = np.zeros_like(p)
    nll, _, _, rc = mo.nll(p0, ev, nm)
    assert rc == -1 and math.isinf(nll)


# ---------------------------------------------------------------- generator
def test_generator_follows_the_model_in_m():
    """Accept-reject events: their m_Kpi histogram matches the 1D density
    p q int S dOmega / I (chi^2 / ndf near 1)."""
    cfg = W.CONFIGS["tiny"]
    res = cfg.resonances
    mo = O.Model(res)
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c)
    (m, _, _, _), used, fmax = mo.generate(p, 20000, 1234)
    I1 = _norm_1d(mo, c)
    edges = np.linspace(W.M_LO, M_END, 41)
    h, _ = np.histogram(m, edges)

    def dens(x):
        return O.breakup(W.M_B, x, W.M_PSI) * O.breakup(x, W.M_K, W.M_PI) * \
            _kstar_angular_closed_form(mo, c, x) / I1
    exp = np.array([integrate.quad(dens, a, b, epsrel=1e-10)[0] for a, b in zip(edges[:-1], edges[1:])])
    exp *= len(m)
    keep = exp > 5
    chi2 = np.sum((h[keep] - exp[keep]) ** 2 / exp[keep])
    ndf = keep.sum()
    assert chi2 / ndf < 2.0
    assert abs(exp.sum() - len(m)) < 1e-6 * len(m)
