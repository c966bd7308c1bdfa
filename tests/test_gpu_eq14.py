"""Efficiency and background (Eq. 14) on the GPU path, against the FP64 oracle.

The templates are seeded 2D Bernstein shapes binned over the two mass variables
and the two angles (the paper's generic real-life shapes), with the purity of
its real-life test (85 %).  Tolerances are those of the signal-only parity tests:
|dNLL| < 1e-3, gradient <= 1e-6 |g|_inf, I relative 1e-8, per-event PDF
relative 2e-5 where the interference is well conditioned."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

# Gradient parity bound: every component within 1e-6 |g|_inf of the oracle's
# gradient (the scope table's "absolute <= 1e-6 |g|_inf" form).
GRAD_TOL = 1e-6


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2007_14931_gb300 as A
    return A


def _dev(pts):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in pts]


def _case(A, name, path, n_ev=20_003, n_mc=60_001, eff=True, bkg=True, purity=W.PURITY,
          float_names=None, data="peaked"):
    cfg = W.CONFIGS[name]
    res = cfg.resonances
    fl = cfg.float_mg if float_names is None else float_names
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed), W.float_mg_values(res, fl))
    em, ea, bm, ba, _ = W.eq14_templates(cfg.template_seed)
    om = O.Model(res, float_names=fl)
    if eff:
        om.set_template(0, em, ea)
    if bkg:
        om.set_template(1, bm, ba, purity=purity)
    if data == "peaked":
        ev = W.peaked_points(n_ev, cfg.data_seed, res)
    else:
        ev = _eq14_data(om, p, n_ev, purity if bkg else 1.0, cfg.data_seed)
    nm = W.uniform_points(n_mc, cfg.norm_seed)
    gm = A.Model(res, float_names=fl, path=path)
    if eff:
        gm.set_efficiency(em, ea)
    gm.set_events(*_dev(ev))
    gm.set_norm_points(*_dev(nm))
    if bkg:   # set after the sets were loaded: the templates apply to loaded sets too
        gm.set_background(bm, ba, purity)
    return res, p, om, gm, ev, nm


def _eq14_data(om, p, n, purity, seed):
    """Events of Eq. 14: signal from the model thinned by the efficiency
    (accepted with probability eps <= 1), and background drawn from p q hb by
    accept-reject over uniform points, in the ratio P : 1 - P."""
    rng = np.random.default_rng(seed)
    n_sig = int(round(purity * n))
    sig, _, _ = om.generate(p, 3 * n_sig + 100, seed)
    eps, _, _ = om.templates(sig)
    keep = rng.uniform(size=len(eps)) < eps
    sig = tuple(np.asarray(a)[keep][:n_sig] for a in sig)
    assert len(sig[0]) == n_sig
    n_bkg = n - n_sig
    u = W.uniform_points(60 * n_bkg + 1000, seed + 1, box=(W.M_LO, W.M_END - 1e-6))
    _, pq = om.density(p, u)
    _, hb, _ = om.templates(u)
    w = pq * hb
    keep = rng.uniform(size=len(w)) * w.max() < w
    bkg = tuple(np.asarray(a)[keep][:n_bkg] for a in u)
    assert len(bkg[0]) == n_bkg
    return tuple(np.concatenate([a, b]).astype(np.float32) for a, b in zip(sig, bkg))


@pytest.mark.parametrize("path", ["plain", "cached"])
@pytest.mark.parametrize("name,fl", [("tiny", None), ("kstar10_2z", None), ("kstar10_2z", []),
                                     ("lass_z", None)])
def test_eq14_nll_grad_parity(A, path, name, fl):
    pth = A.AMP4D_PATH_PLAIN if path == "plain" else A.AMP4D_PATH_CACHED
    res, p, om, gm, ev, nm = _case(A, name, pth, float_names=fl)
    nll_o, g_o, aux, rc = om.nll_eq14(p, ev, nm, grad=True)
    assert rc == 0
    nll, g = gm.eval_nll_grad(p)
    t = gm.eval_terms(p)
    print("%s %s fl=%s: dNLL %.3e  dI/I %.3e  d sum ln g %.3e  max|dg|/|g| %.3e" % (
        name, path, fl, nll - nll_o, t[2] / aux[2] - 1, t[0] - aux[0],
        np.max(np.abs(g - g_o)) / np.max(np.abs(g_o))))
    assert abs(nll - nll_o) < 1e-3
    assert t[2] == pytest.approx(aux[2], rel=1e-8)      # I_eps
    assert t[1] == pytest.approx(aux[1], rel=1e-12)     # sum ln(p q)
    assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))
    # NLL-only kernels and a second parameter point
    assert gm.eval_nll(p) == pytest.approx(nll, abs=1e-4)
    p2 = p.copy()
    p2[2:2 * len(W.columns(res))] *= 1.03
    nll2_o, g2_o, _, _ = om.nll_eq14(p2, ev, nm, grad=True)
    nll2, g2 = gm.eval_nll_grad(p2)
    assert abs(nll2 - nll2_o) < 1e-3
    assert np.max(np.abs(g2 - g2_o)) <= GRAD_TOL * np.max(np.abs(g2_o))


@pytest.mark.parametrize("path", ["plain", "cached"])
def test_efficiency_only(A, path):
    """P = 1: f = p q eps S / I_eps; the data term is ln S plus the constant
    sum ln eps, the points are efficiency-weighted (also in the Gram matrix)."""
    pth = A.AMP4D_PATH_PLAIN if path == "plain" else A.AMP4D_PATH_CACHED
    res, p, om, gm, ev, nm = _case(A, "kstar10_z", pth, bkg=False, float_names=[])
    nll_o, g_o, aux, rc = om.nll_eq14(p, ev, nm, grad=True)
    assert rc == 0
    nll, g = gm.eval_nll_grad(p)
    assert abs(nll - nll_o) < 1e-3
    assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))
    assert gm.eval_terms(p)[2] == pytest.approx(aux[2], rel=1e-8)


def test_eq14_model_distributed_data(A):
    """Signal events from the model, thinned by the efficiency, plus 15 %
    background drawn from the background template: the likelihood of the data
    the fit of the paper's real-life test sees."""
    res, p, om, gm, ev, nm = _case(A, "kstar10_2z", A.AMP4D_PATH_CACHED, n_ev=6000, data="model",
                                   float_names=[])
    nll_o, g_o, aux, rc = om.nll_eq14(p, ev, nm, grad=True)
    nll, g = gm.eval_nll_grad(p)
    assert rc == 0 and abs(nll - nll_o) < 1e-3
    assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))


def test_eq14_pdf_parity(A):
    res, p, om, gm, ev, nm = _case(A, "kstar10_2z", A.AMP4D_PATH_PLAIN)
    P = gm.eval_pdf(p).cpu().numpy().astype(np.float64)
    _, _, aux, rc = om.nll_eq14(p, ev, nm)
    S, pq = om.density(p, ev)
    eps, hb, _ = om.templates(ev)
    f = pq * (W.PURITY * eps * S / aux[2] + (1 - W.PURITY) * hb / aux[3])
    c = W.draw_couplings(res, W.CONFIGS["kstar10_2z"].coupling_seed)
    B, _ = om.basis(p, ev)
    mag = np.sum(np.sum(np.abs(c[None, :, None] * B), axis=1) ** 2, axis=1)
    good = mag / S <= 100
    err = np.abs(P - f)
    assert np.all(err[good] <= 2e-5 * f[good]), np.max(err[good] / f[good])
    bound = 2e-5 * (pq * W.PURITY * eps * mag / aux[2] + pq * (1 - W.PURITY) * hb / aux[3])
    assert np.all(err[~good] <= bound[~good])


@pytest.mark.parametrize("purity", [0.0, 1.0])
def test_eq14_purity_limits(A, purity):
    """P = 0: f = p q hb / B, no coupling dependence (zero gradient in the
    couplings); P = 1 with a background template: the signal-only likelihood."""
    res, p, om, gm, ev, nm = _case(A, "tiny", A.AMP4D_PATH_CACHED, purity=purity)
    nll_o, g_o, aux, rc = om.nll_eq14(p, ev, nm, grad=True)
    nll, g = gm.eval_nll_grad(p)
    assert rc == 0 and abs(nll - nll_o) < 1e-3
    if purity == 0.0:
        assert np.all(g_o == 0.0) and np.all(np.abs(g) == 0.0)
    else:
        assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))


def test_templates_can_be_removed(A):
    res, p, om, gm, ev, nm = _case(A, "tiny", A.AMP4D_PATH_CACHED)
    gm.set_background(None, None, 1.0)
    gm.set_efficiency(None, None)
    plain = O.Model(res)
    nll_o, g_o, _, _ = plain.nll(p, ev, nm, grad=True)
    nll, g = gm.eval_nll_grad(p)
    assert abs(nll - nll_o) < 1e-3
    assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))


def test_eq14_unavailable_calls(A):
    res, p, om, gm, ev, nm = _case(A, "tiny", A.AMP4D_PATH_PLAIN)
    with pytest.raises(A.Amp4dError) as e:
        gm.eval_partials(p)
    assert e.value.code == A.AMP4D_ERR_STATE
    em, ea, bm, ba, _ = W.eq14_templates(1)
    with pytest.raises(A.Amp4dError) as e:
        gm.set_background(bm, ba, 1.5)
    assert e.value.code == A.AMP4D_ERR_ARG
    bad = W.Hist2D(em.h, (1.0, 0.5, 0.0, 1.0))
    with pytest.raises(A.Amp4dError) as e:
        gm.set_efficiency(bad, ea)
    assert e.value.code == A.AMP4D_ERR_ARG
    for v in (-0.1, float("nan"), float("inf")):
        h = em.h.copy()
        h[3, 4] = v
        with pytest.raises(A.Amp4dError) as e:
            gm.set_efficiency(W.Hist2D(h, em.range), ea)
        assert e.value.code == A.AMP4D_ERR_ARG


def test_generator_follows_eq14(A):
    """With templates, amp4d_generate draws from the Eq. 14 PDF: the events'
    mean signal probability is P, and their m_Kpi and cos theta_psi histograms
    match the oracle's expectation (uniform-point integration of f) by chi^2."""
    name = "kstar10_2z"
    cfg = W.CONFIGS[name]
    res = cfg.resonances
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed))
    em, ea, bm, ba, P = W.eq14_templates(cfg.template_seed)
    gm = A.Model(res, path=A.AMP4D_PATH_CACHED)
    nm = W.uniform_points(1 << 20, cfg.norm_seed)
    gm.set_norm_points(*_dev(nm))
    gm.set_efficiency(em, ea)
    gm.set_background(bm, ba, P)
    n = 200_000
    ev = tuple(t.cpu().numpy() for t in gm.generate(p, n, 77))
    om = O.Model(res)
    om.set_template(0, em, ea)
    om.set_template(1, bm, ba, purity=P)
    _, _, aux, rc = om.nll_eq14(p, ev, nm)
    assert rc == 0
    assert abs(aux[4] / n - P) < 4 * 0.5 / math.sqrt(n)
    # expected marginals: f at fresh uniform points
    u = W.uniform_points(1_000_000, 78)
    S, pq = om.density(p, u)
    eps, hb, _ = om.templates(u)
    f = pq * (P * eps * S / aux[2] + (1 - P) * hb / aux[3])
    for var, lo, hi, nb in ((0, W.M_LO, W.M_HI, 30), (2, -1.0, 1.0, 10)):
        edges = np.linspace(lo, hi, nb + 1)
        obs, _ = np.histogram(ev[var], edges)
        wsum, _ = np.histogram(u[var], edges, weights=f)
        w2, _ = np.histogram(u[var], edges, weights=f * f)
        exp = n * wsum / wsum.sum()
        var_exp = (n / wsum.sum()) ** 2 * w2   # Monte Carlo error of the expectation
        ok = exp > 20
        chi2 = np.sum((obs[ok] - exp[ok]) ** 2 / (exp[ok] + var_exp[ok]))
        print("var %d: chi2 %.1f / %d" % (var, chi2, ok.sum()))
        assert chi2 < ok.sum() + 5 * math.sqrt(2 * ok.sum())


def test_efficiency_shards_combine_to_the_union(A):
    """With an efficiency alone the shard partials carry sum ln eps and the
    efficiency-weighted T; combined they give the single model's evaluation."""
    from paper_2007_14931_gb300.shard import shard_range
    cfg = W.CONFIGS["kstar10_z"]
    res = cfg.resonances
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed))
    em, ea, _, _, _ = W.eq14_templates(cfg.template_seed)
    ev = W.peaked_points(30_001, 5, res)
    nm = W.uniform_points(80_003, 6)

    def model(e, n):
        m = A.Model(res, path=A.AMP4D_PATH_CACHED)
        m.set_efficiency(em, ea)
        m.set_events(*_dev(e))
        m.set_norm_points(*_dev(n))
        return m
    whole = model(ev, nm)
    nll_w, g_w = whole.eval_nll_grad(p)
    parts = []
    for r in range(3):
        a, b = shard_range(len(ev[0]), r, 3)
        c, d = shard_range(len(nm[0]), r, 3)
        parts.append(model(tuple(x[a:b] for x in ev), tuple(x[c:d] for x in nm)).eval_partials(p))
    nll, g, out = A.combine_partials(np.stack(parts))
    assert abs(nll - nll_w) < 1e-4
    assert np.max(np.abs(g - g_w)) <= 1e-6 * np.max(np.abs(g_w))
    om = O.Model(res)
    om.set_template(0, em, ea)
    nll_o, _, _, rc = om.nll_eq14(p, ev, nm)
    assert rc == 0 and abs(nll - nll_o) < 1e-3


@pytest.mark.parametrize("path", ["plain", "cached"])
def test_fit_fractions_with_templates_are_those_of_S(A, path):
    """Fit fractions (Eq. 13) are defined on S: with efficiency and background
    set they equal, bit for bit, those of a model without templates on the same
    points, and the Eq. 14 evaluation afterwards is unchanged."""
    pth = A.AMP4D_PATH_PLAIN if path == "plain" else A.AMP4D_PATH_CACHED
    res, p, om, gm, ev, nm = _case(A, "kstar10_2z", pth, float_names=[])
    nll0, g0 = gm.eval_nll_grad(p)
    ff = gm.fit_fractions(p)
    plain = A.Model(res, path=pth)
    plain.set_events(*_dev(ev))
    plain.set_norm_points(*_dev(nm))
    assert np.array_equal(ff, plain.fit_fractions(p))
    nll1, g1 = gm.eval_nll_grad(p)
    assert nll1 == nll0 and np.array_equal(g1, g0)
