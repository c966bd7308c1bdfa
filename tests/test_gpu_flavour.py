"""Flavour tags and mistag (text after Eq. 12) on the GPU path, against the FP64
oracle, which evaluates S at t phi and -t phi from recomputed kinematics (the
GPU conjugates the angular phase factors of the same coupling sums).
Tolerances as in the signal parity tests: |dNLL| < 1e-3, gradient <= 1e-6
|g|_inf, per-event density relative 1e-5 where well conditioned."""
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


def _phi_even(hist):
    return W.Hist2D(((hist.h + hist.h[::-1, :]) / 2).astype(np.float32), hist.range)


def _case(A, name, path, w, fl=None, templates=False, n_ev=15_001, n_mc=40_003):
    cfg = W.CONFIGS[name]
    res = cfg.resonances
    fl = cfg.float_mg if fl is None else fl
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed), W.float_mg_values(res, fl))
    ev = W.peaked_points(n_ev, cfg.data_seed + 3, res)
    nm = W.uniform_points(n_mc, cfg.norm_seed + 3)
    tag = np.where(np.random.default_rng(cfg.index).uniform(size=n_ev) < 0.45, 1.0, -1.0).astype(np.float32)
    om = O.Model(res, float_names=fl)
    om.set_mistag(w)
    gm = A.Model(res, float_names=fl, path=path)
    if templates:
        em, ea, bm, ba, P = W.eq14_templates(cfg.template_seed)
        ea = _phi_even(ea)
        om.set_template(0, em, ea)
        om.set_template(1, bm, ba, purity=P)
        gm.set_efficiency(em, ea)
    gm.set_events(*_dev(ev))
    gm.set_norm_points(*_dev(nm))
    gm.set_flavour(tag, w)
    if templates:
        gm.set_background(bm, ba, P)
    return res, p, om, gm, ev, nm, tag


@pytest.mark.parametrize("path", ["plain", "cached"])
@pytest.mark.parametrize("name,fl", [("tiny", None), ("kstar10_z", None), ("kstar10_2z", []),
                                     ("kstar10_2z", None), ("lass_z", [])])
@pytest.mark.parametrize("w", [0.0, 0.07])
def test_flavour_parity(A, path, name, fl, w):
    pth = A.AMP4D_PATH_PLAIN if path == "plain" else A.AMP4D_PATH_CACHED
    res, p, om, gm, ev, nm, tag = _case(A, name, pth, w, fl)
    nll_o, g_o, aux, rc = om.nll_eq14(p, ev, nm, grad=True, tag=tag)
    assert rc == 0
    nll, g = gm.eval_nll_grad(p)
    print("%s %s fl=%s w=%g: dNLL %.3e max|dg|/|g| %.3e" % (
        name, path, fl, w, nll - nll_o, np.max(np.abs(g - g_o)) / np.max(np.abs(g_o))))
    assert abs(nll - nll_o) < 1e-3
    assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))
    assert gm.eval_nll(p) == pytest.approx(nll, abs=1e-4)


@pytest.mark.parametrize("path", ["plain", "cached"])
def test_flavour_with_efficiency_and_background(A, path):
    pth = A.AMP4D_PATH_PLAIN if path == "plain" else A.AMP4D_PATH_CACHED
    res, p, om, gm, ev, nm, tag = _case(A, "kstar10_2z", pth, 0.05, templates=True)
    nll_o, g_o, aux, rc = om.nll_eq14(p, ev, nm, grad=True, tag=tag)
    nll, g = gm.eval_nll_grad(p)
    assert rc == 0 and abs(nll - nll_o) < 1e-3
    assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))


def test_tagged_density(A):
    """eval_density returns (1 - w) S(t phi) + w S(-t phi)."""
    w = 0.1
    res, p, om, gm, ev, nm, tag = _case(A, "kstar10_2z", A.AMP4D_PATH_PLAIN, w)
    S = gm.eval_density(p, 0).cpu().numpy().astype(np.float64)
    plain = O.Model(res, float_names=W.CONFIGS["kstar10_2z"].float_mg)
    Sa, _ = plain.density(p, (ev[0], ev[1], ev[2], tag * ev[3]))
    Sb, _ = plain.density(p, (ev[0], ev[1], ev[2], -tag * ev[3]))
    ref = (1 - w) * Sa + w * Sb
    mag = np.maximum(ref, 1e-300)
    rel = np.abs(S - ref) / mag
    assert np.quantile(rel, 0.99) < 1e-5
    assert np.all(np.abs(S - ref) <= 1e-5 * np.maximum(ref, np.max(ref) * 1e-6))


def test_tags_equal_mirrored_events(A):
    """w = 0: a B0bar-tagged event is the B0 event at -phi, bit for bit (the
    stored records are the mirrored event's)."""
    res, p, om, gm, ev, nm, tag = _case(A, "kstar10_2z", A.AMP4D_PATH_CACHED, 0.0)
    mir = A.Model(res, float_names=W.CONFIGS["kstar10_2z"].float_mg, path=A.AMP4D_PATH_CACHED)
    mir.set_events(*_dev((ev[0], ev[1], ev[2], (tag * ev[3]).astype(np.float32))))
    mir.set_norm_points(*_dev(nm))
    a, ga = gm.eval_nll_grad(p)
    b, gb = mir.eval_nll_grad(p)
    assert a == b and np.array_equal(ga, gb)
    gm.set_flavour(None, 0.0)   # back to all B0
    plain = A.Model(res, float_names=W.CONFIGS["kstar10_2z"].float_mg, path=A.AMP4D_PATH_CACHED)
    plain.set_events(*_dev(ev))
    plain.set_norm_points(*_dev(nm))
    c, gc = gm.eval_nll_grad(p)
    d, gd = plain.eval_nll_grad(p)
    assert c == d and np.array_equal(gc, gd)


def test_flavour_errors(A):
    res, p, om, gm, ev, nm, tag = _case(A, "tiny", A.AMP4D_PATH_PLAIN, 0.0, n_ev=1001, n_mc=2001)
    bad = tag.copy()
    bad[17] = 0.5
    with pytest.raises(A.Amp4dError) as e:
        gm.set_flavour(bad, 0.0)
    assert e.value.code == A.AMP4D_ERR_ARG
    with pytest.raises(A.Amp4dError) as e:
        gm.set_flavour(tag, 0.6)
    assert e.value.code == A.AMP4D_ERR_ARG
    em, ea, _, _, _ = W.eq14_templates(2)
    asym = W.Hist2D(ea.h.copy(), ea.range)
    asym.h[0, 0] += 0.25
    with pytest.raises(A.Amp4dError) as e:
        gm.set_efficiency(em, asym)
    assert e.value.code == A.AMP4D_ERR_STATE
    gm.set_efficiency(em, _phi_even(ea))   # an even one is accepted
