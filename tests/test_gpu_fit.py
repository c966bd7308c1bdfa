"""Closure fit with the GPU likelihood (Fit validation section): data drawn from
the model by the oracle's generator, fitted from a perturbed start with the
analytic GPU gradient; the result matches the oracle-driven fit within 0.05
sigma and the truth within 3 sigma.  Also checks the autograd bridge."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402
from conftest import load_product_module  # noqa: E402

F = load_product_module("fit")


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2007_14931_gb300 as A
    return A


def _wrap(d):
    d = d.copy()
    d[1::2] = (d[1::2] + math.pi) % (2 * math.pi) - math.pi
    return d


def test_closure_fit_gpu_matches_oracle_fit(A):
    cfg = W.CONFIGS["tiny"]
    res = cfg.resonances
    om = O.Model(res)
    c = W.draw_couplings(res, cfg.coupling_seed)
    p_true = W.couplings_to_params(c)
    ev, _, _ = om.generate(p_true, cfg.n_events, cfg.data_seed)
    nm = W.uniform_points(cfg.n_norm, cfg.norm_seed)
    gm = A.Model(res)
    gm.set_events(*(torch.from_numpy(a).cuda() for a in ev))
    gm.set_norm_points(*(torch.from_numpy(a).cuda() for a in nm))
    fixed = [k for k, (R, l) in enumerate(W.columns(res)) if res[R].name == "K*(892)" and l == 0][0]
    par = F.Parametrization(len(c), 0, fixed_col=fixed, polar=True)
    c0 = W.perturbed_start(c)
    c0[fixed] = 1.0
    p0 = W.couplings_to_params(c0)
    rg = F.fit(gm.eval_nll_grad, par, p0, tol=0.01)

    def fo(p):
        nll, g, _, _ = om.nll(p, ev, nm, grad=True)
        return nll, g
    ro = F.fit(fo, par, p0, tol=0.01)
    assert rg.converged and ro.converged
    dev = _wrap(rg.theta - ro.theta) / ro.errors
    print("GPU vs oracle fit, max |d|/sigma = %.4f" % np.max(np.abs(dev)))
    assert np.max(np.abs(dev)) < 0.05
    pulls = _wrap(rg.theta - par.from_params(p_true)) / rg.errors
    assert np.all(np.abs(pulls) < 3.5)
    assert abs(rg.fval - ro.fval) < 1e-3


def test_autograd_bridge(A):
    cfg = W.CONFIGS["tiny"]
    res = cfg.resonances
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c)
    ev = W.peaked_points(5000, 1, res)
    nm = W.uniform_points(20000, 2)
    gm = A.Model(res)
    gm.set_events(*(torch.from_numpy(a).cuda() for a in ev))
    gm.set_norm_points(*(torch.from_numpy(a).cuda() for a in nm))
    fn = F.nll_function()
    x = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    y = fn.apply(x, gm)
    y.backward()
    nll, g = gm.eval_nll_grad(p)
    assert float(y) == nll
    assert np.array_equal(x.grad.numpy(), g)


def test_large_fit_minimum_agrees_with_oracle(A):
    """Closure fit of 10 K* + Z(4430) at 10^6 events and 2^22 points on the
    cached path (basis cache, tensor-core Gram), then the oracle at the GPU
    minimum.  In every direction the data constrain (Hessian eigenvalue above
    1e-6 of the largest), one Newton step with the oracle's gradient moves the
    minimum by less than 0.05 of that direction's standard error, and the two
    NLLs there agree to 1e-9 of |NLL|.  (This model has weak modes: the K4*(2045)
    helicity-1 couplings are barely constrained near the kinematic edge.)"""
    cfg = W.CONFIGS["large"]
    res = cfg.resonances
    cols = W.columns(res)
    c = W.draw_couplings(res, cfg.coupling_seed)
    fixed = [k for k, (R, l) in enumerate(cols) if res[R].name == "K*(892)" and l == 0][0]
    c = c / c[fixed]
    p_true = W.couplings_to_params(c)
    n_ev, n_mc = 1_000_000, 1 << 22
    gen = A.Model(res)
    ev = gen.generate(p_true, n_ev, 31)
    nm = W.uniform_points(n_mc, cfg.norm_seed)
    gm = A.Model(res, path=A.AMP4D_PATH_CACHED)
    gm.set_events(*ev)
    gm.set_norm_points(*(torch.from_numpy(a).cuda() for a in nm))
    par = F.Parametrization(len(c), 0, fixed_col=fixed, polar=True)
    c0 = W.perturbed_start(c)
    c0[fixed] = 1.0
    rg = F.fit(gm.eval_nll_grad, par, W.couplings_to_params(c0), tol=0.1)
    assert rg.converged
    lam, V = rg.well_constrained()
    ev_h = tuple(t.cpu().numpy() for t in ev)
    om = O.Model(res)
    nll_o, g_o, _, rc = om.nll(rg.params, ev_h, nm, grad=True)
    assert rc == 0
    nll_g, _ = gm.eval_nll_grad(rg.params)
    gt = V.T @ par.grad_to_theta(rg.theta, g_o)
    dev = gt / np.sqrt(2.0 * lam)          # Newton step / standard error, per direction
    print("large fit: nfcn %d, %d of %d directions constrained, |dNLL| at the minimum %.2e, "
          "max oracle Newton step %.4f sigma" % (rg.nfcn, len(lam), len(rg.theta),
                                                  abs(nll_g - nll_o), np.max(np.abs(dev))))
    assert len(lam) >= len(rg.theta) - 5
    assert abs(nll_g - nll_o) <= 1e-9 * abs(nll_o)   # as for the full-size NLL parity
    assert np.max(np.abs(dev)) < 0.05


def test_toy_pull_distributions(A):
    """Toy study (the paper's pull distributions, Figs. 5-8): 40 data sets of 5000
    events drawn by the GPU generator from the two-K* model, each fitted from a
    perturbed start; for every free parameter the pulls (fitted - generated) /
    error have mean within 0.6 of 0 (3.8 standard errors of the mean) and
    standard deviation within [0.6, 1.5].  The 4e5 normalisation points are
    shared by all toys (events / points = 0.0125)."""
    cfg = W.CONFIGS["tiny"]
    res = cfg.resonances
    cols = W.columns(res)
    c = W.draw_couplings(res, cfg.coupling_seed)
    fixed = [k for k, (R, l) in enumerate(cols) if res[R].name == "K*(892)" and l == 0][0]
    c = c / c[fixed]
    p_true = W.couplings_to_params(c)
    par = F.Parametrization(len(c), 0, fixed_col=fixed, polar=True)
    th_true = par.from_params(p_true)
    gen = A.Model(res)
    gm = A.Model(res, path=A.AMP4D_PATH_CACHED)
    gm.set_norm_points(*(torch.from_numpy(a).cuda() for a in W.uniform_points(400_000, 41)))
    pulls = []
    for toy in range(40):
        gm.set_events(*gen.generate(p_true, 5000, 1000 + toy))
        c0 = W.perturbed_start(c, seed=toy)
        c0[fixed] = 1.0
        r = F.fit(gm.eval_nll_grad, par, W.couplings_to_params(c0), tol=0.1)
        assert r.converged
        pulls.append(_wrap(r.theta - th_true) / r.errors)
    pulls = np.array(pulls)
    mean, sd = pulls.mean(axis=0), pulls.std(axis=0, ddof=1)
    print("toy pulls: mean", np.round(mean, 2), "sd", np.round(sd, 2))
    assert np.all(np.abs(mean) < 0.6)
    assert np.all((sd > 0.6) & (sd < 1.5))


def test_z_sensitivity(A):
    """Fit validation, Z sensitivity: events generated with the ten K* alone and
    fitted with the ten K* + Z(4200) + Z(4430) model give Z fit fractions
    consistent with zero (the paper finds about 0.01 %)."""
    res_g = W.CONFIGS["kstar10"].resonances
    res_f = W.CONFIGS["kstar10_2z"].resonances
    assert [r.name for r in res_f[:len(res_g)]] == [r.name for r in res_g]
    cols_g, cols_f = W.columns(res_g), W.columns(res_f)
    fixed = [k for k, (R, l) in enumerate(cols_g) if res_g[R].name == "K*(892)" and l == 0][0]
    c_g = W.draw_couplings(res_g, W.CONFIGS["kstar10"].coupling_seed)
    c_g = c_g / c_g[fixed]
    gen = A.Model(res_g)
    ev = gen.generate(W.couplings_to_params(c_g), 200_000, 909)
    nm = W.uniform_points(1 << 21, 910)
    m = A.Model(res_f, path=A.AMP4D_PATH_CACHED)
    m.set_events(*ev)
    m.set_norm_points(*(torch.from_numpy(a).cuda() for a in nm))
    nz = len(cols_f) - len(cols_g)
    rng = np.random.default_rng(911)
    c0 = np.concatenate([W.perturbed_start(c_g), 0.02 * np.exp(1j * rng.uniform(-np.pi, np.pi, nz))])
    c0[fixed] = 1.0
    par = F.Parametrization(len(c0), 0, fixed_col=fixed, polar=False)
    r = F.fit(m.eval_nll_grad, par, W.couplings_to_params(c0), tol=0.1)
    assert r.converged
    ff = m.fit_fractions(par.to_params(r.theta))
    ffz = ff[len(res_g):]
    print("Z fit fractions on K*-only data: %s" % ", ".join("%.2e" % x for x in ffz))
    assert np.all(ffz < 1e-3)


def test_learned_normalisation_reproduces_the_uniform_minimum(A):
    """The learned normalisation serves the fit: 10 K* + Z(4430), 10^6 events the GPU
    generator draws from the model.  The reference likelihood f = -2 ln L uses 2^26
    uniform normalisation points; its minimum is fitted from the generating point.
    From that minimum, fits with 2^24 uniform points and with two independent
    2^20-point samples of the proposal aimed at the Gram matrix (target
    sum_k |B_k|^2 p q) all converge, and each of their minima lies within one
    standard deviation per free parameter of the reference: on the reference
    likelihood, [f(theta) - f(theta_ref)] / n_free < 1 (for a quadratic f this is
    the mean squared shift in standard deviations).  The measure needs neither a
    Hessian, which finite differences give poorly along this model's nearly flat
    directions, nor convexity between the minima: the likelihood has several nearby
    valleys of almost equal depth, and a fit started at one minimum with another
    normalisation sample can end in a neighbouring one."""
    cfg = W.CONFIGS["learned"]
    res = cfg.resonances
    cols = W.columns(res)
    c = W.draw_couplings(res, cfg.coupling_seed)
    fixed = [k for k, (R, l) in enumerate(cols) if res[R].name == "K*(892)" and l == 0][0]
    c = c / c[fixed]
    p_true = W.couplings_to_params(c)
    m = A.Model(res, path=A.AMP4D_PATH_CACHED)
    ev = m.generate(p_true, 1_000_000, 77)
    m.set_events(*ev)
    one = np.ones(1, dtype=np.float32)

    def uniform(n, seed):     # uniform points, w = V p q (one-cell grid)
        pts, w, _ = A.grid_sample(one, (1, 1, 1, 1), 1.0, seed, n)
        m.set_norm_points(*pts, w=w, volume=1.0)

    par = F.Parametrization(len(c), 0, fixed_col=fixed, polar=True)
    uniform(1 << 26, 9000)
    r_ref = F.fit(m.eval_nll_grad, par, p_true, tol=0.1)
    start = par.to_params(r_ref.theta)
    uniform(1 << 24, 9101)
    fits = {"uniform 2^24": F.fit(m.eval_nll_grad, par, start, tol=0.1)}
    m.proposal_train_gram(p_true, n=1 << 20, seed=12)
    for k, sd in enumerate((201, 202)):
        pts, w = m.proposal_sample(1 << 20, sd)
        m.set_norm_points(*pts, w=w, volume=1.0)
        fits["learned %d" % (k + 1)] = F.fit(m.eval_nll_grad, par, start, tol=0.1)
    uniform(1 << 26, 9000)
    f_ref = m.eval_nll(par.to_params(r_ref.theta))
    loss = {k: (m.eval_nll(par.to_params(r.theta)) - f_ref) / par.n_free for k, r in fits.items()}
    print("reference-likelihood loss per free parameter: " +
          ", ".join("%s %.3f (edm %.1e)" % (k, loss[k], fits[k].edm) for k in fits) +
          "; converged %s" % [bool(r.converged) for r in [r_ref] + list(fits.values())])
    assert r_ref.converged and all(r.converged for r in fits.values())
    assert all(v < 1 for v in loss.values())
