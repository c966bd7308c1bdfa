"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (stated by the method's accuracy targets):
  per-event S: relative 1e-5 where the interference condition number
      kappa = sum_xi (sum_k |c_k B_k,xi|)^2 / S <= 100, else absolute
      1e-5 * sum_xi (sum_k |c_k B_k,xi|)^2;
  NLL: |dNLL| <= 1e-3 (the target at 10^6 events; smaller sets are tighter);
  gradient: per component <= 1e-6 |g|_inf absolute (GRAD_TOL).  The NLL
      gradient is a difference of a data sum and N dI/I, each ~N times larger
      than their difference near the optimum, so a coherent relative error of
      the per-event FP32 terms is amplified by that ratio.  At the generating
      point of a small sample |g|_inf is a statistical fluctuation and can be
      accidentally small; there the scale is max(|g|_inf, the gradient's
      statistical scale) (_gradient_scale);
  normalisation integral I: relative 1e-9.
"""
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


def _setup(A, name, n_ev, n_mc, float_names=None, data="peaked", seed_shift=0, path=None):
    cfg = W.CONFIGS[name]
    res = cfg.resonances
    fl = cfg.float_mg if float_names is None else float_names
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c, W.float_mg_values(res, fl))
    om = O.Model(res, float_names=fl)
    if data == "peaked":
        ev = W.peaked_points(n_ev, cfg.data_seed + seed_shift, res)
    elif data == "uniform":
        ev = W.uniform_points(n_ev, cfg.data_seed + seed_shift, box=(W.M_LO, W.M_END - 1e-6))
    else:
        ev, _, _ = om.generate(p, n_ev, cfg.data_seed + seed_shift)
    nm = W.uniform_points(n_mc, cfg.norm_seed + seed_shift)
    gm = A.Model(res, float_names=fl, path=A.AMP4D_PATH_PLAIN if path is None else path)
    gm.set_events(*_dev(ev))
    gm.set_norm_points(*_dev(nm))
    return cfg, res, c, p, om, gm, ev, nm


def _check_density(om, p, c, pts, S_gpu):
    B, _ = om.basis(p, pts)
    S_o, _ = om.density(p, pts)
    mag = np.sum(np.sum(np.abs(c[None, :, None] * B), axis=1) ** 2, axis=1)
    kappa = mag / S_o
    err = np.abs(S_gpu.astype(np.float64) - S_o)
    good = kappa <= 100
    assert np.all(err[good] <= 1e-5 * S_o[good]), np.max(err[good] / S_o[good])
    assert np.all(err[~good] <= 1e-5 * mag[~good])
    return good.mean(), np.max(err[good] / S_o[good])


@pytest.mark.parametrize("name", ["tiny", "kstar10", "kstar10_z", "kstar10_2z", "lass", "lass_z"])
@pytest.mark.parametrize("data", ["peaked", "uniform"])
def test_density_parity(A, name, data):
    n = 20_003  # several tiles and a ragged tail (n % 4 = 3)
    cfg, res, c, p, om, gm, ev, nm = _setup(A, name, n, 4097, data=data)
    S = gm.eval_density(p, 0).cpu().numpy()
    frac, worst = _check_density(om, p, c, ev, S)
    assert frac > 0.9  # most events are well conditioned; the rest are held to the absolute bound
    Sn = gm.eval_density(p, 1).cpu().numpy()
    _check_density(om, p, c, nm, Sn)


@pytest.mark.parametrize("name", ["tiny", "kstar10", "kstar10_z", "kstar10_2z", "lass", "lass_z"])
def test_nll_terms_parity(A, name):
    cfg, res, c, p, om, gm, ev, nm = _setup(A, name, 50_001, 200_003)
    nll_o, _, aux, rc = om.nll(p, ev, nm)
    assert rc == 0
    t = gm.eval_terms(p)
    assert t[3] == len(ev[0])
    assert t[1] == pytest.approx(aux[1], abs=1e-9 * abs(aux[1]) + 1e-9)   # sum ln(p q), FP64 once
    assert t[2] == pytest.approx(aux[2], rel=1e-8)                         # I
    # sum ln S: 5e-4, widened by three standard deviations of the sum of the
    # per-event errors of ln S if they were independent and unbiased.  A model
    # whose amplitude has a zero (the LASS S-wave, Eq. 7, where thB + dR = pi)
    # has events whose S is ill-conditioned in the FP32 inputs; a bias would
    # still show as |sum d| >> sqrt(sum d^2).
    S_o, _ = om.density(p, ev)
    d = np.log(gm.eval_density(p, 0).cpu().numpy().astype(np.float64) / S_o)
    spread = 3.0 * math.sqrt(np.sum(d * d))
    print("%s: dI/I %.3e  d(sum ln S) %.3e  per-event sum %.3e  3 sigma %.3e" % (
        name, t[2] / aux[2] - 1, t[0] - aux[0], np.sum(d), spread))
    assert abs(t[0] - aux[0]) < 5e-4 + spread                              # sum ln S
    nll = gm.eval_nll(p)
    assert abs(nll - nll_o) < 1e-3 + 2.0 * spread


def _gradient_scale(om, p, ev, k=16):
    """Statistical scale of the -2 ln L gradient of a sample of N events at p:
    2 sqrt(N Var(t)) for the per-event terms t = d ln S / d theta, the largest
    over the components.  Var(t) comes from the spread of the oracle's data sums
    over k equal parts of the sample.  At the generating point the gradient of a
    given sample is a fluctuation of this size; it can happen to be much smaller
    (its largest component, like any other, fluctuates), and the 1e-6 bound is
    then taken relative to this scale."""
    n = len(ev[0])
    P = om.n_params
    empty = tuple(np.zeros(0, np.float32) for _ in range(4))
    sums = np.array([om.partials(p, tuple(a[idx] for a in ev), empty)[6:6 + P]
                     for idx in np.array_split(np.arange(n), k)])
    var_t = sums.var(axis=0, ddof=1) / (n / k)
    return float(np.max(2.0 * np.sqrt(n * var_t)))


@pytest.mark.parametrize("name", ["tiny", "kstar10_z", "kstar10_2z", "lass_z"])
def test_nll_grad_parity_model_data(A, name):
    n = 20_000 if name == "tiny" else 8_000
    cfg, res, c, p, om, gm, ev, nm = _setup(A, name, n, 40_000, data="model")
    nll_o, g_o, _, rc = om.nll(p, ev, nm, grad=True)
    nll, g = gm.eval_nll_grad(p)
    assert abs(nll - nll_o) < 1e-3
    scale = max(np.max(np.abs(g_o)), _gradient_scale(om, p, ev))
    print("%s: max |dg| / |g|inf %.3e, / statistical scale %.3e" % (
        name, np.max(np.abs(g - g_o)) / np.max(np.abs(g_o)), np.max(np.abs(g - g_o)) / scale))
    tol = np.maximum(1e-6 * np.abs(g_o), GRAD_TOL * scale)
    assert np.all(np.abs(g - g_o) <= tol), np.max(np.abs(g - g_o) / scale)
    nll2 = gm.eval_nll(p)
    assert nll2 == pytest.approx(nll, abs=1e-4)  # NLL-only kernel: other summation order


def test_grad_parity_all_masses_floating(A):
    """Gradient with respect to every coupling, mass and width (10 K* + Z)."""
    cfg, res, c, p, om, gm, ev, nm = _setup(A, "kstar10_z", 6_000, 30_000, data="peaked",
                                            float_names=[r.name for r in W.CONFIGS["kstar10_z"].resonances])
    nll_o, g_o, _, rc = om.nll(p, ev, nm, grad=True)
    nll, g = gm.eval_nll_grad(p)
    assert abs(nll - nll_o) < 1e-3
    rel = np.abs(g - g_o) / np.maximum(np.abs(g_o), 1e-3 * np.max(np.abs(g_o)))
    print("all M/G floating: max rel %.3e, max |dg|/|g|inf %.3e" % (np.max(rel), np.max(np.abs(g - g_o)) / np.max(np.abs(g_o))))
    assert np.max(rel) < 1e-3, np.argmax(rel)
    assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))


def test_deterministic(A):
    cfg, res, c, p, om, gm, ev, nm = _setup(A, "kstar10_z", 30_001, 50_000)
    a = gm.eval_nll_grad(p)
    b = gm.eval_nll_grad(p)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_host_pointer_inputs(A):
    """set_events accepts host arrays too (the library copies them)."""
    cfg = W.CONFIGS["tiny"]
    res = cfg.resonances
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed))
    ev = W.peaked_points(1001, 3, res)
    nm = W.uniform_points(2003, 4)
    g1 = A.Model(res)
    g1.set_events(*ev)
    g1.set_norm_points(*nm)
    g2 = A.Model(res)
    g2.set_events(*_dev(ev))
    g2.set_norm_points(*_dev(nm))
    assert g1.eval_nll(p) == g2.eval_nll(p)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_tiny_and_ragged_sizes(A, n):
    cfg = W.CONFIGS["kstar10_z"]
    res = cfg.resonances
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c)
    ev = W.peaked_points(n, 17, res)
    nm = W.uniform_points(n + 2, 18)
    om = O.Model(res)
    gm = A.Model(res)
    gm.set_events(*_dev(ev))
    gm.set_norm_points(*_dev(nm))
    nll_o, g_o, _, _ = om.nll(p, ev, nm, grad=True)
    nll, g = gm.eval_nll_grad(p)
    assert abs(nll - nll_o) < 1e-4
    assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))
    _check_density(om, p, c, ev, gm.eval_density(p, 0).cpu().numpy())


def test_errors(A):
    cfg = W.CONFIGS["tiny"]
    res = cfg.resonances
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed))
    gm = A.Model(res)
    with pytest.raises(A.Amp4dError) as e:
        gm.eval_nll_grad(p)
    assert e.value.code == A.AMP4D_ERR_STATE
    ev = [a.copy() for a in W.uniform_points(100, 1)]
    ev[0][37] = 3.0  # outside the m_Kpi box
    with pytest.raises(A.Amp4dError) as e:
        gm.set_events(*_dev(ev))
    assert e.value.code == A.AMP4D_ERR_INPUT and "37" in str(e.value)
    ev[0][37] = 1.0
    ev[3][12] = float("nan")
    with pytest.raises(A.Amp4dError) as e:
        gm.set_events(*_dev(ev))
    assert e.value.code == A.AMP4D_ERR_INPUT and "12" in str(e.value)
    ev[3][12] = 0.5
    gm.set_events(*_dev(ev))
    gm.set_norm_points(*_dev(W.uniform_points(100, 2)))
    # all couplings zero: S = 0 everywhere -> domain error, NLL = +inf
    nll = gm.eval_nll(np.zeros_like(p))
    assert math.isinf(nll) and nll > 0
    # a good evaluation still works afterwards
    assert math.isfinite(gm.eval_nll(p))
    with pytest.raises(ValueError):
        gm.eval_nll(p[:-1])
    bad = p.copy()
    bad[3] = float("inf")
    with pytest.raises(A.Amp4dError) as e:
        gm.eval_nll_grad(bad)
    assert e.value.code == A.AMP4D_ERR_ARG


def test_bad_model_arguments(A):
    r = W.CONFIGS["tiny"].resonances
    with pytest.raises(A.Amp4dError):
        A.Model(r, box=(0.5, 2.0))      # below the K pi threshold
    zz = [W.Z4430, W.Z4200, W.Z4430]
    with pytest.raises(A.Amp4dError):
        A.Model(r + zz)                  # at most two Z


def test_nll_grad_1e6_model_events(A):
    """The accuracy target at 10^6 events: 10 K* + Z(4430), data drawn from the model by the
    oracle's accept-reject generator, 4e6 uniform normalisation points."""
    cfg, res, c, p, om, gm, ev, nm = _setup(A, "kstar10_z", 1_000_000, 4_000_000, data="model")
    nll_o, g_o, aux, rc = om.nll(p, ev, nm, grad=True)
    nll, g = gm.eval_nll_grad(p)
    t = gm.eval_terms(p)
    print("dNLL %.3e  d(sum lnS) %.3e  dI/I %.3e" % (nll - nll_o, t[0] - aux[0], t[2] / aux[2] - 1))
    assert abs(nll - nll_o) <= 1e-3
    tol = np.maximum(1e-6 * np.abs(g_o), GRAD_TOL * np.max(np.abs(g_o)))
    print("1e6: max |dg|/|g|inf = %.3e" % (np.max(np.abs(g - g_o)) / np.max(np.abs(g_o))))
    assert np.all(np.abs(g - g_o) <= tol), np.max(np.abs(g - g_o)) / np.max(np.abs(g_o))


def test_full_size_benchmarked_path(A):
    """The benchmark's workload and launch configuration: 10 K* + Z(4430), 5e6
    peaked data events, 2^24 uniform normalisation points, every mass and width
    fixed, the cached path (all lineshapes from the basis cache, the two-event
    adjoint kernel over a multi-sweep grid, the tensor-core Gram normalisation).
    NLL and every gradient component against the oracle, at two parameter points
    (the second one after the couplings-only table update)."""
    cfg, res, c, p, om, gm, ev, nm = _setup(A, "large", 5_000_000, 1 << 24, path=A.AMP4D_PATH_CACHED)
    assert not cfg.float_mg
    for k, pk in enumerate([p, p * (1.0 + 1e-3 * math.sin(0.7))]):
        nll_o, g_o, aux, rc = om.nll(pk, ev, nm, grad=True)
        assert rc == 0
        nll, g = gm.eval_nll_grad(pk)
        gi = np.max(np.abs(g_o))
        print("large point %d: dNLL %.3e (NLL %.6f), max |dg|/|g|inf = %.3e" % (
            k, nll - nll_o, nll_o, np.max(np.abs(g - g_o)) / gi))
        # data not drawn from the model: the NLL is 5e7 and its gradient O(N)
        assert abs(nll - nll_o) <= 1e-9 * abs(nll_o)
        assert np.all(np.abs(g - g_o) <= GRAD_TOL * gi), np.argmax(np.abs(g - g_o))
    assert gm.eval_terms(p)[3] == 5_000_000


def test_full_size_floated_z_path(A):
    """The floated-mass benchmark configuration (Z(4430) mass and width free):
    5e6 events and 2^24 points, the per-point adjoint over the normalisation
    points with the Z lineshape computed per event and point; NLL and gradient
    against the oracle."""
    cfg, res, c, p, om, gm, ev, nm = _setup(A, "large_float_z", 5_000_000, 1 << 24,
                                            path=A.AMP4D_PATH_CACHED)
    assert cfg.float_mg
    nll_o, g_o, aux, rc = om.nll(p, ev, nm, grad=True)
    assert rc == 0
    nll, g = gm.eval_nll_grad(p)
    gi = np.max(np.abs(g_o))
    print("large_float_z: dNLL %.3e, max |dg|/|g|inf = %.3e" % (nll - nll_o, np.max(np.abs(g - g_o)) / gi))
    assert abs(nll - nll_o) <= 1e-9 * abs(nll_o)
    assert np.all(np.abs(g - g_o) <= GRAD_TOL * gi), np.argmax(np.abs(g - g_o))


def test_density_bias(A):
    """Mean relative error of S, weighted as in the normalisation integral (w S):
    the FP32 path must not carry a systematic offset (the NLL of data that do not
    follow the model would otherwise shift by N times it)."""
    cfg, res, c, p, om, gm, ev, nm = _setup(A, "kstar10_z", 4, 1_000_000)
    Sg = gm.eval_density(p, 1).cpu().numpy().astype(np.float64)
    So, pq = om.density(p, nm)
    rel = Sg / So - 1
    w = So * pq
    bias = np.sum(rel * w) / np.sum(w)
    sem = np.sqrt(np.sum((rel - bias) ** 2 * w * w)) / np.sum(w)
    print("weighted S bias %.3e +- %.1e, unweighted %.3e" % (bias, sem, rel.mean()))
    assert abs(bias) < 5e-9 + 4 * sem


@pytest.mark.parametrize("name", ["tiny", "kstar10_z", "kstar10_2z", "lass"])
def test_pdf_parity(A, name):
    """P(e) = S p q / I per data event (Eq. 5 with the phase-space density): the
    oracle's S and p q over its own I, per event, with the per-event density
    tolerance and I to 1e-8."""
    cfg, res, c, p, om, gm, ev, nm = _setup(A, name, 20_003, 40_009)
    P = gm.eval_pdf(p).cpu().numpy().astype(np.float64)
    S_o, pq_o = om.density(p, ev)
    I_o = om.norm(p, nm)
    P_o = S_o * pq_o / I_o
    B, _ = om.basis(p, ev)
    mag = np.sum(np.sum(np.abs(c[None, :, None] * B), axis=1) ** 2, axis=1)
    good = mag / S_o <= 100
    err = np.abs(P - P_o)
    assert np.all(err[good] <= 2e-5 * P_o[good]), np.max(err[good] / P_o[good])
    assert np.all(err[~good] <= 2e-5 * mag[~good] * pq_o[~good] / I_o)


@pytest.mark.parametrize("n", [1, 2, 3, 127, 129, 4097, 100_003])
def test_cached_all_fixed_ragged_sizes(A, n):
    """The all-cached adjoint kernel takes two events per thread (e and e + grid
    stride); at these sizes some threads have one real event and one beyond n.
    Its NLL and gradient must match the oracle and the plain path, and repeated
    calls (the Gram path, the couplings-only table update) must give the same bits."""
    cfg = W.CONFIGS["large"]
    res = cfg.resonances
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c)
    ev = W.peaked_points(n, 19, res)
    nm = W.uniform_points(max(n + 5, 70_001), 20)
    om = O.Model(res)
    nll_o, g_o, _, rc = om.nll(p, ev, nm, grad=True)
    assert rc == 0
    gc = A.Model(res, path=A.AMP4D_PATH_CACHED)
    gc.set_events(*_dev(ev))
    gc.set_norm_points(*_dev(nm))
    gp = A.Model(res)
    gp.set_events(*_dev(ev))
    gp.set_norm_points(*_dev(nm))
    nll_c, g_c = gc.eval_nll_grad(p)
    nll_c2, g_c2 = gc.eval_nll_grad(p)
    nll_p, g_p = gp.eval_nll_grad(p)
    assert nll_c2 == nll_c and np.array_equal(g_c2, g_c)
    tol_nll = 1e-4 + 1e-9 * abs(nll_o)
    assert abs(nll_c - nll_o) < tol_nll and abs(nll_p - nll_o) < tol_nll
    assert np.max(np.abs(g_c - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))
    assert np.max(np.abs(g_c - g_p)) <= GRAD_TOL * np.max(np.abs(g_o))


@pytest.mark.parametrize("R", [1.0, 2.0, 0.0])
def test_lass_density_near_threshold_and_pole(A, R):
    """LASS S-wave (Eq. 7-9) with K*(892): events packed near the K pi threshold
    (q -> 0, where the background term tends to m a), at the K0*(1430) pole and
    across the box, for the elastic factor R = 1, the printed R = 2 and the
    background alone (R = 0)."""
    import dataclasses
    res = [dataclasses.replace(W.LASS, lass_R=R), W.RESONANCES["K*(892)"]]
    c = W.draw_couplings(res, 77)
    p = W.couplings_to_params(c)
    rng = np.random.default_rng(78)
    n = 12_007
    m = np.concatenate([W.M_LO + rng.uniform(0, 1e-3, 4000),
                        W.LASS.M + rng.normal(0, 0.02, 4000),
                        rng.uniform(W.M_LO, W.M_END - 1e-6, n - 8000)])
    m = np.clip(m, W.M_LO, W.M_END - 1e-6).astype(np.float32)
    pts = (m, rng.uniform(-1, 1, n).astype(np.float32), rng.uniform(-1, 1, n).astype(np.float32),
           rng.uniform(-math.pi, math.pi, n).astype(np.float32))
    om = O.Model(res)
    gm = A.Model(res)
    gm.set_events(*_dev(pts))
    gm.set_norm_points(*_dev(W.uniform_points(4097, 79)))
    S = gm.eval_density(p, 0).cpu().numpy()
    _check_density(om, p, c, pts, S)
    for path in (A.AMP4D_PATH_PLAIN, A.AMP4D_PATH_CACHED):
        g2 = A.Model(res, path=path)
        g2.set_events(*_dev(pts))
        g2.set_norm_points(*_dev(W.uniform_points(70_001, 80)))
        nll_o, g_o, _, rc = om.nll(p, pts, W.uniform_points(70_001, 80), grad=True)
        assert rc == 0
        nll, g = g2.eval_nll_grad(p)
        assert abs(nll - nll_o) < 1e-4 + 1e-9 * abs(nll_o)
        assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))


def _structure_case(case):
    """Resonance lists that select each compiled variant of the all-cached data
    kernel: the K* count filling its bucket with 0-3 scalars (their positions
    compile-time), with four scalars (run-time spin tests), and with a Z that has
    a single column (run-time column tests)."""
    T = {r.name: r for r in W.KSTAR_TABLE}
    extra_vec = W.Resonance("K*(1550)", W.CHAIN_KSTAR, 1, -1, 1.55, 0.25)
    extra_scalar = W.Resonance("K0*(1200)", W.CHAIN_KSTAR, 0, +1, 1.20, 0.30)
    if case == "bucket2_one_scalar":
        return [T["K*(892)"], T["K0*(1430)"]]
    if case == "bucket10_two_scalars_z":
        return [extra_vec if r.name == "K0*(800)" else r for r in W.KSTAR_TABLE] + [W.Z4430]
    if case == "bucket10_one_scalar_z":
        return [extra_vec if r.name in ("K0*(800)", "K0*(1950)") else r
                for r in W.KSTAR_TABLE[:9]] + [T["K2*(1980)"], W.Z4430]
    if case == "bucket10_four_scalars_z":
        return [extra_scalar if r.name == "K*(1410)" else r for r in W.KSTAR_TABLE] + [W.Z4430]
    if case == "z_one_column":   # J^P = 1^-: no l' = 0 column
        return list(W.KSTAR_TABLE) + [W.Resonance("Z(1-)", W.CHAIN_Z, 1, -1, 4.43, 0.18)]
    raise ValueError(case)


@pytest.mark.parametrize("case", ["bucket2_one_scalar", "bucket10_two_scalars_z", "bucket10_one_scalar_z",
                                  "bucket10_four_scalars_z", "z_one_column"])
def test_structure_variants_match_oracle(A, case):
    """Cached path (the benchmarked data kernel and its variants) against the
    oracle: NLL within 1e-3, every gradient component within 1e-6 of the
    gradient scale; also with the Eq. 14 efficiency and background (the unstaged
    variants), within 1e-6 of |g|_inf as in the Eq. 14 parity tests."""
    res = _structure_case(case)
    nsc = sum(1 for r in res if r.chain == W.CHAIN_KSTAR and r.J == 0)
    c = W.draw_couplings(res, 23)
    p = W.couplings_to_params(c)
    om = O.Model(res)
    ev = W.peaked_points(8_000, 24, res)
    nm = W.uniform_points(40_000, 25)
    gm = A.Model(res, path=A.AMP4D_PATH_CACHED)
    gm.set_events(*_dev(ev))
    gm.set_norm_points(*_dev(nm))
    nll_o, g_o, _, rc = om.nll(p, ev, nm, grad=True)
    nll, g = gm.eval_nll_grad(p)
    scale = max(np.max(np.abs(g_o)), _gradient_scale(om, p, ev))
    print("%s (%d scalars): dNLL %.2e, max |dg| / scale %.3e" % (
        case, nsc, nll - nll_o, np.max(np.abs(g - g_o)) / scale))
    assert abs(nll - nll_o) < 1e-3
    assert np.all(np.abs(g - g_o) <= np.maximum(1e-6 * np.abs(g_o), GRAD_TOL * scale))
    # the same model with the Eq. 14 efficiency and background
    em, ea, bm, ba, _ = W.eq14_templates(26)
    gm.set_efficiency(em, ea)
    gm.set_background(bm, ba, W.PURITY)
    om.set_template(0, em, ea)
    om.set_template(1, bm, ba, purity=W.PURITY)
    nll_o, g_o, _, rc = om.nll_eq14(p, ev, nm, grad=True)
    nll, g = gm.eval_nll_grad(p)
    print("%s with Eq. 14: dNLL %.2e, max |dg| / |g|inf %.3e" % (
        case, nll - nll_o, np.max(np.abs(g - g_o)) / np.max(np.abs(g_o))))
    assert rc == 0
    assert abs(nll - nll_o) < 1e-3
    assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))
    gm.close()
