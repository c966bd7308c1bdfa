"""Tensor-core Gram matrix of the normalisation (tcgen05 path) and the cached
evaluation path that uses it, against the FP64 oracle.

Tolerances: G entries 1e-6 of max|G| (the FP32 basis carries ~1e-7 relative
per-point errors, which the sums average); I from G within 3e-8 of the
oracle's I (the FP32 basis values carry a ~1e-8 weighted offset) and within
5e-9 of sum w S over the GPU's own FP32 per-point densities (the same basis
values: fixed-point quantisation and per-point FP32 rounding only); the
integer digit-product accumulation itself is compared bit for bit; NLL within
1e-3; gradient as the plain path."""
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


def _digits(X):
    d1 = (X + (1 << 23)) >> 24
    r1 = X - (d1 << 24)
    d2 = (r1 + (1 << 15)) >> 16
    r2 = r1 - (d2 << 16)
    d3 = (r2 + 128) >> 8
    d4 = r2 - (d3 << 8)
    return [d1, d2, d3, d4]


def _rnd(v, s):
    return (v + (1 << (s - 1))) >> s


def _gram_int_reference(X):
    """Exact integer reference of the tensor-core Gram accumulation (per 512-point chunk:
    P_ab = D_a^T D_b, combined with weights 2^(8(5-a-b)), a = b = 4 dropped, the
    2^-8 / 2^-16 terms rounded half up)."""
    n = X.shape[0]
    G = np.zeros((64, 64), dtype=np.int64)
    for c0 in range(0, n, 512):
        rows = X[c0:c0 + 512].reshape(-1, 64).astype(np.int64)
        d = _digits(rows)
        P = {(a, b): d[a - 1].T @ d[b - 1] for a in range(1, 5) for b in range(1, 5)}
        assert max(abs(v).max() for v in P.values()) <= (1 << 24)
        G += (P[1, 1] << 24) + (P[1, 2] << 16) + (P[1, 3] << 8) + P[1, 4] + _rnd(P[3, 3], 8)
        G += ((P[1, 3] << 8) + P[1, 4]).T
        G += (P[2, 1] << 16) + (P[2, 2] << 8) + P[2, 3] + _rnd(P[2, 4], 8) + _rnd(P[4, 3], 16)
        G += (P[2, 3] + _rnd(P[2, 4], 8) + _rnd(P[4, 3], 16)).T
    return G


@pytest.mark.parametrize("case", ["random", "extreme", "ragged_small"])
def test_tensor_core_integer_gram_is_exact(A, case):
    """Bit-exact: the tcgen05 digit-product accumulation against integer arithmetic."""
    rng = np.random.default_rng(7)
    if case == "random":
        X = rng.integers(-(1 << 30), (1 << 30) + 1, size=(3000, 2, 64))
    elif case == "extreme":
        base = (63 << 24) + (127 << 16) + (128 << 8) - 128   # digits (63, 127, 128, -128)
        X = np.where(rng.random((2048, 2, 64)) < 0.5, base, -base)
    else:
        X = rng.integers(-(1 << 30), (1 << 30) + 1, size=(5, 2, 64))
    X = X.astype(np.int32)
    Gk = A.gram_selftest(X)
    Gr = _gram_int_reference(X.astype(np.int64))
    bad = np.argwhere(Gk != Gr)
    print("%s: %d of 4096 entries differ; max |diff| %s" % (
        case, len(bad), np.max(np.abs(Gk - Gr)) if len(bad) else 0))
    assert np.array_equal(Gk, Gr)


def _uv(c):
    u = np.empty(2 * len(c)); u[0::2] = c.real; u[1::2] = -c.imag
    v = np.empty(2 * len(c)); v[0::2] = c.imag; v[1::2] = c.real
    return u, v


@pytest.mark.parametrize("name,n_mc", [("tiny", 100_003), ("kstar10", 65_536), ("kstar10_z", 123_457),
                                       ("kstar10_z", 7), ("tiny", 1), ("lass", 65_536)])
def test_gram_matches_oracle(A, name, n_mc):
    cfg = W.CONFIGS[name]
    res = cfg.resonances
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c)
    nm = W.uniform_points(n_mc, cfg.norm_seed)
    gm = A.Model(res, path=A.AMP4D_PATH_CACHED)
    gm.set_events(*_dev(W.peaked_points(100, 1, res)))
    gm.set_norm_points(*_dev(nm))
    gm.build_gram(p)
    G = gm.get_gram()
    om = O.Model(res)
    Go = om.gram(p, nm)
    scale = np.max(np.abs(Go))
    print("%s n=%d: max |dG|/max|G| = %.3e" % (name, n_mc, np.max(np.abs(G - Go)) / scale))
    assert np.max(np.abs(G - Go)) <= 1e-6 * scale
    print("   asymmetry max |G - G^T| / max|G| = %.3e" % (np.max(np.abs(G - G.T)) / scale))
    u, v = _uv(c)
    I_g = W.BOX_VOLUME / n_mc * (u @ G @ u + v @ G @ v)
    I_o = om.norm(p, nm)
    # FP32 basis values: ~1e-8 weighted offset against FP64 (large n), ~1e-7 per point (tiny n)
    assert I_g == pytest.approx(I_o, rel=3e-8 if n_mc > 1000 else 1e-6)
    # same FP32 basis values, summed through the densities: isolates the digit accumulation
    S = gm.eval_density(p, 1).cpu().numpy().astype(np.float64)
    _, pq = om.density(p, nm)
    w = pq.astype(np.float32).astype(np.float64)
    I_s = W.BOX_VOLUME / n_mc * np.sum(w * S)
    print("   I_gram/I_oracle - 1 = %.3e   I_gram/I_gpu_points - 1 = %.3e" % (I_g / I_o - 1, I_g / I_s - 1))
    assert I_g == pytest.approx(I_s, rel=5e-9 if n_mc > 1000 else 1e-6)
    gm.build_gram(p)
    assert np.array_equal(gm.get_gram(), G)  # deterministic


@pytest.mark.parametrize("name", ["tiny", "kstar10", "kstar10_z", "kstar10_2z", "lass", "lass_z"])
def test_cached_path_nll_grad(A, name):
    cfg = W.CONFIGS[name]
    res = cfg.resonances
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c)
    om = O.Model(res)
    ev, _, _ = om.generate(p, 20_000, cfg.data_seed)
    nm = W.uniform_points(300_001, cfg.norm_seed)
    gm = A.Model(res, path=A.AMP4D_PATH_CACHED)
    gm.set_events(*_dev(ev))
    gm.set_norm_points(*_dev(nm))
    nll_o, g_o, aux, _ = om.nll(p, ev, nm, grad=True)
    nll, g = gm.eval_nll_grad(p)
    t = gm.eval_terms(p)
    print("%s cached: dNLL %.3e dI/I %.3e max|dg|/|g|inf %.3e" % (
        name, nll - nll_o, t[2] / aux[2] - 1, np.max(np.abs(g - g_o)) / np.max(np.abs(g_o))))
    assert abs(nll - nll_o) < 1e-3
    assert t[2] == pytest.approx(aux[2], rel=1e-8)
    tol = np.maximum(1e-6 * np.abs(g_o), GRAD_TOL * np.max(np.abs(g_o)))
    assert np.all(np.abs(g - g_o) <= tol)
    # a second parameter point reuses the same Gram
    p2 = p.copy()
    p2[2:] *= 1.01
    nll2, g2 = gm.eval_nll_grad(p2)
    nll2_o, g2_o, _, _ = om.nll(p2, ev, nm, grad=True)
    assert abs(nll2 - nll2_o) < 1e-3
    # the NLL-only and NLL+gradient kernels sum in different orders (FP32 per-thread sums)
    assert gm.eval_nll(p2) == pytest.approx(nll2, abs=1e-5)


def test_cached_path_with_floating_mass_uses_points(A):
    """With a floated mass the Gram cannot be reused; the cached-path model then
    evaluates the normalisation per point and still matches the oracle."""
    cfg = W.CONFIGS["tiny"]
    res = cfg.resonances
    c = W.draw_couplings(res, cfg.coupling_seed)
    fl = ["K*(892)"]
    p = W.couplings_to_params(c, W.float_mg_values(res, fl))
    ev = W.peaked_points(5_000, 3, res)
    nm = W.uniform_points(20_000, 4)
    gm = A.Model(res, float_names=fl, path=A.AMP4D_PATH_CACHED)
    gm.set_events(*_dev(ev))
    gm.set_norm_points(*_dev(nm))
    om = O.Model(res, float_names=fl)
    nll_o, g_o, _, _ = om.nll(p, ev, nm, grad=True)
    nll, g = gm.eval_nll_grad(p)
    assert abs(nll - nll_o) < 1e-3
    assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))


def test_basis_cache_reproduces_recompute_bit_for_bit(A):
    """The per-event basis cache holds the same lineshape values the plain path
    computes, so the cached path's densities equal the plain path's exactly.  With a
    floated Z mass and width (per-point normalisation) the cached path runs the
    two-events-per-thread kernel with the Z lineshape computed per event: its NLL
    and gradient, summed in another order, agree to rounding (NLL 1e-9 relative,
    gradient 1e-6 of |g|_inf), at the start point and after the Z mass moves."""
    cfg = W.CONFIGS["kstar10_z"]
    res = cfg.resonances
    fl = ["Z(4430)"]
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c, W.float_mg_values(res, fl))
    ev = W.peaked_points(30_001, 8, res)
    nm = W.uniform_points(60_003, 9)
    models = []
    for path in (A.AMP4D_PATH_PLAIN, A.AMP4D_PATH_CACHED):
        gm = A.Model(res, float_names=fl, path=path)
        gm.set_events(*_dev(ev))
        gm.set_norm_points(*_dev(nm))
        models.append(gm)
    def close(a, b):
        assert abs(a[0] - b[0]) <= 1e-9 * abs(a[0])
        assert np.max(np.abs(a[1] - b[1])) <= 1e-6 * np.max(np.abs(a[1]))
    r_plain = models[0].eval_nll_grad(p)
    r_cached = models[1].eval_nll_grad(p)          # builds the caches
    close(r_plain, r_cached)
    p2 = p.copy()
    p2[-2] += 0.01                                  # Z mass moves: computed on the fly
    close(models[0].eval_nll_grad(p2), models[1].eval_nll_grad(p2))
    S0 = models[0].eval_density(p2, 0).cpu().numpy()
    S1 = models[1].eval_density(p2, 0).cpu().numpy()
    assert np.array_equal(S0, S1)


@pytest.mark.parametrize("name", ["tiny", "kstar10", "kstar10_z", "kstar10_2z", "lass"])
def test_fit_fractions_match_oracle(A, name):
    """Eq. 13 from the tensor-core Gram matrix against the oracle's definition
    (normalisation integrals with the other couplings zeroed) on the same points;
    with floated masses the Gram is built at the given masses and widths."""
    cfg = W.CONFIGS[name]
    res = cfg.resonances
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c, W.float_mg_values(res, cfg.float_mg))
    nm = W.uniform_points(65_537, 23)
    gm = A.Model(res, float_names=cfg.float_mg, path=A.AMP4D_PATH_CACHED)
    gm.set_events(*_dev(W.uniform_points(1000, 24)))
    gm.set_norm_points(*_dev(nm))
    ff = gm.fit_fractions(p)
    ff_o = O.Model(res, float_names=cfg.float_mg).fit_fractions(p, nm)
    print(name, "fit fractions", np.round(ff, 4), "sum", ff.sum())
    assert np.allclose(ff, ff_o, rtol=1e-7, atol=1e-10)


@pytest.mark.parametrize("name", ["large_float_z", "kstar10_2z", "large_float_kz"])
def test_cached_path_floated_z_matches_oracle(A, name):
    """Fixed lineshapes from the basis cache and some masses and widths floating
    (the Z; or K*(892) and the Z): the all-cached kernel computes the floated
    lineshapes and their mass/width adjoint per event, for the data and the
    per-point normalisation.  NLL and full gradient (couplings, masses and
    widths) against the oracle, at the start point and after the floated masses
    move."""
    cfg = W.CONFIGS[name]
    res = cfg.resonances
    fl = cfg.float_mg
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c, W.float_mg_values(res, fl))
    ev = W.peaked_points(30_001, 5, res)
    nm = W.uniform_points(60_003, 6)
    gm = A.Model(res, float_names=fl, path=A.AMP4D_PATH_CACHED)
    gm.set_events(*_dev(ev))
    gm.set_norm_points(*_dev(nm))
    om = O.Model(res, float_names=fl)
    nz = 2 * len(fl)
    for shift in (0.0, 0.02):
        pp = p.copy()
        pp[-nz::2] += shift            # every floated mass
        nll_o, g_o, _, rc = om.nll(pp, ev, nm, grad=True)
        assert rc == 0
        nll, g = gm.eval_nll_grad(pp)
        assert abs(nll - nll_o) < 1e-4 + 1e-9 * abs(nll_o)
        assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))
        assert np.all(np.abs(g[-nz:] - g_o[-nz:]) <= 1e-5 * np.abs(g_o[-nz:]) + 1e-6 * np.max(np.abs(g_o)))
