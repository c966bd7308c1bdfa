"""The generator and the learned normalisation proposal on the GPU, against the
FP64 oracle: accept-reject events (same Philox candidates), MLP forward and
KL-objective gradient on identical BF16-rounded weights, the grid sampler on
given cell values, and what the trained proposal gains over uniform points."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2007_14931_gb300 as A
    return A


def _bf16(x):
    """Round float32 values to BF16 (nearest even) and back, as __float2bfloat16_rn does."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _theta(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return (rng.normal(scale=scale, size=4545)).astype(np.float32)


def test_generator_matches_oracle_generator(A):
    cfg = W.CONFIGS["tiny"]
    res = cfg.resonances
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed))
    gm = A.Model(res)
    n = 20_000
    ev = [t.cpu().numpy() for t in gm.generate(p, n, 99)]
    om = O.Model(res)
    evo, used, fmax = om.generate(p, n, 99, n_scan=1 << 20)
    a = set(zip(*(e.tolist() for e in ev)))
    b = set(zip(*(e.tolist() for e in evo)))
    common = len(a & b) / n
    print("generator: %.5f of events shared with the oracle's draw" % common)
    assert common > 0.998


def test_generator_follows_the_model(A):
    """GPU accept-reject events of the ten-K* model: their m_Kpi histogram against
    the model's 1D density p q int S dOmega / I, from the exact angular closure and
    adaptive quadrature in m (chi^2 per bin near 1)."""
    from scipy import integrate
    from test_oracle_pins import M_END, _kstar_angular_closed_form, _norm_1d
    cfg = W.CONFIGS["kstar10"]
    res = cfg.resonances
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c)
    mo = O.Model(res)
    gm = A.Model(res)
    m = gm.generate(p, 200_000, 5)[0].cpu().numpy().astype(np.float64)
    I1 = _norm_1d(mo, c)

    def dens(x):
        return O.breakup(W.M_B, x, W.M_PSI) * O.breakup(x, W.M_K, W.M_PI) * \
            _kstar_angular_closed_form(mo, c, x) / I1

    edges = np.linspace(W.M_LO, M_END, 61)
    h, _ = np.histogram(m, edges)
    exp = len(m) * np.array([integrate.quad(dens, a, b, epsrel=1e-10)[0]
                             for a, b in zip(edges[:-1], edges[1:])])
    keep = exp > 10
    chi2 = np.sum((h[keep] - exp[keep]) ** 2 / exp[keep])
    print("generator m_Kpi: chi2 %.1f for %d bins" % (chi2, keep.sum()))
    assert abs(exp.sum() / len(m) - 1) < 1e-6
    assert chi2 / keep.sum() < 1.6


@pytest.mark.parametrize("n", [1, 127, 4099])
def test_mlp_forward_parity(A, n):
    th = _theta(1)
    x = np.random.default_rng(2).uniform(-1, 1, (n, 4)).astype(np.float32)
    g = A.mlp_forward(th, torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    go = O.mlp_forward(_bf16(th).astype(np.float64), x.astype(np.float64))
    assert np.max(np.abs(g / go - 1)) < 1e-5


def test_mlp_loss_grad_parity(A):
    th = _theta(3)
    rng = np.random.default_rng(4)
    xd = rng.uniform(-1, 1, (300, 4)).astype(np.float32)
    xu = rng.uniform(-1, 1, (517, 4)).astype(np.float32)
    loss, g = A.mlp_loss_grad(th, torch.from_numpy(xd).cuda(), torch.from_numpy(xu).cuda())
    lo, go = O.mlp_loss_grad(_bf16(th).astype(np.float64), xd.astype(np.float64), xu.astype(np.float64))
    assert loss == pytest.approx(lo, rel=1e-6, abs=1e-6)
    assert np.max(np.abs(g - go)) <= 1e-4 * np.max(np.abs(go))


def test_grid_sample_parity(A):
    nb = (16, 4, 4, 8)
    gc = np.random.default_rng(5).uniform(0, 1, np.prod(nb)).astype(np.float32) ** 2
    (m, cK, cpsi, phi), w, cell = A.grid_sample(gc, nb, 0.1, 17, 10_001)
    (mo, cKo, cpsio, phio), wo, cello = O.grid_sample(gc.astype(np.float64), nb, 0.1, 17, 10_001)
    cell = cell.cpu().numpy()
    same = cell == cello
    assert same.mean() > 0.9995
    for a, b in ((m, mo), (cK, cKo), (cpsi, cpsio), (phi, phio)):
        a = a.cpu().numpy()
        assert np.all(np.abs(a[same] - b[same]) <= 2 * np.spacing(np.abs(b[same])))
    assert np.allclose(w.cpu().numpy()[same], wo[same], rtol=2e-6)


def test_learned_proposal_meets_the_integral_target(A):
    """The learned normalisation (C4): the proposal trained on 2^20 events the GPU
    generator draws from the 10 K* + Z model; 16 independent samples of 2^20
    importance-sampled points and 16 of 2^24 uniform points, each judged against
    the oracle's 4D product quadrature of I (accurate to about 1e-8).  Target:
    rms relative error <= 1e-4 for the learned estimate, which must also beat
    the uniform one with 16 times fewer points, and no bias beyond its spread."""
    from oracle import quadrature as Q
    cfg = W.CONFIGS["learned"]
    res = cfg.resonances
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c)
    I_q = Q.normalisation_quadrature(O.Model(res), p, 24, 16)
    gm = A.Model(res)
    ev = gm.generate(p, 1 << 20, 3)
    gm.set_events(*ev)
    loss = gm.proposal_train(ev, seed=11)
    one = np.ones(1, dtype=np.float32)
    I_is, I_un = [], []
    for s in range(16):
        pts, w = gm.proposal_sample(1 << 20, 100 + s)
        gm.set_norm_points(*pts, w=w, volume=1.0)
        I_is.append(gm.eval_terms(p)[2])
        pts, w, _ = A.grid_sample(one, (1, 1, 1, 1), 1.0, 500 + s, 1 << 24)   # uniform, w = V p q
        gm.set_norm_points(*pts, w=w, volume=1.0)
        I_un.append(gm.eval_terms(p)[2])
    r_is, r_un = np.array(I_is) / I_q - 1, np.array(I_un) / I_q - 1
    rms_is, rms_un = np.sqrt(np.mean(r_is ** 2)), np.sqrt(np.mean(r_un ** 2))
    print("loss %.4f  rms relative error vs the quadrature: learned 2^20 %.3e (mean %+.2e), "
          "uniform 2^24 %.3e (mean %+.2e); variance reduction per point %.0f" % (
              loss, rms_is, r_is.mean(), rms_un, r_un.mean(), 16 * (rms_un / rms_is) ** 2))
    assert rms_is <= 1e-4
    assert rms_is < rms_un
    assert abs(r_is.mean()) < 4 * r_is.std(ddof=1) / 4.0 + 1e-6


def test_gram_targeted_proposal_is_unbiased_for_every_column(A):
    """The proposal trained on sum_k |B_k|^2 p q: its importance-sampled points
    give each Gram diagonal element (the normalisation of one column alone)
    within Monte Carlo error of the uniform-point value."""
    cfg = W.CONFIGS["kstar10_z"]
    res = cfg.resonances
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed))
    m = A.Model(res, path=A.AMP4D_PATH_CACHED)
    m.set_norm_points(*(torch.from_numpy(a).cuda() for a in W.uniform_points(1 << 22, 31)))
    m.set_events(*(torch.from_numpy(a).cuda() for a in W.uniform_points(1000, 32)))
    m.build_gram(p)
    G_ref = m.get_gram() * W.BOX_VOLUME / (1 << 22)
    m.proposal_train_gram(p, n=1 << 19, seed=3)
    K = m.n_cols
    diag = []
    for sd in range(4):
        pts, w = m.proposal_sample(1 << 20, 40 + sd)
        m.set_norm_points(*pts, w=w, volume=1.0)
        m.build_gram(p)
        G = m.get_gram() / (1 << 20)
        diag.append([G[2 * k, 2 * k] + G[2 * k + 1, 2 * k + 1] for k in range(K)])
    diag = np.array(diag)
    ref = np.array([G_ref[2 * k, 2 * k] + G_ref[2 * k + 1, 2 * k + 1] for k in range(K)])
    mean, sem = diag.mean(0), diag.std(0, ddof=1) / 2.0
    # unbiased within 5 standard errors of the seed spread plus the reference's
    # own Monte Carlo error (about 1e-3 relative for 2^22 uniform points)
    assert np.all(np.abs(mean - ref) <= 5 * sem + 3e-3 * ref), np.max(np.abs(mean / ref - 1))
