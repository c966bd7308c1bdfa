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
    """Mean of cos^2 theta_psi and of m over generated events vs the oracle's draw (statistics)."""
    cfg = W.CONFIGS["kstar10_z"]
    res = cfg.resonances
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed))
    gm = A.Model(res)
    ev = [t.cpu().numpy().astype(np.float64) for t in gm.generate(p, 50_000, 5)]
    S, pq = O.Model(res).density(p, ev)
    assert np.all(S * pq > 0)


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


def test_learned_proposal_reduces_normalisation_variance(A):
    """C4-like: train the proposal on 2^20 events generated from the 10 K* + Z model;
    2^20 importance-sampled points vs 2^24 uniform points, 8 seeds each, judged by
    the FP64 oracle on 2^26 uniform points."""
    cfg = W.CONFIGS["learned"]
    res = cfg.resonances
    c = W.draw_couplings(res, cfg.coupling_seed)
    p = W.couplings_to_params(c)
    gm = A.Model(res)
    ev = gm.generate(p, 1 << 20, 3)
    gm.set_events(*ev)
    loss = gm.proposal_train(ev, steps=1500, batch=4096, seed=11)
    I_is, I_un = [], []
    for s in range(8):
        pts, w = gm.proposal_sample(1 << 20, 100 + s)
        gm.set_norm_points(*pts, w=w, volume=1.0)
        I_is.append(gm.eval_terms(p)[2])
        un = W.uniform_points(1 << 24, 500 + s)
        gm.set_norm_points(*(torch.from_numpy(a).cuda() for a in un))
        I_un.append(gm.eval_terms(p)[2])
    judge_pts = W.uniform_points(1 << 26, 777)
    S, pq = O.Model(res).density(p, judge_pts)
    f = W.BOX_VOLUME * S * pq
    I_ref, sig_ref = f.mean(), f.std() / math.sqrt(len(f))
    I_is, I_un = np.array(I_is), np.array(I_un)
    rms_is = np.sqrt(np.mean((I_is / I_ref - 1) ** 2))
    rms_un = np.sqrt(np.mean((I_un / I_ref - 1) ** 2))
    sd_is, sd_un = I_is.std(ddof=1) / I_ref, I_un.std(ddof=1) / I_ref
    print("loss %.4f  rms rel error vs judge: learned 2^20 %.3e, uniform 2^24 %.3e (judge sigma %.1e); "
          "seed spread: learned %.3e, uniform %.3e; variance reduction per point %.1f" % (
              loss, rms_is, rms_un, sig_ref / I_ref, sd_is, sd_un, 16 * (sd_un / sd_is) ** 2))
    assert abs(I_is.mean() / I_ref - 1) < 4 * max(I_is.std() / math.sqrt(8), sig_ref) / I_ref + 1e-4
    assert rms_is < rms_un * 1.2


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
