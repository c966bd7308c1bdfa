"""Pins of the oracle's learned-proposal pieces: the MLP density (closed-form
special cases, finite-difference gradient of the KL objective), Adam (closed-form
first steps), and the grid proposal sampler (uniform limit, cell frequencies,
unbiased importance-sampling estimate of a known integral)."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O
import workloads as W

NP = 4545
H = 64


def _split(th):
    W1 = th[:256].reshape(64, 4)
    b1 = th[256:320]
    W2 = th[320:320 + 4096].reshape(64, 64)
    b2 = th[4416:4480]
    W3 = th[4480:4544]
    b3 = th[4544:4545]
    return W1, b1, W2, b2, W3, b3


def _softplus(o):
    return np.log1p(np.exp(o))


def test_num_params():
    assert O.mlp_num_params() == NP


def test_mlp_forward_special_cases():
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, (50, 4))
    th = np.zeros(NP)
    th[-1] = 0.37                                   # only b3: g = softplus(b3)
    assert np.allclose(O.mlp_forward(th, x), _softplus(0.37), rtol=1e-15)
    th = np.zeros(NP)
    W1, b1, W2, b2, W3, b3 = _split(th)
    b2[:] = rng.normal(size=64)                     # W2 = 0: h2 = tanh(b2)
    W3[:] = rng.normal(size=64)
    b3[0] = -0.2
    ref = _softplus(W3 @ np.tanh(b2) - 0.2)
    assert np.allclose(O.mlp_forward(th, x), ref, rtol=1e-14)
    th = np.zeros(NP)
    W1, b1, W2, b2, W3, b3 = _split(th)
    W1[0, 0] = 1.7                                  # g = softplus(tanh(tanh(1.7 x0)))
    W2[0, 0] = 1.0
    W3[0] = 1.0
    assert np.allclose(O.mlp_forward(th, x), _softplus(np.tanh(np.tanh(1.7 * x[:, 0]))), rtol=1e-14)


def test_mlp_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    th = rng.normal(scale=0.3, size=NP)
    xd = rng.uniform(-1, 1, (40, 4))
    xu = rng.uniform(-1, 1, (60, 4))
    loss, g = O.mlp_loss_grad(th, xd, xu)
    # loss itself from the forward
    gd, gu = O.mlp_forward(th, xd), O.mlp_forward(th, xu)
    assert loss == pytest.approx(-np.mean(np.log(gd)) + math.log(16 * np.mean(gu)), rel=1e-13)
    idx = list(rng.choice(NP, 60, replace=False)) + [0, 255, 256, 319, 320, 4415, 4416, 4479, 4480, 4543, 4544]
    h = 1e-6
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (O.mlp_loss_grad(tp, xd, xu)[0] - O.mlp_loss_grad(tm, xd, xu)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-6, abs=1e-9), i


def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(2)
    th = rng.normal(size=100)
    g = rng.normal(size=100)
    m, v = np.zeros(100), np.zeros(100)
    t0 = th.copy()
    O.adam_step(th, m, v, g, 1, lr=1e-2)
    # bias-corrected moments at t = 1 are g and g^2: step = lr g / (|g| + eps)
    assert np.allclose(th, t0 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=1e-16)
    t1 = th.copy()
    O.adam_step(th, m, v, g, 2, lr=1e-2)
    assert np.allclose(th, t1 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_grid_sampler_uniform_limit():
    """alpha = 1: the proposal is uniform and w = V p q exactly."""
    nb = (8, 4, 4, 8)
    gc = np.random.default_rng(3).uniform(0, 1, np.prod(nb))
    (m, cK, cpsi, phi), w, cell = O.grid_sample(gc, nb, 1.0, 11, 2000)
    pq = np.array([O.breakup(W.M_B, x, W.M_PSI) * O.breakup(x, W.M_K, W.M_PI) for x in m])
    assert np.allclose(w, W.BOX_VOLUME * pq, rtol=1e-12)
    assert np.all((m >= W.M_LO) & (m <= W.M_HI)) and np.all(np.abs(cK) <= 1) and np.all(np.abs(phi) <= 3.1415927)


def test_grid_sampler_cell_frequencies():
    nb = (4, 2, 2, 4)
    rng = np.random.default_rng(4)
    gc = rng.uniform(0, 1, 64) ** 3
    alpha = 0.2
    n = 200_000
    _, _, cell = O.grid_sample(gc, nb, alpha, 5, n)
    P = alpha / 64 + (1 - alpha) * gc / gc.sum()
    counts = np.bincount(cell, minlength=64)
    # stratified in the CDF: cell c receives the points whose strata [i/n, (i+1)/n)
    # of the total put u in its CDF interval, n P_c of them up to one at each end
    assert np.all(np.abs(counts - n * P) < 2.0)
    # the sampled position lies in the sampled cell
    (m, cK, cpsi, phi), _, cell = O.grid_sample(gc, nb, alpha, 6, 1000)
    x0 = 2 * (m.astype(np.float64) - W.M_LO) / (W.M_HI - W.M_LO) - 1
    i0 = np.minimum((0.5 * (x0 + 1) * nb[0]).astype(int), nb[0] - 1)
    assert np.mean(i0 == cell // (nb[1] * nb[2] * nb[3])) > 0.999


def test_grid_sampler_points_are_marginally_drawn_from_the_proposal():
    """Over independent seeds the cell of point i follows the proposal's cell
    probabilities restricted to its stratum: pooled over the points of many calls
    of a few points each, the cell frequencies are multinomial in P."""
    nb = (4, 2, 2, 4)
    rng = np.random.default_rng(14)
    gc = rng.uniform(0, 1, 64) ** 3
    alpha = 0.2
    P = alpha / 64 + (1 - alpha) * gc / gc.sum()
    cells = np.concatenate([O.grid_sample(gc, nb, alpha, 1000 + s, 1)[2] for s in range(20_000)])
    counts = np.bincount(cells, minlength=64)
    chi2 = np.sum((counts - len(cells) * P) ** 2 / (len(cells) * P))
    assert stats.chi2.sf(chi2, 63) > 1e-3


def test_grid_sampler_is_unbiased_for_the_phase_space_volume():
    """E_q[w] = int p q dPhi = 8 pi int p q dm (importance sampling identity)."""
    nb = (16, 2, 2, 2)
    gc = np.random.default_rng(5).uniform(0.1, 1, np.prod(nb))
    _, w, _ = O.grid_sample(gc, nb, 0.1, 7, 400_000)
    f = lambda x: O.breakup(W.M_B, x, W.M_PSI) * O.breakup(x, W.M_K, W.M_PI)
    ref = 8 * math.pi * integrate.quad(f, W.M_LO, W.M_B - W.M_PSI, epsrel=1e-12, limit=200)[0]
    assert abs(w.mean() - ref) < 4 * w.std() / math.sqrt(len(w))
