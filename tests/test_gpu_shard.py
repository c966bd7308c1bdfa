"""Sharded evaluation on one GPU: the events and points of one fit split into
contiguous shards, one model per shard (as one model per GPU would hold them),
each shard's partial sums through amp4d_eval_partials / amp4d_enqueue_partials,
and the union rebuilt by amp4d_combine_partials.

Checked against the FP64 oracle's partials of the same shards and its -2 ln L
of the union, with the tolerances of the single-model parity tests (NLL
|dNLL| < 1e-3, gradient <= 1e-6 |g|_inf, I relative 1e-8, sum ln S absolute
5e-4 per shard), and against the single-model GPU evaluation of the union."""
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


def _cut(arrs, lo, hi):
    return tuple(a[lo:hi] for a in arrs)


def _workload(name, n_ev, n_mc):
    cfg = W.CONFIGS[name]
    res = cfg.resonances
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed),
                              W.float_mg_values(res, cfg.float_mg))
    ev = W.peaked_points(n_ev, cfg.data_seed, res)
    nm = W.uniform_points(n_mc, cfg.norm_seed)
    return cfg, res, p, ev, nm


def _shard_models(A, cfg, res, ev, nm, world, path):
    from paper_2007_14931_gb300.shard import shard_range
    models, cuts = [], []
    for r in range(world):
        a, b = shard_range(len(ev[0]), r, world)
        c, d = shard_range(len(nm[0]), r, world)
        m = A.Model(res, float_names=cfg.float_mg, path=path)
        m.set_events(*_dev(_cut(ev, a, b)))
        m.set_norm_points(*_dev(_cut(nm, c, d)))
        models.append(m)
        cuts.append(((a, b), (c, d)))
    return models, cuts


@pytest.mark.parametrize("name,world", [("tiny", 3), ("kstar10_z", 2), ("kstar10_z", 5)])
def test_shards_match_oracle_and_union(A, name, world):
    n_ev, n_mc = 100_003, 200_001  # ragged shard sizes
    cfg, res, p, ev, nm = _workload(name, n_ev, n_mc)
    om = O.Model(res, float_names=cfg.float_mg)
    models, cuts = _shard_models(A, cfg, res, ev, nm, world, A.AMP4D_PATH_PLAIN)
    P = models[0].n_params
    parts = np.stack([m.eval_partials(p) for m in models])
    for part, ((a, b), (c, d)) in zip(parts, cuts):
        o = om.partials(p, _cut(ev, a, b), _cut(nm, c, d))
        assert part[2] == b - a and part[4] == d - c and part[5] == 0
        assert abs(part[0] - o[0]) < 5e-4
        assert part[1] == pytest.approx(o[1], abs=1e-9 * abs(o[1]) + 1e-9)
        assert part[3] == pytest.approx(o[3], rel=1e-8)
    nll, g, out = A.combine_partials(parts)
    nll_o, g_o, aux, rc = om.nll(p, ev, nm, grad=True)
    assert rc == 0
    assert abs(nll - nll_o) < 1e-3
    assert out[3] == pytest.approx(aux[2], rel=1e-8)
    assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))
    # the union on one model: the same sums in another order
    whole = A.Model(res, float_names=cfg.float_mg)
    whole.set_events(*_dev(ev))
    whole.set_norm_points(*_dev(nm))
    nll_w, g_w = whole.eval_nll_grad(p)
    assert abs(nll - nll_w) < 1e-3
    assert np.max(np.abs(g - g_w)) <= GRAD_TOL * np.max(np.abs(g_w))
    assert parts.shape == (world, 6 + 2 * P)


def test_shards_on_the_gram_path(A):
    """Cached path: each shard builds its own normalisation Gram matrix."""
    cfg = W.CONFIGS["kstar10"]
    _, res, p, ev, nm = _workload("kstar10", 60_000, 2 * 65_536 + 77)
    models, cuts = _shard_models(A, cfg, res, ev, nm, 3, A.AMP4D_PATH_CACHED)
    parts = np.stack([m.eval_partials(p) for m in models])
    nll, g, out = A.combine_partials(parts)
    om = O.Model(res, float_names=cfg.float_mg)
    nll_o, g_o, aux, rc = om.nll(p, ev, nm, grad=True)
    assert abs(nll - nll_o) < 1e-3
    assert out[3] == pytest.approx(aux[2], rel=1e-8)
    assert np.max(np.abs(g - g_o)) <= GRAD_TOL * np.max(np.abs(g_o))
    for part, ((a, b), (c, d)) in zip(parts, cuts):
        o = om.partials(p, _cut(ev, a, b), _cut(nm, c, d))
        assert part[3] == pytest.approx(o[3], rel=1e-8)
        P = len(g)
        dT, dT_o = part[6 + P:], o[6 + P:]
        assert np.max(np.abs(dT - dT_o)) <= 1e-7 * np.max(np.abs(dT_o))


def test_enqueue_partials_matches_host_call(A):
    cfg, res, p, ev, nm = _workload("kstar10_z", 20_001, 30_011)
    m = A.Model(res, float_names=cfg.float_mg)
    m.set_events(*_dev(ev))
    m.set_norm_points(*_dev(nm))
    host = m.eval_partials(p)
    nll_only = m.eval_partials(p, grad=False)
    p_dev = torch.from_numpy(np.asarray(p, dtype=np.float64)).cuda()
    out = torch.full((6 + 2 * m.n_params,), -7.0, dtype=torch.float64, device="cuda")
    m.enqueue_partials(A.AMP4D_EVAL_NLL_GRAD, p_dev, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), host)
    assert nll_only.shape == (6,)
    assert nll_only[2] == host[2] and nll_only[4] == host[4]
    assert abs(nll_only[0] - host[0]) < 1e-4  # NLL-only kernel sums in another order


def test_partials_report_domain_errors(A):
    """All couplings zero: S = 0 at every event; the shard says so (status bit 1)
    and the combination refuses it."""
    cfg, res, p, ev, nm = _workload("tiny", 4001, 4001)
    m = A.Model(res, float_names=cfg.float_mg)
    m.set_events(*_dev(ev))
    m.set_norm_points(*_dev(nm))
    z = np.zeros_like(p)
    part = m.eval_partials(z)
    assert int(part[5]) & 1
    with pytest.raises(A.Amp4dError) as e:
        A.combine_partials(part[None, :])
    assert e.value.code == A.AMP4D_ERR_DOMAIN
