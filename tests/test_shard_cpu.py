"""Sharded evaluation on the host (no GPU): the split of events and points over
ranks, the oracle's per-shard sums pinned to its own -2 ln L, the native
rank-ordered combination (amp4d_combine_partials), and two gloo ranks that
exchange their blocks with torch.distributed and agree bit for bit.

The likelihood of the unbinned fit (Introduction) is a product over events of
S p q / I (Eq. 5) and I is a sum over points, so a split of both sets changes
only the order of the sums."""
import os
import socket

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


@pytest.fixture(scope="module")
def A():
    import __graft_entry__ as G
    G._build_module().build()
    import paper_2007_14931_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def O():
    import oracle
    return oracle


def _shard_mod():
    from conftest import load_product_module
    return load_product_module("shard")


def _setup(n_ev=3000, n_mc=5000, name="tiny"):
    cfg = W.CONFIGS[name]
    res = cfg.resonances
    c = W.draw_couplings(res, cfg.coupling_seed)
    params = W.couplings_to_params(c, W.float_mg_values(res, cfg.float_mg))
    ev = W.peaked_points(n_ev, cfg.data_seed, res)
    nm = W.uniform_points(n_mc, cfg.norm_seed)
    return cfg, res, params, ev, nm


def _cut(arrs, lo, hi):
    return tuple(a[lo:hi] for a in arrs)


@pytest.mark.parametrize("n,world", [(0, 1), (1, 3), (7, 2), (10, 4), (1000, 8), (5, 5)])
def test_shard_range_covers_contiguously(n, world):
    S = _shard_mod()
    ranges = [S.shard_range(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0


def test_shard_range_rejects_bad_arguments():
    S = _shard_mod()
    for args in [(10, 2, 2), (10, -1, 2), (10, 0, 0), (-1, 0, 1)]:
        with pytest.raises(ValueError):
            S.shard_range(*args)


def test_oracle_partials_reproduce_oracle_nll(O):
    """One shard holding everything: I = T / M and -2 [sum ln S + sum ln pq - N ln I]
    must equal the oracle's -2 ln L, and the gradient -2 [d ln S - N dT / T] its
    gradient (or_nll goes through or_norm, a separate route)."""
    cfg, res, params, ev, nm = _setup(name="kstar10_z")
    om = O.Model(res, float_names=cfg.float_mg)
    nll, g, aux, rc = om.nll(params, ev, nm, grad=True)
    assert rc == 0
    p = om.partials(params, ev, nm, grad=True)
    P = om.n_params
    assert p[2] == len(ev[0]) and p[4] == len(nm[0]) and p[5] == 0
    I = p[3] / p[4]
    assert I == pytest.approx(aux[2], rel=1e-14)
    assert p[0] == pytest.approx(aux[0], rel=1e-14) and p[1] == pytest.approx(aux[1], rel=1e-14)
    nll_p = -2.0 * (p[0] + p[1] - p[2] * np.log(I))
    g_p = -2.0 * (p[6:6 + P] - p[2] * p[6 + P:] / p[3])
    assert nll_p == pytest.approx(nll, rel=1e-13)
    assert np.max(np.abs(g_p - g)) <= 1e-10 * np.max(np.abs(g))


def test_oracle_partials_are_additive_over_shards(O):
    cfg, res, params, ev, nm = _setup()
    om = O.Model(res, float_names=cfg.float_mg)
    full = om.partials(params, ev, nm)
    parts = [om.partials(params, _cut(ev, a, b), _cut(nm, c, d))
             for (a, b), (c, d) in [((0, 1000), (0, 10)), ((1000, 1000), (10, 4000)),
                                     ((1000, 3000), (4000, 5000))]]
    s = np.sum(parts, axis=0)
    assert np.allclose(s, full, rtol=1e-12, atol=1e-9 * np.max(np.abs(full)))


def test_combine_of_oracle_shards_equals_oracle_union(A, O):
    """Native combination of uneven shards (one without events, one without
    points) against the oracle's -2 ln L of the union."""
    cfg, res, params, ev, nm = _setup(name="kstar10_z")
    om = O.Model(res, float_names=cfg.float_mg)
    nll, g, aux, rc = om.nll(params, ev, nm, grad=True)
    cuts = [((0, 1200), (0, 0)), ((1200, 1200), (0, 3100)), ((1200, 3000), (3100, 5000))]
    parts = np.stack([om.partials(params, _cut(ev, a, b), _cut(nm, c, d))
                      for (a, b), (c, d) in cuts])
    nll_c, g_c, out = A.combine_partials(parts)
    assert nll_c == pytest.approx(nll, rel=1e-12)
    assert out[3] == pytest.approx(aux[2], rel=1e-13)
    assert out[4] == len(ev[0]) and out[5] == 0
    assert np.max(np.abs(g_c - g)) <= 1e-9 * np.max(np.abs(g))
    # NLL-only blocks give the same NLL
    nll_n, g_n, _ = A.combine_partials(parts[:, :6])
    assert g_n is None and nll_n == nll_c


def test_combine_is_deterministic_and_order_only_rounds(A, O):
    cfg, res, params, ev, nm = _setup()
    om = O.Model(res, float_names=cfg.float_mg)
    parts = np.stack([om.partials(params, _cut(ev, 1000 * r, 1000 * r + 1000),
                                  _cut(nm, 1250 * r, 1250 * r + 1250)) for r in range(3)] +
                     [om.partials(params, _cut(ev, 3000, 3000), _cut(nm, 3750, 5000))])
    a = A.combine_partials(parts)
    b = A.combine_partials(parts.copy())
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    c = A.combine_partials(parts[::-1].copy())
    assert c[0] == pytest.approx(a[0], rel=1e-14)
    assert np.allclose(c[1], a[1], rtol=1e-12, atol=1e-12 * np.max(np.abs(a[1])))


def test_combine_error_paths(A):
    P = 4
    ok = np.zeros((2, 6 + 2 * P))
    ok[:, 2] = 10.0
    ok[:, 3] = 5.0
    ok[:, 4] = 100.0
    nll, g, out = A.combine_partials(ok)
    assert np.isfinite(nll) and out[3] == pytest.approx(0.05)
    no_pts = ok.copy()
    no_pts[:, 4] = 0.0
    with pytest.raises(A.Amp4dError) as e:
        A.combine_partials(no_pts)
    assert e.value.code == A.AMP4D_ERR_STATE
    bad = ok.copy()
    bad[1, 5] = 1.0
    with pytest.raises(A.Amp4dError) as e:
        A.combine_partials(bad)
    assert e.value.code == A.AMP4D_ERR_DOMAIN
    inval = ok.copy()
    inval[0, 5] = 2.0
    with pytest.raises(A.Amp4dError) as e:
        A.combine_partials(inval)
    assert e.value.code == A.AMP4D_ERR_ARG
    neg = ok.copy()
    neg[0, 2] = -1.0
    with pytest.raises(A.Amp4dError) as e:
        A.combine_partials(neg)
    assert e.value.code == A.AMP4D_ERR_ARG
    zeroI = ok.copy()
    zeroI[:, 3] = 0.0
    with pytest.raises(A.Amp4dError) as e:
        A.combine_partials(zeroI)
    assert e.value.code == A.AMP4D_ERR_DOMAIN
    with pytest.raises(ValueError):
        A.combine_partials(np.zeros((2, 9)), what=A.AMP4D_EVAL_NLL_GRAD)


# ------------------------------------------------------------------ gloo ranks
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir, fail_rank):
    """One CPU rank: its contiguous shard of the events and points, the oracle's
    partials, the all-gather over gloo, the native combination."""
    import sys
    import datetime
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, os.path.join(root, "tests"))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import oracle
    import workloads as W
    import paper_2007_14931_gb300.shard as S
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    try:
        cfg = W.CONFIGS["kstar10_z"]
        res = cfg.resonances
        params = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed),
                                       W.float_mg_values(res, cfg.float_mg))
        ev = W.peaked_points(3000, cfg.data_seed, res)
        nm = W.uniform_points(5000, cfg.norm_seed)
        a, b = S.shard_range(len(ev[0]), rank, world)
        c, d = S.shard_range(len(nm[0]), rank, world)
        om = oracle.Model(res, float_names=cfg.float_mg)
        part = om.partials(params, tuple(x[a:b] for x in ev), tuple(x[c:d] for x in nm))
        if rank == fail_rank:
            raise RuntimeError("rank %d fails before the exchange" % rank)
        gathered = S.gather_partials(part)
        nll, g = S.combine_gathered(gathered)
        np.save(os.path.join(outdir, "r%d.npy" % rank), np.concatenate([[nll], g]))
    except RuntimeError as e:
        with open(os.path.join(outdir, "r%d.err" % rank), "w") as f:
            f.write(type(e).__name__ + ": " + str(e))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run_ranks(tmp_path, world, fail_rank=-1, timeout=180):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path), fail_rank))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
        p.join()
    assert not alive, "a rank did not finish"
    return procs


def test_two_gloo_ranks_agree_with_the_union(A, O, tmp_path):
    _run_ranks(tmp_path, 2)
    r = [np.load(tmp_path / ("r%d.npy" % k)) for k in range(2)]
    assert np.array_equal(r[0], r[1]), "ranks combined different bits"
    cfg = W.CONFIGS["kstar10_z"]
    res = cfg.resonances
    params = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed),
                                   W.float_mg_values(res, cfg.float_mg))
    ev = W.peaked_points(3000, cfg.data_seed, res)
    nm = W.uniform_points(5000, cfg.norm_seed)
    nll, g, aux, rc = O.Model(res, float_names=cfg.float_mg).nll(params, ev, nm, grad=True)
    assert r[0][0] == pytest.approx(nll, rel=1e-12)
    assert np.max(np.abs(r[0][1:] - g)) <= 1e-9 * np.max(np.abs(g))


def test_a_failing_rank_ends_the_exchange_with_an_error(A, tmp_path):
    """Rank 1 raises before the all-gather and leaves; rank 0 must get an error
    from the collective (closed connection or the 20 s process-group timeout),
    not hang."""
    _run_ranks(tmp_path, 2, fail_rank=1)
    assert (tmp_path / "r1.err").exists()
    assert not (tmp_path / "r0.npy").exists()
    assert (tmp_path / "r0.err").exists(), "rank 0 neither failed nor finished"
