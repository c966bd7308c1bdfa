"""Synchronous evaluations replayed as CUDA graphs.

From the second call at one model state, amp4d_eval_nll_grad / amp4d_eval_nll
replay a captured graph of the parameter copy, the evaluation's launches and the
result copy.  The kernels' sums are exact 128-bit fixed-point accumulations of
per-CTA values in a fixed order, so a replay must return the first (direct)
call's bits; after a call that changes the model's state (new points, new
events, flavour tags) the results must equal those of a model built from
scratch in that state."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2007_14931_gb300 as A
    return A


def _dev(pts):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in pts]


def _model(A, res, path, ev, nm, tag=None, mistag=0.0):
    m = A.Model(res, path=path)
    m.set_events(*_dev(ev))
    m.set_norm_points(*_dev(nm))
    if tag is not None:
        m.set_flavour(tag, mistag)
    return m


@pytest.mark.parametrize("path", ["cached", "plain"])
def test_replayed_evaluations_return_the_direct_results(A, path):
    cfg = W.CONFIGS["kstar10_z"]
    res = cfg.resonances
    p = W.couplings_to_params(W.draw_couplings(res, cfg.coupling_seed))
    p2 = p.copy()
    p2[2:] *= 1.01
    ev = W.peaked_points(30_001, 11, res)
    nm = W.uniform_points(65_536, 12)
    pth = A.AMP4D_PATH_CACHED if path == "cached" else A.AMP4D_PATH_PLAIN
    m = _model(A, res, pth, ev, nm)
    first = [m.eval_nll_grad(q) for q in (p, p2)]          # direct, then captured
    again = [m.eval_nll_grad(q) for q in (p, p2, p)]        # replays
    for (f, g), (f2, g2) in zip(first + first[:1], again):
        assert f2 == f
        assert np.array_equal(g2, g)
    n1 = m.eval_nll(p)
    assert m.eval_nll(p) == n1 and m.eval_nll(p) == n1

    # state changes between replays: new points, new events, flavour tags
    nm_b = W.uniform_points(40_000, 13)
    m.set_norm_points(*_dev(nm_b))
    ref = _model(A, res, pth, ev, nm_b)
    for q in (p, p2, p):
        f, g = m.eval_nll_grad(q)
        fr, gr = ref.eval_nll_grad(q)
        assert f == fr and np.array_equal(g, gr)
    ref.close()
    ev_b = W.peaked_points(20_000, 14, res)
    m.set_events(*_dev(ev_b))
    ref = _model(A, res, pth, ev_b, nm_b)
    for q in (p2, p, p2):
        f, g = m.eval_nll_grad(q)
        fr, gr = ref.eval_nll_grad(q)
        assert f == fr and np.array_equal(g, gr)
        assert m.eval_nll(q) == ref.eval_nll(q)
    ref.close()
    tag = np.where(np.random.default_rng(15).random(len(ev_b[0])) < 0.5, 1.0, -1.0).astype(np.float32)
    m.set_flavour(tag, 0.05)
    ref = _model(A, res, pth, ev_b, nm_b, tag, 0.05)
    for q in (p, p, p2):
        f, g = m.eval_nll_grad(q)
        fr, gr = ref.eval_nll_grad(q)
        assert f == fr and np.array_equal(g, gr)
    ref.close()
    m.close()


def test_default_stream_is_torchs_current_stream(A):
    """The binding's stream for stream=None is torch's current stream, also inside
    a torch.cuda.stream context."""
    assert A._stream_ptr(None) == torch.cuda.current_stream().cuda_stream
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert A._stream_ptr(None) == s.cuda_stream == torch.cuda.current_stream().cuda_stream
    assert A._stream_ptr(None) == torch.cuda.current_stream().cuda_stream
