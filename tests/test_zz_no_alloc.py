"""The allocation-free proposal-gradient entry point, called through the C ABI.

Callers that may not allocate device memory (a component whose memory budget is
owned by another pool, or code that must avoid the synchronisation an
allocation can cause) use amp4d_mlp_loss_grad_noalloc, whose scratch is a
static device array.  It must give the same result as the allocating entry
point, on consecutive calls that reuse that array, and reject sizes beyond
its limit before touching the GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2007_14931_gb300 as A
    return A


def _inputs(seed, nd, nu):
    rng = np.random.default_rng(seed)
    th = rng.normal(scale=0.3, size=4545).astype(np.float32)
    xd = torch.from_numpy(rng.uniform(-1, 1, (nd, 4)).astype(np.float32)).cuda()
    xu = torch.from_numpy(rng.uniform(-1, 1, (nu, 4)).astype(np.float32)).cuda()
    return th, xd, xu


def test_noalloc_matches_allocating_entry_on_consecutive_calls(A):
    for seed, nd, nu in [(1, 300, 517), (2, 4096, 4096), (3, 1, 129)]:
        th, xd, xu = _inputs(seed, nd, nu)
        ref_loss, ref_grad = A.mlp_loss_grad(th, xd, xu)
        out = torch.full((4546,), float("nan"), dtype=torch.float64, device="cuda")
        A.mlp_loss_grad_noalloc(torch.from_numpy(th).cuda(), xd, xu, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        # same kernels and summation order as the allocating entry point
        assert o[-1] == pytest.approx(ref_loss, rel=1e-12, abs=1e-12)
        assert np.allclose(o[:-1], ref_grad, rtol=1e-12, atol=1e-12 * np.max(np.abs(ref_grad)))


def test_noalloc_rejects_sizes_beyond_its_scratch(A):
    th, xd, xu = _inputs(4, A.AMP4D_NOALLOC_MAX_ROWS + 1, 8)
    out = torch.zeros(4546, dtype=torch.float64, device="cuda")
    with pytest.raises(A.Amp4dError) as e:
        A.mlp_loss_grad_noalloc(torch.from_numpy(th).cuda(), xd, xu, out)
    assert e.value.code == A.AMP4D_ERR_ARG and "4096" in str(e.value)


def test_noalloc_back_to_back_calls_share_the_scratch_in_stream_order(A):
    """Two calls with different inputs enqueued on one stream with no synchronisation
    between them reuse the same static scratch: stream order alone must keep them
    apart.  A loop of further calls must leave the device's free memory unchanged."""
    inputs = [_inputs(seed, nd, nu) for seed, nd, nu in [(5, 777, 1500), (6, 2048, 333)]]
    refs = [A.mlp_loss_grad(th, xd, xu) for th, xd, xu in inputs]
    ths = [torch.from_numpy(th).cuda() for th, _, _ in inputs]
    outs = [torch.full((4546,), float("nan"), dtype=torch.float64, device="cuda") for _ in inputs]
    st = torch.cuda.current_stream()
    A.mlp_loss_grad_noalloc(ths[0], inputs[0][1], inputs[0][2], outs[0], stream=st)   # warm-up
    torch.cuda.synchronize()
    for out in outs:
        out.fill_(float("nan"))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for th, (_, xd, xu), out in zip(ths, inputs, outs):
            A.mlp_loss_grad_noalloc(th, xd, xu, out, stream=st)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for out, (ref_loss, ref_grad) in zip(outs, refs):
        o = out.cpu().numpy()
        assert o[-1] == pytest.approx(ref_loss, rel=1e-12, abs=1e-12)
        assert np.allclose(o[:-1], ref_grad, rtol=1e-12, atol=1e-12 * np.max(np.abs(ref_grad)))


def test_noalloc_binding_rejects_tensors_the_abi_cannot_check(A):
    th, xd, xu = _inputs(7, 64, 64)
    thd = torch.from_numpy(th).cuda()
    out = torch.zeros(4546, dtype=torch.float64, device="cuda")
    wide = torch.zeros((64, 6), dtype=torch.float32, device="cuda")
    for args in [(thd.double(), xd, xu, out), (thd, wide[:, :4], xu, out), (thd, xd, xu, out[:100]),
                 (thd, xd, xu, out.float()), (thd, xd.cpu(), xu, out), (thd[:-1], xd, xu, out)]:
        with pytest.raises(ValueError):
            A.mlp_loss_grad_noalloc(*args)
