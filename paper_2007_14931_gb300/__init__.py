"""Python binding of libamp4d (the GB300 amplitude-fit hot path).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libamp4d.so, reached through its C ABI (include/amp4d.h) with
ctypes.  The functions below carry the C names; ``Model`` wraps them for
convenience.  PyTorch supplies device memory and the current stream.

There is no CPU fallback: importing this package fails if the library has not
been built (``python -m paper_2007_14931_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamp4d.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libamp4d.so is not built; run `python -m paper_2007_14931_gb300.build` "
                      "(needs nvcc) -- there is no CPU fallback")

_lib = C.CDLL(LIB_PATH)

AMP4D_OK = 0
AMP4D_ERR_ARG = -1
AMP4D_ERR_CUDA = -2
AMP4D_ERR_OOM = -3
AMP4D_ERR_INPUT = -4
AMP4D_ERR_DOMAIN = -5
AMP4D_ERR_TIMEOUT = -6
AMP4D_ERR_STATE = -7
AMP4D_CHAIN_KSTAR = 0
AMP4D_CHAIN_Z = 1
AMP4D_SHAPE_BW = 0
AMP4D_SHAPE_LASS = 1
AMP4D_PATH_PLAIN = 0
AMP4D_PATH_CACHED = 1
AMP4D_MAX_RES = 16
AMP4D_EVAL_NLL = 0
AMP4D_EVAL_NLL_GRAD = 1

_ERRNAMES = {AMP4D_ERR_ARG: "ARG", AMP4D_ERR_CUDA: "CUDA", AMP4D_ERR_OOM: "OOM",
             AMP4D_ERR_INPUT: "INPUT", AMP4D_ERR_DOMAIN: "DOMAIN",
             AMP4D_ERR_TIMEOUT: "TIMEOUT", AMP4D_ERR_STATE: "STATE"}


def gram_selftest(X, stream=None):
    """Integer Gram of fixed-point values X (int32 array [n, 2, 64]) on the tensor cores."""
    X = np.ascontiguousarray(X, dtype=np.int32)
    out = np.zeros((64, 64), dtype=np.int64)
    rc = amp4d_gram_selftest(X.ctypes.data, X.shape[0], out.ctypes.data, _stream_ptr(stream))
    if rc != 0:
        raise Amp4dError(rc, amp4d_last_error(None).decode())
    return out


def _check_global(rc):
    if rc != 0:
        raise Amp4dError(rc, amp4d_last_error(None).decode())


def mlp_forward(theta, x, stream=None):
    """g(x) of the proposal MLP for FP32 weights theta (4545, host) and rows x (torch cuda n x 4)."""
    import torch
    th = np.ascontiguousarray(theta, dtype=np.float32)
    x = x.contiguous()
    g = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    _check_global(amp4d_mlp_forward(th.ctypes.data, x.data_ptr(), x.shape[0], g.data_ptr(),
                                    _stream_ptr(stream)))
    return g


def mlp_loss_grad(theta, xd, xu, stream=None):
    """(loss, gradient) of the KL objective on rows xd (data) and xu (uniform), torch cuda."""
    th = np.ascontiguousarray(theta, dtype=np.float32)
    out = np.zeros(MLP_NUM_PARAMS + 1)
    xd, xu = xd.contiguous(), xu.contiguous()
    _check_global(amp4d_mlp_loss_grad(th.ctypes.data, xd.data_ptr(), xd.shape[0], xu.data_ptr(),
                                      xu.shape[0], out.ctypes.data_as(_d), _stream_ptr(stream)))
    return out[-1], out[:-1]


def mlp_loss_grad_noalloc(theta_dev, xd, xu, out_dev, stream=None):
    """Allocation-free KL gradient: all arguments are torch cuda tensors; out_dev (4546
    float64) receives the gradient and then the loss.  Stream-ordered, no sync.

    The C entry point sees only raw pointers, so every tensor is checked here and a
    mismatch raises ValueError; nothing is converted or copied, since a copy would
    allocate."""
    import torch

    def need(ok, what):
        if not ok:
            raise ValueError("mlp_loss_grad_noalloc: " + what)

    ts = {"theta_dev": theta_dev, "xd": xd, "xu": xu, "out_dev": out_dev}
    for k, t in ts.items():
        need(isinstance(t, torch.Tensor) and t.is_cuda, "%s must be a CUDA tensor" % k)
        need(t.is_contiguous(), "%s must be contiguous" % k)
    need(len({t.device for t in ts.values()}) == 1, "all tensors must be on one device")
    need(theta_dev.dtype == torch.float32 and theta_dev.numel() == MLP_NUM_PARAMS,
         "theta_dev must hold %d float32" % MLP_NUM_PARAMS)
    for k, x in (("xd", xd), ("xu", xu)):
        need(x.dtype == torch.float32 and x.dim() == 2 and x.shape[1] == 4,
             "%s must be float32 of shape (n, 4)" % k)
    need(out_dev.dtype == torch.float64 and out_dev.numel() >= MLP_NUM_PARAMS + 1,
         "out_dev must hold at least %d float64" % (MLP_NUM_PARAMS + 1))
    rc = amp4d_mlp_loss_grad_noalloc(theta_dev.data_ptr(), xd.data_ptr(), xd.shape[0],
                                     xu.data_ptr(), xu.shape[0], out_dev.data_ptr(),
                                     _stream_ptr(stream))
    if rc != 0:
        raise Amp4dError(rc, amp4d_noalloc_last_error().decode())


def combine_partials(parts, what=None):
    """Evaluation of the union of shards from their partial blocks (rows, in shard
    order): returns (nll, gradient or None, out) with out in the enqueue_eval layout.
    Raises Amp4dError on a domain error, like Model.eval_nll."""
    parts = np.ascontiguousarray(np.atleast_2d(parts), dtype=np.float64)
    n_shards, width = parts.shape
    if what is None:
        what = AMP4D_EVAL_NLL if width == 6 else AMP4D_EVAL_NLL_GRAD
    n_param = (width - 6) // 2 if what == AMP4D_EVAL_NLL_GRAD else 0
    if width != 6 + 2 * n_param:
        raise ValueError("partial blocks of width %d do not match what=%d" % (width, what))
    out = np.zeros(6 + n_param)
    rc = amp4d_combine_partials(parts.ctypes.data_as(_d), n_shards, n_param, what,
                                out.ctypes.data_as(_d))
    if rc != 0:
        raise Amp4dError(rc, amp4d_shard_last_error().decode())
    return out[0], (out[6:].copy() if what == AMP4D_EVAL_NLL_GRAD else None), out


def grid_sample(gcell, nb, alpha, seed, n, masses=None, box=None, stream=None):
    """Sampler of the grid proposal on given cell values: (m, cK, cpsi, phi), w, cell (torch cuda)."""
    import torch
    import workloads as W
    masses = W.PARTICLE_MASSES if masses is None else masses
    box = (W.M_LO, W.M_HI) if box is None else box
    gc = np.ascontiguousarray(gcell, dtype=np.float32)
    nbv = (C.c_int * 4)(*nb)
    outs = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(5)]
    cell = torch.empty(n, dtype=torch.int64, device="cuda")
    pm = amp4d_particle_masses(*masses)
    _check_global(amp4d_grid_sample(gc.ctypes.data, nbv, float(alpha), int(seed), int(n), box[0], box[1],
                                    C.byref(pm), *(o.data_ptr() for o in outs), cell.data_ptr(),
                                    _stream_ptr(stream)))
    return tuple(outs[:4]), outs[4], cell


class amp4d_particle_masses(C.Structure):
    _fields_ = [("mB", C.c_double), ("mpsi", C.c_double), ("mK", C.c_double), ("mpi", C.c_double)]


class amp4d_resonance(C.Structure):
    _fields_ = [("chain", C.c_int), ("J", C.c_int), ("P", C.c_int), ("LB", C.c_int),
                ("LR", C.c_int), ("M", C.c_double), ("G0", C.c_double), ("r", C.c_double),
                ("float_mg", C.c_int), ("shape", C.c_int), ("lass_a", C.c_double),
                ("lass_b", C.c_double), ("lass_R", C.c_double)]


class amp4d_hist2d(C.Structure):
    _fields_ = [("h", C.c_void_p), ("nx", C.c_int), ("ny", C.c_int), ("x_lo", C.c_double),
                ("x_hi", C.c_double), ("y_lo", C.c_double), ("y_hi", C.c_double)]


class amp4d_mlp_cfg(C.Structure):
    _fields_ = [("nb", C.c_int * 4), ("alpha", C.c_double), ("steps", C.c_int64),
                ("batch", C.c_int), ("lr", C.c_double)]


_vp = C.c_void_p
_d = C.POINTER(C.c_double)
_f = C.POINTER(C.c_float)


def _proto(name, res, args):
    fn = getattr(_lib, name)
    fn.restype = res
    fn.argtypes = args
    return fn


amp4d_model_create = _proto("amp4d_model_create", C.c_int,
                            [C.POINTER(amp4d_particle_masses), C.POINTER(amp4d_resonance), C.c_int,
                             C.c_double, C.c_double, C.c_int, C.POINTER(_vp)])
amp4d_model_destroy = _proto("amp4d_model_destroy", C.c_int, [_vp])
amp4d_last_error = _proto("amp4d_last_error", C.c_char_p, [_vp])
amp4d_num_columns = _proto("amp4d_num_columns", C.c_int, [_vp])
amp4d_num_params = _proto("amp4d_num_params", C.c_int, [_vp])
amp4d_set_events = _proto("amp4d_set_events", C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_int64, _vp])
amp4d_set_norm_points = _proto("amp4d_set_norm_points", C.c_int,
                               [_vp, _vp, _vp, _vp, _vp, _vp, C.c_int64, C.c_double, _vp])
amp4d_eval_nll = _proto("amp4d_eval_nll", C.c_int, [_vp, _vp, _vp, _vp])
amp4d_eval_nll_grad = _proto("amp4d_eval_nll_grad", C.c_int, [_vp, _vp, _vp, _vp, _vp])
amp4d_eval_terms = _proto("amp4d_eval_terms", C.c_int, [_vp, _d, _d, _vp])
amp4d_eval_density = _proto("amp4d_eval_density", C.c_int, [_vp, _d, C.c_int, _vp, _vp])
amp4d_enqueue_eval = _proto("amp4d_enqueue_eval", C.c_int, [_vp, C.c_int, _vp, _vp, _vp])
amp4d_eval_pdf = _proto("amp4d_eval_pdf", C.c_int, [_vp, _d, _vp, _vp])
amp4d_build_gram = _proto("amp4d_build_gram", C.c_int, [_vp, _d, _vp])
amp4d_get_gram = _proto("amp4d_get_gram", C.c_int, [_vp, _d, _vp])
amp4d_fit_fractions = _proto("amp4d_fit_fractions", C.c_int, [_vp, _d, _d, _vp])
amp4d_set_efficiency = _proto("amp4d_set_efficiency", C.c_int,
                              [_vp, C.POINTER(amp4d_hist2d), C.POINTER(amp4d_hist2d), _vp])
amp4d_set_background = _proto("amp4d_set_background", C.c_int,
                              [_vp, C.POINTER(amp4d_hist2d), C.POINTER(amp4d_hist2d), C.c_double, _vp])
amp4d_set_flavour = _proto("amp4d_set_flavour", C.c_int, [_vp, _vp, C.c_double, _vp])
amp4d_gram_selftest = _proto("amp4d_gram_selftest", C.c_int, [_vp, C.c_int64, _vp, _vp])
amp4d_generate = _proto("amp4d_generate", C.c_int, [_vp, _d, C.c_uint64, C.c_int64, _vp, _vp, _vp, _vp, _vp])
amp4d_proposal_train = _proto("amp4d_proposal_train", C.c_int,
                              [_vp, _vp, _vp, _vp, _vp, C.c_int64, C.POINTER(amp4d_mlp_cfg), C.c_uint64,
                               _d, _vp])
amp4d_proposal_train_gram = _proto("amp4d_proposal_train_gram", C.c_int,
                                   [_vp, _d, C.c_int64, C.POINTER(amp4d_mlp_cfg), C.c_uint64, C.c_uint64,
                                    _d, _vp])
amp4d_proposal_sample = _proto("amp4d_proposal_sample", C.c_int,
                               [_vp, C.c_int64, C.c_uint64, _vp, _vp, _vp, _vp, _vp, _vp])
amp4d_mlp_forward = _proto("amp4d_mlp_forward", C.c_int, [_vp, _vp, C.c_int64, _vp, _vp])
amp4d_mlp_loss_grad = _proto("amp4d_mlp_loss_grad", C.c_int, [_vp, _vp, C.c_int64, _vp, C.c_int64, _d, _vp])
amp4d_grid_sample = _proto("amp4d_grid_sample", C.c_int,
                           [_vp, _vp, C.c_double, C.c_uint64, C.c_int64, C.c_double, C.c_double,
                            C.POINTER(amp4d_particle_masses), _vp, _vp, _vp, _vp, _vp, _vp, _vp])
amp4d_mlp_loss_grad_noalloc = _proto("amp4d_mlp_loss_grad_noalloc", C.c_int,
                                     [_vp, _vp, C.c_int64, _vp, C.c_int64, _vp, _vp])
amp4d_noalloc_last_error = _proto("amp4d_noalloc_last_error", C.c_char_p, [])
AMP4D_NOALLOC_MAX_ROWS = 4096
amp4d_eval_partials = _proto("amp4d_eval_partials", C.c_int, [_vp, C.c_int, _d, _d, _vp])
amp4d_enqueue_partials = _proto("amp4d_enqueue_partials", C.c_int, [_vp, C.c_int, _vp, _vp, _vp])
amp4d_combine_partials = _proto("amp4d_combine_partials", C.c_int, [_d, C.c_int, C.c_int, C.c_int, _d])
amp4d_shard_last_error = _proto("amp4d_shard_last_error", C.c_char_p, [])
amp4d_profile_enable = _proto("amp4d_profile_enable", C.c_int, [_vp, C.c_int])
amp4d_profile_read = _proto("amp4d_profile_read", C.c_int, [_vp, _d, C.POINTER(C.c_int64)])

EXPORTED = ["amp4d_set_efficiency", "amp4d_set_background", "amp4d_set_flavour",
            "amp4d_model_create", "amp4d_model_destroy", "amp4d_last_error", "amp4d_num_columns",
            "amp4d_num_params", "amp4d_set_events", "amp4d_set_norm_points", "amp4d_eval_nll",
            "amp4d_eval_nll_grad", "amp4d_eval_terms", "amp4d_eval_density", "amp4d_enqueue_eval",
            "amp4d_profile_enable", "amp4d_profile_read", "amp4d_build_gram", "amp4d_get_gram",
            "amp4d_gram_selftest", "amp4d_generate", "amp4d_proposal_train",
            "amp4d_proposal_train_gram", "amp4d_proposal_sample", "amp4d_mlp_forward", "amp4d_mlp_loss_grad", "amp4d_grid_sample",
            "amp4d_mlp_loss_grad_noalloc", "amp4d_noalloc_last_error", "amp4d_eval_partials",
            "amp4d_enqueue_partials", "amp4d_combine_partials", "amp4d_shard_last_error",
            "amp4d_eval_pdf", "amp4d_fit_fractions"]

MLP_NUM_PARAMS = 4545


class Amp4dError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("amp4d %s (%d): %s" % (_ERRNAMES.get(code, "?"), code, msg))
        self.code = code


_torch_cuda = None
_raw_stream = None


def _stream_ptr(stream):
    """cudaStream_t of a torch stream, an int, or (None) torch's current stream.
    The current stream's handle is read with torch's raw getter where it exists
    (it builds no Stream object: 0.06 us against about 3-8 us per call)."""
    global _torch_cuda, _raw_stream
    if stream is None:
        if _torch_cuda is None:
            import torch
            _torch_cuda = torch.cuda
            _raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        if _raw_stream is not None:
            return _raw_stream(_torch_cuda.current_device())
        return _torch_cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _ptr(a):
    """Device or host pointer of a float32 contiguous torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        if a.dtype.__repr__() != "torch.float32" or not a.is_contiguous():
            raise TypeError("expected a contiguous float32 tensor")
        return a.data_ptr()
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous):
        raise TypeError("expected a contiguous float32 array")
    return a.ctypes.data


class Model:
    """A model built from ``workloads.Resonance`` records (one per resonance)."""

    def __init__(self, res_list, float_names=(), path=AMP4D_PATH_PLAIN, masses=None, box=None):
        import workloads as W
        masses = W.PARTICLE_MASSES if masses is None else masses
        box = (W.M_LO, W.M_HI) if box is None else box
        self.res_list = list(res_list)
        arr = (amp4d_resonance * len(res_list))()
        for i, r in enumerate(res_list):
            arr[i] = amp4d_resonance(r.chain, r.J, r.P, r.LB, r.LR, r.M, r.G0, r.r,
                                     1 if r.name in float_names else 0,
                                     getattr(r, "shape", AMP4D_SHAPE_BW),
                                     getattr(r, "lass_a", 0.0), getattr(r, "lass_b", 0.0),
                                     getattr(r, "lass_R", 0.0))
        pm = amp4d_particle_masses(*masses)
        h = _vp()
        rc = amp4d_model_create(C.byref(pm), arr, len(res_list), box[0], box[1], path, C.byref(h))
        if rc != 0:
            raise Amp4dError(rc, amp4d_last_error(None).decode())
        self.h = h
        self.n_cols = amp4d_num_columns(h)
        self.n_params = amp4d_num_params(h)
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            amp4d_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise Amp4dError(rc, amp4d_last_error(self.h).decode())

    def set_events(self, m, cK, cpsi, phi, stream=None):
        n = len(m)
        self._check(amp4d_set_events(self.h, _ptr(m), _ptr(cK), _ptr(cpsi), _ptr(phi), n,
                                     _stream_ptr(stream)))
        self.n_events = n

    def set_norm_points(self, m, cK, cpsi, phi, w=None, volume=None, stream=None):
        import workloads as W
        volume = W.BOX_VOLUME if volume is None else volume
        n = len(m)
        self._check(amp4d_set_norm_points(self.h, _ptr(m), _ptr(cK), _ptr(cpsi), _ptr(phi),
                                          _ptr(w) if w is not None else None, n, float(volume),
                                          _stream_ptr(stream)))
        self.n_norm = n

    def _params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        if p.shape != (self.n_params,):
            raise ValueError("expected %d parameters" % self.n_params)
        return p

    def eval_nll(self, params, stream=None, check=True):
        p = self._params(params)
        out = np.empty(1)
        rc = amp4d_eval_nll(self.h, p.ctypes.data, out.ctypes.data, _stream_ptr(stream))
        if check and rc not in (0, AMP4D_ERR_DOMAIN):
            self._check(rc)
        return float(out[0])

    def eval_nll_grad(self, params, stream=None):
        p = self._params(params)
        out = np.empty(1 + self.n_params)   # NLL, then the gradient
        rc = amp4d_eval_nll_grad(self.h, p.ctypes.data, out.ctypes.data, out[1:].ctypes.data,
                                 _stream_ptr(stream))
        if rc not in (0, AMP4D_ERR_DOMAIN):
            self._check(rc)
        return float(out[0]), out[1:]

    def eval_terms(self, params, stream=None):
        p = self._params(params)
        o = np.zeros(4)
        self._check(amp4d_eval_terms(self.h, p.ctypes.data_as(_d), o.ctypes.data_as(_d),
                                     _stream_ptr(stream)))
        return o

    def eval_partials(self, params, grad=True, stream=None):
        """Shard partials of this model's events and points (host float64 array of
        6 or 6 + 2P values; layout in include/amp4d.h)."""
        p = self._params(params)
        what = AMP4D_EVAL_NLL_GRAD if grad else AMP4D_EVAL_NLL
        o = np.zeros(6 + (2 * self.n_params if grad else 0))
        self._check(amp4d_eval_partials(self.h, what, p.ctypes.data_as(_d), o.ctypes.data_as(_d),
                                        _stream_ptr(stream)))
        return o

    def enqueue_partials(self, what, params_dev, out_dev, stream=None):
        """Enqueue the shard partials with device parameters/outputs (torch float64)."""
        self._check(amp4d_enqueue_partials(self.h, what, params_dev.data_ptr(), out_dev.data_ptr(),
                                           _stream_ptr(stream)))

    def enqueue_eval(self, what, params_dev, out_dev, stream=None):
        """Enqueue an evaluation with device parameters/outputs (torch float64 tensors)."""
        self._check(amp4d_enqueue_eval(self.h, what, params_dev.data_ptr(), out_dev.data_ptr(),
                                       _stream_ptr(stream)))

    def build_gram(self, params, stream=None):
        p = self._params(params)
        self._check(amp4d_build_gram(self.h, p.ctypes.data_as(_d), _stream_ptr(stream)))

    @staticmethod
    def _hist(t):
        """ctypes record of a template with h[iy, ix] contents (FP32, kept alive by the caller)."""
        h = np.ascontiguousarray(t.h, dtype=np.float32)
        r = t.range
        return amp4d_hist2d(h.ctypes.data, int(h.shape[1]), int(h.shape[0]), *map(float, r)), h

    def set_efficiency(self, mass, angle, stream=None):
        """Eq. 14 relative efficiency: templates over (m^2_Kpi, m^2_psipi) and
        (cos theta_psi, phi) (objects with .h [ny, nx] and .range); None removes it."""
        if mass is None:
            self._check(amp4d_set_efficiency(self.h, None, None, _stream_ptr(stream)))
            return
        (hm, km), (ha, ka) = self._hist(mass), self._hist(angle)
        self._check(amp4d_set_efficiency(self.h, C.byref(hm), C.byref(ha), _stream_ptr(stream)))

    def set_background(self, mass, angle, purity, stream=None):
        """Eq. 14 background templates with signal purity P; None removes it."""
        if mass is None:
            self._check(amp4d_set_background(self.h, None, None, 1.0, _stream_ptr(stream)))
            return
        (hm, km), (ha, ka) = self._hist(mass), self._hist(angle)
        self._check(amp4d_set_background(self.h, C.byref(hm), C.byref(ha), float(purity),
                                         _stream_ptr(stream)))

    def set_flavour(self, tag, mistag=0.0, stream=None):
        """Flavour tags of the data events (+1 B0, -1 B0bar; FP32 host array or
        CUDA tensor, None for all B0) and the mistag fraction w."""
        if tag is None:
            ptr = None
        elif hasattr(tag, "data_ptr"):
            ptr = tag.data_ptr()
        else:
            tag = np.ascontiguousarray(tag, dtype=np.float32)
            ptr = tag.ctypes.data
        self._check(amp4d_set_flavour(self.h, ptr, float(mistag), _stream_ptr(stream)))

    def fit_fractions(self, params, stream=None):
        """Fit fraction of every resonance (Eq. 13), in creation order (host float64)."""
        p = self._params(params)
        ff = np.zeros(len(self.res_list))
        self._check(amp4d_fit_fractions(self.h, p.ctypes.data_as(_d), ff.ctypes.data_as(_d),
                                        _stream_ptr(stream)))
        return ff

    def get_gram(self, stream=None):
        d = 2 * self.n_cols
        G = np.zeros((d, d))
        self._check(amp4d_get_gram(self.h, G.ctypes.data_as(_d), _stream_ptr(stream)))
        return G

    def generate(self, params, n, seed, stream=None):
        """n events drawn from the model at params (device float32 tensors m, cK, cpsi, phi)."""
        import torch
        p = self._params(params)
        outs = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(4)]
        self._check(amp4d_generate(self.h, p.ctypes.data_as(_d), int(seed), int(n),
                                   *(o.data_ptr() for o in outs), _stream_ptr(stream)))
        return tuple(outs)

    def proposal_train(self, events, nb=(128, 32, 16, 32), alpha=0.05, steps=4000, batch=8192,
                       lr=2e-3, seed=1, stream=None):
        cfg = amp4d_mlp_cfg((C.c_int * 4)(*nb), alpha, steps, batch, lr)
        loss = C.c_double()
        ev = [e.contiguous() for e in events]
        self._check(amp4d_proposal_train(self.h, *(e.data_ptr() for e in ev), ev[0].shape[0],
                                         C.byref(cfg), int(seed), C.byref(loss), _stream_ptr(stream)))
        return loss.value

    def proposal_train_gram(self, params, n=1 << 20, seed=12, gen_seed=5000, nb=(128, 32, 16, 32),
                            alpha=0.05, steps=4000, batch=8192, lr=2e-3, stream=None):
        """Train the proposal toward the whole normalisation Gram matrix (target
        sum_k |B_k|^2 p q; amp4d_proposal_train_gram).  params gives the masses
        and widths (its couplings are not used).  Returns the training loss."""
        p = self._params(params)
        cfg = amp4d_mlp_cfg((C.c_int * 4)(*nb), alpha, steps, batch, lr)
        loss = C.c_double()
        self._check(amp4d_proposal_train_gram(self.h, p.ctypes.data_as(_d), int(n), C.byref(cfg),
                                              int(seed), int(gen_seed), C.byref(loss),
                                              _stream_ptr(stream)))
        return loss.value

    def proposal_sample(self, n, seed, stream=None):
        """n importance-sampled points and weights w = p q / q (device float32 tensors)."""
        import torch
        outs = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(5)]
        self._check(amp4d_proposal_sample(self.h, int(n), int(seed), *(o.data_ptr() for o in outs),
                                          _stream_ptr(stream)))
        return tuple(outs[:4]), outs[4]

    def profile(self, on=True):
        self._check(amp4d_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        ms = np.zeros(4)
        cnt = np.zeros(4, dtype=np.int64)
        self._check(amp4d_profile_read(self.h, ms.ctypes.data_as(_d),
                                       cnt.ctypes.data_as(C.POINTER(C.c_int64))))
        return ms, cnt

    def eval_density(self, params, which=0, out=None, stream=None):
        import torch
        p = self._params(params)
        n = self.n_events if which == 0 else self.n_norm
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device="cuda")
        self._check(amp4d_eval_density(self.h, p.ctypes.data_as(_d), which, out.data_ptr(),
                                       _stream_ptr(stream)))
        return out

    def eval_pdf(self, params, out=None, stream=None):
        """Normalised PDF S p q / I of every data event (torch cuda float32)."""
        import torch
        p = self._params(params)
        if out is None:
            out = torch.empty(self.n_events, dtype=torch.float32, device="cuda")
        self._check(amp4d_eval_pdf(self.h, p.ctypes.data_as(_d), out.data_ptr(), _stream_ptr(stream)))
        return out
