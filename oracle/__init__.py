"""FP64 CPU oracle for the B0 -> J/psi K pi four-dimensional amplitude fit.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's timed
CPU baseline use it; the product path never imports it.  The arithmetic lives
in ``amp4d_oracle.c`` (plain C, double precision, OpenMP over events); this
module compiles it with gcc on first use and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amp4d_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = C.POINTER(C.c_double)
_f = C.POINTER(C.c_float)
_i = C.POINTER(C.c_int)
_u32 = C.POINTER(C.c_uint32)


def build(force=False):
    """Compile the oracle shared library with gcc (no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.or_model_new.restype = C.c_void_p
            L.or_model_new.argtypes = [_d, C.c_double, C.c_double, C.c_int, _i, _i, _i, _i, _i,
                                       _d, _d, _d, _i]
            L.or_model_free.argtypes = [C.c_void_p]
            L.or_model_set_lass.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double,
                                            C.c_double]
            L.or_num_cols.argtypes = [C.c_void_p]
            L.or_num_params.argtypes = [C.c_void_p]
            L.or_columns.argtypes = [C.c_void_p, _i, _i]
            L.or_wigner_d.restype = C.c_double
            L.or_wigner_d.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double]
            L.or_bw_poly.restype = C.c_double
            L.or_bw_poly.argtypes = [C.c_int, C.c_double]
            L.or_breakup.restype = C.c_double
            L.or_breakup.argtypes = [C.c_double, C.c_double, C.c_double]
            L.or_lineshape.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double, _d]
            L.or_kinematics.argtypes = [C.c_void_p, _d, _d, _d, _d, C.c_int64, _d]
            L.or_basis.argtypes = [C.c_void_p, _d, _d, _d, _d, _d, C.c_int64, _d, _d]
            L.or_density.argtypes = [C.c_void_p, _d, _d, _d, _d, _d, C.c_int64, _d, _d]
            L.or_norm.argtypes = [C.c_void_p, _d, _d, _d, _d, _d, _d, C.c_int64, C.c_double,
                                  _d, _d]
            L.or_nll.argtypes = [C.c_void_p, _d, _d, _d, _d, _d, C.c_int64, _d, _d, _d, _d, _d,
                                 C.c_int64, C.c_double, _d, _d, _d]
            L.or_gram.argtypes = [C.c_void_p, _d, _d, _d, _d, _d, _d, C.c_int64, _d]
            L.or_nll_eq14.argtypes = [C.c_void_p, _d, _d, _d, _d, _d, _d, C.c_int64, _d, _d, _d,
                                      _d, _d, C.c_int64, C.c_double, _d, _d, _d]
            L.or_model_set_mistag.argtypes = [C.c_void_p, C.c_double]
            L.or_model_set_template.argtypes = [C.c_void_p, C.c_int, _d, C.c_int, C.c_int, _d,
                                                _d, C.c_int, C.c_int, _d, C.c_double]
            L.or_tpl_value.restype = C.c_double
            L.or_tpl_value.argtypes = [_d, C.c_int, C.c_int, _d, C.c_double, C.c_double]
            L.or_templates.argtypes = [C.c_void_p, _d, _d, _d, _d, C.c_int64, _d]
            L.or_partials.argtypes = [C.c_void_p, _d, _d, _d, _d, _d, C.c_int64, _d, _d, _d, _d,
                                      _d, C.c_int64, C.c_double, C.c_int, _d]
            L.or_generate.restype = C.c_int64
            L.or_generate.argtypes = [C.c_void_p, _d, C.c_uint64, C.c_int64, C.c_int64,
                                      C.c_int64, _f, _f, _f, _f, _d]
            L.or_philox4x32_10.argtypes = [_u32, _u32, _u32]
            L.or_mlp_num_params.restype = C.c_int
            L.or_mlp_forward.argtypes = [_d, _d, C.c_int64, _d]
            L.or_mlp_loss_grad.argtypes = [_d, _d, C.c_int64, _d, C.c_int64, _d, _d]
            L.or_adam_step.argtypes = [_d, _d, _d, _d, C.c_int64, C.c_double, C.c_double,
                                       C.c_double, C.c_double, C.c_int64]
            L.or_grid_sample.argtypes = [_d, _i, C.c_double, C.c_uint64, C.c_int64, C.c_double,
                                         C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                         _f, _f, _f, _f, _d, C.POINTER(C.c_int64)]
            L.or_num_threads.restype = C.c_int
            L.or_set_num_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _pd(a):
    return a.ctypes.data_as(_d)


def _pf(a):
    return a.ctypes.data_as(_f)


def _pi(a):
    return a.ctypes.data_as(_i)


def _f64(a):
    """Coordinates enter the oracle in double; FP32 event arrays promote exactly."""
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads():
    return lib().or_num_threads()


def set_num_threads(n):
    lib().or_set_num_threads(int(n))


def wigner_d(j, mp, m, cosb):
    """Wigner small-d d^j_{mp m}(beta) at cos(beta), by the general factorial sum."""
    return lib().or_wigner_d(int(j), int(mp), int(m), float(cosb))


def bw_poly(L, z):
    """Blatt-Weisskopf barrier polynomial P_L(z)."""
    return lib().or_bw_poly(int(L), float(z))


def breakup(Mp, m1, m2):
    """Two-body momentum of a parent of mass Mp decaying to m1, m2 (0 if closed)."""
    return lib().or_breakup(float(Mp), float(m1), float(m2))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(c.ctypes.data_as(_u32), k.ctypes.data_as(_u32), o.ctypes.data_as(_u32))
    return o


class Model:
    """Oracle model built from a list of ``workloads.Resonance`` records."""

    def __init__(self, res_list, float_names=(), masses=None, box=None):
        import workloads as W
        masses = W.PARTICLE_MASSES if masses is None else masses
        box = (W.M_LO, W.M_HI) if box is None else box
        self.res_list = list(res_list)
        self.masses = tuple(masses)
        self.box = tuple(box)
        n = len(self.res_list)
        ia = lambda xs: np.ascontiguousarray(xs, dtype=np.int32)
        self._arrs = dict(
            masses=_f64(masses),
            chain=ia([r.chain for r in res_list]), J=ia([r.J for r in res_list]),
            P=ia([r.P for r in res_list]), LB=ia([r.LB for r in res_list]),
            LR=ia([r.LR for r in res_list]), M=_f64([r.M for r in res_list]),
            G0=_f64([r.G0 for r in res_list]), r=_f64([r.r for r in res_list]),
            flt=ia([1 if r.name in float_names else 0 for r in res_list]))
        a = self._arrs
        self.h = lib().or_model_new(_pd(a["masses"]), box[0], box[1], n, _pi(a["chain"]),
                                    _pi(a["J"]), _pi(a["P"]), _pi(a["LB"]), _pi(a["LR"]),
                                    _pd(a["M"]), _pd(a["G0"]), _pd(a["r"]), _pi(a["flt"]))
        if not self.h:
            raise ValueError("oracle: bad model")
        for i, r in enumerate(res_list):
            if r.shape == W.SHAPE_LASS:
                if lib().or_model_set_lass(self.h, i, r.lass_a, r.lass_b, r.lass_R) != 0:
                    lib().or_model_free(self.h)
                    self.h = None
                    raise ValueError(f"oracle: bad LASS record {r.name}")
        self.n_cols = lib().or_num_cols(self.h)
        self.n_params = lib().or_num_params(self.h)
        res = np.zeros(self.n_cols, np.int32)
        lam = np.zeros(self.n_cols, np.int32)
        lib().or_columns(self.h, _pi(res), _pi(lam))
        self.col_res, self.col_lam = res, lam

    def __del__(self):
        try:
            if self.h:
                lib().or_model_free(self.h)
        except Exception:
            pass

    def lineshape(self, R, mrun, M=None, G0=None):
        """(A, dA/dM, dA/dG0) of resonance R at running mass mrun."""
        r = self.res_list[R]
        o = np.zeros(6)
        lib().or_lineshape(self.h, int(R), float(mrun), float(r.M if M is None else M),
                           float(r.G0 if G0 is None else G0), _pd(o))
        return complex(o[0], o[1]), complex(o[2], o[3]), complex(o[4], o[5])

    def kinematics(self, pts):
        m, cK, cpsi, phi = (_f64(a) for a in pts)
        out = np.zeros((len(m), 24))
        lib().or_kinematics(self.h, _pd(m), _pd(cK), _pd(cpsi), _pd(phi), len(m), _pd(out))
        return out

    def basis(self, params, pts):
        """B[e, k, xi] complex (xi index 0 = +1, 1 = -1) and p q per point."""
        m, cK, cpsi, phi = (_f64(a) for a in pts)
        n = len(m)
        out = np.zeros((n, self.n_cols, 2, 2))
        pq = np.zeros(n)
        pr = _f64(params)
        lib().or_basis(self.h, _pd(pr), _pd(m), _pd(cK), _pd(cpsi), _pd(phi), n, _pd(out), _pd(pq))
        return out[..., 0] + 1j * out[..., 1], pq

    def density(self, params, pts):
        """(S, p q) per point."""
        m, cK, cpsi, phi = (_f64(a) for a in pts)
        n = len(m)
        S = np.zeros(n)
        pq = np.zeros(n)
        pr = _f64(params)
        lib().or_density(self.h, _pd(pr), _pd(m), _pd(cK), _pd(cpsi), _pd(phi), n, _pd(S), _pd(pq))
        return S, pq

    def norm(self, params, pts, w=None, volume=None, grad=False):
        import workloads as W
        volume = W.BOX_VOLUME if volume is None else volume
        m, cK, cpsi, phi = (_f64(a) for a in pts)
        wf = _f64(w) if w is not None else None
        I = C.c_double()
        g = np.zeros(self.n_params) if grad else None
        pr = _f64(params)
        lib().or_norm(self.h, _pd(pr), _pd(m), _pd(cK), _pd(cpsi), _pd(phi),
                      _pd(wf) if wf is not None else None, len(m), float(volume), C.byref(I),
                      _pd(g) if grad else None)
        return (I.value, g) if grad else I.value

    def nll(self, params, events, norm_pts, w=None, volume=None, grad=False):
        """(-2 ln L, gradient or None, aux = [sum ln S, sum ln pq, I], status)."""
        import workloads as W
        volume = W.BOX_VOLUME if volume is None else volume
        ev = [_f64(a) for a in events]
        nm = [_f64(a) for a in norm_pts]
        wf = _f64(w) if w is not None else None
        out = C.c_double()
        g = np.zeros(self.n_params) if grad else None
        aux = np.zeros(3)
        pr = _f64(params)
        rc = lib().or_nll(self.h, _pd(pr), *(_pd(a) for a in ev), len(ev[0]),
                          *(_pd(a) for a in nm), _pd(wf) if wf is not None else None,
                          len(nm[0]), float(volume), C.byref(out), _pd(g) if grad else None,
                          _pd(aux))
        return out.value, g, aux, rc

    def partials(self, params, events, norm_pts, w=None, volume=None, grad=True):
        """Sums of one shard (either set may be empty): [sum ln S, sum ln pq, N,
        T = V sum w S, M, bad, d sum ln S (P), dT (P)]; I = sum T / sum M over shards."""
        import workloads as W
        volume = W.BOX_VOLUME if volume is None else volume
        ev = [_f64(a) for a in events]
        nm = [_f64(a) for a in norm_pts]
        wf = _f64(w) if w is not None else None
        out = np.zeros(6 + (2 * self.n_params if grad else 0))
        pr = _f64(params)
        lib().or_partials(self.h, _pd(pr), *(_pd(a) for a in ev), len(ev[0]),
                          *(_pd(a) for a in nm), _pd(wf) if wf is not None else None,
                          len(nm[0]), float(volume), 1 if grad else 0, _pd(out))
        return out

    def fit_fractions(self, params, pts, w=None, volume=None):
        """Fit fractions (Eq. 13) by their definition: FF_j = I_j / I, I_j the
        normalisation integral over pts with every helicity coupling outside
        resonance j set to zero (masses and widths unchanged)."""
        pr = _f64(params)
        I = self.norm(pr, pts, w=w, volume=volume)
        out = np.zeros(len(self.res_list))
        for R in range(len(self.res_list)):
            pj = pr.copy()
            for k, r in enumerate(self.col_res):
                if r != R:
                    pj[2 * k] = pj[2 * k + 1] = 0.0
            out[R] = self.norm(pj, pts, w=w, volume=volume) / I
        return out

    def set_template(self, which, mass, angle, purity=1.0):
        """Eq. 14 templates: which 0 = efficiency, 1 = background (with purity).
        mass, angle: workloads.Hist2D (contents [ny, nx], x and y ranges)."""
        hm, ha = _f64(np.ravel(mass.h)), _f64(np.ravel(angle.h))
        rm, ra = _f64(mass.range), _f64(angle.range)
        self._keep_tpl = getattr(self, "_keep_tpl", []) + [hm, ha, rm, ra]
        rc = lib().or_model_set_template(self.h, int(which), _pd(hm), mass.nx, mass.ny, _pd(rm),
                                         _pd(ha), angle.nx, angle.ny, _pd(ra), float(purity))
        if rc != 0:
            raise ValueError("oracle: bad template")

    def templates(self, pts):
        """(eps, hb, m^2_psipi) per point."""
        m, cK, cpsi, phi = (_f64(a) for a in pts)
        out = np.zeros((len(m), 3))
        lib().or_templates(self.h, _pd(m), _pd(cK), _pd(cpsi), _pd(phi), len(m), _pd(out))
        return out[:, 0], out[:, 1], out[:, 2]

    def set_mistag(self, w):
        if lib().or_model_set_mistag(self.h, float(w)) != 0:
            raise ValueError("oracle: mistag must lie in [0, 0.5]")

    def nll_eq14(self, params, events, norm_pts, w=None, volume=None, grad=False, tag=None):
        """Eq. 14: (-2 ln L, gradient or None, aux, status); aux = [sum ln(f/pq),
        sum ln pq, I_eps, B, sum of signal probabilities].  tag: +1 (B0) / -1
        (B0bar) per event, None for all B0."""
        import workloads as W
        volume = W.BOX_VOLUME if volume is None else volume
        ev = [_f64(a) for a in events]
        tg = _f64(tag) if tag is not None else None
        nm = [_f64(a) for a in norm_pts]
        wf = _f64(w) if w is not None else None
        out = C.c_double()
        g = np.zeros(self.n_params) if grad else None
        aux = np.zeros(5)
        pr = _f64(params)
        rc = lib().or_nll_eq14(self.h, _pd(pr), *(_pd(a) for a in ev),
                               _pd(tg) if tg is not None else None, len(ev[0]),
                               *(_pd(a) for a in nm), _pd(wf) if wf is not None else None,
                               len(nm[0]), float(volume), C.byref(out), _pd(g) if grad else None,
                               _pd(aux))
        return out.value, g, aux, rc

    def gram(self, params, pts, w=None):
        m, cK, cpsi, phi = (_f64(a) for a in pts)
        D = 2 * self.n_cols
        G = np.zeros((D, D))
        wf = _f64(w) if w is not None else None
        pr = _f64(params)
        lib().or_gram(self.h, _pd(pr), _pd(m), _pd(cK), _pd(cpsi), _pd(phi),
                      _pd(wf) if wf is not None else None, len(m), _pd(G))
        return G

    def generate(self, params, n, seed, n_scan=200_000, max_cand=None):
        """Accept-reject pseudo-data distributed as S p q (FP32 SoA)."""
        max_cand = max_cand or 4000 * n + (1 << 20)
        outs = [np.zeros(n, np.float32) for _ in range(4)]
        fmax = C.c_double()
        pr = _f64(params)
        used = lib().or_generate(self.h, _pd(pr), int(seed), int(n), int(n_scan), int(max_cand),
                                 *(_pf(a) for a in outs), C.byref(fmax))
        if used < 0:
            raise RuntimeError("oracle generator: candidate budget exhausted")
        return tuple(outs), used, fmax.value


# ---------------------------------------------------------------- learned proposal
def mlp_num_params():
    return lib().or_mlp_num_params()


def mlp_forward(theta, x):
    """g(x) of the proposal MLP (x: n x 4 in [-1, 1]^4)."""
    th = _f64(theta)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 4)
    g = np.zeros(len(x))
    lib().or_mlp_forward(_pd(th), _pd(x), len(x), _pd(g))
    return g


def mlp_loss_grad(theta, xd, xu):
    """KL objective -mean ln g(xd) + ln(16 mean g(xu)) and its gradient."""
    th = _f64(theta)
    xd = np.ascontiguousarray(xd, dtype=np.float64).reshape(-1, 4)
    xu = np.ascontiguousarray(xu, dtype=np.float64).reshape(-1, 4)
    g = np.zeros(mlp_num_params())
    loss = C.c_double()
    lib().or_mlp_loss_grad(_pd(th), _pd(xd), len(xd), _pd(xu), len(xu), C.byref(loss), _pd(g))
    return loss.value, g


def adam_step(theta, m, v, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of theta, m, v (float64 arrays)."""
    lib().or_adam_step(_pd(theta), _pd(m), _pd(v), _pd(_f64(grad)), len(theta), lr, beta1, beta2,
                       eps, int(t))


def tpl_value(hist, x, y):
    """Content of a workloads.Hist2D template at (x, y) by the oracle's bin rule."""
    h = _f64(np.ravel(hist.h))
    r = _f64(hist.range)
    return lib().or_tpl_value(_pd(h), hist.nx, hist.ny, _pd(r), float(x), float(y))


def grid_sample(gc, nb, alpha, seed, n, masses=None, box=None):
    """Samples of the grid proposal: (m, cK, cpsi, phi) FP32, weights p q / density, cells."""
    import workloads as W
    masses = W.PARTICLE_MASSES if masses is None else masses
    box = (W.M_LO, W.M_HI) if box is None else box
    gcv = _f64(gc)
    nbv = np.ascontiguousarray(nb, dtype=np.int32)
    outs = [np.zeros(n, np.float32) for _ in range(4)]
    w = np.zeros(n)
    cell = np.zeros(n, np.int64)
    lib().or_grid_sample(_pd(gcv), _pi(nbv), float(alpha), int(seed), int(n), box[0], box[1],
                         *masses, *(_pf(a) for a in outs), _pd(w),
                         cell.ctypes.data_as(C.POINTER(C.c_int64)))
    return tuple(outs), w, cell
