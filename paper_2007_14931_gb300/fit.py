"""Host-side fit loop: a MIGRAD-style variable-metric minimiser fed by the
analytic gradient of the GPU likelihood.

The paper's fit (Introduction) runs MINUIT on the host and evaluates the NLL on
the device at every step.  Here the device returns the NLL *and* its adjoint
gradient, so each iteration costs one evaluation instead of 2P + 1.

Minimiser (after the MINUIT reference manual's description of MIGRAD):
  * inverse-Hessian estimate V, started from finite differences of the
    analytic gradient along each axis (diagonal second derivatives);
  * step dx = -V g, parabolic line search on the step length;
  * BFGS update of V from (dx, dg);
  * stop when the estimated distance to minimum EDM = g^T V g / 2 is below
    0.002 * tolerance * errordef (errordef = 1 for -2 ln L, tolerance 0.1).
HESSE: the covariance 2 H^-1 (errordef 1 for -2 ln L) with H from central
differences of the analytic gradient.

Parametrisation: the couplings can be fitted as (|H|, arg H) -- the amplitudes
and phases the paper reports (Figs. 5-6) -- or as (Re, Im); the K*(892)
lambda = 0 coupling is fixed to 1 (Eq. 6).  Masses and widths of floated
resonances are fitted directly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Parametrization:
    """Maps free fit variables theta <-> the ABI parameter vector p."""
    n_cols: int
    n_mg: int
    fixed_col: int | None = None       # column with the fixed coupling (Eq. 6)
    polar: bool = True

    @property
    def n_free(self):
        return 2 * self.n_cols - (2 if self.fixed_col is not None else 0) + self.n_mg

    def _cols(self):
        return [k for k in range(self.n_cols) if k != self.fixed_col]

    def to_params(self, theta, fixed_value=1.0 + 0j):
        theta = np.asarray(theta, dtype=np.float64)
        p = np.empty(2 * self.n_cols + self.n_mg)
        i = 0
        for k in range(self.n_cols):
            if k == self.fixed_col:
                c = fixed_value
            elif self.polar:
                c = theta[i] * complex(math.cos(theta[i + 1]), math.sin(theta[i + 1]))
                i += 2
            else:
                c = complex(theta[i], theta[i + 1])
                i += 2
            p[2 * k], p[2 * k + 1] = c.real, c.imag
        p[2 * self.n_cols:] = theta[i:]
        return p

    def from_params(self, p):
        th = []
        for k in self._cols():
            c = complex(p[2 * k], p[2 * k + 1])
            th += [abs(c), math.atan2(c.imag, c.real)] if self.polar else [c.real, c.imag]
        th += list(p[2 * self.n_cols:])
        return np.array(th)

    def grad_to_theta(self, theta, gp):
        """Chain rule dNLL/dtheta from dNLL/dp."""
        theta = np.asarray(theta)
        g = np.empty(self.n_free)
        i = 0
        for k in self._cols():
            gr, gi = gp[2 * k], gp[2 * k + 1]
            if self.polar:
                r, ph = theta[i], theta[i + 1]
                c, s = math.cos(ph), math.sin(ph)
                g[i] = gr * c + gi * s
                g[i + 1] = r * (-gr * s + gi * c)
            else:
                g[i], g[i + 1] = gr, gi
            i += 2
        g[i:] = gp[2 * self.n_cols:]
        return g


@dataclass
class MinResult:
    x: np.ndarray
    fval: float
    edm: float
    nfcn: int
    niter: int
    converged: bool
    V: np.ndarray
    history: list = field(default_factory=list)


def migrad(fg, x0, tol=0.1, errordef=1.0, maxiter=500, init_step=None, V0=None, f_noise=None):
    """Minimise f with gradient: fg(x) -> (f, g).  Returns a MinResult.  V0: an
    initial inverse-Hessian estimate (positive definite), e.g. from HESSE.

    f_noise: the absolute rounding noise of f (default 1e-9 |f(x0)|).  A sum of
    millions of single-precision log-likelihood terms carries noise of order
    1e-3, as large as the decreases left near the minimum, where the sufficient-
    decrease test on f alone then fails at random.  A step whose expected
    decrease is below 10 f_noise is therefore also accepted when f has not risen
    by more than the noise and the directional derivative has shrunk,
    |g(x + a dx) . dx| < |g(x) . dx|: the gradient is accurate where f is not.
    """
    x = np.array(x0, dtype=np.float64)
    n = len(x)
    f, g = fg(x)
    nfcn = 1
    if not math.isfinite(f):
        raise ValueError("starting point has a non-finite function value")
    if f_noise is None:
        f_noise = 1e-9 * max(abs(f), 1.0)
    if V0 is not None:
        V = np.array(V0, dtype=np.float64)
        diag = 1.0 / np.maximum(np.diag(V), 1e-300)
    else:
        # Initial V from the diagonal of the Hessian (forward differences of the gradient).
        h = np.array(init_step if init_step is not None else 1e-4 * np.maximum(np.abs(x), 1e-2))
        diag = np.empty(n)
        for i in range(n):
            xp = x.copy()
            xp[i] += h[i]
            fp, gpi = fg(xp)
            nfcn += 1
            d = (gpi[i] - g[i]) / h[i]
            diag[i] = d if d > 0 else abs(g[i]) / max(abs(h[i]), 1e-12) + 1.0
        V = np.diag(1.0 / diag)
    edm_stop = 0.002 * tol * errordef
    hist = []
    converged = False
    it = 0
    for it in range(1, maxiter + 1):
        edm = 0.5 * g @ V @ g
        hist.append((f, edm))
        if edm < edm_stop:
            converged = True
            break
        dx = -V @ g
        slope = g @ dx
        if slope >= 0:  # V lost positive definiteness: restart from the diagonal
            V = np.diag(1.0 / diag)
            dx = -V @ g
            slope = g @ dx
        # Parabolic line search on alpha in f(x + alpha dx).
        alpha, f_new, g_new = 1.0, None, None
        for _ in range(8):
            xn = x + alpha * dx
            fn, gn = fg(xn)
            nfcn += 1
            if math.isfinite(fn) and fn <= f + 1e-4 * alpha * slope:
                f_new, g_new = fn, gn
                break
            if (math.isfinite(fn) and -alpha * slope < 10.0 * f_noise and fn <= f + 10.0 * f_noise
                    and abs(gn @ dx) < abs(slope)):
                f_new, g_new = fn, gn   # within the noise of f: decided by the gradient
                break
            if math.isfinite(fn):
                # minimum of the parabola through f(0), f'(0) = slope, f(alpha)
                den = 2.0 * (fn - f - slope * alpha)
                a2 = -slope * alpha * alpha / den if den > 0 else 0.1 * alpha
                alpha = min(max(a2, 0.1 * alpha), 0.5 * alpha)
            else:
                alpha *= 0.25
        if f_new is None:
            break
        s = xn - x
        y = g_new - g
        sy = s @ y
        if sy > 1e-300:
            rho = 1.0 / sy
            I = np.eye(n)
            V = (I - rho * np.outer(s, y)) @ V @ (I - rho * np.outer(y, s)) + rho * np.outer(s, s)
        x, f, g = xn, f_new, g_new
    edm = 0.5 * g @ V @ g
    return MinResult(x, f, edm, nfcn, it, converged or edm < edm_stop, V, hist)


def hesse(gfun, x, step=None):
    """Covariance of -2 ln L fit results: 2 H^-1 with H from central differences of
    the gradient (errordef = 1)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    h = step if step is not None else 1e-4 * np.maximum(np.abs(x), 1e-2)
    H = np.empty((n, n))
    for i in range(n):
        xp, xm = x.copy(), x.copy()
        xp[i] += h[i]
        xm[i] -= h[i]
        H[:, i] = (gfun(xp) - gfun(xm)) / (2 * h[i])
    H = 0.5 * (H + H.T)
    return 2.0 * np.linalg.inv(H), H


def nll_function():
    """torch.autograd.Function computing -2 ln L and its gradient with the GPU model."""
    import torch

    class Amp4dNLL(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params, model):
            p = params.detach().cpu().numpy().astype(np.float64)
            nll, g = model.eval_nll_grad(p)
            ctx.save_for_backward(torch.from_numpy(g).to(params.device, params.dtype))
            return torch.tensor(nll, dtype=params.dtype, device=params.device)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g, None

    return Amp4dNLL


@dataclass
class FitResult:
    params: np.ndarray
    theta: np.ndarray
    errors: np.ndarray
    cov: np.ndarray
    fval: float
    edm: float
    nfcn: int
    converged: bool
    hessian: np.ndarray | None = None   # H of -2 ln L at the minimum (HESSE), if computed

    def well_constrained(self, rel=1e-6):
        """Eigen-decomposition of the Hessian restricted to the directions the data
        constrain: (eigenvalues, eigenvectors as columns) with lambda > rel lambda_max.
        Weak modes (a spin-4 state near the kinematic edge, interference ambiguities)
        have curvature near zero or, within the gradient's rounding noise, below it."""
        w, V = np.linalg.eigh(self.hessian)
        keep = w > rel * w.max()
        return w[keep], V[:, keep]


def _two_pass_hesse(gfun, x):
    """H of -2 ln L at x from central differences of the gradient, in two passes
    (as MINUIT scales its steps to the curvature): a small fixed step gives the
    diagonal of H (large signal), then the full H is differenced over 0.2 of each
    parameter's conditional standard error sqrt(2 / H_ii).  A step of a fixed
    small fraction of |theta| leaves the off-diagonal differences too close to
    the gradient's FP32 rounding noise once the data set is large."""
    h0 = 1e-4 * np.maximum(np.abs(x), 1e-2)
    hd = np.empty(len(x))
    for i in range(len(x)):
        xp, xm = x.copy(), x.copy()
        xp[i] += h0[i]
        xm[i] -= h0[i]
        hd[i] = (gfun(xp)[i] - gfun(xm)[i]) / (2 * h0[i])
    step = np.where(hd > 0, 0.2 * np.sqrt(2.0 / np.where(hd > 0, hd, 1.0)), h0)
    cov, H = hesse(gfun, x, step=step)
    return cov, H, 4 * len(x)


def _regularised_inverse(H, rel=1e-6):
    """H^-1 with every eigenvalue floored at rel lambda_max: weak modes (curvature
    near zero, or below it within the gradient's noise) take bounded steps."""
    w, V = np.linalg.eigh(H)
    w = np.maximum(w, rel * w.max())
    return (V / w) @ V.T


def fit(eval_nll_grad, par: Parametrization, start_params, tol=0.1, with_hesse=True, maxiter=500,
        max_rounds=4):
    """Fit with a model's NLL + gradient callable (params -> (nll, grad)).

    MIGRAD, then HESSE; as in MINUIT, when the estimated distance to the minimum
    computed with the HESSE matrix (EDM = g^T H^-1 g / 2) is above the tolerance,
    MIGRAD runs again from the HESSE matrix (the variable-metric estimate can be
    far from the curvature in strongly correlated directions).  Works with the
    GPU model (``Model.eval_nll_grad``) or any other callable of the same
    signature.
    """
    def fg(theta):
        p = par.to_params(theta)
        f, gp = eval_nll_grad(p)
        return f, par.grad_to_theta(theta, gp)

    gfun = lambda t: fg(t)[1]
    edm_stop = 0.002 * tol
    th0 = par.from_params(start_params)
    r = migrad(fg, th0, tol=tol, maxiter=maxiter)
    cov = r.V * 2.0
    nf = r.nfcn
    H = None
    edm, converged = r.edm, r.converged
    if with_hesse:
        for _ in range(max_rounds):
            cov, H, k = _two_pass_hesse(gfun, r.x)
            nf += k
            Hinv = _regularised_inverse(H)
            g = gfun(r.x)
            nf += 1
            edm = 0.5 * g @ Hinv @ g
            converged = edm < edm_stop
            if converged:
                break
            r = migrad(fg, r.x, tol=tol, maxiter=maxiter, V0=Hinv)
            nf += r.nfcn
    err = np.sqrt(np.maximum(np.diag(cov), 0.0))
    return FitResult(par.to_params(r.x), r.x, err, cov, r.fval, edm, nf, converged, H)
