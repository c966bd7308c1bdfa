"""Benchmark of the amplitude-fit hot path: NLL + gradient evaluations per second.

One step = one evaluation of -2 ln L and its full gradient (couplings and the
floated masses/widths) over every data event and every normalisation point of
the workload, at a new parameter point.  Default workload: 10 K* + Z(4430),
5e6 data events, 2^24 uniform normalisation points, Z mass and width floating.

  value      device throughput: steps enqueued back to back through the C ABI
             (amp4d_enqueue_eval, parameters already in device memory), timed
             with CUDA events on the launching stream.
  e2e        the same steps through the synchronous user call
             amp4d_eval_nll_grad: parameters copied from pinned host memory and
             NLL + gradient read back to the host inside every step.
  roofline   the dominant kernel (the data-side adjoint kernel), with its mean
             launch time from CUDA events recorded around it inside the timed
             region, against both ceilings: algorithmic bytes per event (FP32
             records + cached lineshapes) x events / time against the measured
             HBM copy bandwidth, and formula flops per event x events / time
             against the FP32 FMA peak of 152 SMs x 128 lanes x 2 flop x
             2.07 GHz.  The line reports the larger fraction as the bound and
             keeps the other as alu_frac / hbm_frac.
  cpu_baseline  the FP64 oracle on a bounded sample of the same workload, scaled
             to the full workload; the GPU's NLL and gradient on that sample at
             the same parameter point are compared with the oracle's.
  fit        a closure fit at full size (events drawn from the model by the GPU
             generator, 50 free parameters from a perturbed start): time, function
             calls, convergence and pulls against the generating values.

--impl reference times the FP64 oracle (the reference arm) on the same config.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # FMA lanes x 2 flop x max SM clock
METRIC = "NLL+grad evals/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# Formula flop count per event of the adjoint kernel (FP32, FMA = 2 flop,
# special-function ops counted as 1 each).  Derived from the per-event
# arithmetic of Eq. 2-5, 10-12 as written in the kernels:
#   per lineshape (Eq. 2-3):      barrier polynomials, 1/sqrt, powers, width,
#                                 (M-m)(M+m), 1/|D|^2, A            ~ 46 + 4 SFU
#   per K* column (Eq. 4-5):      d_l scaling + hi/lo complex MAC      14
#   K* angular set-up:            sqrt x2, d^1 table, Psi              ~ 40 + 2 SFU
#   coherent sum a_xi:            3 complex MAC x 2 xi                 24
#   Z angular set-up (Eq. 10):    sqrt x2, d^1 table                    ~ 20 + 3 SFU
#   per Z (Eq. 10-11):            Om0, Om1 (x 2 xi), hi/lo MAC          ~ 70
#   |a|^2, ln S (split)           ~ 12 + 2 SFU
# adjoint (gradient):
#   v_l                           3 x 2 complex conj-MAC               24
#   per K* column                 complex scale + mul + 2 accumulates  14
#   per floated K* (M, G0)        y, dA/dM, dA/dG0, 2 accumulates      ~ 40
#   per Z                         w0, w1, 2 complex mul, 4 accumulates  ~ 40 (+ 40 if floated)
# ---------------------------------------------------------------------------
def flops_per_event(res_list, float_names, grad=True, cached=False):
    """cached: lineshapes of fixed resonances come from the basis cache."""
    nK = sum(1 for r in res_list if r.chain == W.CHAIN_KSTAR)
    nZ = len(res_list) - nK
    colsK = sum(1 if r.J == 0 else 3 for r in res_list if r.chain == W.CHAIN_KSTAR)
    n_line = sum(1 for r in res_list if r.name in float_names) if cached else nK + nZ
    f = 50 * n_line + 14 * colsK + 44 + 24 + 14
    if nZ:
        f += 23 + 70 * nZ
    if grad:
        f += 24 + 14 * colsK
        f += sum(40 for r in res_list if r.chain == W.CHAIN_KSTAR and r.name in float_names)
        f += 40 * nZ + sum(40 for r in res_list if r.chain == W.CHAIN_Z and r.name in float_names)
    return f


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) per data event of the cached adjoint kernel, from one
# ncu capture on 4e6 events of the same model, with the SHA-256 (first 16 hex
# digits) of the kernel sources it was taken on.  Scaled by events to the
# launch; reported as null when the sources have changed since.
K_GRAD_SOURCES = ("paper_2007_14931_gb300/csrc/amp4d_eval.cuh",
                  "paper_2007_14931_gb300/csrc/amp4d_device.cuh",
                  "paper_2007_14931_gb300/csrc/amp4d_finish.cuh")
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_grad_fx launch on 4e6
# events of `large` (544.12 MB + 3.27 MB), per event; valid for these sources only
K_GRAD_TRAFFIC = {"bytes_per_event": (544.121856e6 + 3.26912e6) / 4e6, "sources_sha16": "af101cab03cc6bf9"}


def kernel_sources_sha16():
    import hashlib
    h = hashlib.sha256()
    for f in K_GRAD_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def bytes_per_event(res_list, cached=True, float_names=(), norm=False):
    """Algorithmic bytes read per event (or normalisation point) by the adjoint
    kernel: the FP32 records it reads and, on the cached path, one complex FP32
    lineshape per fixed resonance and the four complex Z-chain angular factors of
    each Z.  Records: 17 with a Z, 8 without.  The cached kernel reads cos/sin phi
    instead of phi, none of the six Z-chain angle records, the K pi mass and
    momenta only when a K* lineshape is computed per event, and the J/psi pi mass
    and momenta only when a Z lineshape is; normalisation points add their weight."""
    n_z = sum(1 for r in res_list if r.chain == W.CHAIN_Z)
    nrec = 17 if n_z else 8
    n_fixed = len(res_list)
    if cached:
        fl = [r for r in res_list if r.name in float_names]
        n_fixed -= len(fl)
        nrec -= 1                                                  # phi
        if not any(r.chain == W.CHAIN_KSTAR for r in fl):
            nrec -= 3                                              # m, p, q
        if n_z:
            nrec -= 6                                              # the Z angles (cached factors)
            if not any(r.chain == W.CHAIN_Z for r in fl):
                nrec -= 3                                          # m_psi pi, p_Z, q_Z
    return 4 * (nrec + (1 if norm else 0)) + ((8 * n_fixed + 32 * n_z) if cached else 0)


def make_workload(cfg, rank=0):
    res = cfg.resonances
    c = W.draw_couplings(res, cfg.coupling_seed)
    params = W.couplings_to_params(c, W.float_mg_values(res, cfg.float_mg))
    ev = W.peaked_points(cfg.n_events, cfg.data_seed + 1000 * rank, res)
    nm = W.uniform_points(cfg.n_norm, cfg.norm_seed + 1000 * rank)
    return res, params, ev, nm


def step_params(params, k, n_col):
    """Parameter point of step k: couplings rotated/scaled slightly (a new point per step)."""
    p = params.copy()
    s = 1.0 + 1e-3 * math.sin(0.7 * k)
    p[:2 * n_col] *= s
    return p


def oracle_baseline(cfg, frac, A=None, reps_min_s=10.0, max_reps=30):
    """FP64 oracle NLL+grad on a 1/frac sample of the workload; evals/s scaled to full size.
    With the GPU package A, the GPU's NLL and gradient on the same sample at the
    oracle's last parameter point are compared with the oracle's."""
    import oracle as O
    res, params, ev, nm = make_workload(cfg)
    n_s = max(1, cfg.n_events // frac)
    m_s = max(1, cfg.n_norm // frac)
    evs = tuple(a[:n_s] for a in ev)
    nms = tuple(a[:m_s] for a in nm)
    om = O.Model(res, float_names=cfg.float_mg)
    t0 = time.perf_counter()
    reps = 0
    while True:
        p_last = step_params(params, reps, om.n_cols)
        nll_o, g_o, _, rc = om.nll(p_last, evs, nms, grad=True)
        reps += 1
        if time.perf_counter() - t0 > reps_min_s or reps >= max_reps:
            break
    dt = (time.perf_counter() - t0) / reps
    full = dt * (cfg.n_events + cfg.n_norm) / (n_s + m_s)
    out = {"value": 1.0 / full, "unit": METRIC, "cores": O.num_threads(), "kind": "oracle",
           "sample": "%d events + %d normalisation points per eval (1/%d of the workload), "
                     "%d evals, time scaled by events+points" % (n_s, m_s, frac, reps),
           "extrapolated": True, "sec_per_sample_eval": dt}
    if A is not None and rc == 0:
        import torch
        gm = A.Model(res, float_names=cfg.float_mg, path=A.AMP4D_PATH_CACHED)
        gm.set_events(*(torch.from_numpy(a).cuda() for a in evs))
        gm.set_norm_points(*(torch.from_numpy(a).cuda() for a in nms))
        nll_g, g_g = gm.eval_nll_grad(p_last)
        out["gpu_vs_oracle_on_sample"] = {
            "nll_oracle": float(nll_o), "delta_nll": float(nll_g - nll_o),
            "max_abs_dgrad_over_gradmax": float(np.max(np.abs(g_g - g_o)) / np.max(np.abs(g_o)))}
    return out


def full_fit(cfg, A, seed=2718, tol=0.1):
    """Closure fit at the workload's full size: events drawn from the model at the
    workload's couplings by the GPU generator, fitted from a perturbed start by
    the variable-metric minimiser with the analytic GPU gradient."""
    import torch
    import paper_2007_14931_gb300.fit as F
    res = cfg.resonances
    cols = W.columns(res)
    c = W.draw_couplings(res, cfg.coupling_seed)
    fixed = [k for k, (R, l) in enumerate(cols) if res[R].name == "K*(892)" and l == 0][0]
    c = c / c[fixed]     # reference coupling 1 (Eq. 6); the NLL is invariant under a global scale
    mg = W.float_mg_values(res, cfg.float_mg)
    p_true = W.couplings_to_params(c, mg)
    gen = A.Model(res, float_names=cfg.float_mg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev = gen.generate(p_true, cfg.n_events, seed)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    del gen
    nm = W.uniform_points(cfg.n_norm, cfg.norm_seed)
    m = A.Model(res, float_names=cfg.float_mg, path=A.AMP4D_PATH_CACHED)
    m.set_events(*ev)
    m.set_norm_points(*(torch.from_numpy(a).cuda() for a in nm))
    par = F.Parametrization(len(c), len(mg), fixed_col=fixed, polar=True)
    c0 = W.perturbed_start(c)
    c0[fixed] = 1.0
    p0 = W.couplings_to_params(c0, mg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = F.fit(m.eval_nll_grad, par, p0, tol=tol)
    t_fit = time.perf_counter() - t0
    d = r.theta - par.from_params(p_true)
    nph = 2 * (len(c) - 1)
    d[1:nph:2] = (d[1:nph:2] + math.pi) % (2 * math.pi) - math.pi
    # Pulls along the Hessian eigen-directions the data constrain (eigenvalue above
    # 1e-6 of the largest): this model has weak modes (the K4*(2045) helicity-1
    # couplings near the kinematic edge) whose errors are not meaningful.
    lam, V = r.well_constrained()
    pulls = (V.T @ d) * np.sqrt(lam / 2.0)
    # The normalisations are compared from one reference minimum: the fit with the
    # first uniform sample started at the generating point.  The likelihood of this
    # 50-parameter model has secondary minima, and a fit from the perturbed start can
    # reach one of them depending on the normalisation sample, which says nothing
    # about the accuracy of the normalisation itself (chi2 measure below:
    # perturbed_start_vs_reference).
    r_t = F.fit(m.eval_nll_grad, par, p_true, tol=tol)
    p_u = par.to_params(r_t.theta)
    # The same fit with an independent uniform normalisation sample: the spread
    # between the two minima, in the same units, is the statistical error of the
    # Monte Carlo normalisation integral (N/M = events / points).
    nm2 = W.uniform_points(cfg.n_norm, cfg.norm_seed + 7919)
    m.set_norm_points(*(torch.from_numpy(a).cuda() for a in nm2))
    r2 = F.fit(m.eval_nll_grad, par, p_u, tol=tol)
    d2 = r2.theta - r_t.theta
    d2[1:nph:2] = (d2[1:nph:2] + math.pi) % (2 * math.pi) - math.pi
    spread = (V.T @ d2) * np.sqrt(lam / 2.0)
    # The same fit normalised by the learned proposal: the MLP density trained on
    # 2^20 of the generated events, 2^24 importance-sampled points with weights
    # p q / q (two independent samples).
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m.proposal_train(tuple(t[:1 << 20] for t in ev), seed=11)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # The learned-normalisation fits start from the reference minimum.
    learned = []
    for sd in (101, 102):
        pts, w = m.proposal_sample(cfg.n_norm, sd)
        m.set_norm_points(*pts, w=w, volume=1.0)
        rl = F.fit(m.eval_nll_grad, par, p_u, tol=tol)
        dl = rl.theta - par.from_params(p_true)
        dl[1:nph:2] = (dl[1:nph:2] + math.pi) % (2 * math.pi) - math.pi
        learned.append((rl, dl))
    pl = [(V.T @ dl) * np.sqrt(lam / 2.0) for _, dl in learned]
    dll = learned[1][0].theta - learned[0][0].theta
    dll[1:nph:2] = (dll[1:nph:2] + math.pi) % (2 * math.pi) - math.pi
    spread_l = (V.T @ dll) * np.sqrt(lam / 2.0)
    # A proposal aimed at the whole Gram matrix rather than at S: trained on the
    # mixture sum_k |B_k|^2 p q (per-column samples mixed by the Gram diagonal).
    m.set_norm_points(*(torch.from_numpy(a).cuda() for a in nm))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m.proposal_train_gram(p_true, n=1 << 20, seed=12)
    torch.cuda.synchronize()
    t_train_g = time.perf_counter() - t0
    gram_t = []
    for sd in (201, 202):
        pts, w = m.proposal_sample(cfg.n_norm, sd)
        m.set_norm_points(*pts, w=w, volume=1.0)
        rg = F.fit(m.eval_nll_grad, par, p_u, tol=tol)
        dg = rg.theta - par.from_params(p_true)
        dg[1:nph:2] = (dg[1:nph:2] + math.pi) % (2 * math.pi) - math.pi
        gram_t.append((rg, dg))
    pg = [(V.T @ dg) * np.sqrt(lam / 2.0) for _, dg in gram_t]
    # the first Gram-targeted sample, fitted from the perturbed start instead
    pts, w = m.proposal_sample(cfg.n_norm, 201)
    m.set_norm_points(*pts, w=w, volume=1.0)
    rp = F.fit(m.eval_nll_grad, par, p0, tol=tol)
    dp = rp.theta - par.from_params(p_true)
    dp[1:nph:2] = (dp[1:nph:2] + math.pi) % (2 * math.pi) - math.pi
    zp = (V.T @ dp) * np.sqrt(lam / 2.0)
    du = rp.theta - r_t.theta
    du[1:nph:2] = (du[1:nph:2] + math.pi) % (2 * math.pi) - math.pi
    zu = (V.T @ du) * np.sqrt(lam / 2.0)
    dgg = gram_t[1][0].theta - gram_t[0][0].theta
    dgg[1:nph:2] = (dgg[1:nph:2] + math.pi) % (2 * math.pi) - math.pi
    spread_g = (V.T @ dgg) * np.sqrt(lam / 2.0)
    shift_u = []
    for rg, _ in gram_t:
        dd = rg.theta - r_t.theta
        dd[1:nph:2] = (dd[1:nph:2] + math.pi) % (2 * math.pi) - math.pi
        shift_u.append(float(np.sqrt(np.mean(((V.T @ dd) * np.sqrt(lam / 2.0)) ** 2))))
    gram_out = {"proposal_train_s": t_train_g,
                "converged": [bool(rg.converged) for rg, _ in gram_t],
                "rms_pull_vs_truth": [float(np.sqrt(np.mean(x ** 2))) for x in pg],
                "max_abs_pull_vs_truth": [float(np.max(np.abs(x))) for x in pg],
                "rms_shift_between_normalisation_samples": float(np.sqrt(np.mean(spread_g ** 2))),
                "rms_shift_to_uniform_minimum": shift_u,
                "from_perturbed_start": {"converged": bool(rp.converged),
                                         "rms_pull_vs_truth": float(np.sqrt(np.mean(zp ** 2))),
                                         "rms_shift_to_uniform_minimum": float(np.sqrt(np.mean(zu ** 2))),
                                         "fval_minus_uniform_fit_fval_on_this_sample":
                                             float(rp.fval - gram_t[0][0].fval)},
                "note": "proposal trained on sum_k |B_k|^2 p q (per-column samples mixed by G_kk); "
                        "fits start from the reference minimum"}
    # Hessian-free measures on the likelihood of the first uniform sample (f = -2 ln L):
    # the sum of squared pulls of a minimum against the truth is f(truth) - f(min),
    # and the squared distance between two minima a, b in units of the errors is
    # 2 [f(a) + f(b) - 2 f((a + b) / 2)] (exact for a quadratic f), each per free
    # parameter.  Unlike the eigen-direction pulls they do not depend on the
    # finite-difference HESSE matrix.
    m.set_norm_points(*(torch.from_numpy(a).cuda() for a in nm))

    def f_at(th):
        return m.eval_nll(par.to_params(th))

    def midpoint(a, b):
        dd = b - a
        dd[1:nph:2] = (dd[1:nph:2] + math.pi) % (2 * math.pi) - math.pi
        return a + 0.5 * dd

    def shift_chi2(a, b):
        return 2.0 * (f_at(a) + f_at(b) - 2.0 * f_at(midpoint(a, b))) / par.n_free

    th_true = par.from_params(p_true)
    f_ref = f_at(r_t.theta)

    def loss(th):
        return (f_at(th) - f_ref) / par.n_free

    chi2 = {"loss_vs_reference": {
                "note": "[f(theta) - f(reference)] / n_free on the first uniform sample's "
                        "likelihood: the mean squared shift in standard deviations for a "
                        "quadratic f; needs neither a Hessian nor convexity between minima",
                "perturbed_start": loss(r.theta), "uniform_sample_2": loss(r2.theta),
                "learned_S": [loss(x.theta) for x, _ in learned],
                "gram_targeted": [loss(x.theta) for x, _ in gram_t]},
            "truth_vs_uniform_fit": (f_at(th_true) - f_at(r.theta)) / par.n_free,
            "perturbed_start_vs_reference": shift_chi2(r.theta, r_t.theta),
            "uniform_sample_shift": shift_chi2(r_t.theta, r2.theta),
            "learned_S_vs_reference": [shift_chi2(r_t.theta, x.theta) for x, _ in learned],
            "learned_S_sample_shift": shift_chi2(learned[0][0].theta, learned[1][0].theta),
            "gram_targeted_vs_reference": [shift_chi2(r_t.theta, x.theta) for x, _ in gram_t],
            "gram_targeted_sample_shift": shift_chi2(gram_t[0][0].theta, gram_t[1][0].theta),
            "note": "per free parameter, on the first uniform sample's likelihood; 1 is one "
                    "standard deviation per parameter, negative means another valley; the "
                    "reference is the first uniform sample's fit from the generating point"}
    learned_out = {"proposal_train_s": t_train,
                   "converged": [bool(rl.converged) for rl, _ in learned],
                   "rms_pull_vs_truth": [float(np.sqrt(np.mean(x ** 2))) for x in pl],
                   "max_abs_pull_vs_truth": [float(np.max(np.abs(x))) for x in pl],
                   "rms_shift_between_normalisation_samples": float(np.sqrt(np.mean(spread_l ** 2)))}
    return {"events": cfg.n_events, "normalisation_points": cfg.n_norm, "free_parameters": par.n_free,
            "generation_s": t_gen, "fit_s": t_fit, "nfcn": int(r.nfcn), "converged": bool(r.converged),
            "edm": float(r.edm), "fval": float(r.fval),
            "evals_per_s_in_fit": r.nfcn / t_fit,
            "constrained_directions": int(len(lam)),
            "max_abs_pull_vs_truth": float(np.max(np.abs(pulls))),
            "rms_pull_vs_truth": float(np.sqrt(np.mean(pulls ** 2))),
            "rms_shift_between_normalisation_samples": float(np.sqrt(np.mean(spread ** 2))),
            "events_over_points": cfg.n_events / cfg.n_norm,
            "learned_normalisation": learned_out,
            "gram_targeted_normalisation": gram_out,
            "chi2_per_free_parameter": chi2,
            "note": "GPU closure fit: MIGRAD-style variable metric with the analytic adjoint gradient, "
                    "HESSE (re-run from the HESSE matrix until its EDM is below tolerance); pulls in "
                    "units of the statistical error along the Hessian directions the data constrain; "
                    "the uniform-MC normalisation error adds to them (shift between two "
                    "normalisation samples reported beside)"}


def real_life_fit(A, seed=3141, tol=0.1):
    """The paper's real-life test (Eq. 14): 10 K* + Z(4200) + Z(4430) with a
    relative efficiency and 15 % background.  10^6 events are drawn from the Eq. 14
    PDF by the GPU generator and fitted from a perturbed start with the same
    efficiency and background model; the evaluation rate of the Eq. 14 path and
    the Z fit fractions (defined on S, from a model without templates) are reported."""
    import torch
    import paper_2007_14931_gb300.fit as F
    cfg = W.CONFIGS["real_life"]
    res = cfg.resonances
    cols = W.columns(res)
    c = W.draw_couplings(res, cfg.coupling_seed, z_scale=cfg.z_scale)
    fixed = [k for k, (R, l) in enumerate(cols) if res[R].name == "K*(892)" and l == 0][0]
    c = c / c[fixed]
    p_true = W.couplings_to_params(c)
    em, ea, bm, ba, P = W.eq14_templates(cfg.template_seed)

    def model(points_seed, path=A.AMP4D_PATH_CACHED, templates=True):
        m = A.Model(res, path=path)
        m.set_norm_points(*(torch.from_numpy(a).cuda() for a in W.uniform_points(cfg.n_norm, points_seed)))
        if templates:
            m.set_efficiency(em, ea)
            m.set_background(bm, ba, P)
        return m

    gen = model(cfg.norm_seed + 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev = gen.generate(p_true, cfg.n_events, seed)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    gen.close()
    m = model(cfg.norm_seed)
    m.set_events(*ev)
    # evaluation rate of the Eq. 14 path (NLL + gradient, parameters on the device)
    P_ = m.n_params
    K = 30
    pts = np.stack([step_params(p_true, k, m.n_cols) for k in range(K + 5)])
    p_dev = torch.from_numpy(pts).cuda()
    out_dev = torch.zeros((K + 5, 6 + P_), dtype=torch.float64, device="cuda")
    ms = _timed(m, A, p_dev, out_dev, A.AMP4D_EVAL_NLL_GRAD, K, 5, torch.cuda.current_stream())
    par = F.Parametrization(len(c), 0, fixed_col=fixed, polar=True)
    c0 = W.perturbed_start(c)
    c0[fixed] = 1.0
    p0 = W.couplings_to_params(c0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = F.fit(m.eval_nll_grad, par, p0, tol=tol)
    t_fit = time.perf_counter() - t0
    d = r.theta - par.from_params(p_true)
    nph = 2 * (len(c) - 1)
    d[1:nph:2] = (d[1:nph:2] + math.pi) % (2 * math.pi) - math.pi
    lam, V = r.well_constrained()
    pulls = (V.T @ d) * np.sqrt(lam / 2.0)
    p_fit = par.to_params(r.theta)
    m.close()
    ffm = model(cfg.norm_seed, templates=False)
    ff_true = ffm.fit_fractions(p_true)
    ff_fit = ffm.fit_fractions(p_fit)
    zi = [i for i, rr in enumerate(res) if rr.chain == W.CHAIN_Z]
    ffm.close()
    return {"events": cfg.n_events, "normalisation_points": cfg.n_norm, "purity": P,
            "free_parameters": par.n_free, "generation_s": t_gen,
            "eq14_evals_per_s": K / (ms / 1e3),
            "fit_s": t_fit, "nfcn": int(r.nfcn), "converged": bool(r.converged),
            "constrained_directions": int(len(lam)),
            "rms_pull_vs_truth": float(np.sqrt(np.mean(pulls ** 2))),
            "max_abs_pull_vs_truth": float(np.max(np.abs(pulls))),
            "fit_fraction_Z": {res[i].name: {"generated": float(ff_true[i]), "fitted": float(ff_fit[i])}
                               for i in zi},
            "note": "events drawn from the Eq. 14 PDF (efficiency x signal + 15 % background, "
                    "Bernstein templates binned 2D masses x 2D angles) and fitted with it; pulls along "
                    "the constrained Hessian directions, the uniform-MC normalisation error included"}


def z_sensitivity_fit(A, n_events=1_000_000, n_norm=1 << 22, seed=2020, tol=0.1):
    """The paper's Z-sensitivity test: events generated with the ten K* alone,
    fitted with the ten K* + Z(4200) + Z(4430) model (Cartesian couplings, the Z
    starting at |H| = 0.02); the fitted Z fit fractions should be near zero."""
    import torch
    import paper_2007_14931_gb300.fit as F
    res_g = W.CONFIGS["kstar10"].resonances
    res_f = W.CONFIGS["kstar10_2z"].resonances
    cols_g, cols_f = W.columns(res_g), W.columns(res_f)
    fixed = [k for k, (R, l) in enumerate(cols_g) if res_g[R].name == "K*(892)" and l == 0][0]
    c_g = W.draw_couplings(res_g, W.CONFIGS["kstar10"].coupling_seed)
    c_g = c_g / c_g[fixed]
    gen = A.Model(res_g)
    ev = gen.generate(W.couplings_to_params(c_g), n_events, seed)
    gen.close()
    m = A.Model(res_f, path=A.AMP4D_PATH_CACHED)
    m.set_events(*ev)
    m.set_norm_points(*(torch.from_numpy(a).cuda() for a in W.uniform_points(n_norm, seed + 1)))
    nz = len(cols_f) - len(cols_g)
    rng = np.random.default_rng(seed + 2)
    c0 = np.concatenate([W.perturbed_start(c_g), 0.02 * np.exp(1j * rng.uniform(-np.pi, np.pi, nz))])
    c0[fixed] = 1.0
    par = F.Parametrization(len(c0), 0, fixed_col=fixed, polar=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = F.fit(m.eval_nll_grad, par, W.couplings_to_params(c0), tol=tol)
    t_fit = time.perf_counter() - t0
    ff = m.fit_fractions(par.to_params(r.theta))
    m.close()
    return {"events": n_events, "normalisation_points": n_norm, "free_parameters": par.n_free,
            "fit_s": t_fit, "nfcn": int(r.nfcn), "converged": bool(r.converged),
            "fit_fraction_Z": {res_f[i].name: float(ff[i]) for i in range(len(res_g), len(res_f))},
            "note": "K*-only data fitted with the K* + 2 Z model; the paper reports Z fit fractions "
                    "of about 1e-4"}


def roofline_of(units, bpe, fpe, mean_launch_s, kernel):
    """The larger of the HBM and FP32 fractions of one kernel launch over `units`
    events or points (algorithmic bytes and formula flops per unit)."""
    achieved_tf = fpe * units / mean_launch_s / 1e12
    achieved_gbs = bpe * units / mean_launch_s / 1e9
    hbm_peak = _peaks().get("hbm_gbs") or 6800.0
    frac_alu, frac_hbm = achieved_tf / FP32_PEAK_TFLOPS, achieved_gbs / hbm_peak
    if frac_hbm >= frac_alu:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": frac_hbm, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    else:
        roof = {"bound": "alu", "achieved": achieved_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": frac_alu,
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (of nominal)"}
    roof.update({"kernel": kernel, "units_per_launch": units, "bytes_per_unit": bpe,
                 "flops_per_unit": fpe, "alu_frac": frac_alu, "hbm_frac": frac_hbm,
                 "mean_launch_ms": mean_launch_s * 1e3})
    return roof


def floated_z(A, res, c, dev, devn, K, Wm, stream, n_norm, proposal_seeds=16):
    """The benchmark workload with the Z(4430) mass and width floating: the Gram
    matrix cannot be reused while a mass moves, so I and dI/dtheta come from the
    per-point adjoint pass every evaluation.  Timed like the headline (device and
    end to end), then again with 2^20 points of the learned proposal in place of
    the 2^24 uniform ones, with the equality of their normalisation accuracy
    measured as the seed-to-seed spread of I over independent samples."""
    import torch
    fl = ["Z(4430)"]
    p = W.couplings_to_params(c, W.float_mg_values(res, fl))
    m = A.Model(res, float_names=fl, path=A.AMP4D_PATH_CACHED)
    P = m.n_params
    m.set_events(*dev)
    m.set_norm_points(*devn)
    pts = np.stack([step_params(p, k, m.n_cols) for k in range(K + Wm)])
    p_dev = torch.from_numpy(pts).cuda()
    out_dev = torch.zeros((K + Wm, 6 + P), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    m.profile(True)
    ms = _timed(m, A, p_dev, out_dev, A.AMP4D_EVAL_NLL_GRAD, K, Wm, stream)
    prof_ms, prof_n = m.profile_read()
    m.profile(False)
    assert np.all(out_dev.cpu().numpy()[:, 5] == 0), "evaluation reported an error status"
    host_pts = torch.from_numpy(pts).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(K):
        m.eval_nll_grad(host_pts[Wm + k])
    t_e2e = time.perf_counter() - t0
    n_ev = int(dev[0].shape[0])
    dom = 1 if prof_ms[1] >= prof_ms[2] else 2
    units = n_ev if dom == 1 else n_norm
    roof = roofline_of(units, bytes_per_event(res, True, fl, norm=dom == 2),
                       flops_per_event(res, fl, grad=True, cached=True),
                       prof_ms[dom] / max(1, prof_n[dom]) / 1e3,
                       "k_grad_fx<..., LFM = 1> over the %s (K* lineshapes cached, Z computed per %s)"
                       % (("data events", "event") if dom == 1 else ("normalisation points", "point")))
    out = {"workload": "large with the Z(4430) mass and width floating", "params": P,
           "value": K / (ms / 1e3), "unit": "evals/s", "ms_per_step": ms / K,
           "e2e": {"value": K / t_e2e, "unit": "evals/s", "h2d_bytes_per_step": 8 * P,
                   "d2h_bytes_per_step": 8 * (6 + P)},
           "gpu_launches": 4 * K,
           "phases_ms_per_step": {nm: float(prof_ms[i] / max(1, prof_n[i]))
                                  for i, nm in enumerate(["table", "data_kernel", "norm_kernel", "finish"])},
           "roofline": roof}
    # Learned proposal: trained on 2^20 events the model generates at its start point.
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev = m.generate(p, 1 << 20, 31)
    m.proposal_train(ev, seed=11)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    def spread(sampler, n):
        vals = []
        for s_ in range(proposal_seeds):
            pts_, w_ = sampler(s_)
            m.set_norm_points(*pts_, w=w_, volume=1.0)
            vals.append(m.eval_terms(p)[2])
        v = np.array(vals)
        return float(v.std(ddof=1) / v.mean()), float(v.mean())

    one = np.ones(1, dtype=np.float32)
    sd_u, I_u = spread(lambda s_: A.grid_sample(one, (1, 1, 1, 1), 1.0, 900 + s_, n_norm)[:2], n_norm)
    sd_l, I_l = spread(lambda s_: m.proposal_sample(1 << 20, 100 + s_), 1 << 20)
    pts_l, w_l = m.proposal_sample(1 << 20, 99)
    m.set_norm_points(*pts_l, w=w_l, volume=1.0)
    ms_l = _timed(m, A, p_dev, out_dev, A.AMP4D_EVAL_NLL_GRAD, K, Wm, stream)
    m.close()
    out["learned_proposal"] = {
        "train_s": t_train, "train_events": 1 << 20, "points": 1 << 20,
        "I_seed_sd_rel": sd_l, "uniform_points": n_norm, "uniform_I_seed_sd_rel": sd_u,
        "seeds": proposal_seeds, "I_learned_over_uniform": I_l / I_u,
        "variance_reduction_per_point": (sd_u / sd_l) ** 2 * n_norm / (1 << 20),
        "equal_or_better_accuracy": bool(sd_l <= sd_u),
        "value": K / (ms_l / 1e3), "unit": "evals/s",
        "speedup_vs_uniform_points": (K / (ms_l / 1e3)) / out["value"],
        "note": "normalisation error measured as the relative spread of I over independent "
                "point samples (learned 2^20 vs uniform 2^24); the bias against the 4D quadrature "
                "is checked in the GPU tests"}
    return out


def oracle_rates(max_events=50_000, max_points=200_000, min_s=0.5):
    """The FP64 oracle's NLL and NLL + gradient rates on the three workloads of the
    plan (two K*; ten K*; ten K* + Z with every mass and width floating), with all
    threads and with one, each on a bounded sample and scaled to the workload's
    events + points (evaluation time is linear in them)."""
    import oracle as O
    out = {}
    nthr = O.num_threads()
    for name in ("tiny", "kstar10", "kstar10_z"):
        cfg = W.CONFIGS[name]
        res, params, ev, nm = make_workload(cfg)
        n_s, m_s = min(cfg.n_events, max_events), min(cfg.n_norm, max_points)
        evs = tuple(a[:n_s] for a in ev)
        nms = tuple(a[:m_s] for a in nm)
        om = O.Model(res, float_names=cfg.float_mg)
        scale = (cfg.n_events + cfg.n_norm) / (n_s + m_s)
        r = {"events": cfg.n_events, "points": cfg.n_norm, "sample_events": n_s, "sample_points": m_s,
             "float_mg": len(cfg.float_mg), "params": om.n_params}
        for threads in (nthr, 1):
            O.set_num_threads(threads)
            for grad in (False, True):
                t0 = time.perf_counter()
                reps = 0
                while reps < 1 or time.perf_counter() - t0 < min_s:
                    om.nll(step_params(params, reps, om.n_cols), evs, nms, grad=grad)
                    reps += 1
                dt = (time.perf_counter() - t0) / reps * scale
                r["%s_evals_per_s_%s" % ("nll_grad" if grad else "nll",
                                         "all_threads" if threads == nthr else "1_thread")] = 1.0 / dt
        O.set_num_threads(nthr)
        out[name] = r
    out["threads"] = nthr
    out["note"] = ("each rate timed on the bounded sample and scaled to the workload's events + points "
                   "(extrapolated, not measured at full size)")
    return out


def run_reference(args, cfg):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    res, params, ev, nm = make_workload(cfg)
    frac = args.ref_frac
    n_s, m_s = cfg.n_events // frac, cfg.n_norm // frac
    evs = tuple(a[:n_s] for a in ev)
    nms = tuple(a[:m_s] for a in nm)
    om = O.Model(res, float_names=cfg.float_mg)
    for k in range(args.warmup):
        om.nll(step_params(params, k, om.n_cols), evs, nms, grad=True)
    t0 = time.perf_counter()
    for k in range(args.steps):
        om.nll(step_params(params, k, om.n_cols), evs, nms, grad=True)
    dt = (time.perf_counter() - t0) / args.steps
    full = dt * (cfg.n_events + cfg.n_norm) / (n_s + m_s)
    val = 1.0 / full
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": full * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg.name, "n_events": cfg.n_events, "n_norm": cfg.n_norm,
                       "resonances": len(res), "float_mg": cfg.float_mg},
            "cpu_baseline": {"value": val, "unit": "evals/s", "cores": O.num_threads(),
                             "kind": "oracle",
                             "sample": "each step: %d events + %d points (1/%d), scaled" % (n_s, m_s, frac),
                             "extrapolated": True},
            "e2e": {"value": val, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _timed(model, A, pts_dev, out_dev, what, K, W0, stream):
    """K back-to-back enqueued evaluations timed with CUDA events on the stream."""
    import torch
    for k in range(W0):
        model.enqueue_eval(what, pts_dev[k % len(pts_dev)], out_dev[k % len(out_dev)])
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(K):
        model.enqueue_eval(what, pts_dev[(W0 + k) % len(pts_dev)], out_dev[(W0 + k) % len(out_dev)])
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large", choices=sorted(W.CONFIGS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain GPU path")
    ap.add_argument("--no-fit", action="store_true", help="skip the full-size closure fit")
    ap.add_argument("--no-floated", action="store_true",
                    help="skip the floated-Z configuration and its learned-proposal timing")
    ap.add_argument("--cpu-frac", type=int, default=16)
    ap.add_argument("--ref-frac", type=int, default=64)
    ap.add_argument("--events", type=int, default=None, help="override the number of data events")
    ap.add_argument("--norm", type=int, default=None, help="override the number of normalisation points")
    args = ap.parse_args()
    cfg = W.CONFIGS[args.config]
    if args.events or args.norm:
        import dataclasses
        cfg = dataclasses.replace(cfg, n_events=args.events or cfg.n_events,
                                  n_norm=args.norm or cfg.n_norm)
    if args.impl == "reference":
        run_reference(args, cfg)
        return

    import torch
    import paper_2007_14931_gb300 as A

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()

    res, params, ev, nm = make_workload(cfg, rank)
    dev = [torch.from_numpy(a).cuda() for a in ev]
    devn = [torch.from_numpy(a).cuda() for a in nm]
    # Optimised form: adjoint gradient + tensor-core Gram normalisation (masses and
    # widths fixed); falls back to per-point normalisation when some float.
    model = A.Model(res, float_names=cfg.float_mg, path=A.AMP4D_PATH_CACHED)
    P = model.n_params
    model.set_events(*dev)
    model.set_norm_points(*devn)
    gram_ms = gram_first_ms = None
    if not cfg.float_mg:
        # the first build allocates the basis-matrix scratch; a repeat build (the
        # cost of a new Gram between mass steps) finds it allocated
        gev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        gev[0].record(stream)
        model.build_gram(params)
        gev[1].record(stream)
        gev[2].record(stream)
        model.build_gram(params)
        gev[3].record(stream)
        torch.cuda.synchronize()
        gram_first_ms = gev[0].elapsed_time(gev[1])
        gram_ms = gev[2].elapsed_time(gev[3])

    K, Wm = args.steps, args.warmup
    pts = np.stack([step_params(params, k, model.n_cols) for k in range(K + Wm)])
    p_dev = torch.from_numpy(pts).cuda()
    out_dev = torch.zeros((K + Wm, 6 + P), dtype=torch.float64, device="cuda")

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    model.profile(True)
    ms = _timed(model, A, p_dev, out_dev, A.AMP4D_EVAL_NLL_GRAD, K, Wm, stream)
    prof_ms, prof_n = model.profile_read()
    model.profile(False)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    outs = out_dev.cpu().numpy()
    assert np.all(outs[:, 5] == 0), "evaluation reported an error status"

    # end-to-end through the synchronous user call (host params in, host NLL + grad out)
    host_pts = torch.from_numpy(pts).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(K):
        model.eval_nll_grad(host_pts[Wm + k])
    t_e2e = time.perf_counter() - t0
    clk = clocks.stop()
    if dist:
        t = torch.tensor([t_e2e], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_e2e = float(t.item())

    value = world * K / (ms / 1e3)
    e2e_value = world * K / t_e2e
    names = ["table", "data_kernel", "norm_kernel", "finish"]
    # The dominant kernel is the adjoint over the data events or over the
    # normalisation points.  The table phase opens with an event recorded before
    # the host launches the table kernel, so it also holds host launch gaps.
    dom = 1 if prof_ms[1] >= prof_ms[2] else 2
    units = cfg.n_events if dom == 1 else cfg.n_norm
    fpe = flops_per_event(res, cfg.float_mg, grad=True, cached=True)
    bpe = bytes_per_event(res, cached=True, float_names=cfg.float_mg)
    mean_launch_s = prof_ms[dom] / max(1, prof_n[dom]) / 1e3
    achieved_tf = fpe * units / mean_launch_s / 1e12
    achieved_gbs = bpe * units / mean_launch_s / 1e9
    hbm_peak = _peaks().get("hbm_gbs") or 6800.0
    frac_alu, frac_hbm = achieved_tf / FP32_PEAK_TFLOPS, achieved_gbs / hbm_peak
    if frac_hbm >= frac_alu:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": frac_hbm, "bytes_per_event": bpe,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    else:
        roof = {"bound": "alu", "achieved": achieved_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": frac_alu,
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (of nominal)"}
    same_model = (not cfg.float_mg and [r.name for r in res] ==
                  [r.name for r in W.CONFIGS["large"].resonances])
    fresh = K_GRAD_TRAFFIC["sources_sha16"] == kernel_sources_sha16()
    traffic = (K_GRAD_TRAFFIC["bytes_per_event"] * units
               if (fresh and K_GRAD_TRAFFIC["bytes_per_event"] and same_model and dom == 1) else None)
    kname = ("k_grad_fx data (adjoint, all lineshapes from the basis cache)" if dom == 1 else
             "adjoint over the normalisation points (per-point normalisation)")
    roof.update({"kernel": kname,
                 "traffic": traffic,
                 "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum on 4e6 events, "
                                    "scaled by events" if traffic else
                                    "null: no ncu capture of the current kernel sources (sha16 %s)"
                                    % kernel_sources_sha16()),
                 "units_per_launch": units, "flops_per_event": fpe, "alu_frac": frac_alu,
                 "hbm_frac": frac_hbm})
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": K,
        "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": cfg.name, "n_events": cfg.n_events, "n_norm": cfg.n_norm,
                   "resonances": len(res), "params": P, "float_mg": cfg.float_mg,
                   "path": ("adjoint gradient + basis cache + tensor-core Gram normalisation"
                            if not cfg.float_mg else
                            "adjoint gradient + basis cache, per-point normalisation"),
                   "l2": "inputs larger than L2 (%.2f GB of event records)" % (
                       (17 * cfg.n_events + 18 * cfg.n_norm) * 4 / 1e9)},
        "events_per_s": value * cfg.n_events,
        "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": 8 * P,
                "d2h_bytes_per_step": 8 * (6 + P)},
        # per step on the Gram path: the table update and the data adjoint, whose
        # last CTA finishes the evaluation; with floated masses the table build, the
        # data adjoint, the point adjoint and the finish
        "gpu_launches": int(K * (2 if not cfg.float_mg else 4)),
        "phases_ms_per_step": {n: float(prof_ms[i] / max(1, prof_n[i])) for i, n in enumerate(names)},
        "roofline": roof,
        "clocks": clk,
        "nll_last": float(outs[-1, 0]),
    }
    if gram_ms is not None:
        rows = 2 * cfg.n_norm
        mma_flops = rows / 16 * 2 * 128 * (256 + 64) * 16
        line["gram"] = {"build_ms": gram_ms, "first_build_ms": gram_first_ms, "rows": rows,
                        "basis_matrix_gb": rows * 2 * model.n_cols * 4 / 1e9,
                        "tensor_tflops_executed": mma_flops / (gram_ms / 1e3) / 1e12,
                        "bf16_peak_measured": _peaks().get("bf16_tflops"),
                        "note": "per mass/width setting: basis pass (FP32 basis matrix + column maxima), "
                                "tcgen05 digit-product kernel, reduce; build_ms is a repeat build, "
                                "first_build_ms includes allocating the basis matrix"}
    model.close()
    del model
    if not args.no_plain:
        # The plain GPU path on the same data: every amplitude recomputed per evaluation,
        # uniform normalisation points summed per evaluation, adjoint gradient; and the
        # GooFit-like form with the gradient by central differences (2P + 1 NLL evaluations).
        plain = A.Model(res, float_names=cfg.float_mg, path=A.AMP4D_PATH_PLAIN)
        plain.set_events(*dev)
        plain.set_norm_points(*devn)
        Kp = max(3, K // 2)
        ms_g = _timed(plain, A, p_dev, out_dev, A.AMP4D_EVAL_NLL_GRAD, Kp, 2, stream)
        ms_n = _timed(plain, A, p_dev, out_dev, A.AMP4D_EVAL_NLL, Kp, 2, stream)
        nll_rate = Kp / (ms_n / 1e3)
        line["plain_gpu"] = {
            "adjoint_evals_per_s": world * Kp / (ms_g / 1e3),
            "nll_evals_per_s": world * nll_rate,
            "fd_grad_evals_per_s": world * nll_rate / (2 * P + 1),
            "note": "same GPU, recompute per evaluation, uniform points; fd = 2P+1 NLL evaluations"}
        line["speedup_vs_plain_fd"] = value / line["plain_gpu"]["fd_grad_evals_per_s"]
        plain.close()
    if rank == 0 and world == 1 and not args.no_floated and cfg.name == "large":
        line["floated_z"] = floated_z(A, res, W.draw_couplings(res, cfg.coupling_seed), dev, devn,
                                      K, Wm, stream, cfg.n_norm)
    if rank == 0 and world == 1 and not args.no_fit:
        line["fit"] = full_fit(cfg, A)
        line["real_life"] = real_life_fit(A)
        line["z_sensitivity"] = z_sensitivity_fit(A)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(cfg, args.cpu_frac, A)
        line["cpu_baseline"]["oracle_rates"] = oracle_rates()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
