"""Seeded synthetic inputs for the B0 -> J/psi K+ pi- four-dimensional amplitude fit.

This module is the only code shared by the FP64 oracle tests and the GPU path.
It holds inputs, never the method's arithmetic: particle masses, the observable
box, resonance tables with their spin/orbital assignments, seeded coupling
draws and seeded point draws (uniform in the box, or with Cauchy-shaped
m_Kpi peaks at the resonance poles).  Nothing here evaluates a lineshape, an
angular function or a density.

Observables (Eq. 1 with the K* helicity angle of Eq. 4 in place of m_J/psi pi):
    m      = m_Kpi in [0.6336, 2.1828] GeV
    cK     = cos(theta_K*) in [-1, 1]
    cpsi   = cos(theta_J/psi) in [-1, 1]
    phi    = angle between the two decay planes, in [-pi, pi]
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Particle masses in GeV (B0, J/psi, K+, pi-).
M_B = 5.27966
M_PSI = 3.0969
M_K = 0.493677
M_PI = 0.13957
PARTICLE_MASSES = (M_B, M_PSI, M_K, M_PI)

# Observable box.  The upper m_Kpi edge lies 4e-5 GeV above m_B - m_psi; the
# phase-space weight is zero on that sliver.
M_LO = 0.6336
M_HI = 2.1828
BOX_VOLUME = (M_HI - M_LO) * 2.0 * 2.0 * (2.0 * math.pi)

CHAIN_KSTAR = 0
CHAIN_Z = 1

# Blatt-Weisskopf radius (GeV^-1) used for both barrier factors.
R_BW = 1.6

# Lineshape kinds: the Breit-Wigner of Eq. 2-3, or the LASS K pi S-wave of Eq. 7-8.
SHAPE_BW = 0
SHAPE_LASS = 1
# Effective-range constants of Eq. 8 (GeV^-1), and the factor on the resonant
# term of Eq. 7: 1 for the elastic (unitary) form; the paper prints 2.
LASS_A = 1.95
LASS_B = 1.76
LASS_R = 1.0


@dataclass(frozen=True)
class Resonance:
    name: str
    chain: int      # CHAIN_KSTAR (-> K pi) or CHAIN_Z (-> J/psi pi)
    J: int
    P: int          # intrinsic parity (+1 / -1)
    M: float        # pole mass, GeV
    G0: float       # nominal width, GeV
    r: float = R_BW
    shape: int = SHAPE_BW   # SHAPE_LASS: the K0*(1430) pole inside the LASS S-wave
    lass_a: float = LASS_A
    lass_b: float = LASS_B
    lass_R: float = LASS_R

    @property
    def LB(self) -> int:
        """Lowest orbital angular momentum in the B0 decay (Sec. 'The K*-only model').

        B0(0-) -> J/psi(1-) K*(J): L in {|J-1|, ..., J+1}, lowest is |J-1|.
        B0(0-) -> Z(J) K(0-): L = J.
        """
        if self.chain == CHAIN_KSTAR:
            return abs(self.J - 1)
        return self.J

    @property
    def LR(self) -> int:
        """Orbital angular momentum in the resonance decay.

        K*(J) -> K pi: L = J.
        Z(J^P) -> J/psi(1-) pi(0-): lowest L in {|J-1|, ..., J+1} with (-1)^L = P.
        """
        if self.chain == CHAIN_KSTAR:
            return self.J
        for L in range(abs(self.J - 1), self.J + 2):
            if (-1) ** L == self.P:
                return L
        raise ValueError(f"{self.name}: no orbital wave for J^P={self.J}^{self.P}")


# K* states allowed up to m_Kpi = 2.183 GeV (Sec. 'The K*-only model').  The
# paper fixes masses and widths to world averages without printing them; these
# are synthetic stand-ins near those values.
KSTAR_TABLE = [
    Resonance("K0*(800)", CHAIN_KSTAR, 0, +1, 0.682, 0.470),
    Resonance("K*(892)", CHAIN_KSTAR, 1, -1, 0.8955, 0.0473),
    Resonance("K*(1410)", CHAIN_KSTAR, 1, -1, 1.414, 0.232),
    Resonance("K0*(1430)", CHAIN_KSTAR, 0, +1, 1.425, 0.270),
    Resonance("K2*(1430)", CHAIN_KSTAR, 2, +1, 1.4324, 0.109),
    Resonance("K*(1680)", CHAIN_KSTAR, 1, -1, 1.717, 0.322),
    Resonance("K3*(1780)", CHAIN_KSTAR, 3, -1, 1.776, 0.159),
    Resonance("K0*(1950)", CHAIN_KSTAR, 0, +1, 1.945, 0.201),
    Resonance("K2*(1980)", CHAIN_KSTAR, 2, +1, 1.974, 0.376),
    Resonance("K4*(2045)", CHAIN_KSTAR, 4, +1, 2.045, 0.198),
]
Z4430 = Resonance("Z(4430)", CHAIN_Z, 1, +1, 4.43, 0.18)
Z4200 = Resonance("Z(4200)", CHAIN_Z, 1, +1, 4.196, 0.37)
# LASS K pi S-wave (Eq. 7-9): the effective-range amplitude with the K0*(1430)
# pole inside it.  In Eq. 9 it replaces the two scalar Breit-Wigners K0*(800)
# and K0*(1430); the other K* states keep theirs.
LASS = Resonance("LASS", CHAIN_KSTAR, 0, +1, 1.425, 0.270, shape=SHAPE_LASS)
RESONANCES = {r.name: r for r in KSTAR_TABLE + [Z4430, Z4200, LASS]}
KSTAR_PRIME = [r.name for r in KSTAR_TABLE if r.name not in ("K0*(800)", "K0*(1430)")]

# Z helicity couplings are drawn like the K* ones, then scaled by this factor
# so that the Z fit fraction is a few percent.
Z_COUPLING_SCALE = 0.2


def columns(res_list):
    """Basis columns (resonance index, helicity label) in the order the ABI uses.

    K*(J=0): lambda = 0 only.  K*(J>=1): lambda = -1, 0, +1.
    Z(J^P): the parity relation H_{-l} = eta H_{+l}, eta = -P(-1)^J (Eq. 11),
    ties lambda' = +-1 into one column (label 1); lambda' = 0 (label 0) exists
    only when eta = +1.
    """
    cols = []
    for i, r in enumerate(res_list):
        if r.chain == CHAIN_KSTAR:
            lams = (0,) if r.J == 0 else (-1, 0, 1)
        else:
            eta = -r.P * (-1) ** r.J
            lams = ((0,) if eta == 1 else ()) + ((1,) if r.J >= 1 else ())
        cols.extend((i, l) for l in lams)
    return cols


@dataclass
class Config:
    """One workload: resonance list, sizes and seeds."""
    name: str
    index: int
    res_names: list
    n_events: int
    n_norm: int
    float_mg: list = field(default_factory=list)   # names whose M, Gamma float
    eq14: bool = False   # efficiency and background templates (Eq. 14)
    z_scale: float = Z_COUPLING_SCALE   # factor on the drawn Z couplings

    @property
    def template_seed(self):
        return 1400 + self.index

    @property
    def resonances(self):
        return [RESONANCES[n] for n in self.res_names]

    @property
    def coupling_seed(self):
        return 14931 + self.index

    @property
    def data_seed(self):
        return 2007 + self.index

    @property
    def norm_seed(self):
        return 4931 + self.index


ALL_KSTAR = [r.name for r in KSTAR_TABLE]
CONFIGS = {
    "tiny": Config("tiny", 0, ["K*(892)", "K2*(1430)"], 10_000, 100_000),
    "kstar10": Config("kstar10", 1, ALL_KSTAR, 200_000, 2_000_000),
    "kstar10_z": Config("kstar10_z", 2, ALL_KSTAR + ["Z(4430)"], 1_000_000, 4_000_000,
                        float_mg=ALL_KSTAR + ["Z(4430)"]),
    "learned": Config("learned", 3, ALL_KSTAR + ["Z(4430)"], 1 << 20, 1 << 20),
    "large": Config("large", 4, ALL_KSTAR + ["Z(4430)"], 5_000_000, 1 << 24),
    "large_float_z": Config("large_float_z", 5, ALL_KSTAR + ["Z(4430)"], 5_000_000, 1 << 24,
                            float_mg=["Z(4430)"]),
    # The benchmark model with the K*(892) and Z(4430) masses and widths floating.
    "large_float_kz": Config("large_float_kz", 10, ALL_KSTAR + ["Z(4430)"], 5_000_000, 1 << 24,
                             float_mg=["K*(892)", "Z(4430)"]),
    # Z-sensitivity model: both Z states, their masses and widths floating.
    "kstar10_2z": Config("kstar10_2z", 6, ALL_KSTAR + ["Z(4200)", "Z(4430)"], 200_000, 2_000_000,
                         float_mg=["Z(4200)", "Z(4430)"]),
    # Eq. 9: the LASS S-wave and the eight other K* states.
    "lass": Config("lass", 7, ["LASS"] + KSTAR_PRIME, 200_000, 2_000_000),
    # Eq. 9 with Z(4430); every mass and width but the LASS pole's floating.
    "lass_z": Config("lass_z", 8, ["LASS"] + KSTAR_PRIME + ["Z(4430)"], 200_000, 2_000_000,
                     float_mg=KSTAR_PRIME + ["Z(4430)"]),
    # The paper's real-life test (Eq. 14): 10 K* + Z(4200) + Z(4430) with a
    # relative efficiency and 15 % background.
    # Z couplings scaled so that the Z fit fractions are a few percent, as the
    # paper reports for its real-life test.
    "real_life": Config("real_life", 9, ALL_KSTAR + ["Z(4200)", "Z(4430)"], 1_000_000, 1 << 22,
                        eq14=True, z_scale=3.0),
}


# ---------------------------------------------------------------- Eq. 14 templates
@dataclass
class Hist2D:
    """Binned template: contents h[iy, ix] (FP32) over [x_lo, x_hi] x [y_lo, y_hi]."""
    h: np.ndarray
    range: tuple

    @property
    def nx(self):
        return int(self.h.shape[1])

    @property
    def ny(self):
        return int(self.h.shape[0])


# Template axes: the two mass variables (m^2_Kpi, m^2_psipi over the Dalitz
# plot's bounding box) and the two angles (cos theta_psi, phi).
MASS2_RANGE = (M_LO ** 2, M_HI ** 2, (M_PSI + M_PI) ** 2, (M_B - M_K) ** 2)
ANGLE_RANGE = (-1.0, 1.0, -math.pi, math.pi)
PURITY = 0.85   # signal purity of the paper's real-life test (15 % background)


def bernstein_hist(nx, ny, rng_xy, degree, seed, floor=0.2):
    """A 2D Bernstein polynomial of the given degree with seeded coefficients in
    [floor, 1], binned at the bin centres and scaled to a maximum of 1: the
    generic template shape of the paper's efficiency and background tests."""
    rng = np.random.Generator(np.random.Philox(seed))
    coef = rng.uniform(floor, 1.0, size=(degree + 1, degree + 1))
    u = (np.arange(nx) + 0.5) / nx
    v = (np.arange(ny) + 0.5) / ny
    bu = np.array([math.comb(degree, i) * u ** i * (1 - u) ** (degree - i) for i in range(degree + 1)])
    bv = np.array([math.comb(degree, j) * v ** j * (1 - v) ** (degree - j) for j in range(degree + 1)])
    h = bv.T @ coef.T @ bu          # [ny, nx]
    h = h / h.max()
    return Hist2D(h.astype(np.float32), tuple(float(x) for x in rng_xy))


def eq14_templates(seed):
    """(efficiency x masses, efficiency x angles, background x masses,
    background x angles, purity), seeded."""
    return (bernstein_hist(40, 40, MASS2_RANGE, 3, seed),
            bernstein_hist(20, 24, ANGLE_RANGE, 2, seed + 1),
            bernstein_hist(30, 30, MASS2_RANGE, 2, seed + 2, floor=0.05),
            bernstein_hist(16, 16, ANGLE_RANGE, 2, seed + 3, floor=0.3),
            PURITY)


def draw_couplings(res_list, seed, z_scale=Z_COUPLING_SCALE):
    """Complex helicity couplings, one per basis column.

    |H| ~ U(0.2, 1), arg H ~ U(-pi, pi); the K*(892) lambda = 0 coupling is
    fixed to 1 (Eq. 6).  Z couplings are scaled by z_scale.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    cols = columns(res_list)
    c = np.empty(len(cols), dtype=np.complex128)
    for k, (i, lam) in enumerate(cols):
        mag = rng.uniform(0.2, 1.0)
        ph = rng.uniform(-math.pi, math.pi)
        if res_list[i].chain == CHAIN_Z:
            mag *= z_scale
        c[k] = mag * complex(math.cos(ph), math.sin(ph))
        if res_list[i].name == "K*(892)" and lam == 0:
            c[k] = 1.0
    return c


def couplings_to_params(c, mg=()):
    """ABI parameter vector: [Re c_k, Im c_k]_k, then [M_R, Gamma_R] of floated R."""
    out = np.empty(2 * len(c) + len(mg), dtype=np.float64)
    out[0:2 * len(c):2] = c.real
    out[1:2 * len(c):2] = c.imag
    out[2 * len(c):] = np.asarray(mg, dtype=np.float64).ravel()
    return out


def float_mg_values(res_list, float_names):
    """[M, Gamma] of each floated resonance, in resonance-list order."""
    vals = []
    for r in res_list:
        if r.name in float_names:
            vals += [r.M, r.G0]
    return vals


M_END = M_B - M_PSI   # kinematic limit of m_Kpi (the box edge lies 4e-5 GeV above it)


def _f32_in(x, lo, hi):
    """Round to FP32 and keep the result inside [lo, hi] (as double)."""
    f = np.asarray(x, dtype=np.float32)
    lo32 = np.float32(lo)
    if float(lo32) < lo:
        lo32 = np.nextafter(lo32, np.float32(np.inf))
    hi32 = np.float32(hi)
    if float(hi32) > hi:
        hi32 = np.nextafter(hi32, np.float32(-np.inf))
    return np.ascontiguousarray(np.clip(f, lo32, hi32))


def _angles(u1, u2, u3):
    return (_f32_in(2.0 * u1 - 1.0, -1.0, 1.0), _f32_in(2.0 * u2 - 1.0, -1.0, 1.0),
            _f32_in(math.pi * (2.0 * u3 - 1.0), -math.pi, math.pi))


def uniform_points(n, seed, box=(M_LO, M_HI)):
    """n points uniform in the observable box, FP32 SoA (m, cK, cpsi, phi).

    Use box=(M_LO, M_END) for data-like events: beyond M_END the phase space
    vanishes and no real event can lie there."""
    rng = np.random.Generator(np.random.Philox(seed))
    u = rng.random((4, n))
    m = _f32_in(box[0] + (box[1] - box[0]) * u[0], box[0], box[1])
    return (m,) + _angles(u[1], u[2], u[3])


def peaked_points(n, seed, res_list, f_uniform=0.3, box=(M_LO, M_END)):
    """n points whose m_Kpi has Cauchy peaks at the K* poles (truncated to the box).

    A fraction f_uniform is uniform in m; the rest picks a K* in res_list with
    equal probability and draws m from a Cauchy of location M and half-width
    Gamma0/2 restricted to the box by inverse-CDF sampling.  Angles are uniform.
    The result has the peaked m_Kpi structure of real B0 -> J/psi K pi data
    without evaluating the amplitude model.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    ks = [r for r in res_list if r.chain == CHAIN_KSTAR]
    u = rng.random((6, n))
    m = box[0] + (box[1] - box[0]) * u[0]
    pick = np.minimum((u[4] * len(ks)).astype(np.int64), len(ks) - 1)
    peaked = u[5] >= f_uniform
    for j, r in enumerate(ks):
        sel = peaked & (pick == j)
        hw = 0.5 * r.G0
        a = math.atan((box[0] - r.M) / hw)
        b = math.atan((box[1] - r.M) / hw)
        m[sel] = r.M + hw * np.tan(a + (b - a) * u[0][sel])
    # strictly below the kinematic edge, where p q > 0
    m = _f32_in(m, box[0], min(box[1], M_END - 1e-6))
    return (m,) + _angles(u[1], u[2], u[3])


def perturbed_start(c, seed=7, amount=0.1):
    """Fit start: each |H| scaled by 1 + U(-amount, amount), each phase shifted by
    U(-amount, amount) rad; the fixed K*(892) lambda = 0 coupling is kept (by
    the caller's fixed mask)."""
    rng = np.random.Generator(np.random.Philox(seed))
    mag = np.abs(c) * (1.0 + rng.uniform(-amount, amount, len(c)))
    ph = np.angle(c) + rng.uniform(-amount, amount, len(c))
    return mag * np.exp(1j * ph)
