"""FP64 CPU theory tool for the Carnahan-Starling pseudopotential model.

TEST INFRASTRUCTURE ONLY.  This module belongs to the oracle: only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  The CUDA library has its own, independent host-side equation-of-state
code and never calls anything here.

What it computes (Li, Luo & Li, Sec. III C and Sec. IV):

* the Carnahan-Starling pressure (Eq. 23) and its exact critical point
  (dp/drho = d^2p/drho^2 = 0), with a = 1, b = 4, R = 1 as in the paper;
* the pseudopotential psi(rho) that reproduces that pressure (Eq. 8);
* coexistence densities (rho_g, rho_l, p0) from an equal-"area" condition
      int_{rho_g}^{rho_l} (p0 - p(rho)) w(rho) drho = 0,   p(rho_g) = p(rho_l) = p0
  with w = 1/rho^2 for the Maxwell construction (Eq. 7) and
  w = psi'/psi^(1+eps) for the mechanical-stability condition (Eq. 26; Eq. 6
  is eps = 0);
* the eps = 2 condition in the integrated-by-parts form of Eq. 30, used only
  as an independent cross-check of the general solver;
* eps as a function of sigma for the improved forcing scheme,
  eps = -2(alpha + 24 G sigma)/beta with alpha = 0, beta = 3 (Sec. IV B,
  text after Eq. 35; alpha and beta from the text after Eq. 25).

Everything is plain numpy/scipy: polynomial arithmetic for exact derivatives,
brentq for roots and composite Gauss-Legendre quadrature for the integrals.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from numpy.polynomial import Polynomial
from scipy.optimize import brentq

CS2 = 1.0 / 3.0          # c_s^2 for D2Q9 with c = 1 (Eq. 2)
TC_PAPER = 0.094         # Tc as printed with the constants of Eq. 23
RHOC_PAPER = 0.13044     # rho_c as printed with the constants of Eq. 23


# ---------------------------------------------------------------------------
# Carnahan-Starling equation of state (Eq. 23)
# ---------------------------------------------------------------------------

def _cs_h_polys(b: float):
    """h(rho) = rho * Z(eta), eta = b rho / 4, as a ratio of polynomials in rho.

    Z(eta) = (1 + eta + eta^2 - eta^3) / (1 - eta)^3 is the Carnahan-Starling
    compressibility factor of Eq. 23, so p = R T h(rho) - a rho^2.
    """
    eta = Polynomial([0.0, b / 4.0])
    num = Polynomial([0.0, 1.0]) * (1 + eta + eta ** 2 - eta ** 3)
    den = (1 - eta) ** 3
    return num, den


def critical_point(a: float = 1.0, b: float = 4.0, R: float = 1.0):
    """Exact critical point (rho_c, T_c, p_c) of Eq. 23.

    With p = R T h(rho) - a rho^2 the two conditions dp/drho = 0 and
    d^2p/drho^2 = 0 give R T = 2a / h'' and h' - rho h'' = 0.  h' and h'' are
    taken exactly with polynomial arithmetic (quotient rule), and the root of
    the numerator polynomial of h' - rho h'' in (0, 4/b) is rho_c.
    """
    num, den = _cs_h_polys(b)
    d1n = num.deriv() * den - num * den.deriv()
    d1d = den ** 2
    d2n = d1n.deriv() * d1d - d1n * d1d.deriv()
    # h' - rho h'' = d1n/d1d - rho d2n/d1d^2 ; multiply by d1d^2 > 0
    cond = d1n * d1d - Polynomial([0.0, 1.0]) * d2n
    lo, hi = 1e-6, 4.0 / b * (1 - 1e-9)
    roots = [r.real for r in cond.roots()
             if abs(r.imag) < 1e-9 and lo < r.real < hi]
    if not roots:
        raise ValueError("no critical point found")
    # polish the smallest admissible root (the physical branch) with brentq
    r0 = min(roots)
    f = lambda x: cond(x)
    rho_c = brentq(f, r0 * (1 - 1e-6), r0 * (1 + 1e-6), xtol=1e-17, rtol=1e-15) \
        if f(r0 * (1 - 1e-6)) * f(r0 * (1 + 1e-6)) < 0 else r0
    h2 = d2n(rho_c) / d1d(rho_c) ** 2
    T_c = 2.0 * a / (R * h2)
    eos = CarnahanStarling(T_c, a=a, b=b, R=R)
    return rho_c, T_c, eos.p(rho_c)


def temperature(T_over_Tc: float, tc_mode: int = 0, a: float = 1.0,
                b: float = 4.0, R: float = 1.0) -> float:
    """Absolute T for a reduced temperature.

    tc_mode 0 uses the exact critical temperature; tc_mode 1 uses the rounded
    T_c = 0.094 printed with Eq. 23 (only meaningful for a = 1, b = 4, R = 1).
    """
    if tc_mode == 0:
        return T_over_Tc * critical_point(a, b, R)[1]
    if tc_mode == 1:
        return T_over_Tc * TC_PAPER
    raise ValueError("tc_mode must be 0 or 1")


@dataclass
class CarnahanStarling:
    """p_EOS of Eq. 23 with psi from Eq. 8 (c = 1)."""

    T: float
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    G: float = -1.0

    def p(self, rho):
        eta = self.b * rho / 4.0
        return (rho * self.R * self.T * (1 + eta + eta ** 2 - eta ** 3)
                / (1 - eta) ** 3 - self.a * rho ** 2)

    def dp(self, rho):
        # d/drho [rho Z(eta)] = Z + eta Z'(eta),
        # Z'(eta) = (4 + 4 eta - 2 eta^2)/(1 - eta)^4
        eta = self.b * rho / 4.0
        Z = (1 + eta + eta ** 2 - eta ** 3) / (1 - eta) ** 3
        dZ = (4 + 4 * eta - 2 * eta ** 2) / (1 - eta) ** 4
        return self.R * self.T * (Z + eta * dZ) - 2 * self.a * rho

    def psi2(self, rho):
        """psi^2 = 2 (p_EOS - rho c_s^2) / (G c^2)  (Eq. 8)."""
        return 2.0 * (self.p(rho) - rho * CS2) / self.G

    def psi(self, rho):
        return np.sqrt(self.psi2(rho))

    def dpsi(self, rho):
        """psi' from 2 psi psi' = 2 (p' - c_s^2) / G."""
        return (self.dp(rho) - CS2) / (self.G * self.psi(rho))

    def rho_max(self) -> float:
        return 4.0 / self.b


@dataclass
class ExpPsiModel:
    """Original Shan-Chen potential psi = psi0 exp(-rho0/rho).

    The pressure is the model EOS of Eq. 5, p = rho c_s^2 + (G/2) psi^2.  For
    this psi the mechanical-stability condition (Eq. 6) coincides with the
    Maxwell construction (Eq. 7), which the tests use as a pin.
    """

    G: float = -3.0
    psi0: float = 1.0
    rho0: float = 1.0
    rmax: float = 50.0

    def psi(self, rho):
        return self.psi0 * np.exp(-self.rho0 / rho)

    def dpsi(self, rho):
        return self.psi(rho) * self.rho0 / rho ** 2

    def psi2(self, rho):
        return self.psi(rho) ** 2

    def p(self, rho):
        return rho * CS2 + 0.5 * self.G * self.psi2(rho)

    def dp(self, rho):
        return CS2 + self.G * self.psi(rho) * self.dpsi(rho)

    def rho_max(self) -> float:
        return self.rmax


# ---------------------------------------------------------------------------
# coexistence from an equal-area condition (Eqs. 6, 7, 26)
# ---------------------------------------------------------------------------

def spinodal(eos, n: int = 20001):
    """The two zeros of dp/drho (local max, then local min of p)."""
    rmax = eos.rho_max()
    grid = np.linspace(rmax * 1e-6, rmax * (1 - 1e-6), n)
    d = eos.dp(grid)
    idx = np.nonzero(np.sign(d[:-1]) * np.sign(d[1:]) < 0)[0]
    if len(idx) < 2:
        return None
    s1 = brentq(eos.dp, grid[idx[0]], grid[idx[0] + 1], xtol=1e-16, rtol=1e-15)
    s2 = brentq(eos.dp, grid[idx[1]], grid[idx[1] + 1], xtol=1e-16, rtol=1e-15)
    return s1, s2


def _branch_roots(eos, p0, s1, s2):
    """rho_g < s1 and rho_l > s2 with p(rho) = p0."""
    f = lambda r: eos.p(r) - p0
    lo = 1e-300
    while f(lo) > 0 and lo < s1:
        lo *= 10.0
    rho_g = brentq(f, lo, s1, xtol=1e-300, rtol=1e-15, maxiter=500)
    hi = eos.rho_max() * (1 - 1e-12)
    rho_l = brentq(f, s2, hi, xtol=1e-16, rtol=1e-15, maxiter=500)
    return rho_g, rho_l


_GL_X, _GL_W = np.polynomial.legendre.leggauss(20)


def _log_quad(g, lo, hi, panels: int = 64):
    """int_lo^hi g(rho) drho by composite 20-point Gauss-Legendre in s = ln(rho).

    The vapour end of the coexistence integrals sits at small rho where the
    Maxwell weight 1/rho^2 varies fast; in ln(rho) (drho = rho ds) the
    integrand is smooth and analytic, so a fixed composite rule converges to
    rounding level (the tests compare 64 against 128 panels).
    """
    if hi <= lo:
        return 0.0
    edges = np.linspace(math.log(lo), math.log(hi), panels + 1)
    mid = 0.5 * (edges[1:] + edges[:-1])[:, None]
    half = 0.5 * (edges[1:] - edges[:-1])[:, None]
    s = mid + half * _GL_X[None, :]
    r = np.exp(s)
    vals = g(r) * r
    return float(np.sum(half * _GL_W[None, :] * vals))


def coexistence(eos, weight, panels: int = 64):
    """Solve int (p0 - p) weight drho = 0 with p(rho_g) = p(rho_l) = p0.

    Parametrised by p0 between the spinodal extrema: for each p0 the two
    outer roots of p = p0 give (rho_g, rho_l), and brentq finds the p0 whose
    weighted area vanishes.  Returns (rho_g, rho_l, p0) or None when the area
    does not change sign (no solution, e.g. eps = 0 at low T).
    """
    sp = spinodal(eos)
    if sp is None:
        return None
    s1, s2 = sp
    p_hi = eos.p(s1)
    p_lo = max(eos.p(s2), 0.0)
    span = p_hi - p_lo
    # stay clear of the spinodal extrema, where two roots merge
    p_hi -= span * 1e-7
    p_lo += span * 1e-7

    def area(p0):
        rg, rl = _branch_roots(eos, p0, s1, s2)
        g = lambda r: (p0 - eos.p(r)) * weight(r)
        # split at the middle root of p = p0 so each piece has one sign and
        # the relative tolerance is reachable; the pieces cancel in the sum
        rm = brentq(lambda r: eos.p(r) - p0, s1, s2, xtol=1e-16, rtol=1e-15)
        return _log_quad(g, rg, rm, panels) + _log_quad(g, rm, rl, panels)

    a_hi = area(p_hi)
    a_lo = area(p_lo)
    if a_hi * a_lo > 0:
        return None
    p0 = brentq(area, p_lo, p_hi, xtol=1e-300, rtol=1e-15, maxiter=300)
    rg, rl = _branch_roots(eos, p0, s1, s2)
    return rg, rl, p0


def maxwell(eos):
    """Maxwell equal-area construction, Eq. 7: weight 1/rho^2."""
    return coexistence(eos, lambda r: 1.0 / r ** 2)


def mechanical_stability(eos, eps: float):
    """Mechanical-stability solution of Eq. 26: weight psi'/psi^(1+eps)."""
    return coexistence(eos, lambda r: eos.dpsi(r) / eos.psi(r) ** (1.0 + eps))


def eq30_residual(eos, rho_g: float, rho_l: float, p0: float) -> float:
    """Left-hand side of Eq. 30 (eps = 2 after integration by parts), c = 1."""
    def bracket(r):
        return (p0 - r * CS2) * (-0.5 / eos.psi2(r)) - 0.5 * eos.G * math.log(eos.psi(r))
    integral = _log_quad(lambda r: CS2 * (-0.5 / eos.psi2(r)), rho_g, rho_l, 128)
    return bracket(rho_l) - bracket(rho_g) + integral


def mechanical_stability_eq30(eos):
    """eps = 2 coexistence from Eq. 30 instead of the Eq. 26 quadrature."""
    sp = spinodal(eos)
    s1, s2 = sp
    p_hi = eos.p(s1)
    p_lo = max(eos.p(s2), 0.0)
    span = p_hi - p_lo
    p_hi -= span * 1e-7
    p_lo += span * 1e-7

    def resid(p0):
        rg, rl = _branch_roots(eos, p0, s1, s2)
        return eq30_residual(eos, rg, rl, p0)

    p0 = brentq(resid, p_lo, p_hi, xtol=1e-300, rtol=1e-15)
    rg, rl = _branch_roots(eos, p0, s1, s2)
    return rg, rl, p0


def eps_of_sigma(sigma: float, alpha: float = 0.0, beta: float = 3.0,
                 G: float = -1.0) -> float:
    """eps = -2 (alpha + 24 G sigma) / beta (Sec. IV B, after Eq. 35)."""
    return -2.0 * (alpha + 24.0 * G * sigma) / beta


def cs_chemical_potential(eos: CarnahanStarling, rho):
    """Chemical potential of the Carnahan-Starling fluid (up to a constant).

    From the CS excess free energy per particle R T (4 eta - 3 eta^2)/(1-eta)^2
    and the mean-field attraction -a rho: mu = f + p/rho with
    f/N = R T [ln rho - 1 + (4 eta - 3 eta^2)/(1 - eta)^2] - a rho.  Equal mu
    and p in both phases is the Maxwell rule in closed form; the tests use it
    to pin the quadrature-based ``maxwell``.
    """
    eta = eos.b * rho / 4.0
    f = eos.R * eos.T * (np.log(rho) - 1.0 + (4 * eta - 3 * eta ** 2) / (1 - eta) ** 2) \
        - eos.a * rho
    return f + eos.p(rho) / rho


def coexistence_table(T_over_Tc, tc_mode: int = 0, eps=None):
    """(rho_g, rho_l) from Maxwell (eps None) or Eq. 26 at each T/Tc."""
    out = []
    for t in np.atleast_1d(T_over_Tc):
        eos = CarnahanStarling(temperature(float(t), tc_mode))
        sol = maxwell(eos) if eps is None else mechanical_stability(eos, eps)
        out.append(None if sol is None else sol[:2])
    return out
