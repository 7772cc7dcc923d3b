"""Coexistence densities from the equation of state alone (FP64, host).

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).

* Maxwell equal-area construction, Eq. 19 (Sec. 3.1):
      int_{rho_g}^{rho_l} (p_c - p0(rho)) / rho^2 drho = 0,
      p0(rho_g) = p0(rho_l) = p_c.
* Mechanical stability condition, Eq. 18 (Sec. 3.1):
      int_{rho_g}^{rho_l} (p_c - p0(rho)) psi'(rho) / psi(rho)^(1+eps) drho = 0,
  with eps = -2a/b = -2A for Kupershtokh's force (Table 1).

p0 is the K-scaled Carnahan-Starling EOS of Eq. 30 (taken from the C oracle)
and psi = sqrt(2 (rho/3 - p0)) (Eq. 7 with G = -1).  Library primitives do
the numerics: scipy ``brentq`` for roots, ``quad`` for integrals (in log rho),
``minimize_scalar`` for the spinodal extrema.  The solvers also accept any
(p0, psi) pair, which the tests use for the Sbragaglia-Shan psi of Eq. 33.
"""
from __future__ import annotations

import math
import warnings
from typing import Callable

from scipy import integrate, optimize

from . import Tc, pressure

_RHO_MAX = 1.0 - 1e-9   # CS pole at eta = b rho / 4 = 1


def _spinodals(p: Callable[[float], float], lo=1e-6, hi=0.95, n=4000):
    """Local maximum (gas spinodal) and following local minimum (liquid spinodal) of p."""
    xs = [lo + (hi - lo) * i / n for i in range(n + 1)]
    ps = [p(x) for x in xs]
    imax = next(i for i in range(1, n) if ps[i] >= ps[i - 1] and ps[i] > ps[i + 1])
    imin = next(i for i in range(imax + 1, n) if ps[i] <= ps[i - 1] and ps[i] < ps[i + 1])
    r1 = optimize.minimize_scalar(lambda x: -p(x), bounds=(xs[imax - 1], xs[imax + 1]),
                                  method="bounded", options={"xatol": 1e-13}).x
    r2 = optimize.minimize_scalar(p, bounds=(xs[imin - 1], xs[imin + 1]),
                                  method="bounded", options={"xatol": 1e-13}).x
    return r1, r2


def _branches(p, pc, r1, r2, rho_max, rho_min=1e-14):
    """Gas and liquid densities with p(rho) = pc, on either side of the spinodals."""
    rg = optimize.brentq(lambda r: p(r) - pc, rho_min, r1, xtol=1e-16, rtol=1e-15, maxiter=500)
    hi = r2
    while p(hi) < pc:
        hi = 0.5 * (hi + rho_max)
        if rho_max - hi < 1e-12:
            raise ValueError("no liquid branch")
    rl = optimize.brentq(lambda r: p(r) - pc, r2, hi, xtol=1e-16, rtol=1e-15, maxiter=500)
    return rg, rl


def _integral(fn, a, b):
    """int_a^b fn(rho) drho, integrated in s = log(rho)."""
    with warnings.catch_warnings():   # quad's roundoff notice at the 1e-15 floor
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        val, _err = integrate.quad(lambda s: fn(math.exp(s)) * math.exp(s), math.log(a),
                                   math.log(b), epsabs=1e-15, epsrel=1e-12, limit=500)
    return val


def _solve(p, weight, scan_hi=0.95, rho_max=_RHO_MAX):
    r1, r2 = _spinodals(p, hi=scan_hi)
    p_hi = p(r1)
    p_lo = max(p(r2), 1e-300)

    def area(pc):
        rg, rl = _branches(p, pc, r1, r2, rho_max)
        return _integral(lambda r: (pc - p(r)) * weight(r), rg, rl)

    # area(pc) < 0 just above p_lo and > 0 at p_hi; bracket away from the ends.
    a = p_lo * (1 + 1e-9) if p_lo > 1e-300 else p_hi * 1e-12
    while area(a) > 0:
        a *= 0.5
    b = p_hi * (1 - 1e-12)
    pc = optimize.brentq(area, a, b, xtol=1e-18, rtol=1e-14, maxiter=500)
    rg, rl = _branches(p, pc, r1, r2, rho_max)
    return rg, rl, pc


def cs_pressure(T_over_Tc: float, K: float = 1.0):
    T = T_over_Tc * Tc()
    return lambda r: pressure(r, T, K)


def maxwell(T_over_Tc: float, K: float = 1.0):
    """Eq. 19 for the Eq. 30 EOS: returns (rho_g, rho_l, p_c)."""
    return maxwell_for(cs_pressure(T_over_Tc, K))


def maxwell_for(p: Callable[[float], float], **kw):
    """Eq. 19 for any isotherm p(rho); kw: scan_hi, rho_max (search range)."""
    return _solve(p, lambda r: 1.0 / (r * r), **kw)


def mechanical(T_over_Tc: float, K: float, eps: float):
    """Eq. 18 with psi = sqrt(2(rho/3 - p0)), p0 from Eq. 30: returns (rho_g, rho_l, p_c)."""
    p = cs_pressure(T_over_Tc, K)
    psi = lambda r: math.sqrt(2.0 * (r / 3.0 - p(r)))
    return mechanical_for(p, psi, eps)


def mechanical_for(p: Callable[[float], float], psi: Callable[[float], float], eps: float, **kw):
    """Eq. 18 for any isotherm p(rho) and effective density psi(rho)."""
    def weight(r):
        h = 1e-6 * r
        dpsi = (psi(r + h) - psi(r - h)) / (2.0 * h)   # central difference for psi'
        return dpsi / psi(r) ** (1.0 + eps)
    return _solve(p, weight, **kw)
