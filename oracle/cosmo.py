"""Background cosmology and leapfrog factors (Section 2.3.3, "timestep").

Units: H0 = 1, lengths in fine cells.  With p = a^2 dx/dt = a^3 E dx/da and
lap Phi = (3/2) Omega_m (rho - 1):
    dx/da = p / (a^3 E(a)),     dp/da = -grad Phi / (a^2 E(a)).
(The paper is silent on the equations of motion; these are the comoving
equations in the units above.)  The kick over [a0, a1] multiplies -grad Phi
by int da / (a^2 E); the drift over [a0, a1] multiplies p by int da / (a^3 E).
"""
import math

from scipy import integrate


def E(a, om, ol):
    """H(a)/H0."""
    ok = 1.0 - om - ol
    return math.sqrt(om / a ** 3 + ok / a ** 2 + ol)


def kick_factor(a0, a1, om, ol):
    """int_{a0}^{a1} da / (a^2 E(a))   (adaptive quadrature, FP64)."""
    if a1 == a0:
        return 0.0
    return integrate.quad(lambda a: 1.0 / (a * a * E(a, om, ol)), a0, a1,
                          epsabs=0.0, epsrel=1e-13, limit=200)[0]


def drift_factor(a0, a1, om, ol):
    """int_{a0}^{a1} da / (a^3 E(a))   (adaptive quadrature, FP64)."""
    if a1 == a0:
        return 0.0
    return integrate.quad(lambda a: 1.0 / (a ** 3 * E(a, om, ol)), a0, a1,
                          epsabs=0.0, epsrel=1e-13, limit=200)[0]


def _heath(a, om, ol):
    return integrate.quad(lambda x: 1.0 / (x * E(x, om, ol)) ** 3, 0.0, a,
                          epsabs=0.0, epsrel=1e-13, limit=200)[0]


def growth(a, om, ol):
    """Linear growth D(a) (Heath integral), normalised to D(1) = 1."""
    d = lambda x: 2.5 * om * E(x, om, ol) * _heath(x, om, ol)
    return d(a) / d(1.0)


def growth_rate(a, om, ol):
    """f = dlnD/dlna for the Heath solution."""
    e = E(a, om, ol)
    ok = 1.0 - om - ol
    dlnE = (-1.5 * om / a ** 3 - ok / a ** 2) / (e * e)
    return dlnE + 1.0 / (a * a * e ** 3 * _heath(a, om, ol))


def momentum_growth(a, om, ol):
    """g(a) = a^2 E f D: growth of p in linear theory (p = g Psi)."""
    return a * a * E(a, om, ol) * growth_rate(a, om, ol) * growth(a, om, ol)
