"""Fit the circular Gaussian-mixture stand-ins for the exponential and de Vaucouleurs
galaxy light profiles.

The paper describes each galaxy by a shape/scale/morphology vector and defers the
profile formulas to its single-threaded predecessor; that predecessor's mixture
tables are not available here, so this script fits its own.  Each profile is a
Sersic law I(r) ~ exp(-b_n r^(1/n)) (n = 1 exponential, n = 4 de Vaucouleurs) with
b_n chosen so that the half-light radius is 1.  It is approximated by
    M(r) = sum_j nu_j N(r; 0, tau_j I_2),   sum_j nu_j = 1,
with 6 components for the exponential and 8 for de Vaucouleurs, by least squares of
(M - I) in the flux-weighted 2-D L2 norm on r in (0, r_max].  The fitted variances
are then rescaled by one common factor so that the mixture's own half-light radius is
exactly 1.

Run:  python -m synth.fit_mixtures   (prints the tables pasted into synth/mixtures.py)
"""
import math

import numpy as np
from scipy import optimize, special


def sersic_b(n):
    """b_n with P(2n, b_n) = 1/2 (regularised lower incomplete gamma), i.e. unit half-light radius."""
    return optimize.brentq(lambda b: special.gammainc(2 * n, b) - 0.5, 1e-3, 50.0)


def sersic_profile(r, n):
    """Unit-flux Sersic surface brightness with half-light radius 1."""
    b = sersic_b(n)
    total = 2.0 * math.pi * n * math.gamma(2 * n) / b ** (2 * n)
    return np.exp(-b * r ** (1.0 / n)) / total


def mixture_profile(r, nu, tau):
    return (nu[None, :] / (2 * math.pi * tau[None, :]) * np.exp(-0.5 * r[:, None] ** 2 / tau[None, :])).sum(1)


def mixture_half_light_radius(nu, tau):
    nu = nu / nu.sum()
    g = lambda r: (nu * (1.0 - np.exp(-0.5 * r * r / tau))).sum() - 0.5
    return optimize.brentq(g, 1e-6, 1e3)


def fit(n, K, r_max, seed=0):
    r = np.geomspace(1e-4, r_max, 4000)
    dr = np.gradient(r)
    w = np.sqrt(2 * math.pi * r * dr)
    target = sersic_profile(r, n)

    def unpack(p):
        z, lt = p[:K], p[K:]
        nu = np.exp(z - z.max())
        return nu / nu.sum(), np.exp(lt)

    def resid(p):
        nu, tau = unpack(p)
        return w * (mixture_profile(r, nu, tau) - target)

    best = None
    rng = np.random.default_rng(seed)
    for trial in range(12):
        lt0 = np.sort(np.linspace(-9 if n == 4 else -5, 2.5, K) + rng.normal(0, 0.3, K))
        p0 = np.concatenate([np.zeros(K), lt0])
        sol = optimize.least_squares(resid, p0, method="lm", max_nfev=20000, xtol=1e-15, ftol=1e-15)
        if best is None or sol.cost < best.cost:
            best = sol
    nu, tau = unpack(best.x)
    order = np.argsort(tau)
    nu, tau = nu[order], tau[order]
    hlr = mixture_half_light_radius(nu, tau)
    tau = tau / hlr ** 2
    return nu, tau, best.cost


if __name__ == "__main__":
    for name, n, K, rmax in (("EXP", 1, 6, 8.0), ("DEV", 4, 8, 10.0)):
        nu, tau, cost = fit(n, K, rmax)
        print(f"# {name}: residual cost {cost:.3e}, half-light radius {mixture_half_light_radius(nu, tau):.12f}")
        print(f"{name}_NU = np.array([{', '.join(repr(float(v)) for v in nu)}])")
        print(f"{name}_TAU = np.array([{', '.join(repr(float(v)) for v in tau)}])")
