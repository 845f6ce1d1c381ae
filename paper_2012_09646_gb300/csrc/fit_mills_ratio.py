"""Derivation of the Mills-ratio approximation used by the B&S kernel.

The standard normal CDF is written as N(x) = phi(x) R(-x) for x < 0 and
N(x) = 1 - phi(x) R(x) for x >= 0, where R(z) = (1 - N(z)) / phi(z) is the
Mills ratio (smooth and decreasing on z >= 0, R(0) = sqrt(pi/2), R(z) ~ 1/z).
R is approximated by a rational function P(u)/Q(u), u = z/4, deg P = 4,
deg Q = 5, with every coefficient constrained to be >= 0 so that fp32 Horner
evaluation has no cancellation.  (Degree 4/5 reaches a relative error of
about 4e-8 on [0, 4] and 1e-6 beyond, where the tail it multiplies is below
3e-5, so its share of a call price's error stays far below fp32 rounding.)  The fit is a linearised least-squares
problem y Q(u) - P(u) = 0 (y = R(z) from scipy.special.erfcx) with Lawson
re-weighting towards minimax relative error; the coefficients are printed
rescaled to z (P also multiplied by 1/sqrt(2 pi), the constant of phi) in
the form k_bs.cu uses.  Run: python fit_mills_ratio.py
"""
import numpy as np
import scipy.special as sp
from scipy.optimize import lsq_linear

SCALE = 4.0


def mills(z):
    return sp.erfcx(z / np.sqrt(2.0)) * np.sqrt(np.pi / 2.0)


def fit(m=4, zmax=40.0, iters=60):
    z = np.concatenate([np.linspace(0, 8, 6000), np.geomspace(8, zmax, 3000)])
    u = z / SCALE
    y = mills(z)
    lw = np.ones_like(z)
    den = np.ones_like(z)
    best = None
    for _ in range(iters):
        A = np.zeros((z.size, 2 * m + 2))
        for k in range(m + 1):
            A[:, k] = u ** k
        for k in range(1, m + 2):
            A[:, m + k] = -y * u ** k
        w = lw / (y * den)
        c = lsq_linear(A * w[:, None], y * w, bounds=(0, np.inf), method="bvls").x
        p, q = c[: m + 1], np.concatenate([[1.0], c[m + 1:]])
        den = np.polyval(q[::-1], u)
        e = np.abs(np.polyval(p[::-1], u) / den - y) / y
        if best is None or e.max() < best[0]:
            best = (e.max(), p.copy(), q.copy())
        lw = lw * np.maximum(e / e.max(), 1e-3)
        lw /= lw.mean()
    return best


if __name__ == "__main__":
    err, p, q = fit()
    zz = np.concatenate([np.linspace(0, 8, 400001), np.geomspace(8, 1e5, 20000)])
    e = np.abs(np.polyval(p[::-1], zz / SCALE) / np.polyval(q[::-1], zz / SCALE) - mills(zz)) / mills(zz)
    print("max relative error on [0, 1e5]: %.3g, on [0, 4]: %.3g" % (e.max(), e[zz <= 4].max()))
    k = np.arange(p.size)
    pz = p / SCALE ** k / np.sqrt(2.0 * np.pi)
    qz = q / SCALE ** np.arange(q.size)
    print("P (z, highest first):", ", ".join("%.9ef" % v for v in pz[::-1]))
    print("Q (z, highest first):", ", ".join("%.9ef" % v for v in qz[::-1]))
