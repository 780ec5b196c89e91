"""Coefficients of the normal CDF used by the surrogate's GELU epilogues.

The kernels evaluate Phi(z) as a logistic of an odd polynomial,

    Phi_a(z) = 1 / (1 + 2^(z q(z^2))),   q(u) = c0 + c1 u + c2 u^2 + c3 u^3 + c4 u^4,

one hardware exp2 and one hardware reciprocal per element (the logistic
approximation of the normal CDF with a cubic exponent is a textbook form;
the quartic q here only adds terms).  GELU(z) = z Phi(z), so the fit
minimises the largest |z (Phi_a(z) - Phi(z))| over [-14, 14] (beyond it
Phi_a is 0 or 1 to float32 precision, as Phi is): a least-squares fit
re-weighted toward the largest residuals (Lawson's iteration toward the
minimax fit), started from the logistic form's usual exponent
-2 log2(e) sqrt(2/pi) (z + 0.044715 z^3).

Run: python fit_normal_cdf.py  -- prints the float32 coefficients and the
largest errors of GELU and Phi over a fine grid (the kernels' constants are
these values).
"""
import numpy as np
from scipy.optimize import least_squares
from scipy.special import ndtr


def phi_a(c, z):
    s = z * np.polyval(np.asarray(c)[::-1], z * z)
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp2(s))


def fit(degree=4, lo=-14.0, hi=14.0, n=112001, rounds=60):
    z = np.linspace(lo, hi, n)
    ref = ndtr(z)
    k = -2.0 * np.log2(np.e) * np.sqrt(2.0 / np.pi)
    c = np.zeros(degree + 1)
    c[0], c[1] = k, k * 0.044715

    def resid(cv):
        return np.abs(z) * (phi_a(cv, z) - ref)

    c = least_squares(resid, c, xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000).x
    w = np.ones_like(z)
    for _ in range(rounds):
        c = least_squares(lambda cv: w * resid(cv), c, xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=5000).x
        r = np.abs(resid(c))
        w = w * (1.0 + r / r.max()) ** 2
        w /= w.max()
    c32 = c.astype(np.float32)
    e = resid(c32.astype(np.float64))
    return c32, float(np.abs(e).max()), float(np.abs(phi_a(c32.astype(np.float64), z) - ref).max())


if __name__ == "__main__":
    c, eg, ep = fit()
    print("coefficients (float32):", ", ".join(f"{x:.9e}" for x in c))
    print(f"max |z (Phi_a - Phi)| = {eg:.3e}, max |Phi_a - Phi| = {ep:.3e}")
