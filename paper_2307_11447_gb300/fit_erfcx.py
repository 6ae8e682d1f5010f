"""Coefficients of the scaled complementary error function used by the aqueous pair term.

erfcx(x) = exp(x^2) erfc(x) is smooth and slowly varying on [0, X]; it is approximated as
t * sum_k c_k t^k with t = 1 / (1 + x / 2), fitted here by least squares in relative error
and reweighted toward the minimax solution (Lawson's iteration), against SciPy's erfcx
(double precision) on a fine grid.  The engine then forms erfc(x) = exp(-x^2) erfcx(x),
sharing exp(-x^2) with the force term.  Run to print the coefficients and the fit's
relative error (exact arithmetic and a float32 evaluation with fused multiply-adds).
"""
import numpy as np
from scipy import special

X_MAX = 3.2   # the pair term needs x = alpha r4 < alpha rc (2.5 for the aqueous system)
DEGREE = 9
P = 0.5


def fit(x_max=X_MAX, degree=DEGREE, p=P, n=40001, rounds=30):
    x = np.linspace(0.0, x_max, n)
    t = 1.0 / (1.0 + p * x)
    f = special.erfcx(x)
    V = np.vander(t, degree + 1, increasing=True)
    w = 1.0 / f
    for _ in range(rounds):
        c, *_ = np.linalg.lstsq(V * (t * w)[:, None], f * w, rcond=None)
        err = (t * (V @ c) - f) / f
        w = w * (1.0 + 50.0 * np.abs(err) / np.abs(err).max())
    return c, float(np.abs(err).max())


def float32_error(c, x_max=X_MAX, p=P, n=40001):
    x = np.linspace(0.0, x_max, n).astype(np.float32)
    den = (np.float64(p) * x.astype(np.float64) + 1.0).astype(np.float32)
    t = (1.0 / den.astype(np.float64)).astype(np.float32)
    cf = np.asarray(c, np.float64).astype(np.float32)
    acc = np.full_like(t, cf[-1])
    for k in range(len(cf) - 2, -1, -1):
        acc = (acc.astype(np.float64) * t.astype(np.float64) + np.float64(cf[k])).astype(np.float32)
    v = (acc.astype(np.float64) * t.astype(np.float64)).astype(np.float32)
    f = special.erfcx(x.astype(np.float64))
    return float((np.abs(v.astype(np.float64) - f) / f).max())


if __name__ == "__main__":
    c, e = fit()
    print("coefficients c_0 .. c_%d:" % DEGREE)
    for k, v in enumerate(np.asarray(c, np.float64).astype(np.float32)):
        print(f"  c{k} = {float(v):.9e}")
    print(f"max relative error: fit {e:.2e}, float32 evaluation {float32_error(c):.2e}")
