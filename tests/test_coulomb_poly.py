"""The polynomial form of the screened-Coulomb force term that the LJ-electrolyte force pass
evaluates (Eqs. 9-11: -du/dr / r of K q_i q_j erfc(alpha r)/r is
K q_i q_j (erfc(x) + 2x/sqrt(pi) e^{-x^2}) / r^3 with x = alpha r), checked on the host
against scipy's erfc in FP64: r^-3 + C(r^2) with the library's float32 coefficients
reproduces the erfc form within 5e-7 relative on (0, rc] for the configurations'
alpha = 0.3, rc = 4 and across the range where the form is used; outside it the
library reports that the engine keeps the erfc form.  No GPU is needed."""
import numpy as np
import pytest
from scipy.special import erfc

from paper_2307_11447_gb300 import lib as h4d


def erfc_force_term(alpha, r):
    x = alpha * r
    return (erfc(x) + 2.0 * x / np.sqrt(np.pi) * np.exp(-x * x)) / r**3


def poly_force_term(coef, r):
    s = r * r
    p = np.zeros_like(s)
    for c in coef[::-1].astype(np.float64):
        p = p * s + c
    return 1.0 / r**3 + p


@pytest.mark.parametrize("alpha,rc", [(0.3, 4.0), (0.1, 4.0), (0.3, 2.5), (0.5, 2.5), (0.0, 4.0), (0.325, 4.0)])
def test_polynomial_matches_erfc_form(alpha, rc):
    coef, used = h4d.h4d_coulomb_poly(alpha, rc)
    assert used
    r = np.linspace(rc / 4000.0, rc, 4000)
    exact = erfc_force_term(alpha, r)
    rel = np.abs(poly_force_term(coef, r) - exact) / exact
    assert rel.max() < 5e-7, rel.max()


def test_unscreened_limit_is_plain_coulomb():
    """alpha = 0: erfc(0) = 1, the force term is r^-3 and C vanishes"""
    coef, used = h4d.h4d_coulomb_poly(0.0, 4.0)
    assert used and np.all(coef == 0.0)


def test_beyond_the_range_the_erfc_form_is_kept():
    coef, used = h4d.h4d_coulomb_poly(0.3, 5.0)  # alpha rc = 1.5
    assert not used and np.all(coef == 0.0)
    coef, used = h4d.h4d_coulomb_poly(0.3, 0.0)
    assert not used


def test_leading_coefficient_is_the_series_term():
    """C(s) = alpha^3 H(alpha^2 s), H(0) = -4/(3 sqrt(pi)): the constant term of the
    interpolant approaches it (the fit is not a Taylor expansion, so only closely)"""
    alpha = 0.3
    coef, _ = h4d.h4d_coulomb_poly(alpha, 4.0)
    assert coef[0] == pytest.approx(alpha**3 * (-4.0 / (3.0 * np.sqrt(np.pi))), rel=1e-5)
