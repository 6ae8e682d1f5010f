"""The fitted erfcx of the aqueous pair term (the engine forms erfc(x) = exp(-x^2)
erfcx(x) on [0, 3.2]): the coefficients compiled into the engine are those the committed
generator fits, the fit is accurate to 1e-9 relative in exact arithmetic, and its float32
evaluation (the engine's fused multiply-adds) to 4e-7 relative, about the library erfcf's
error.  CPU only."""
import os
import re

import numpy as np

from paper_2307_11447_gb300 import fit_erfcx as fx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _engine_coefficients():
    src = open(os.path.join(ROOT, "paper_2307_11447_gb300", "csrc", "h4d_engine.cu")).read()
    body = src[src.index("float erfcx_poly(float x)"):]
    body = body[: body.index("return p * t;")]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    return np.array(vals[::-1], np.float64)  # Horner runs from c_9 down to c_0


def test_engine_coefficients_are_the_fit():
    c, err = fx.fit()
    assert err < 1e-9
    eng = _engine_coefficients()
    assert len(eng) == fx.DEGREE + 1
    assert np.array_equal(eng.astype(np.float32), np.asarray(c, np.float64).astype(np.float32))


def test_float32_evaluation_error():
    c, _ = fx.fit()
    assert fx.float32_error(c) < 4e-7
    # erfcx(0) = 1 and the sum of the coefficients is erfcx(0)
    assert abs(np.sum(c) - 1.0) < 1e-9
