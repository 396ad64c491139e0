"""The tensor-core surrogate's GELU: the logistic fit of the normal CDF declared in
paper_2210_06713_gb300/csrc/gelu_fit.h, checked against erf over [-30, 30]."""
import os
import re

import numpy as np
from scipy.special import erf

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2210_06713_gb300", "csrc", "gelu_fit.h")


def _constants():
    text = open(HDR).read()
    out = {}
    for name in ("C0", "C1", "C2", "Z2MAX"):
        m = re.search(r"#define DFP2S_GELU_%s\s+(\S+)f" % name, text)
        lit = m.group(1)
        out[name] = float.fromhex(lit) if "0x" in lit else float(lit)
    return out


def _phi_fit(z, c):
    s = np.minimum(z * z, c["Z2MAX"])
    q = (c["C2"] * s + c["C1"]) * s + c["C0"]
    return 1.0 / (1.0 + np.exp2(-z * q))


def test_logistic_fit_of_the_normal_cdf():
    c = _constants()
    z = np.linspace(-30.0, 30.0, 600001)
    phi = 0.5 * (1.0 + erf(z / np.sqrt(2.0)))
    fit = _phi_fit(z, c)
    assert np.max(np.abs(fit - phi)) < 2e-5
    assert np.max(np.abs(z * (fit - phi))) < 6e-5  # GELU error
    assert np.all(np.diff(fit) >= 0)               # monotone, 0 and 1 at the ends
    assert fit[0] < 1e-30 and fit[-1] == 1.0
