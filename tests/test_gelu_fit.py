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
    for name in ("C0", "C1", "C2", "Z2MAX", "TANH_SCALE"):
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


def test_tanh_form_of_the_fit():
    """The kernel's form (z / 2)(1 + tanh(z q')) with q' = q ln2 / 2, its three
    coefficients rounded to float32 as the device computes them."""
    c = _constants()
    assert abs(c["TANH_SCALE"] - np.log(2.0) / 2) < 2e-8
    h = np.float32(c["TANH_SCALE"])
    c0, c1, c2 = (float(np.float32(c[k]) * h) for k in ("C0", "C1", "C2"))
    z = np.linspace(-30.0, 30.0, 600001)
    s = np.minimum(z * z, c["Z2MAX"])
    q = (c2 * s + c1) * s + c0
    g = 0.5 * z * (1.0 + np.tanh(z * q))
    gelu = z * 0.5 * (1.0 + erf(z / np.sqrt(2.0)))
    assert np.max(np.abs(g - gelu)) < 6e-5
    assert np.max(np.abs(g - z * _phi_fit(z, c))) < 1e-6  # the same function as the base-2 form
