"""Host analysis routines of the study runners (CPU only)."""
import json
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_vft_fit_recovers_the_papers_parameters():
    from paper_1004_5058_gb300.studies import vft_fit
    g = GOLD["vft_fit_reciprocal_response"]["value"]
    r0 = np.array([0.70, 0.74, 0.78, 0.81, 0.83, 0.85, 0.86])
    inv = g["A"] * np.exp(g["B"] / (g["rho_c"] - r0))
    f = vft_fit(r0, inv)
    assert f["A"] == pytest.approx(g["A"], rel=1e-8)
    assert f["B"] == pytest.approx(g["B"], rel=1e-8)
    assert f["rho_c"] == pytest.approx(g["rho_c"], rel=1e-10)


def test_kolmogorov_forcing_amplitude():
    """F0 = rho nu k^2 U0 reproduces the paper's sigma_0 = rho nu U0 2 pi / L = F0 / k
    ~ 2.5e-4 at U0 = 0.1, L = 512, tau = 1, rho = 2 x 0.61."""
    from paper_1004_5058_gb300 import inputs as I
    import math
    L = 512
    f0 = I.kolmogorov_f0(0.1, L, rho=1.22, tau=1.0)
    sigma0 = f0 / (2 * math.pi / L)
    assert sigma0 == pytest.approx(GOLD["kolmogorov_sigma0"]["value"], rel=0.01)
