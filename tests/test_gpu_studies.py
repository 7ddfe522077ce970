"""The study runners (paper_1004_5058_gb300/studies.py) at toy sizes: each
returns its documented keys with finite values, so the full-size runs whose
results the docs quote stay runnable."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def finite(x):
    return x is not None and math.isfinite(float(x))


def test_precision_study_small():
    from paper_1004_5058_gb300 import studies
    r = studies.precision_study(n=128, steps=400, every=10, g_ab=0.045)
    assert set(r) >= {"fp64", "fp32", "fp16", "fp16sr"}
    for p in ("fp32", "fp16", "fp16sr"):
        assert finite(r[p]["sigma_rel_err"]) and finite(r[p]["max_abs_drho"]) and r[p]["mlups"] > 0
    assert r["fp64"]["mass_drift"] < 1e-12


def test_couette_flow_curves_small():
    from paper_1004_5058_gb300 import studies
    r = studies.couette_flow_curve(n=64, n_speeds=4, steps=2000, every=10)
    assert len(r["sigma_xy"]) == 4 and r["samples"] == 100 and r["points_per_s"] > 0
    b = studies.flow_curve(L=64, steps=1000, n_speeds=4, g_abs=(0.3, 0.405))
    s = studies.flow_curve(L=64, steps=1000, n_speeds=4, g_abs=(0.3, 0.405), sequential=True)
    for g in ("0.3", "0.405"):  # batching changes nothing but the rounding of the FP64 sums
        np.testing.assert_allclose(b["curves"][g]["sigma_xy"], s["curves"][g]["sigma_xy"], rtol=1e-9, atol=1e-15)


def test_kolmogorov_runners_small():
    from paper_1004_5058_gb300 import studies
    r = studies.kolmogorov(L=64, steps=3000, every=50, rho0s=(0.83,), u0s=(0.1, 0.4))
    assert len(r["runs"]) == 2 and all(finite(x["R"]) for x in r["runs"])
    assert "0.83" in r["master"]
    s = studies.kolmogorov_rho0_sweep(L=64, steps=3000, rho0s=(0.70, 0.74, 0.78, 0.82, 0.86), r_floor=0.0)
    assert len(s["runs"]) == 5 and "vft" in s


def test_surrogate_study_small():
    from paper_1004_5058_gb300 import studies
    r = studies.surrogate_study(n_train=24, n_test=8, n_speeds=8, L=32, steps=2000, epochs=30, batch=64)
    assert r["train_points"] > 0 and 0.0 <= r["served_fraction"] <= 1.0
    assert r["network_queries_per_s"] > 0 and len(r["error_table_by_logS_bin"]) == 8


def test_two_time_flow_curve_small():
    """One batch over three tau_B values, one curve and fit slot per value; the
    relaxation time of B changes the stresses.  (The sign of the wall stress is
    not asserted: in a short run of a demixing cell the rearranging domains give
    stresses of either sign even at the highest wall speed.)"""
    from paper_1004_5058_gb300 import studies
    r = studies.two_time_flow_curve(L=64, steps=2000, every=10, n_speeds=4, tau_bs=(0.7, 1.0, 1.5))
    assert set(r["curves"]) == {"0.7", "1.0", "1.5"} and r["mlups"] > 0
    for c in r["curves"].values():
        assert len(c["sigma_xy"]) == 4 and all(finite(v) for v in c["sigma_xy"] + c["shear_rate"])
    assert r["curves"]["0.7"]["sigma_xy"][-1] != r["curves"]["1.5"]["sigma_xy"][-1]


def test_mrt_flow_curve_small():
    """Multiple relaxation times beside BGK in one batch: in the mixed fluid
    (G_AB = 0.3) the Newtonian ratio sigma/S is rho nu with nu = (1/s_nu - 1/2)/3,
    a quarter of the BGK value at tau = 1 for s_nu = 1.6 (tau still 1)."""
    from paper_1004_5058_gb300 import studies
    r = studies.mrt_flow_curve(L=32, steps=3000, every=10, n_speeds=4)
    assert set(r["curves"]) == {c[0] for c in studies.MRT_CONFIGS} and r["mlups"] > 0
    for label, nu in (("BGK, G_AB 0.30", 1 / 6), ("MRT s_nu 1.6, G_AB 0.30", (1 / 1.6 - 0.5) / 3)):
        for ratio in r["curves"][label]["sigma_over_S"][-2:]:
            assert ratio == pytest.approx(1.2 * nu, rel=0.05)
