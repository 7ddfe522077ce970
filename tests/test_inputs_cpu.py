"""The seeded input generator shared by the oracle and the CUDA path
(paper_1004_5058_gb300/inputs.py): SplitMix64 against its published test
vector, and the input recipe's closed forms (CPU only)."""
import json
import math
import os

import numpy as np

from paper_1004_5058_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.json")))


def test_splitmix64_published_vector():
    got = [int(v) for v in I.splitmix64(GOLD["seed"], 5)]
    assert got == GOLD["first_outputs"]
    # counter form: any window of the stream equals the same slice of the whole
    whole = I.splitmix64(GOLD["seed"], 40)
    assert np.array_equal(I.splitmix64(GOLD["seed"], 7, offset=20), whole[20:27])


def test_uniform_doubles_are_the_top_53_bits():
    z = I.splitmix64(99, 1000)
    u = I.uniform01(99, 1000)
    assert np.all((u >= 0.0) & (u < 1.0))
    assert np.array_equal(u, (z >> np.uint64(11)).astype(np.float64) / 2.0 ** 53)
    assert abs(u.mean() - 0.5) < 0.03  # 1000 draws: 3.5 standard errors


def test_random_fields_recipe():
    ra, rb = I.random_fields(16, 8, n_cells=3, rho_bar=0.6, amp=0.1, seed=5)
    assert ra.shape == rb.shape == (3, 8, 16)
    xi = 2.0 * I.uniform01(5, 3 * 8 * 16) - 1.0
    np.testing.assert_array_equal(ra.ravel(), 0.6 * (1.0 + 0.1 * xi))
    np.testing.assert_array_equal(rb.ravel(), 0.6 * (1.0 - 0.1 * xi))
    assert np.all(np.abs(ra + rb - 1.2) < 1e-15)


def test_couette_start_and_speeds():
    ux, uy = I.couette_velocity(4, 10, [1e-3, 2e-3], n_cells=2)
    y = np.arange(10)
    np.testing.assert_allclose(ux[1, :, 0], 2e-3 * (2 * (y + 0.5) / 10 - 1), rtol=0, atol=1e-18)
    assert np.all(uy == 0.0) and np.all(ux[:, :, 0:1] == ux)  # x-invariant
    # walls at y = -1/2 and ny - 1/2 move at -U and +U: the profile reaches them linearly
    assert math.isclose(ux[0, 0, 0] - (ux[0, 1, 0] - ux[0, 0, 0]) / 2, -1e-3, rel_tol=1e-12)
    s = I.log_spaced(1e-4, 1e-2, 8)
    assert s[0] == 1e-4 and math.isclose(s[-1], 1e-2, rel_tol=1e-15)
    assert np.allclose(np.diff(np.log10(s)), 2.0 / 7.0)


def test_paper_sine_start():
    ra, rb = I.sine_fields(8, 128)  # k_in = 64 pi / L = pi / 2 (at L = 64 it would vanish on the lattice)
    k = 64 * math.pi / 128
    y = np.arange(128)
    assert np.ptp(ra[0, :, 3]) > 0.1
    np.testing.assert_allclose(ra[0, :, 3], 0.61 * (1 + 0.1 * np.sin(k * y)), rtol=0, atol=1e-15)
    np.testing.assert_allclose(rb[0, :, 3], 0.61 * (1 + 0.01 * np.sin(k * y)), rtol=0, atol=1e-15)
    na, nb = I.sine_fields(8, 128, noise=1e-3, seed=3)
    assert 0 < np.abs(na / ra - 1).max() <= 1e-3 and 0 < np.abs(nb / rb - 1).max() <= 1e-3
