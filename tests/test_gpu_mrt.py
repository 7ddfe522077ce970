"""GPU parity of the multiple-relaxation-time collision (a method variant, not
in the paper: the orthogonal D2Q9 moments of Lallemand and Luo, density and
momentum relaxing with 1/tau_s, e, eps, q and p with the cell's s_e, s_eps,
s_q, s_nu) against the FP64 oracle on the same seeded inputs, through the C ABI.

Tolerances are those of the BGK model (test_gpu_parity.py, test_gpu_two_tau.py):
the correction adds a few operations on the non-equilibrium parts f - f^eq,
which are small next to f, so the rounding stays that of the BGK update.
"""
import struct

import numpy as np
import pytest

from paper_1004_5058_gb300 import inputs as I
from tests._util import max_abs, oracle_runs

pytestmark = pytest.mark.gpu

KERNELS = ["generic", "tiled"]
RATES = dict(s_e=1.4, s_eps=1.1, s_q=1.2, s_nu=1.1)  # stable with the demixing couplings


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def lattice(cells, prec, kernel):
    from paper_1004_5058_gb300 import Lattice
    lat = Lattice(cells, prec)
    lat.set_kernel(kernel)
    return lat


def evolved(cell, steps, seed):
    from oracle import lb as orc
    ra, rb = I.random_fields(cell.nx, cell.ny, seed=seed)
    ux = uy = None
    if cell.bc == 1:
        ux, uy = I.couette_velocity(cell.nx, cell.ny, cell.u_wall)
        ux, uy = ux[0], uy[0]
    return orc.Run(cell, ra[0], rb[0], ux, uy).step(steps).f.copy()


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec,tol", [("fp64", 2e-15), ("fp32", 4e-7), ("fp16", 2.0 ** -11), ("fp16sr", 2.0 ** -10)])
@pytest.mark.parametrize("case", ["couette", "kolmogorov"])
@pytest.mark.parametrize("taus", [(1.0, 0.0), (0.8, 1.3)], ids=["tau1", "0.8-1.3"])
def test_one_step_mrt(kernel, prec, tol, case, taus):
    """One step from an evolved demixing state, with all four rates set; tau = 1
    would take f* = f^eq under BGK and must take the general update here."""
    from oracle import lb as orc
    bc = 1 if case == "couette" else 0
    cell = I.make_cell("paper", nx=64, ny=48, g_ab=0.405, bc=bc, u_wall=0.02 if bc else 0.0,
                       f0=0.0 if bc else I.kolmogorov_f0(0.05, 48), tau=taus[0], tau_b=taus[1], **RATES)
    f0 = evolved(cell, 300, seed=61)
    with lattice([cell], prec, kernel) as lat:
        lat.set_populations(f0[None])
        start = lat.get_populations()[0]
        lat.set_sampling(0, 1).step(1)
        g1 = lat.get_populations()[0]
        sigma, _, _ = lat.shear_stress()
        ub, ns = lat.profile()
    f1, obs, prof = orc.step(cell, start, want_profile=True)
    if prec.startswith("fp16"):
        w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[None, :, None, None]
        shift = w * np.array([cell.rho_bar_a, cell.rho_bar_b])[:, None, None, None]
        gmag = np.maximum(np.abs(g1 - shift), np.abs(f1 - shift))
        excess = np.abs(g1 - f1) - (tol * gmag + 5e-7)
        assert excess.max() <= 0.0, (excess.max(), gmag.max())
    else:
        assert max_abs(g1, f1) <= tol
    assert ns == 1
    otol = 1e-14 if prec == "fp64" else 1e-6
    np.testing.assert_allclose(ub[0], prof / cell.nx, rtol=0, atol=otol)
    if bc == 1:
        assert abs(sigma[0] - 0.5 * (obs["pi_top"] - obs["pi_bot"]) / cell.nx) <= otol


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_1000_steps_mrt_conserve_mass_and_momentum(kernel, prec, tol):
    """64 x 64 periodic, footnote couplings, two times and all four rates: fields
    against the oracle after 1000 steps, species masses and total momentum kept."""
    cell = I.make_cell("paper", nx=64, ny=64, tau=0.7, tau_b=1.3, **RATES)
    ra, rb = I.random_fields(64, 64, seed=1004)
    with lattice([cell], prec, kernel) as lat:
        lat.init_fields(ra, rb).step(1000)
        ga, gb, gu, gv = lat.fields()
        mass, mom = lat.reductions()
    (r,) = oracle_runs([cell], ra, rb, steps=1000)
    oa, ob, ou, ov = r.fields()
    assert max_abs(ga[0], oa) <= tol and max_abs(gb[0], ob) <= tol
    assert max_abs(gu[0], ou) <= tol and max_abs(gv[0], ov) <= tol
    m0 = (ra.sum(), rb.sum())
    mtol = 1e-13 if prec == "fp64" else 2e-6
    assert abs(mass[0, 0] - m0[0]) / m0[0] <= mtol and abs(mass[0, 1] - m0[1]) / m0[1] <= mtol
    assert abs(mom[0]).max() / (m0[0] + m0[1]) <= (1e-13 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-14), ("fp32", 1e-6)])
def test_rates_equal_to_one_over_tau_give_bgk(kernel, prec, tol):
    """Rates all 1/tau take the MRT kernels with a zero correction: the BGK run
    to rounding."""
    out = []
    ra, rb = I.random_fields(64, 48, seed=7)
    ux, uy = I.couette_velocity(64, 48, 0.01)
    for rates in ({}, dict(s_e=1 / 0.8, s_eps=1 / 0.8, s_q=1 / 0.8, s_nu=1 / 0.8)):
        cell = I.make_cell("paper", nx=64, ny=48, g_ab=0.405, bc=1, u_wall=0.01, tau=0.8, **rates)
        with lattice([cell], prec, kernel) as lat:
            lat.init_fields(ra, rb, ux, uy).set_sampling(10, 5).step(40)
            out.append((lat.get_populations(), lat.shear_stress()[0]))
    assert max_abs(out[0][0], out[1][0]) <= tol
    assert abs(out[0][1][0] - out[1][1][0]) <= 1e-3 * abs(out[0][1][0]) + 1e-15


@pytest.mark.parametrize("kernel", KERNELS)
def test_batch_mixing_bgk_and_mrt_cells(kernel):
    """BGK cells (one and two times) and MRT cells in one launch, each against its
    own oracle run (FP64), with stress and shear rate."""
    nx, ny = 64, 32
    spec = [(1e-3, 1.0, 0.0, {}), (3e-3, 1.0, 0.7, {}), (1e-2, 0.8, 1.3, RATES),
            (2e-2, 1.0, 0.0, dict(s_nu=1.6)), (5e-3, 0.9, 0.0, dict(s_e=1.2, s_q=1.3))]
    cells = [I.make_cell("paper", nx=nx, ny=ny, bc=1, u_wall=u, g_ab=0.405, tau=ta, tau_b=tb, **rt)
             for u, ta, tb, rt in spec]
    n = len(cells)
    ra, rb = I.random_fields(nx, ny, n_cells=n, seed=19)
    ux, uy = I.couette_velocity(nx, ny, [c.u_wall for c in cells], n_cells=n)
    with lattice(cells, "fp64", kernel) as lat:
        lat.init_fields(ra, rb, ux, uy).set_sampling(50, 10).step(120)
        ga, gb, _, _ = lat.fields()
        sigma, S, _ = lat.shear_stress()
    for c, r in enumerate(oracle_runs(cells, ra, rb, ux, uy, steps=120, sampling=(50, 10))):
        oa, ob, _, _ = r.fields()
        assert max_abs(ga[c], oa) <= 1e-12 and max_abs(gb[c], ob) <= 1e-12
        osig, oS, _, _ = r.shear()
        assert sigma[c] == pytest.approx(osig, rel=1e-9, abs=1e-16)
        assert S[c] == pytest.approx(oS, rel=1e-9, abs=1e-16)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_mrt_narrow_last_strip(prec, tol):
    """MRT with tiles that do not divide nx (80 = 64 + 16), against the oracle
    after 20 steps, with the sampled profile."""
    from paper_1004_5058_gb300 import Lattice
    nx, ny = 80, 40
    cell = I.make_cell("paper", nx=nx, ny=ny, g_ab=0.405, bc=1, u_wall=0.01, tau=0.9, **RATES)
    ra, rb = I.random_fields(nx, ny, seed=29)
    ux, uy = I.couette_velocity(nx, ny, 0.01)
    with Lattice([cell], prec) as lat:
        lat.set_kernel("tiled", 64, 0)
        assert lat.kernel()[:2] == ("tiled", 64)
        lat.init_fields(ra, rb, ux, uy).set_sampling(5, 5).step(20)
        ga, gb, gu, _ = lat.fields()
        ub, ns = lat.profile()
    (r,) = oracle_runs([cell], ra, rb, ux, uy, steps=20, sampling=(5, 5))
    oa, ob, ou, _ = r.fields()
    assert max_abs(ga[0], oa) <= tol and max_abs(gb[0], ob) <= tol and max_abs(gu[0], ou) <= tol
    _, _, _, oub = r.shear()
    assert ns == 3
    np.testing.assert_allclose(ub[0], oub, rtol=0, atol=tol)


def fnv1a64(data: bytes) -> int:
    h = 1469598103934665603
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_checkpoint_carries_the_rates_and_reads_version_2(tmp_path):
    """A checkpoint holds the four rates: a BGK handle continues with the file's
    MRT collision.  A version-2 file (15 float64 per cell, before the rates)
    loads with rates 0, i.e. BGK."""
    from paper_1004_5058_gb300 import Lattice
    nx, ny = 64, 48
    mrt = [I.make_cell("paper", nx=nx, ny=ny, g_ab=0.405, bc=1, u_wall=0.01, tau=0.8, **RATES)]
    bgk = [I.make_cell("paper", nx=nx, ny=ny, g_ab=0.405, bc=1, u_wall=0.01, tau=0.8)]
    ra, rb = I.random_fields(nx, ny, seed=23)
    ux, uy = I.couette_velocity(nx, ny, 0.01)
    path = tmp_path / "mrt.ckpt"
    with Lattice(mrt, "fp32") as a:
        a.init_fields(ra, rb, ux, uy).step(20)
        f20 = a.get_populations()
        a.save(path)
        a.step(15)
        fa = a.get_populations()
    with Lattice(bgk, "fp32") as b:
        b.load(path).step(15)
        assert np.array_equal(b.get_populations(), fa)
    raw = path.read_bytes()
    assert struct.unpack_from("<I", raw, 8)[0] == 3
    n_cells = struct.unpack_from("<i", raw, 16)[0]
    payload = raw[128:]
    payload_v2 = b"".join(payload[c * 152:c * 152 + 120] for c in range(n_cells)) + payload[n_cells * 152:]
    head = bytearray(raw[:128])
    struct.pack_into("<I", head, 8, 2)
    struct.pack_into("<QQ", head, 72, len(payload_v2), fnv1a64(payload_v2))
    v2 = tmp_path / "v2.ckpt"
    v2.write_bytes(bytes(head) + payload_v2)
    with Lattice(mrt, "fp32") as c:
        c.load(v2).step(15)
        got = c.get_populations()
    with Lattice(bgk, "fp32") as d:
        d.set_populations(f20).step(15)
        ref = d.get_populations()
    assert np.array_equal(got, ref)
    assert not np.array_equal(got, fa)


@pytest.mark.parametrize("kernel", KERNELS)
def test_mrt_fp16_stochastic_rounding_keeps_mass(kernel):
    """The multiple-relaxation-time collision in FP16 storage: over 3000 steps of
    a near-uniform mixed state, stochastic rounding keeps the species masses to
    2e-6 and well below round to nearest, and both stay close to the FP64 oracle
    (the bounds of the BGK test)."""
    cell = I.make_cell("paper", nx=64, ny=64, **RATES)
    ra, rb = I.random_fields(64, 64, seed=21)
    m0 = np.array([ra.sum(), rb.sum()])
    (r,) = oracle_runs([cell], ra, rb, steps=3000)
    oa = r.fields()[0]
    drift, dev = {}, {}
    for prec in ("fp16", "fp16sr"):
        with lattice([cell], prec, kernel) as lat:
            lat.init_fields(ra, rb).step(3000)
            mass, _ = lat.reductions()
            ga = lat.fields()[0]
        drift[prec] = np.abs(mass[0] - m0) / m0
        dev[prec] = max_abs(ga[0], oa)
    assert np.all(drift["fp16sr"] <= 2e-6)
    assert np.max(drift["fp16sr"]) < 0.2 * np.max(drift["fp16"])
    assert dev["fp16sr"] <= 2e-3 and dev["fp16"] <= 2e-3


@pytest.mark.parametrize("kernel", KERNELS)
def test_mrt_kolmogorov_sine_start_against_oracle(kernel):
    """The paper's Kolmogorov start (sine densities, 128^2) under the MRT
    collision, 300 steps with the sampled line profile, FP64 against the oracle."""
    L = 128
    cell = I.make_cell("paper", nx=L, ny=L, g_ab=0.405, f0=I.kolmogorov_f0(0.1, L), **RATES)
    ra, rb = I.sine_fields(L, L, noise=1e-3, seed=3)
    with lattice([cell], "fp64", kernel) as lat:
        lat.init_fields(ra, rb).set_sampling(100, 10).step(300)
        ga, gb, gu, _ = lat.fields()
        ub, ns = lat.profile()
    (r,) = oracle_runs([cell], ra, rb, steps=300, sampling=(100, 10))
    oa, ob, ou, _ = r.fields()
    assert max_abs(ga[0], oa) <= 1e-12 and max_abs(gb[0], ob) <= 1e-12 and max_abs(gu[0], ou) <= 1e-12
    _, _, _, oub = r.shear()
    assert ns == 20
    np.testing.assert_allclose(ub[0], oub, rtol=0, atol=1e-13)
