"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, on the
same seeded inputs.

Tolerances (written per test) follow from the arithmetic:
  * FP64 storage/arithmetic: differences come only from the order of additions
    and fused multiply-adds; one step stays within ~1e-15 of f, and 1000 steps
    of a relaxing state within 1e-12 of rho.
  * FP32 (eps = 6e-8): one step differs by the rounding of the loaded f
    (|f| < 0.5) plus the force/shift error, a few ulp; 4e-7 absolute bounds it.
    Over 1000 steps of a relaxing (non-demixing) state, max |d rho| <= 1e-5.
  * FP16-shifted storage: one rounding of the stored g = f - w rho_bar per step,
    element by element at most 2^-11 |g| (round to nearest, half an ulp) or
    2^-10 |g| (stochastic rounding, one ulp), plus the FP32 arithmetic (5e-7);
    on the evolved state of these tests |g| <= 0.06, so <= 3.5e-5 / 7e-5.
A demixing state (spinodal growth) amplifies any difference exponentially;
there the comparison stops before the growth phase, and longer runs are
compared through exact invariants (mass) instead.
"""
import numpy as np
import pytest

from paper_1004_5058_gb300 import inputs as I
from tests._util import max_abs, oracle_runs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def lattice(cells, prec, kernel="generic", tile=(0, 0)):
    from paper_1004_5058_gb300 import Lattice
    lat = Lattice(cells, prec)
    if kernel == "tiled":
        from paper_1004_5058_gb300._lib import LBError
        try:
            lat.set_kernel("tiled", *tile)
        except LBError as e:
            lat.close()
            pytest.skip("tiled kernel unsupported here: %s" % e)
    else:
        lat.set_kernel(kernel)
    return lat


KERNELS = ["generic", "tiled"]


def evolved_state(cell, steps, seed):
    from oracle import lb as orc
    ra, rb = I.random_fields(cell.nx, cell.ny, seed=seed)
    ux = uy = None
    if cell.bc == 1:
        ux, uy = I.couette_velocity(cell.nx, cell.ny, cell.u_wall)
    r = orc.Run(cell, ra[0], rb[0], None if ux is None else ux[0], None if uy is None else uy[0])
    r.step(steps)
    return r


# ------------------------------------------------------------ one step --
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec,tol", [("fp64", 2e-15), ("fp32", 4e-7), ("fp16", 2.0 ** -11), ("fp16sr", 2.0 ** -10)])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_one_step_from_evolved_state(kernel, prec, tol, bc, tau):
    """tau = 1 takes the kernels' f* = f^eq path, tau = 0.8 the general BGK update."""
    cell = I.make_cell("paper", nx=64, ny=48, g_ab=0.405, bc=bc, u_wall=0.02 if bc else 0.0, tau=tau)
    from oracle import lb as orc
    r = evolved_state(cell, 400, seed=31)
    f0 = r.f.copy()
    f1, obs, prof = orc.step(cell, f0, want_profile=True)
    with lattice([cell], prec, kernel) as lat:
        lat.set_populations(f0[None])
        start = lat.get_populations()[0]
        lat.set_sampling(0, 1).step(1)
        g1 = lat.get_populations()[0]
        sigma, S, _ = lat.shear_stress()
        ub, ns = lat.profile()
    # compare the update itself, from the state the device holds after rounding
    f1_from_start, obs_s, prof_s = orc.step(cell, start, want_profile=True)
    if prec.startswith("fp16"):
        # tol is relative to the stored shifted value g (one rounding of it)
        w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[None, :, None, None]
        shift = w * np.array([cell.rho_bar_a, cell.rho_bar_b])[:, None, None, None]
        gmag = np.maximum(np.abs(g1 - shift), np.abs(f1_from_start - shift))
        excess = np.abs(g1 - f1_from_start) - (tol * gmag + 5e-7)
        assert excess.max() <= 0.0, (excess.max(), gmag.max())
    else:
        assert max_abs(g1, f1_from_start) <= tol
    if prec == "fp64":
        assert max_abs(g1, f1) <= tol
    assert ns == 1
    # observables of the step, from the same start: FP64 sums of FP32/FP64 site values
    otol = 1e-14 if prec == "fp64" else 1e-6
    np.testing.assert_allclose(ub[0], prof_s / cell.nx, rtol=0, atol=otol)
    if bc == 1:
        ref_sigma = 0.5 * (obs_s["pi_top"] - obs_s["pi_bot"]) / cell.nx
        assert abs(sigma[0] - ref_sigma) <= otol


# ------------------------------------------------------------- C1 runs --
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_c1_periodic_1000_steps_paper_couplings(kernel, prec, tol):
    """64x64 fully periodic, the paper's footnote couplings, random init, 1000 steps."""
    cell = I.make_cell("paper", nx=64, ny=64)
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
    # mass: FP64 to round-off.  FP32: the collision closes the rest population on
    # the loaded populations, f*_0 = f_0 + sum_i (f_i - f*_i) with each difference
    # exact (Sterbenz), so a site and step change a species' mass only by the one
    # rounding of f*_0 (at most 2^-25 f*_0, 1.7e-8 of rho_s), with a sign that
    # varies from site to site.  The earlier closure rho_s - sum_i f*_i inherited
    # the rounding of the FP32 sum rho_s, which in this near-uniform mixed state is
    # the same at every site: it drifted 3.9e-6 per 1000 steps, reproduced by an
    # FP32 emulation of the bookkeeping, which gives 6e-9 with the new closure.
    mtol = 1e-13 if prec == "fp64" else 2e-6
    assert abs(mass[0, 0] - m0[0]) / m0[0] <= mtol and abs(mass[0, 1] - m0[1]) / m0[1] <= mtol
    assert abs(mom[0]).max() / (m0[0] + m0[1]) <= (1e-13 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec,tol,steps", [("fp64", 1e-11, 1000), ("fp32", 1e-5, 150)])
def test_c1_periodic_demixing(kernel, prec, tol, steps):
    """Same box with G_AB = 0.405 (demixing).  FP64 follows the oracle through the
    spinodal growth; FP32 is compared before the growth phase, and mass is
    checked after 1000 steps."""
    cell = I.make_cell("paper", nx=64, ny=64, g_ab=0.405)
    ra, rb = I.random_fields(64, 64, seed=1004)
    with lattice([cell], prec, kernel) as lat:
        lat.init_fields(ra, rb).step(steps)
        ga, gb, _, _ = lat.fields()
        lat.step(1000 - steps)
        mass, _ = lat.reductions()
    (r,) = oracle_runs([cell], ra, rb, steps=steps)
    oa, ob, _, _ = r.fields()
    assert max_abs(ga[0], oa) <= tol and max_abs(gb[0], ob) <= tol
    mtol = 1e-13 if prec == "fp64" else 2e-6  # the closure of the rest population, as above
    assert abs(mass[0, 0] - ra.sum()) / ra.sum() <= mtol


# ------------------------------------------------------------- Couette --
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec,tol,sig_tol", [("fp64", 1e-12, 1e-13), ("fp32", 2e-5, 1e-7)])
def test_couette_fields_and_stress(kernel, prec, tol, sig_tol):
    """sig_tol: absolute on sigma_xy (~6e-5 here): each wall link's momentum is
    a difference of O(0.03) populations, so FP32 leaves ~1e-8 per site and the
    FP32/FP64 field drift over 400 steps adds to it."""
    nx, ny, U = 64, 64, 0.01
    cell = I.make_cell("paper", nx=nx, ny=ny, bc=1, u_wall=U)
    ra, rb = I.random_fields(nx, ny, seed=3)
    ux, uy = I.couette_velocity(nx, ny, U)
    with lattice([cell], prec, kernel) as lat:
        lat.init_fields(ra, rb, ux, uy).set_sampling(100, 5).step(400)
        ga, gb, gu, _ = lat.fields()
        sigma, S, Sb = lat.shear_stress()
        ub, ns = lat.profile()
    (r,) = oracle_runs([cell], ra, rb, ux, uy, steps=400, sampling=(100, 5))
    oa, ob, ou, _ = r.fields()
    osig, oS, oSb, oub = r.shear()
    assert ns == r.acc.n_samples == 60  # t = 100, 105, ..., 395
    assert max_abs(ga[0], oa) <= tol and max_abs(gu[0], ou) <= tol
    np.testing.assert_allclose(ub[0], oub, rtol=0, atol=tol * U * 10)
    assert abs(sigma[0] - osig) <= sig_tol
    assert abs(S[0] - oS) <= tol * abs(oS) * 10 + 1e-15
    assert abs(Sb[0] - oSb) <= tol * abs(oSb) * 10 + 1e-15


@pytest.mark.parametrize("kernel", KERNELS)
def test_batched_cells_each_match_own_oracle(kernel):
    """Four cells with different wall speeds, couplings and relaxation times
    (tau = 1 and others in one launch) in one handle."""
    nx, ny = 64, 32
    cells = [I.make_cell("paper", nx=nx, ny=ny, bc=1, u_wall=u, g_ab=g, tau=t)
             for u, g, t in [(1e-3, 0.3, 0.8), (3e-3, 0.35, 1.0), (1e-2, 0.405, 1.3), (2e-2, 0.45, 1.0)]]
    ra, rb = I.random_fields(nx, ny, n_cells=4, seed=9)
    ux, uy = I.couette_velocity(nx, ny, [c.u_wall for c in cells], n_cells=4)
    with lattice(cells, "fp64", kernel) as lat:
        lat.init_fields(ra, rb, ux, uy).set_sampling(50, 10).step(120)
        ga, gb, _, _ = lat.fields()
        sigma, S, _ = lat.shear_stress()
    runs = oracle_runs(cells, ra, rb, ux, uy, steps=120, sampling=(50, 10))
    for c, r in enumerate(runs):
        oa, ob, _, _ = r.fields()
        assert max_abs(ga[c], oa) <= 1e-12 and max_abs(gb[c], ob) <= 1e-12
        osig, oS, _, _ = r.shear()
        assert sigma[c] == pytest.approx(osig, rel=1e-9, abs=1e-16)
        assert S[c] == pytest.approx(oS, rel=1e-9, abs=1e-16)


# -------------------------------------------------------- ragged shapes --
@pytest.mark.parametrize("nx,ny,bc", [(37, 23, 0), (37, 23, 1), (5, 5, 0), (130, 9, 1), (96, 70, 1)])
@pytest.mark.parametrize("kernel", KERNELS)
def test_ragged_and_small_shapes(nx, ny, bc, kernel):
    cell = I.make_cell("paper", nx=nx, ny=ny, g_ab=0.405, bc=bc, u_wall=0.01 if bc else 0.0)
    ra, rb = I.random_fields(nx, ny, seed=nx * 100 + ny)
    with lattice([cell], "fp64", kernel) as lat:
        lat.init_fields(ra, rb).step(50)
        ga, gb, _, _ = lat.fields()
    (r,) = oracle_runs([cell], ra, rb, steps=50)
    oa, ob, _, _ = r.fields()
    assert max_abs(ga[0], oa) <= 1e-13 and max_abs(gb[0], ob) <= 1e-13


# ----------------------------------------------------------- the ABI --
def test_error_paths_and_state():
    from paper_1004_5058_gb300 import Lattice
    from paper_1004_5058_gb300._lib import LBError, LB_ERR_NONFINITE, LB_ERR_STATE
    cell = I.make_cell("paper", nx=32, ny=32)
    with Lattice([cell], "fp32") as lat:
        with pytest.raises(LBError) as e:
            lat.step(1)  # nothing loaded yet
        assert e.value.status == LB_ERR_STATE
        ra, rb = I.random_fields(32, 32)
        lat.init_fields(ra, rb).step(0).sync()
        assert lat.steps_done == 0
        bad = ra.copy()
        bad[0, 3, 4] = np.nan
        lat.init_fields(bad, rb).step(3)
        with pytest.raises(LBError) as e:
            lat.fields()
        assert e.value.status == LB_ERR_NONFINITE
        with pytest.raises(LBError) as e:
            lat.step(1)
        assert e.value.status == LB_ERR_STATE
        lat.init_fields(ra, rb).step(5)  # a fresh state clears the error
        lat.fields()
        assert lat.steps_done == 5
        assert lat.kernel_launches > 0


@pytest.mark.parametrize("kernel", KERNELS)
def test_unsampled_steps_report_bad_density(kernel):
    """The watchdog runs on every step, sampled or not: a NaN or a non-positive
    total density planted in the initial fields is reported by the next
    synchronising call with sampling off and no field read, and the handle then
    refuses to step until a new state is loaded."""
    from paper_1004_5058_gb300._lib import LBError, LB_ERR_NONFINITE, LB_ERR_STATE
    cell = I.make_cell("paper", nx=64, ny=32)
    ra, rb = I.random_fields(64, 32)
    nan_a = ra.copy()
    nan_a[0, 5, 7] = np.nan
    neg_a, neg_b = ra.copy(), rb.copy()
    neg_a[0, 20, 40], neg_b[0, 20, 40] = -0.5, 0.2  # finite, total -0.3
    with lattice([cell], "fp32", kernel) as lat:
        for bad_a, bad_b in ((nan_a, rb), (neg_a, neg_b)):
            lat.init_fields(bad_a, bad_b).step(3)
            with pytest.raises(LBError) as e:
                lat.sync()
            assert e.value.status == LB_ERR_NONFINITE
            with pytest.raises(LBError) as e:
                lat.step(1)
            assert e.value.status == LB_ERR_STATE
        lat.init_fields(ra, rb).step(20).sync()  # a good state runs clean
        assert lat.steps_done == 20


def test_autotune_keeps_state_and_caches(tmp_path):
    from paper_1004_5058_gb300 import Lattice
    cell = I.make_cell("paper", nx=256, ny=128, g_ab=0.405)
    ra, rb = I.random_fields(256, 128)
    cache = str(tmp_path / "tune.txt")
    with Lattice([cell], "fp32") as lat:
        lat.init_fields(ra, rb).step(7)
        before = lat.get_populations()
        choice = lat.autotune(cache)
        after = lat.get_populations()
        assert np.array_equal(before, after)
        assert lat.steps_done == 7
    with Lattice([cell], "fp32") as lat2:
        lat2.init_fields(ra, rb)
        assert lat2.autotune(cache) == choice


# ----------------------------------------------------- Kolmogorov forcing --
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec,tol", [("fp64", 2e-15), ("fp32", 4e-7)])
def test_one_step_kolmogorov_forcing(kernel, prec, tol):
    from oracle import lb as orc
    cell = I.make_cell("paper", nx=64, ny=64, g_ab=0.405, f0=I.kolmogorov_f0(0.05, 64))
    r = evolved_state(cell, 300, seed=41)
    f0 = r.f.copy()
    with lattice([cell], prec, kernel) as lat:
        lat.set_populations(f0[None])
        start = lat.get_populations()[0]
        lat.set_sampling(0, 1).step(1)
        g1 = lat.get_populations()[0]
        ub, ns = lat.profile()
    f1, _, prof = orc.step(cell, start, want_profile=True)
    assert max_abs(g1, f1) <= tol
    np.testing.assert_allclose(ub[0], prof / cell.nx, rtol=0, atol=1e-14 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_kolmogorov_flow_paper_start(kernel, prec, tol):
    """The paper's workload in small: fully periodic box, body force
    F0 sin(2 pi y / L), the sinusoidal initial densities of the paper
    (k_in = 64 pi / L: L = 128 gives k_in = pi/2; at L = 64 the sine would vanish
    on every lattice row)."""
    L = 128
    cell = I.make_cell("paper", nx=L, ny=L, f0=I.kolmogorov_f0(0.02, L))
    ra, rb = I.sine_fields(L, L)
    with lattice([cell], prec, kernel) as lat:
        lat.init_fields(ra, rb).set_sampling(200, 5).step(500)
        ga, gb, gu, _ = lat.fields()
        ub, ns = lat.profile()
        mass, mom = lat.reductions()
    (r,) = oracle_runs([cell], ra, rb, steps=500, sampling=(200, 5))
    oa, ob, ou, _ = r.fields()
    _, _, _, oub = r.shear()
    assert max_abs(ga[0], oa) <= tol and max_abs(gu[0], ou) <= tol
    np.testing.assert_allclose(ub[0], oub, rtol=0, atol=tol)
    # sin(k y) forcing injects no net momentum
    assert abs(mom[0, 0]) <= (1e-12 if prec == "fp64" else 1e-4) * (ra.sum() + rb.sum())


# ------------------------------------------------- stochastic rounding --
@pytest.mark.parametrize("kernel", KERNELS)
def test_fp16_stochastic_rounding_removes_mass_drift(kernel):
    """A near-uniform mixed state (footnote couplings, G_AB = 0.045) relaxing
    for 3000 steps: round-to-nearest FP16 storage repeats the same rounding
    error at every site and the mass drifts; stochastic rounding makes each
    error zero-mean, so the drift is a random walk far below it.  The fields
    stay close to the FP64 oracle in both."""
    cell = I.make_cell("paper", nx=64, ny=64)
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
    print("mass drift", drift, "max |d rho_A| vs FP64", dev)
    assert np.all(drift["fp16sr"] <= 2e-6)
    assert np.max(drift["fp16sr"]) < 0.2 * np.max(drift["fp16"])
    assert dev["fp16sr"] <= 2e-3 and dev["fp16"] <= 2e-3


def test_fp16_stochastic_rounding_is_reproducible():
    """The random bits come from the sites and their densities: two runs from
    the same start agree bit for bit."""
    cell = I.make_cell("paper", nx=64, ny=48, g_ab=0.405, bc=1, u_wall=0.01)
    ra, rb = I.random_fields(64, 48, seed=4)
    ux, uy = I.couette_velocity(64, 48, 0.01)
    out = []
    for _ in range(2):
        with lattice([cell], "fp16sr", "tiled") as lat:
            lat.init_fields(ra, rb, ux, uy).step(50)
            out.append(lat.get_populations())
    assert np.array_equal(out[0], out[1])


# ------------------------------------------------------- initial state --
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec,rel,absol", [("fp64", 1e-15, 0.0), ("fp32", 4e-7, 0.0), ("fp16", 0.0, 2.0 ** -11),
                                             ("fp16sr", 0.0, 2.0 ** -11)])
def test_initial_equilibrium(kernel, prec, rel, absol):
    """lb_init_fields stores f^eq(rho_s, u): FP64 to round-off, FP32 within a few
    ulp (it is evaluated in FP32), FP16 within one rounding of g = f - w rho_bar
    (round to nearest there in both FP16 modes)."""
    from oracle import lb as orc
    cell = I.make_cell("paper", nx=64, ny=40, g_ab=0.405, bc=1, u_wall=0.03)
    ra, rb = I.random_fields(64, 40, seed=17)
    ux, uy = I.couette_velocity(64, 40, 0.03)
    uy = 0.01 * np.sin(np.arange(64 * 40).reshape(1, 40, 64))
    with lattice([cell], prec, kernel) as lat:
        lat.init_fields(ra, rb, ux, uy)
        got = lat.get_populations()[0]
    ref = orc.equilibrium(cell, ra[0], rb[0], ux[0], uy[0])
    if absol:
        w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[None, :, None, None]
        g = np.abs(ref - w * np.array([cell.rho_bar_a, cell.rho_bar_b])[:, None, None, None])
        assert np.all(np.abs(got - ref) <= absol * g + 2e-7)
    else:
        assert np.all(np.abs(got - ref) <= rel * np.abs(ref) + 1e-18)


# ------------------------------------------------ ragged tiled strips --
@pytest.mark.parametrize("nx,ny,tile,bc", [(80, 40, 64, 1), (200, 24, 128, 0), (136, 30, 128, 1), (36, 20, 32, 1),
                                           (100, 16, 64, 1)])
def test_tiled_narrow_last_strip(nx, ny, tile, bc):
    """Widths that are not a multiple of the tile: the last strip is narrower,
    its extra columns read zeros and store nothing, and the partial sums of the
    sampled observables cover only lattice columns.  FP64 against the oracle to
    round-off, fields and sampled stress and profile."""
    cell = I.make_cell("paper", nx=nx, ny=ny, g_ab=0.405, bc=bc, u_wall=0.01 if bc else 0.0)
    ra, rb = I.random_fields(nx, ny, seed=nx + ny)
    ux = uy = None
    if bc:
        ux, uy = I.couette_velocity(nx, ny, 0.01)
    with lattice([cell], "fp64", "tiled", (tile, 8)) as lat:
        assert lat.kernel() == ("tiled", tile, 8)
        lat.init_fields(ra, rb, ux, uy).set_sampling(10, 5).step(30)
        ga, gb, _, _ = lat.fields()
        sigma, S, _ = lat.shear_stress()
        ub, ns = lat.profile()
    (r,) = oracle_runs([cell], ra, rb, ux, uy, steps=30, sampling=(10, 5))
    oa, ob, _, _ = r.fields()
    assert max_abs(ga[0], oa) <= 1e-13 and max_abs(gb[0], ob) <= 1e-13
    osig, oS, _, oub = r.shear()
    assert ns == 4  # steps 10, 15, 20, 25
    np.testing.assert_allclose(ub[0], oub, rtol=0, atol=1e-14)
    if bc:
        assert sigma[0] == pytest.approx(osig, rel=1e-9, abs=1e-16)


@pytest.mark.parametrize("prec,tol", [("fp32", 4e-7), ("fp16", 2.0 ** -11)])
def test_tiled_narrow_last_strip_reduced_precision(prec, tol):
    cell = I.make_cell("paper", nx=200, ny=32, g_ab=0.405, bc=1, u_wall=0.02)
    from oracle import lb as orc
    r = evolved_state(cell, 200, seed=44)
    f0 = r.f.copy()
    with lattice([cell], prec, "tiled", (128, 0)) as lat:
        lat.set_populations(f0[None])
        start = lat.get_populations()[0]
        lat.step(1)
        g1 = lat.get_populations()[0]
    f1, _, _ = orc.step(cell, start)
    if prec == "fp16":
        w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[None, :, None, None]
        shift = w * np.array([cell.rho_bar_a, cell.rho_bar_b])[:, None, None, None]
        gmag = np.maximum(np.abs(g1 - shift), np.abs(f1 - shift))
        assert np.all(np.abs(g1 - f1) <= tol * gmag + 5e-7)
    else:
        assert max_abs(g1, f1) <= tol
