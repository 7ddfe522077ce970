"""Parity at the full workload sizes, in the launch configuration the benchmark
uses (tiled kernel, persistent grid, CUDA-graph chunks):

  * 8 Couette cells of 1024 x 1024 (the benchmark batch): sampled cells
    compared with the oracle site by site after 1 and 10 steps; mass of every
    cell after 100 steps;
  * one 4096 x 4096 cell (the precision-study size) in FP32, FP16-shifted (both
    roundings) and FP64: one step against the oracle;
  * 64 cells of 512 x 512 (the batched flow-curve size): two sampled cells
    against the oracle after 5 steps;
  * properties at any size: G = 0 Couette from the linear profile stays linear.

Tolerances as in test_gpu_parity.py (FP64 to round-off, FP32 a few ulp per
step, FP16 one rounding of the shifted value)."""
import numpy as np
import pytest

from paper_1004_5058_gb300 import inputs as I
from tests._util import max_abs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def couette_batch(n_cells, L, seed=1004):
    cells = [I.make_cell("paper", nx=L, ny=L, g_ab=0.405, bc=1, u_wall=u)
             for u in I.log_spaced(1e-4, 1e-2, n_cells)]
    ra, rb = I.random_fields(L, L, n_cells=n_cells, seed=seed)
    ux, uy = I.couette_velocity(L, L, [c.u_wall for c in cells], n_cells=n_cells)
    return cells, ra, rb, ux, uy


def oracle_fields(cell, ra, rb, ux, uy, steps):
    from oracle import lb as orc
    r = orc.Run(cell, ra, rb, ux, uy).step(steps)
    return r.fields()


def test_bench_batch_8x1024():
    from paper_1004_5058_gb300 import Lattice
    cells, ra, rb, ux, uy = couette_batch(8, 1024)
    with Lattice(cells, "fp32") as lat:
        lat.init_fields(ra, rb, ux, uy).set_kernel("tiled", 128, 147)
        assert lat.kernel() == ("tiled", 128, 147)
        lat.step(1)
        a1, b1, u1, _ = lat.fields()
        lat.step(9)
        a10, b10, u10, _ = lat.fields()
        lat.step(90)
        mass, _ = lat.reductions()
    for c in (0, 7):
        oa, ob, ou, _ = oracle_fields(cells[c], ra[c], rb[c], ux[c], uy[c], 1)
        assert max_abs(a1[c], oa) <= 1e-6 and max_abs(b1[c], ob) <= 1e-6 and max_abs(u1[c], ou) <= 1e-6
    oa, ob, ou, _ = oracle_fields(cells[3], ra[3], rb[3], ux[3], uy[3], 10)
    assert max_abs(a10[3], oa) <= 3e-6 and max_abs(u10[3], ou) <= 3e-6
    m0 = ra.reshape(8, -1).sum(axis=1)
    assert np.all(np.abs(mass[:, 0] - m0) / m0 <= 1e-6)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("fp16", 5e-5), ("fp16sr", 1e-4), ("fp64", 1e-14)])
def test_precision_study_cell_4096(prec, tol):
    from paper_1004_5058_gb300 import Lattice
    cells = [I.make_cell("paper", nx=4096, ny=4096, g_ab=0.405, bc=1, u_wall=1e-3)]
    ra, rb = I.random_fields(4096, 4096, n_cells=1, seed=77)
    ux, uy = I.couette_velocity(4096, 4096, [1e-3], n_cells=1)
    with Lattice(cells, prec) as lat:
        lat.init_fields(ra, rb, ux, uy)
        assert lat.kernel()[0] == "tiled"
        lat.step(1)
        a, b, u, v = lat.fields()
    oa, ob, ou, ov = oracle_fields(cells[0], ra[0], rb[0], ux[0], uy[0], 1)
    assert max_abs(a[0], oa) <= tol and max_abs(b[0], ob) <= tol
    assert max_abs(u[0], ou) <= tol and max_abs(v[0], ov) <= tol


def test_flow_curve_batch_64x512():
    from paper_1004_5058_gb300 import Lattice
    speeds = I.log_spaced(1e-5, 1e-2, 16)
    cells = [I.make_cell("paper", nx=512, ny=512, g_ab=g, bc=1, u_wall=u)
             for g in (0.3, 0.35, 0.405, 0.45) for u in speeds]
    ra, rb = I.random_fields(512, 512, n_cells=64, seed=5)
    ux, uy = I.couette_velocity(512, 512, [c.u_wall for c in cells], n_cells=64)
    with Lattice(cells, "fp32") as lat:
        lat.init_fields(ra, rb, ux, uy).step(5)
        a, b, u, _ = lat.fields()
    for c in (9, 50):
        oa, ob, ou, _ = oracle_fields(cells[c], ra[c], rb[c], ux[c], uy[c], 5)
        assert max_abs(a[c], oa) <= 2e-6 and max_abs(u[c], ou) <= 2e-6


def test_g0_couette_stays_linear_at_1024():
    """With no interactions the linear profile is the steady state of halfway
    bounce-back (exactly), so the line profile stays linear at any size."""
    from paper_1004_5058_gb300 import Lattice
    L, U = 1024, 1e-3
    cell = I.make_cell("ideal", nx=L, ny=L, bc=1, u_wall=U)
    ux, uy = I.couette_velocity(L, L, U)
    with Lattice([cell], "fp32") as lat:
        lat.init_fields(np.full((L, L), 0.6), np.full((L, L), 0.6), ux, uy)
        lat.set_sampling(0, 10).step(200)
        ub, ns = lat.profile()
        sigma, S, Sb = lat.shear_stress()
    y = np.arange(L)
    # FP32 rounding only: u = j/rho from differences of f ~ 0.3 (3e-8) -> 3e-5 U per site
    np.testing.assert_allclose(ub[0], U * (2 * (y + 0.5) / L - 1), rtol=0, atol=1e-4 * U)
    assert S[0] == pytest.approx(2 * U / L, rel=1e-4)


def test_no_samples_and_zero_steps():
    from paper_1004_5058_gb300 import Lattice
    cells, ra, rb, ux, uy = couette_batch(2, 64)
    with Lattice(cells, "fp32") as lat:
        lat.init_fields(ra, rb, ux, uy).step(0)
        sigma, S, Sb = lat.shear_stress()
        assert np.all(np.isnan(sigma)) and np.all(np.isnan(S))
        ub, ns = lat.profile()
        assert ns == 0 and np.all(np.isnan(ub))
        lat.set_sampling(5, 0).step(20)  # every = 0: sampling off
        assert lat.profile()[1] == 0


def test_largest_tiled_cell():
    """The largest cell the tiled kernel takes (18 planes of ny x pitch just
    under 2^31 elements: 32-bit offsets inside a cell): a uniform periodic
    background stays bitwise uniform, and a seeded bump placed near the far
    end of the arrays evolves as the oracle's same bump in a small cell
    (translation invariance), which checks the high addresses."""
    from oracle import lb as orc
    from paper_1004_5058_gb300 import Lattice
    nx, ny = 10240, 11648
    assert 18 * ny * nx < 2 ** 31
    cell = I.make_cell("paper", nx=nx, ny=ny, g_ab=0.405, bc=0)
    bump = 0.05 * (2.0 * I.uniform01(8, 36).reshape(6, 6) - 1.0)
    ra = np.full((1, ny, nx), 0.6)
    rb = np.full((1, ny, nx), 0.6)
    ra[0, ny - 30:ny - 24, nx - 30:nx - 24] += bump
    with Lattice([cell], "fp32") as lat:
        lat.init_fields(ra, rb)
        assert lat.kernel()[0] == "tiled"
        lat.step(2)
        ga, gb, gu, _ = lat.fields()
        mass, _ = lat.reductions()
    del ra, rb
    win = (slice(ny - 40, ny - 14), slice(nx - 40, nx - 14))
    small = I.make_cell("paper", nx=64, ny=64, g_ab=0.405, bc=0)
    sa = np.full((64, 64), 0.6)
    sb = np.full((64, 64), 0.6)
    sa[34:40, 34:40] += bump
    r = orc.Run(small, sa, sb).step(2)
    oa, ob, ou, _ = r.fields()
    assert max_abs(ga[0][win], oa[24:50, 24:50]) <= 1e-6
    assert max_abs(gb[0][win], ob[24:50, 24:50]) <= 1e-6
    assert max_abs(gu[0][win], ou[24:50, 24:50]) <= 1e-6
    bg = ga[0].copy()
    bg[ny - 40:ny - 14, nx - 40:nx - 14] = bg[0, 0]
    assert np.ptp(bg) == 0.0  # the untouched background is bitwise uniform
    assert abs(mass[0, 0] - (0.6 * nx * ny + bump.sum())) <= 1e-6 * 0.6 * nx * ny


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("fp16", 5e-5)])
def test_bench_batch_8x1024_multiple_relaxation_times(prec, tol):
    """The bench batch with the multiple-relaxation-time collision (bench.py
    --mrt 1.4,1.1,1.2,1.1), in the bench's tile: two cells against the oracle
    after 1 step and one after 10; mass of every cell after 100 steps."""
    from paper_1004_5058_gb300 import Lattice
    cells, ra, rb, ux, uy = couette_batch(8, 1024)
    for c in cells:
        c.s_e, c.s_eps, c.s_q, c.s_nu = 1.4, 1.1, 1.2, 1.1
    with Lattice(cells, prec) as lat:
        lat.init_fields(ra, rb, ux, uy).set_kernel("tiled", 128, 147)
        lat.step(1)
        a1, b1, u1, _ = lat.fields()
        lat.step(9)
        a10, _, u10, _ = lat.fields()
        lat.step(90)
        mass, _ = lat.reductions()
    for c in (0, 7):
        oa, ob, ou, _ = oracle_fields(cells[c], ra[c], rb[c], ux[c], uy[c], 1)
        assert max_abs(a1[c], oa) <= tol and max_abs(b1[c], ob) <= tol and max_abs(u1[c], ou) <= tol
    oa, _, ou, _ = oracle_fields(cells[3], ra[3], rb[3], ux[3], uy[3], 10)
    assert max_abs(a10[3], oa) <= 3 * tol and max_abs(u10[3], ou) <= 3 * tol
    m0 = ra.reshape(8, -1).sum(axis=1)
    assert np.all(np.abs(mass[:, 0] - m0) / m0 <= (1e-6 if prec == "fp32" else 1e-4))
