"""One cell split into horizontal slabs (lb_create_slab, lb_slab_get/put), all
slabs on one GPU, each with its own handle and buffers, trading their edge rows
and outflow populations by device-to-device copies between steps
(paper_1004_5058_gb300.slabs.LocalExchange).  The slabs' rows must equal the
whole-cell run bit for bit, every precision, periodic and Couette, even and
ragged splits; and the FP64 slabs match the FP64 oracle."""
import numpy as np
import pytest

from paper_1004_5058_gb300 import inputs as I

from ._util import CudaBuffer, max_abs, oracle_runs

pytestmark = pytest.mark.gpu


def setup(bc, nx=64, ny=40, f0=0.0, seed=11):
    cell = I.make_cell("paper", nx=nx, ny=ny, g_ab=0.405, bc=bc, u_wall=0.02 if bc else 0.0, f0=f0)
    ra, rb = I.random_fields(nx, ny, seed=seed)
    if bc:
        ux, uy = I.couette_velocity(nx, ny, 0.02)
    else:
        ux, uy = np.zeros_like(ra), np.zeros_like(ra)
    return cell, ra, rb, ux, uy


def run_whole(cell, prec, fields, steps, sampling=None):
    from paper_1004_5058_gb300 import Lattice
    with Lattice([cell], prec) as lat:
        lat.init_fields(*fields)
        if sampling:
            lat.set_sampling(*sampling)
        lat.step(steps)
        f = lat.get_populations()[0]
        prof = lat.profile()[0][0] if sampling else None
        wall = lat.wall_momentum()[0][0] if sampling else None
    return f, prof, wall


def run_slabs(cell, prec, fields, steps, world, sampling=None):
    from paper_1004_5058_gb300.slabs import LocalExchange, SlabLattice, split_rows
    parts = split_rows(cell.ny, world)
    slabs = [SlabLattice([cell], y0, rows, prec) for y0, rows in parts]
    try:
        for s, (y0, rows) in zip(slabs, parts):
            s.lat.init_fields(*[a[:, y0:y0 + rows] for a in fields])
            if sampling:
                s.lat.set_sampling(*sampling)
        LocalExchange(slabs, periodic=cell.bc == 0).step(steps)
        f = np.concatenate([s.lat.get_populations()[0] for s in slabs], axis=2)
        prof = np.concatenate([s.lat.profile()[0][0] for s in slabs]) if sampling else None
        wall = sum(s.lat.wall_momentum()[0][0] for s in slabs) if sampling else None
    finally:
        for s in slabs:
            s.close()
    return f, prof, wall


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16sr"])
@pytest.mark.parametrize("bc,world", [(0, 2), (0, 3), (0, 4), (1, 1), (1, 2), (1, 3), (1, 4)])
def test_slabs_equal_whole_cell_bitwise(prec, bc, world):
    cell, ra, rb, ux, uy = setup(bc)
    fields = (ra, rb, ux, uy)
    whole, _, _ = run_whole(cell, prec, fields, 25)
    got, _, _ = run_slabs(cell, prec, fields, 25, world)
    assert np.array_equal(got, whole)


def test_slabs_kolmogorov_sampled_observables_bitwise():
    """Body force on the global rows, and the sampled observables: the slabs'
    line profiles, stacked, and their wall momentum sums equal the whole cell's."""
    nx, ny = 64, 48
    k = 2 * np.pi / ny
    cell, ra, rb, ux, uy = setup(0, nx=nx, ny=ny, f0=I.kolmogorov_f0(2e-3, ny, rho=1.2, tau=1.0))
    fields = (ra, rb, ux, uy)
    w_f, w_prof, _ = run_whole(cell, "fp64", fields, 30, sampling=(10, 4))
    s_f, s_prof, _ = run_slabs(cell, "fp64", fields, 30, 3, sampling=(10, 4))
    assert np.array_equal(s_f, w_f) and np.array_equal(s_prof, w_prof)
    assert np.abs(w_prof).max() > 0 and k > 0
    cc, ra, rb, ux, uy = setup(1, nx=nx, ny=ny)
    w_f, w_prof, w_wall = run_whole(cc, "fp64", (ra, rb, ux, uy), 30, sampling=(10, 4))
    s_f, s_prof, s_wall = run_slabs(cc, "fp64", (ra, rb, ux, uy), 30, 4, sampling=(10, 4))
    assert np.array_equal(s_prof, w_prof) and np.array_equal(s_wall, w_wall) and np.all(w_wall != 0)


@pytest.mark.parametrize("bc", [0, 1])
def test_slabs_match_the_oracle(bc):
    cell, ra, rb, ux, uy = setup(bc, ny=36)
    got, _, _ = run_slabs(cell, "fp64", (ra, rb, ux, uy), 40, 3)
    (r,) = oracle_runs([cell], ra, rb, ux, uy, steps=40)
    assert max_abs(got, r.f) <= 1e-12


def test_slab_errors():
    import ctypes as C
    import torch
    from paper_1004_5058_gb300 import Lattice
    from paper_1004_5058_gb300._lib import (LBError, LB_ERR_INVALID, LB_ERR_UNSUPPORTED, LB_SLAB_EDGE_LO,
                                            LB_SLAB_FLOW_HI)
    cell, ra, rb, ux, uy = setup(1)
    with pytest.raises(LBError) as e:  # rows beyond the cell
        Lattice([cell], "fp32", slab=(30, 20))
    assert e.value.status == LB_ERR_INVALID
    with pytest.raises(LBError) as e:  # a periodic cell of 40 rows cannot hold 37 rows + 4 ghosts
        Lattice([setup(0)[0]], "fp32", slab=(0, 37))
    assert e.value.status == LB_ERR_INVALID
    with pytest.raises(LBError) as e:  # an odd width: the tiled kernel (a slab's only one) does not take it
        Lattice([I.make_cell("paper", nx=63, ny=40, bc=1)], "fp32", slab=(0, 20))
    assert e.value.status == LB_ERR_UNSUPPORTED
    with Lattice([cell], "fp32", slab=(10, 12)) as lat:
        y0, rows, nyg = C.c_int(), C.c_int(), C.c_int()
        assert lat.lib.lb_slab_info(lat.h, C.byref(y0), C.byref(rows), C.byref(nyg)) == 0
        assert (y0.value, rows.value, nyg.value) == (10, 12, 40)
        assert lat.message_bytes(LB_SLAB_EDGE_LO) == 18 * 2 * 64 * 4
        assert lat.message_bytes(LB_SLAB_FLOW_HI) == 6 * 64 * 4
        lat.init_fields(ra[:, 10:22], rb[:, 10:22])
        with pytest.raises(LBError) as e:  # one step per call
            lat.step(2)
        assert e.value.status == LB_ERR_INVALID
        with pytest.raises(LBError) as e:  # the stress needs both walls
            lat.shear_stress()
        assert e.value.status == LB_ERR_UNSUPPORTED
        with CudaBuffer(100) as small, pytest.raises(LBError) as e:  # refused before anything is enqueued
            lat.slab_get(LB_SLAB_EDGE_LO, small.ptr.value)
        assert e.value.status == LB_ERR_INVALID
        host = np.zeros(18 * 2 * 64, dtype=np.float32)
        with pytest.raises(LBError) as e:
            lat.slab_put(LB_SLAB_EDGE_LO, host.ctypes.data)
        assert e.value.status == LB_ERR_INVALID
    with Lattice([cell], "fp32") as whole:
        whole.init_fields(ra, rb)
        buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
        with pytest.raises(LBError) as e:
            whole.slab_get(LB_SLAB_EDGE_LO, buf.data_ptr())
        assert e.value.status == LB_ERR_UNSUPPORTED


@pytest.mark.parametrize("bc,world", [(0, 3), (1, 2)])
def test_slabs_multiple_relaxation_times_bitwise(bc, world):
    """The multiple-relaxation-time collision runs in slabs as in the whole cell."""
    cell, ra, rb, ux, uy = setup(bc)
    cell.s_e, cell.s_eps, cell.s_q, cell.s_nu = 1.4, 1.1, 1.2, 1.1
    fields = (ra, rb, ux, uy)
    whole, _, _ = run_whole(cell, "fp32", fields, 25)
    got, _, _ = run_slabs(cell, "fp32", fields, 25, world)
    assert np.array_equal(got, whole)


@pytest.mark.parametrize("bc,world", [(0, 2), (0, 4), (1, 3)])
def test_stream_exchange_equals_whole_cell_bitwise(bc, world):
    """All slabs on one stream, the exchange stream-ordered (no host waits):
    the same rows as the whole cell, bit for bit."""
    import torch
    from paper_1004_5058_gb300.slabs import SlabLattice, StreamExchange, split_rows
    cell, ra, rb, ux, uy = setup(bc)
    fields = (ra, rb, ux, uy)
    whole, _, _ = run_whole(cell, "fp32", fields, 25)
    stream = torch.cuda.Stream()
    parts = split_rows(cell.ny, world)
    slabs = [SlabLattice([cell], y0, rows, "fp32", stream=stream) for y0, rows in parts]
    try:
        for s, (y0, rows) in zip(slabs, parts):
            s.lat.init_fields(*[a[:, y0:y0 + rows] for a in fields])
        StreamExchange(slabs, periodic=bc == 0).step(25)
        got = np.concatenate([s.lat.get_populations()[0] for s in slabs], axis=2)
    finally:
        for s in slabs:
            s.close()
    assert np.array_equal(got, whole)
