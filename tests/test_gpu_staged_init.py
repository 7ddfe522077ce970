"""lb_stage_fields / lb_init_fields_staged: lb_init_fields in two halves, so
that the copy of the next run's fields overlaps the current run's time steps.
The staged path must set the same populations, bit for bit, as lb_init_fields,
and a pipelined sequence of runs must give the results of the same runs one
after another."""
import numpy as np
import pytest
import torch

from paper_1004_5058_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def workload(n_cells=3, nx=64, ny=48, seed=5):
    speeds = I.log_spaced(1e-3, 1e-2, n_cells)
    cells = [I.make_cell("paper", nx=nx, ny=ny, g_ab=0.405, bc=1, u_wall=u) for u in speeds]
    ra, rb = I.random_fields(nx, ny, n_cells=n_cells, seed=seed)
    ux, uy = I.couette_velocity(nx, ny, speeds, n_cells=n_cells)
    return cells, [pinned(a) for a in (ra, rb, ux, uy)]


@pytest.mark.parametrize("prec", ["fp32", "fp16sr", "fp64"])
def test_staged_init_equals_init_fields(prec):
    from paper_1004_5058_gb300 import Lattice
    cells, fields = workload()
    with Lattice(cells, prec) as a, Lattice(cells, prec) as b:
        a.init_fields(*fields)
        b.stage_fields(*fields).init_fields_staged()
        assert np.array_equal(a.get_populations(), b.get_populations())
        a.set_sampling(5, 5).step(30)
        b.set_sampling(5, 5).step(30)
        assert np.array_equal(a.get_populations(), b.get_populations())
        for x, y in zip(a.shear_stress(), b.shear_stress()):
            assert np.array_equal(x, y)


def test_pipelined_runs_equal_serial_runs():
    """Three runs with different fields: staged copies of run k+1 issued while
    run k steps, against the same runs with lb_init_fields."""
    from paper_1004_5058_gb300 import Lattice
    cells, _ = workload()
    runs = [workload(seed=s)[1] for s in (11, 12, 13)]
    serial, piped = [], []
    with Lattice(cells, "fp32") as lat:
        lat.set_kernel("tiled")
        for f in runs:
            lat.init_fields(*f).set_sampling(20, 5).step(60)
            serial.append((lat.get_populations(), lat.shear_stress()[0]))
        lat.stage_fields(*runs[0])
        for k in range(len(runs)):
            lat.init_fields_staged()
            if k + 1 < len(runs):
                lat.stage_fields(*runs[k + 1])
            lat.set_sampling(20, 5).step(60)
            piped.append((lat.get_populations(), lat.shear_stress()[0]))
    for (fs, ss), (fp, sp) in zip(serial, piped):
        assert np.array_equal(fs, fp) and np.array_equal(ss, sp)
    assert not np.array_equal(serial[0][0], serial[1][0])


def test_staged_errors_and_discard():
    from paper_1004_5058_gb300 import Lattice
    from paper_1004_5058_gb300._lib import LBError, LB_ERR_INVALID, LB_ERR_STATE
    cells, fields = workload()
    with Lattice(cells, "fp32") as lat:
        with pytest.raises(LBError) as e:  # nothing staged
            lat.init_fields_staged()
        assert e.value.status == LB_ERR_STATE
        assert lat.lib.lb_stage_fields(lat.h, None, None, None, None) == LB_ERR_INVALID
        lat.stage_fields(*fields)
        lat.init_fields(*fields)  # the synchronous path discards the staged copy
        with pytest.raises(LBError) as e:
            lat.init_fields_staged()
        assert e.value.status == LB_ERR_STATE
        # pageable host arrays also work (the copy may then wait)
        lat.stage_fields(*[np.array(a) for a in fields]).init_fields_staged().step(5)
        ref = Lattice(cells, "fp32")
        ref.init_fields(*fields).step(5)
        assert np.array_equal(lat.get_populations(), ref.get_populations())
        ref.close()
