"""Failure detection on the GPU without a GPU fault: the test hook
lb_test_inject arms a stalled row copy (the kernel's bounded waits run out,
it records a timeout and returns) or a failed launch (reported on the host).
Each test checks the status the host reads, that the wait was bounded in wall
time, and that the device keeps working afterwards."""
import time

import numpy as np
import pytest

from paper_1004_5058_gb300 import inputs as I
from tests._util import max_abs, oracle_runs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def setup():
    cell = I.make_cell("paper", nx=64, ny=48, g_ab=0.405, bc=1, u_wall=0.01)
    ra, rb = I.random_fields(64, 48, seed=3)
    ux, uy = I.couette_velocity(64, 48, 0.01)
    return cell, ra, rb, ux, uy


def test_stalled_copy_times_out_and_recovers():
    from paper_1004_5058_gb300 import Lattice
    from paper_1004_5058_gb300._lib import LBError, LB_ERR_STATE, LB_ERR_TIMEOUT
    cell, ra, rb, ux, uy = setup()
    with Lattice([cell], "fp32") as lat:
        lat.set_kernel("tiled", 64, 16)
        lat.init_fields(ra, rb, ux, uy).step(3).sync()
        assert lat.lib.lb_test_inject(lat.h, 1) == 0
        t0 = time.perf_counter()
        lat.step(40)  # one stalled launch, then 39 that see the flag and return
        with pytest.raises(LBError) as e:
            lat.sync()
        waited = time.perf_counter() - t0
        assert e.value.status == LB_ERR_TIMEOUT
        assert waited < 10.0, waited  # one bounded wait (1.5 s), not one per launch
        with pytest.raises(LBError) as e:
            lat.step(1)
        assert e.value.status == LB_ERR_STATE
        # a fresh state runs normally and matches the oracle
        lat.init_fields(ra, rb, ux, uy).step(10)
        ga, gb, _, _ = lat.fields()
    (r,) = oracle_runs([cell], ra, rb, ux, uy, steps=10)
    oa, ob, _, _ = r.fields()
    assert max_abs(ga[0], oa) <= 3e-6 and max_abs(gb[0], ob) <= 3e-6


def test_failed_launch_is_reported_and_state_kept():
    from paper_1004_5058_gb300 import Lattice
    from paper_1004_5058_gb300._lib import LBError, LB_ERR_CUDA, LB_ERR_INVALID, LB_ERR_UNSUPPORTED
    cell, ra, rb, ux, uy = setup()
    with Lattice([cell], "fp64") as a, Lattice([cell], "fp64") as b:
        a.init_fields(ra, rb, ux, uy).step(7)
        b.init_fields(ra, rb, ux, uy).step(7)
        assert a.lib.lb_test_inject(a.h, 2) == 0
        with pytest.raises(LBError) as e:
            a.step(5)
        assert e.value.status == LB_ERR_CUDA
        assert a.steps_done == 7
        a.step(5)
        b.step(5)
        assert np.array_equal(a.get_populations(), b.get_populations())
        assert a.lib.lb_test_inject(a.h, 9) == LB_ERR_INVALID
        a.set_kernel("generic")
        assert a.lib.lb_test_inject(a.h, 1) == LB_ERR_UNSUPPORTED
