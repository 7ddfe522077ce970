"""Checkpoint and resume (lb_save / lb_load): a run continued from a saved
state equals the uninterrupted run bit for bit (populations, sampled stress
and profile), in every storage precision and both kernel families; files of
another shape, truncated or corrupted files are refused."""
import os

import numpy as np
import pytest

from paper_1004_5058_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def cells_and_fields(nx=64, ny=48, n=3):
    cells = [I.make_cell("paper", nx=nx, ny=ny, g_ab=0.405, bc=1, u_wall=u) for u in (0.004, 0.01, 0.02)[:n]]
    ra, rb = I.random_fields(nx, ny, n_cells=n, seed=12)
    ux, uy = I.couette_velocity(nx, ny, [c.u_wall for c in cells], n_cells=n)
    return cells, ra, rb, ux, uy


@pytest.mark.parametrize("prec", ["fp32", "fp16", "fp16sr", "fp64"])
@pytest.mark.parametrize("kernel", ["generic", "tiled"])
def test_resume_equals_uninterrupted_run(tmp_path, prec, kernel):
    from paper_1004_5058_gb300 import Lattice
    cells, ra, rb, ux, uy = cells_and_fields()
    path = tmp_path / "state.ckpt"
    with Lattice(cells, prec) as a:
        a.set_kernel(kernel)
        a.init_fields(ra, rb, ux, uy).set_sampling(20, 3).step(37)
        a.save(path)
        a.step(41)
        fa = a.get_populations()
        sa = a.shear_stress()
        pa = a.profile()
        ta = a.steps_done
    with Lattice(cells, prec) as b:
        b.set_kernel(kernel)
        b.load(path).step(41)
        fb = b.get_populations()
        sb = b.shear_stress()
        pb = b.profile()
        tb = b.steps_done
    assert ta == tb == 78
    assert np.array_equal(fa, fb)
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)
    assert np.array_equal(pa[0], pb[0]) and pa[1] == pb[1]


def test_load_refuses_other_shapes_and_damaged_files(tmp_path):
    from paper_1004_5058_gb300 import Lattice
    from paper_1004_5058_gb300._lib import LBError
    cells, ra, rb, ux, uy = cells_and_fields()
    path = tmp_path / "state.ckpt"
    with Lattice(cells, "fp32") as a:
        a.init_fields(ra, rb, ux, uy).step(5).save(path)
    raw = path.read_bytes()
    other, *_ = cells_and_fields(nx=96)
    with Lattice(other, "fp32") as b, pytest.raises(LBError):
        b.load(path)
    with Lattice(cells, "fp64") as b, pytest.raises(LBError):
        b.load(path)
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(raw[:-100])                      # truncated
    with Lattice(cells, "fp32") as b:
        with pytest.raises(LBError):
            b.load(bad)
        with pytest.raises(LBError):                  # no state after a failed load
            b.step(1)
    flipped = bytearray(raw)
    flipped[len(raw) // 2] ^= 0x40                    # one bit in the populations
    bad.write_bytes(bytes(flipped))
    with Lattice(cells, "fp32") as b, pytest.raises(LBError):
        b.load(bad)
    bad.write_bytes(b"not a checkpoint" * 20)
    with Lattice(cells, "fp32") as b, pytest.raises(LBError):
        b.load(bad)
    with Lattice(cells, "fp32") as b:                 # the intact file still loads
        b.load(path).step(1)
    os.remove(bad)
