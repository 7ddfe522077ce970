"""Pin of the slab decomposition of one cell (oracle/slab.py): stepping a cell
as 2, 3 or 4 horizontal slabs that trade ghost rows and streamed-out
populations every step gives the whole-cell oracle state bit for bit, periodic,
Couette and Kolmogorov-forced, with even and ragged splits."""
import numpy as np
import pytest

from paper_1004_5058_gb300 import inputs as I


def case(bc, f0=0.0, nx=16, ny=24, seed=3):
    from oracle import lb
    cell = I.make_cell("paper", nx=nx, ny=ny, g_ab=0.405, bc=bc, u_wall=0.01 if bc == 1 else 0.0)
    cell.f0 = f0
    ra, rb = I.random_fields(nx, ny, n_cells=1, seed=seed)
    if bc == 1:
        ux, uy = I.couette_velocity(nx, ny, 0.01)
        ux, uy = ux.reshape(ny, nx), uy.reshape(ny, nx)
    else:
        ux = uy = None
    return cell, lb.equilibrium(cell, ra[0], rb[0], ux, uy)


def whole(cell, f, n):
    from oracle import lb
    for _ in range(n):
        f, o, _ = lb.step(cell, f)
    return f, o


@pytest.mark.parametrize("bc,f0", [(0, 0.0), (1, 0.0), (0, 2e-4)], ids=["periodic", "couette", "kolmogorov"])
@pytest.mark.parametrize("world", [2, 3, 4])
def test_slabs_equal_whole_cell_bitwise(bc, f0, world):
    from oracle import slab
    cell, f = case(bc, f0)
    ref, o = whole(cell, f, 12)
    got, obs = slab.run_in_process(cell, f, 12, world)
    assert np.array_equal(got, ref)
    for s in range(2):  # per-rank sums add in another order: round-off only
        assert obs["mass"][s] == pytest.approx(o["mass"][s], rel=1e-14)
    assert obs["pi_top"] == pytest.approx(o["pi_top"], rel=1e-12, abs=1e-18)


def test_slabs_two_relaxation_times():
    """The slab step restates the per-species relaxation times too."""
    from oracle import slab
    cell, f = case(1, seed=5)
    cell.tau, cell.tau_b = 0.7, 1.3
    ref, _ = whole(cell, f, 10)
    got, _ = slab.run_in_process(cell, f, 10, 3)
    assert np.array_equal(got, ref)


def test_ragged_split():
    from oracle import slab
    assert slab.split_rows(26, 4) == [(0, 7), (7, 7), (14, 6), (20, 6)]
    cell, f = case(1, ny=26, seed=8)
    ref, _ = whole(cell, f, 8)
    got, _ = slab.run_in_process(cell, f, 8, 4)
    assert np.array_equal(got, ref)


def test_each_exchange_is_needed():
    """Dropping either trade breaks the equality, so the test above sees them."""
    from oracle import slab
    cell, f = case(0)
    ref, _ = whole(cell, f, 2)
    parts = slab.split_rows(cell.ny, 2)
    for drop in ("ghost", "inflow"):
        slabs = [slab.scatter(f, y0, r) for y0, r in parts]
        for _ in range(2):
            sends = [slab.ghost_send(s) for s in slabs]
            if drop != "ghost":
                for r in range(2):
                    b, a = slab.neighbours(cell, r, 2)
                    slab.ghost_recv(slabs[r], sends[b][1], sends[a][0])
            outs = [slab.step_slab(cell, parts[r][0], slabs[r])[0] for r in range(2)]
            flows = [slab.outflow_send(o) for o in outs]
            if drop != "inflow":
                for r in range(2):
                    b, a = slab.neighbours(cell, r, 2)
                    slab.inflow_recv(outs[r], flows[b][1], flows[a][0])
            slabs = outs
        assert not np.array_equal(slab.gather(slabs, cell.ny), ref), drop


def test_rejects_thin_slabs():
    from oracle import slab
    cell, f = case(0, ny=6)
    with pytest.raises(ValueError):
        slab.run_in_process(cell, f, 1, 4)
