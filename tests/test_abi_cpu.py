"""CPU-only checks of the C ABI library: it loads without a GPU, exports every
function include/lbhb.h declares, and its host-only routines (argument
validation, the Herschel-Bulkley fit) behave.  No kernel is launched here."""
import ctypes as C

import numpy as np
import pytest

from tests._util import header_functions


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1004_5058_gb300 import _lib
    return _lib.load()


def test_exports_every_declared_function(lib):
    from paper_1004_5058_gb300 import _lib
    names = header_functions()
    assert "lb_create" in names and "lb_step" in names and "lb_hb_fit" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, "binding lacks a signature for %s" % n


def test_null_and_invalid_arguments_rejected_before_device_work(lib):
    from paper_1004_5058_gb300 import _lib as L
    h = L._H()
    assert lib.lb_create(None, 1, 0, None, C.byref(h)) == L.LB_ERR_INVALID
    assert not h.value
    cell = L.lb_cell_params(64, 64, 0.5, 0.83, -9, 8.1, -8, 7.1, 0.045, 0, 0, 0.6, 0.6, 0)
    assert lib.lb_create(C.byref(cell), 1, 0, None, C.byref(h)) == L.LB_ERR_INVALID  # tau = 1/2
    assert b"tau" in lib.lb_last_error(None)
    cell.tau, cell.tau_b = 1.0, 0.5
    assert lib.lb_create(C.byref(cell), 1, 0, None, C.byref(h)) == L.LB_ERR_INVALID  # tau_B = 1/2
    assert b"tau_b" in lib.lb_last_error(None)
    cell.tau_b = 0.0
    for rate in (2.0, -0.1, float("nan")):  # multiple-relaxation-time rates live in (0, 2); 0 is 1/tau
        cell.s_q = rate
        assert lib.lb_create(C.byref(cell), 1, 0, None, C.byref(h)) == L.LB_ERR_INVALID
        assert b"multiple-relaxation-time rate" in lib.lb_last_error(None)
    cell.s_q, cell.nx = 0.0, 4
    assert lib.lb_create(C.byref(cell), 1, 0, None, C.byref(h)) == L.LB_ERR_INVALID  # nx < 5
    cell.nx, cell.bc = 64, 7
    assert lib.lb_create(C.byref(cell), 1, 0, None, C.byref(h)) == L.LB_ERR_INVALID
    cell.bc = 0
    assert lib.lb_create(C.byref(cell), 1, 9, None, C.byref(h)) == L.LB_ERR_INVALID  # precision
    cells = (L.lb_cell_params * 2)(cell, L.lb_cell_params(32, 64, 1.0, 0.83, 0, 0, 0, 0, 0, 0, 0, 0.6, 0.6, 0))
    assert lib.lb_create(cells, 2, 0, None, C.byref(h)) == L.LB_ERR_INVALID  # mixed shapes
    assert lib.lb_create(C.byref(cell), 1, 0, None, None) == L.LB_ERR_INVALID
    # NULL handles
    assert lib.lb_step(None, 1) == L.LB_ERR_INVALID
    assert lib.lb_sync(None) == L.LB_ERR_INVALID
    assert lib.lb_steps_done(None) == 0
    lib.lb_destroy(None)
    assert lib.lb_test_inject(None, 1) == L.LB_ERR_INVALID
    assert lib.lb_save(None, b"x.ckpt") == L.LB_ERR_INVALID
    assert lib.lb_load(None, b"x.ckpt") == L.LB_ERR_INVALID
    e = (C.c_float * 4)()
    assert lib.mlp_set_error_budget(None, e, 4, -10.0, -2.0, 1.0) == L.LB_ERR_INVALID
    assert lib.mlp_create(None, None, C.byref(h)) == L.LB_ERR_INVALID
    lib.mlp_destroy(None)


def test_every_handle_call_refuses_a_null_handle(lib):
    """Each call that takes a handle, given NULL (and zeros or NULLs for the
    rest), returns LB_ERR_INVALID before any device work; the queries return
    their documented neutral values and the destructors do nothing."""
    from paper_1004_5058_gb300 import _lib as L
    neutral = {"lb_steps_done": 0, "lb_kernel_launches": 0, "mlp_kernel_launches": 0, "lb_stream": None,
               "lb_destroy": None, "mlp_destroy": None}
    seen = 0
    for name, (res, args) in L.SIGNATURES.items():
        if not args or args[0] is not L._H:
            continue  # creators, the fit and the handle-free reduction take no handle
        zeros = [0.0 if a is C.c_double else 0 if a in (C.c_int, C.c_longlong) else None for a in args[1:]]
        got = getattr(lib, name)(None, *zeros)
        if name == "lb_last_error":
            assert got, name  # a static message
        elif name in neutral:
            assert got == neutral[name], (name, got)
        else:
            assert got == L.LB_ERR_INVALID, (name, got)
        seen += 1
    assert seen >= 35


def test_slab_geometry_rejected_before_device_work(lib):
    """lb_create_slab refuses rows that do not fit the cell (and periodic slabs
    too tall for their four ghost rows) before touching a device."""
    from paper_1004_5058_gb300 import _lib as L
    h = L._H()
    cell = L.lb_cell_params(64, 32, 1.0, 0.83, -9, 8.1, -8, 7.1, 0.045, 0, 0, 0.6, 0.6, 0)
    for y0, rows in ((0, 1), (-1, 8), (28, 8), (0, 29)):  # too few rows, outside, past the top, no room for ghosts
        assert lib.lb_create_slab(C.byref(cell), 1, 0, y0, rows, None, C.byref(h)) == L.LB_ERR_INVALID, (y0, rows)
        assert not h.value
        assert b"lb_create_slab" in lib.lb_last_error(None)
    assert lib.lb_create_slab(C.byref(cell), 1, 0, 0, -3, None, C.byref(h)) == L.LB_ERR_INVALID


def test_hb_fit_recovers_noiseless_law(lib):
    from paper_1004_5058_gb300 import hb_fit
    S = np.logspace(-5, -2, 16)
    for sy, A, beta in [(1.5e-4, 2e-2, 0.5), (1.5e-4, 5e-3, 0.25), (0.0, 0.3, 1.0)]:
        r = hb_fit(S, sy + A * S ** beta)
        assert r["beta"] == pytest.approx(beta, rel=1e-7)
        assert r["A"] == pytest.approx(A, rel=1e-6)
        assert r["sigma_y"] == pytest.approx(sy, abs=1e-9 * A)


def test_hb_fit_matches_oracle_on_noisy_points(lib):
    from oracle import hbfit as ohb
    from paper_1004_5058_gb300 import hb_fit
    from paper_1004_5058_gb300.inputs import uniform01
    S = np.logspace(-5, -2, 16)
    noise = 1.0 + 0.05 * (2 * uniform01(77, S.size) - 1)
    sig = (1.5e-4 + 1e-2 * S ** 0.4) * noise
    r = hb_fit(S, sig, 0.02, 3.0)
    o = ohb.fit(S, sig, 0.02, 3.0)
    assert r["beta"] == pytest.approx(o["beta"], rel=1e-6)
    assert r["A"] == pytest.approx(o["A"], rel=1e-5)
    assert r["sigma_y"] == pytest.approx(o["sigma_y"], rel=1e-5, abs=1e-12)
    assert r["rss"] <= o["rss"] * (1 + 1e-9)


def test_hb_fit_rejects_bad_input(lib):
    from paper_1004_5058_gb300 import _lib as L
    S = np.array([1e-3, -1e-3, 2e-3])
    s = np.array([1.0, 2.0, 3.0])
    out = np.empty(4)
    D = L._D
    assert lib.lb_hb_fit(S.ctypes.data_as(D), s.ctypes.data_as(D), 3, 0.1, 2.0, out.ctypes.data_as(D)) == L.LB_ERR_INVALID
    assert lib.lb_hb_fit(S.ctypes.data_as(D), s.ctypes.data_as(D), 2, 0.1, 2.0, out.ctypes.data_as(D)) == L.LB_ERR_INVALID
