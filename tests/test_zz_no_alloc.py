"""lb_reductions_noalloc: the FP64 state sums for callers that cannot allocate
device memory (their memory is owned by another allocator or a fixed budget,
or they cannot accept the synchronisation cudaMalloc/cudaFree may cause).
It takes the caller's device buffers and keeps its partial sums in a scratch
array compiled into the library.  Checked against lb_reductions, which works on
a handle and its own allocations, on two calls in a row.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_1004_5058_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# same tolerance as the FP64 reductions elsewhere: relative 1e-13 on mass,
# 1e-13 of the total mass on momentum
REL = 1e-13


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1004_5058_gb300 import _lib
    return torch, _lib, _lib.load()


def device_copy(torch, lat, pitch, dtype):
    """The handle's populations as the caller's own device buffer
    [cells][18][ny][pitch] (pitch >= nx, padding zero)."""
    f = lat.get_populations().reshape(lat.n_cells, 18, lat.ny, lat.nx)
    buf = torch.zeros((lat.n_cells, 18, lat.ny, pitch), dtype=dtype, device="cuda")
    buf[..., :lat.nx] = torch.from_numpy(f).to(device="cuda", dtype=dtype)
    return buf


def noalloc_sums(torch, L, lib, buf, prec, nx, ny, pitch, n_cells):
    out = torch.full((n_cells, 4), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.lb_reductions_noalloc(C.c_void_p(buf.data_ptr()), prec, nx, ny, pitch, n_cells,
                                   C.c_void_p(out.data_ptr()), C.c_void_p(stream))
    assert st == L.LB_OK, lib.lb_last_error(None)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec,dtype_name", [("fp32", "float32"), ("fp64", "float64")])
def test_noalloc_matches_handle_reductions_twice(env, prec, dtype_name):
    torch, L, lib = env
    from paper_1004_5058_gb300 import Lattice
    nx, ny, pitch = 90, 64, 96
    cells = [I.make_cell("paper", nx=nx, ny=ny, g_ab=0.405, bc=1, u_wall=u) for u in (1e-3, 5e-3, 2e-2)]
    ra, rb = I.random_fields(nx, ny, n_cells=3, seed=2024)
    ux, uy = I.couette_velocity(nx, ny, [c.u_wall for c in cells], n_cells=3)
    code = {"fp32": L.LB_FP32, "fp64": L.LB_FP64}[prec]
    dtype = getattr(torch, dtype_name)
    with Lattice(cells, prec) as lat:
        lat.init_fields(ra, rb, ux, uy)
        for steps in (30, 25):  # two calls in a row, on different states
            lat.step(steps)
            mass, mom = lat.reductions()
            buf = device_copy(torch, lat, pitch, dtype)
            got = noalloc_sums(torch, L, lib, buf, code, nx, ny, pitch, 3)
            total = mass.sum(axis=1, keepdims=True)
            np.testing.assert_allclose(got[:, :2], mass, rtol=REL, atol=0)
            assert np.all(np.abs(got[:, 2:] - mom) <= REL * total)


def test_noalloc_rejects_what_it_cannot_do(env):
    torch, L, lib = env
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    p, o = C.c_void_p(buf.data_ptr()), C.c_void_p(out.data_ptr())
    # beyond the compiled-in scratch: 17 cells of 4096 x 4096 (checked before any launch)
    assert lib.lb_reductions_noalloc(p, L.LB_FP32, 4096, 4096, 4096, 17, o, None) == L.LB_ERR_INVALID
    assert b"scratch" in lib.lb_last_error(None)
    assert lib.lb_reductions_noalloc(p, L.LB_FP16_SHIFTED, 8, 8, 8, 1, o, None) == L.LB_ERR_UNSUPPORTED
    assert lib.lb_reductions_noalloc(p, L.LB_FP16_SHIFTED_SR, 8, 8, 8, 1, o, None) == L.LB_ERR_UNSUPPORTED
    assert lib.lb_reductions_noalloc(None, L.LB_FP32, 8, 8, 8, 1, o, None) == L.LB_ERR_INVALID
    assert lib.lb_reductions_noalloc(p, L.LB_FP32, 8, 8, 4, 1, o, None) == L.LB_ERR_INVALID  # pitch < nx
    # host memory, for either buffer: refused before anything is enqueued
    host = np.zeros(18 * 64, dtype=np.float64)
    hp = C.c_void_p(host.ctypes.data)
    assert lib.lb_reductions_noalloc(hp, L.LB_FP32, 8, 8, 8, 1, o, None) == L.LB_ERR_INVALID
    assert b"host memory" in lib.lb_last_error(None)
    assert lib.lb_reductions_noalloc(p, L.LB_FP32, 8, 8, 8, 1, hp, None) == L.LB_ERR_INVALID
    assert b"host memory" in lib.lb_last_error(None)


def _cudart():
    for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return C.CDLL(name)
        except OSError:
            pass
    pytest.skip("CUDA runtime library not found for a plain cudaMalloc")


def test_noalloc_checks_the_allocation_extent(env):
    """Buffers from a plain cudaMalloc of a known size: a request that needs more
    bytes than the allocation holds from the given pointer is refused before any
    launch; one that fits runs."""
    torch, L, lib = env
    rt = _cudart()
    rt.cudaMalloc.argtypes = [C.POINTER(C.c_void_p), C.c_size_t]
    rt.cudaFree.argtypes = [C.c_void_p]
    torch.cuda.synchronize()
    pops, sums = C.c_void_p(), C.c_void_p()
    nx = ny = 8
    need = 18 * ny * nx * 4  # one FP32 cell
    assert rt.cudaMalloc(C.byref(pops), need) == 0
    assert rt.cudaMalloc(C.byref(sums), 4 * 8) == 0
    try:
        host = np.ones((18, ny, nx), dtype=np.float32)
        rt.cudaMemcpy.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
        assert rt.cudaMemcpy(pops, C.c_void_p(host.ctypes.data), need, 1) == 0  # host to device
        # a 1024 x 1024 cell needs 75 MB; the allocation holds 4.6 kB
        assert lib.lb_reductions_noalloc(pops, L.LB_FP32, 1024, 1024, 1024, 1, sums, None) == L.LB_ERR_INVALID
        assert b"allocation holds" in lib.lb_last_error(None)
        # the same buffer read from 4 bytes past its start no longer holds one cell
        late = C.c_void_p(pops.value + 4)
        assert lib.lb_reductions_noalloc(late, L.LB_FP32, nx, ny, nx, 1, sums, None) == L.LB_ERR_INVALID
        # two cells' sums do not fit a buffer of one cell's
        assert lib.lb_reductions_noalloc(pops, L.LB_FP32, nx, ny // 2, nx, 2, sums, None) == L.LB_ERR_INVALID
        # exactly one cell fits: every population is 1, so rho_s = 9 per site and j = 0
        assert lib.lb_reductions_noalloc(pops, L.LB_FP32, nx, ny, nx, 1, sums, None) == L.LB_OK
        assert rt.cudaDeviceSynchronize() == 0
        out = np.zeros(4)
        assert rt.cudaMemcpy(C.c_void_p(out.ctypes.data), sums, 32, 2) == 0  # device to host
        np.testing.assert_array_equal(out, [9.0 * nx * ny, 9.0 * nx * ny, 0.0, 0.0])
    finally:
        rt.cudaFree(pops)
        rt.cudaFree(sums)
