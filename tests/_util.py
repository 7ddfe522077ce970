"""Shared helpers of the test suite (no method arithmetic here)."""
import glob
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def header_functions(paths=None):
    """Names of the functions the headers under include/ declare."""
    out = set()
    for path in paths or HEADERS:
        src = open(path).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M)
        out |= {n for n in names if n.startswith("lb_") or n.startswith("mlp_")}
    return sorted(out)


def oracle_runs(cells, ra, rb, ux=None, uy=None, steps=0, sampling=None):
    """One oracle run per cell (test infrastructure)."""
    from oracle import lb as orc
    runs = []
    for c, cell in enumerate(cells):
        r = orc.Run(cell, ra[c], rb[c], None if ux is None else ux[c], None if uy is None else uy[c])
        if sampling:
            r.set_sampling(*sampling)
        r.step(steps)
        runs.append(r)
    return runs


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


class CudaBuffer:
    """A device buffer from a plain cudaMalloc of exactly `nbytes` (the caching
    allocator of torch hands out pieces of larger allocations, which hides a
    too small buffer from an extent check).  Use as a context manager."""

    def __init__(self, nbytes):
        import ctypes as C
        import pytest
        self.rt = None
        for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
            try:
                self.rt = C.CDLL(name)
                break
            except OSError:
                pass
        if self.rt is None:
            pytest.skip("CUDA runtime library not found for a plain cudaMalloc")
        self.rt.cudaMalloc.argtypes = [C.POINTER(C.c_void_p), C.c_size_t]
        self.rt.cudaFree.argtypes = [C.c_void_p]
        self.ptr = C.c_void_p()
        assert self.rt.cudaMalloc(C.byref(self.ptr), int(nbytes)) == 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.rt.cudaDeviceSynchronize()
        self.rt.cudaFree(self.ptr)
