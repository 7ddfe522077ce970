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
