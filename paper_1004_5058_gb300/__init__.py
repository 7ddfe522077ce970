"""GB300 (sm_103a) implementation of the two-species multirange lattice
Boltzmann update of Benzi, Bernaschi, Sbragaglia and Succi (arXiv 1004.5058).

The CUDA library liblbhb.so (C ABI in include/lbhb.h) does all lattice work;
this package only marshals arguments.  Importing the package does not load the
library; the first Lattice(...) does, and fails loudly if it was not built.
"""
from .inputs import CellParams, make_cell, PRESETS  # noqa: F401


def __getattr__(name):
    if name in ("Lattice", "hb_fit"):
        from . import lattice
        return getattr(lattice, name)
    raise AttributeError(name)
