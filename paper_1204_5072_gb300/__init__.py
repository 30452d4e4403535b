"""GB300-native engine for the 2+1-dimensional octahedron KPZ growth model.

The hot path (sweeps of the decomposed stochastic update, exact roughness) runs
in hand-written CUDA kernels for sm_103a behind the C ABI of include/kpz.h;
this package is the thin Python binding. See Kelling, Odor, Nagy, Schulz,
Heinig, arXiv:1204.5072, Sec. 2.1 (model) and Sec. 3 (decomposition).
"""
from ._lib import Batch, KpzError, Lattice, load  # noqa: F401

__all__ = ["Lattice", "Batch", "KpzError", "load"]
