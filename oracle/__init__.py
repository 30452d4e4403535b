"""CPU oracle of the octahedron KPZ model (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
import this package; the CUDA library never does.
"""
