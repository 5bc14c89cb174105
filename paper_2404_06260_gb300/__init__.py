"""GB300-native localized model-order reduction (Gustafsson, Hannukainen, Kohonen,
"Distributed finite element solution using model order reduction"): the per-subdomain
optimal local bases, the interface-only projection Q^T A Q and the reduced solve, as
hand-written sm_103a CUDA behind the C ABI of include/mor.h.

``build()`` compiles libmor.so in-tree; ``paper_2404_06260_gb300.mor`` is the Python
binding (importing it loads the library and fails loudly if it is missing).
"""
from ._build import LIB, build  # noqa: F401
