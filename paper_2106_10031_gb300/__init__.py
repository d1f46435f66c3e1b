"""GB300-native analytic marching (arXiv 2106.10031): a CUDA library behind a C ABI.

Importing this package loads nothing; ``Mesher`` loads the CUDA library on first use and
fails loudly if it is missing.
"""
from .mesher import AMError, Mesh, Mesher, canonicalize, mesh_net, triangulate  # noqa: F401
