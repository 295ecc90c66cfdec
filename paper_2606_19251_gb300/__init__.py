"""GB300-native GNN-smoothed algebraic multigrid pressure solver.

``paper_2606_19251_gb300.api`` is the Python face of the C ABI declared in
``include/amg_gnn.h`` (library ``libamggnn.so``, hand-written sm_103a CUDA).
"""
from . import api  # noqa: F401
from .api import *  # noqa: F401,F403
