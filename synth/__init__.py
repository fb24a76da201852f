"""Seeded synthetic inputs shared by the CUDA path and the oracle.

Nothing here computes shadows: the sun-direction table, the city meshes and the
receiver sets are the method's inputs.
"""
from .sun import SunTable, sun_direction, sun_table  # noqa: F401
from .city import City, Mesh, GroundGrid, extrude, facade_samples  # noqa: F401
