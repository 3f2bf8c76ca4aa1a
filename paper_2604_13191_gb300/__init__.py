"""GB300 (sm_103a) sparse voxelization, LoD and SGGX-H clustering of microgeometry.

Implements the data-parallel path of "Fast Voxelization and Level of Detail for
Microgeometry Rendering" (Fabre et al.): triangles and fiber segments -> sparse
Morton-keyed level 0 with 8^3 sub-cell occupancy, mass and SGGX second moments
(Sec. 3, 4.1) -> bottom-up pyramid with hierarchical SGGX clustering (Sec. 4.2-4.4).
The compute runs in hand-written CUDA kernels behind the C ABI of include/vx.h.
"""
from .api import Context, Level, VxError, VoxelizeLoD, load, library_path, EXPORTS  # noqa: F401

__all__ = ["Context", "Level", "VxError", "VoxelizeLoD", "load", "library_path", "EXPORTS"]
