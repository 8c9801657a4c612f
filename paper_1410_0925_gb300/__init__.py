"""GB300-native voxel-block TSDF depth fusion (InfiniTAM, arXiv 1410.0925).

The fusion hot path -- ray-band block allocation into a spatial hash with an
excess list, visible-block compaction and the per-voxel running-average
update -- is hand-written CUDA for sm_103a in ``csrc/`` behind the C ABI of
``include/tsdf.h`` (libtsdf.so). ``tsdf`` is the ctypes binding.
"""

from .tsdf import (Admission, Batch, Blocks, Engine, Icp, Intrinsics, Scene, SceneDesc, Server,
                   TsdfError, load_library, make_intrinsics, scene_device_bytes,
                   status_string, swap_merge_voxels, swap_visibility, STORAGE_F32, STORAGE_I16, STORAGE_F16)

__all__ = ["Admission", "Batch", "Blocks", "Engine", "Icp", "Intrinsics", "Scene", "SceneDesc", "Server",
           "TsdfError", "load_library", "make_intrinsics", "scene_device_bytes",
           "status_string", "swap_merge_voxels", "swap_visibility", "STORAGE_F32", "STORAGE_I16", "STORAGE_F16"]
