"""GB300 (sm_103a) C-AMS pressure solver: a C-ABI CUDA library (libcams.so,
declared in include/cams.h) and its ctypes binding.

    from paper_1705_05783_gb300 import cams
    h = cams.cams_setup(grid, fluid, opts, kx, ky, kz)

The binding loads the in-tree library on import and raises ImportError when
it has not been built (see paper_1705_05783_gb300.build).
"""
__all__ = ["cams", "build"]
