"""GB300 (sm_103a) implementation of the FUSE-Flow per-frame fusion path (arXiv 2602.01035).

* ``paper_2602_01035_gb300.fuseflow``: ctypes binding of the C ABI (``include/fuseflow.h``)
  implemented by ``libfuseflow.so`` (CUDA kernels in ``csrc/``).
* ``paper_2602_01035_gb300.scenes``: seeded synthetic multi-camera RGB-D inputs.
* ``paper_2602_01035_gb300.build``: in-tree nvcc build of ``libfuseflow.so``.
"""
__all__ = ["fuseflow", "scenes", "build"]
