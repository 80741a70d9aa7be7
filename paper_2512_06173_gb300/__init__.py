"""GB300-native coupled Yee FDTD / molecular-ensemble time step (arXiv 2512.06173).

The compute path is `libmaxlink.so` (hand-written CUDA for sm_103a behind a C ABI,
declared in `include/maxlink.h`).  `paper_2512_06173_gb300.maxlink` is the thin
ctypes binding with the same entry-point names; `workloads` describes seeded
synthetic problems.  Importing this package does not load the CUDA library; the
binding loads it on first use and raises if it is missing.
"""
__all__ = ["workloads", "maxlink"]
