"""GB300 (sm_103a) K-GRAPE hot path: Krylov propagation of an XXZ-chain state through a
piecewise-constant pulse, the backward co-state sweep and the per-slice gradient overlaps.

``workloads`` (seeded inputs) imports nothing else; ``api`` binds the CUDA library
(libkgrape.so, built by ``build.build()``) and needs torch.  Importing this package does
not load the library: it is loaded, or a clear error raised, on first use.
"""

__all__ = ["workloads", "api", "build"]
