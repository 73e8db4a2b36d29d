"""GB300-native fastCAT CBCT hot path: polyenergetic cone-beam projector,
detector blur + scatter, counter-based Poisson noise and FDK reconstruction,
as hand-written sm_103a CUDA kernels behind a C ABI (``include/fastcat.h``).

``fastcat`` is the thin ctypes binding of that library; ``workloads`` holds
the seeded synthetic inputs.  Importing the package loads neither.
"""
__all__ = ["fastcat", "workloads"]
