"""GB300-native (sm_103a) 2-D TM FDTD forward model and exact discrete adjoint for
dual-parameter GPR full waveform inversion (arXiv 2506.20513).

Layout: ``csrc/`` CUDA kernels and the C-ABI runtime (``include/gprfwi.h``), ``_lib``
(ctypes binding under the C names), ``fdtd`` (PyTorch-facing API and autograd Function),
``workloads`` (seeded synthetic inputs), ``build`` (nvcc build of ``libgprfwi.so``).
Heavy modules are imported lazily so that ``workloads`` can be used without torch/CUDA.
"""

__all__ = ["FDTD", "FDTDBatch", "FDTDFunction", "TEMode", "Tiling", "autotune", "ricker"]


def __getattr__(name):
    if name in __all__:
        from . import fdtd
        return getattr(fdtd, name)
    raise AttributeError(name)
