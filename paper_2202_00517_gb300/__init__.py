"""GB300 (sm_103a) K-nearest-neighbour descent with the Kullback-Leibler
comparator (Baron & Darling, arXiv:2202.00517).

The compute path is the CUDA library libknnd.so (C ABI in include/knnd.h);
this package holds its ctypes binding (``_lib``), a thin PyTorch adapter
(``api``), the build step (``build_ext``) and the seeded input generator
(``datagen``).  Importing the package does not load the library; the first
``Handle`` does, and fails loudly when it has not been built.
"""
__version__ = "0.1.0"


def __getattr__(name):
    if name in ("Handle", "build", "build_batched"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
