"""GB300-native explicit material point method step (arXiv 1909.13380).

The compute path is libmpm.so (hand-written CUDA for sm_103a behind the C-ABI
of include/mpm.h); ``mpm`` is its ctypes binding and ``workloads`` builds
seeded synthetic inputs.  Import of ``mpm`` is lazy so that the workload
generators are usable on machines without the compiled library.
"""
__all__ = ["mpm", "workloads", "build"]


def __getattr__(name):
    if name in ("mpm", "workloads", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
