"""GB300-native cascaded central-moment lattice Boltzmann step (arXiv:1202.6074).

    from paper_1202_6074_gb300 import cmlbm      # ctypes binding of libcmlbm.so (CUDA, sm_103a)
    from paper_1202_6074_gb300 import rollout    # autograd.Function with step checkpointing
    from paper_1202_6074_gb300 import workloads  # seeded synthetic input fields

The binding is imported on demand so that the input generators work without the library.
"""
import importlib

__all__ = ["cmlbm", "rollout", "workloads", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
