"""GB300-native two-component colour-gradient lattice Boltzmann step with reaction-limited
evaporation (Nath, Aouane and Harting, arXiv:2412.14859).

The compute path is the CUDA library ``libcgevap.so`` (C ABI declared in ``include/cgevap.h``);
``binding`` marshals arguments to it through ctypes, with PyTorch used for device memory and
streams only.  ``inputs`` generates seeded synthetic workloads; ``adjoint`` wraps the library's
reverse sweep as a torch.autograd.Function of the flux field.  Importing the package does not
load the library; ``binding.lib()`` does, and fails loudly if it is missing.
"""
import importlib

__all__ = ["adjoint", "binding", "inputs", "Sim"]


def __getattr__(name):
    if name in ("adjoint", "binding", "inputs"):
        return importlib.import_module(f"{__name__}.{name}")
    if name == "Sim":
        return importlib.import_module(f"{__name__}.binding").Sim
    raise AttributeError(name)
