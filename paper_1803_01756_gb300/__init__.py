"""GB300-native D2Q9 pseudopotential MRT lattice Boltzmann update with the
finite-difference energy equation (Zhao, Xu & Zhang, arXiv:1803.01756).

Importing the package loads nothing native; ``Lattice`` loads the CUDA library
on first use and raises if it is missing.
"""
from .inputs import base_params, workload, initial_density  # noqa: F401

__all__ = ["Lattice", "base_params", "workload", "initial_density"]


def __getattr__(name):
    if name == "Lattice":
        from .lattice import Lattice
        return Lattice
    raise AttributeError(name)
