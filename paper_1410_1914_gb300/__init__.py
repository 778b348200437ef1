"""GB300-native reactive-diffusion lattice Boltzmann (D3Q7 and the paper's
D3Q19) for catalyst layers (after Chen et al., arXiv:1410.1914).

The solver is the CUDA library behind include/cl_lbm.h; ``Solver`` and the
``cl_*`` functions of ``_lib`` are its Python binding.  ``inputs`` generates
seeded synthetic structures.  Submodules load lazily so that importing the
package never needs a GPU.
"""

__all__ = ["Solver", "inputs", "build"]


def __getattr__(name):
    if name == "Solver":
        from .solver import Solver
        return Solver
    if name in ("inputs", "build", "_lib", "solver"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
