"""GB300-native deviational Monte Carlo solver for the linearised phonon BTE
(arXiv:2104.03573, MCBTE): C-ABI CUDA library + thin PyTorch binding."""
from . import _lib  # noqa: F401

__all__ = ["api", "autograd", "batch", "autotune", "build"]


def __getattr__(name):
    if name in ("api", "autograd", "batch", "autotune", "build"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
