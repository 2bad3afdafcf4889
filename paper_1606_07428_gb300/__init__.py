"""GB300-native rigid-body Stokes mobility solver (second-kind single-layer boundary integral
method of Corona, Greengard, Rachh and Veerapaneni, arXiv:1606.07428).

The computation lives in the CUDA library csrc/ -> librbs.so behind the C ABI of include/rbs.h;
rbs.py is its Python binding.
"""
from . import rbs  # noqa: F401
from .rbs import Context  # noqa: F401
