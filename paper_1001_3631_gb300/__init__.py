"""GB300-native (sm_103a) Lax-Wendroff solver of the (2+1)D Teukolsky equation for one
azimuthal mode, with a smeared particle source (Khanna & McKennon, arXiv 1001.3631).

The product path is libteuk.so (include/teuk.h); this package only binds it."""
from . import _lib, inputs
from ._lib import (TEUK_FP32, TEUK_FP32_KAHAN, TEUK_FP64, TeukError)
from .solver import TeukSolver, make_params, set_allocator, use_torch_allocator

__all__ = ["TeukSolver", "make_params", "set_allocator", "use_torch_allocator", "TeukError", "TEUK_FP64", "TEUK_FP32",
           "TEUK_FP32_KAHAN", "inputs"]
