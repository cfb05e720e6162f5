"""GB300-native DG-SWEM hot path: C-ABI library (libdgswem.so) and its Python binding."""
from . import synth  # noqa: F401
from .dgswem import DgswemError, Ensemble, Model, load_library  # noqa: F401
