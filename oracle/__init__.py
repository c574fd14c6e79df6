"""CPU FP64 oracle for the BU-MBAR hot path (test infrastructure only).

Imported by the tests, the smoke check and the benchmark's CPU baseline; never
by the library or its Python binding.
"""
from .bumbar import *  # noqa: F401,F403
from .bumbar import __all__  # noqa: F401
