"""GB300-native correction-function KFBI solver (Zhou & Ying, arXiv 2309.05965).

``kfbi`` is the Python binding of the C ABI in ``include/kfbi.h``; ``build``
compiles the CUDA library in tree.  The binding loads ``libkfbi.so`` lazily and
raises if it is missing (no CPU fallback).
"""
from . import kfbi  # noqa: F401

__all__ = ["kfbi"]
