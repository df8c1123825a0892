"""GB300-native Aho-Corasick multiple-pattern scan.

The product is ``libacgb300.so`` (CUDA for sm_103a behind the C ABI in
``include/ac.h``); :mod:`paper_1403_1305_gb300.ac` is its Python binding.
"""
from .ac import *  # noqa: F401,F403
from .ac import AcError, Automaton, Server, lib  # noqa: F401
