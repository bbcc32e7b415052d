"""GB300-native Swendsen-Wang engine (Komura & Okabe, arXiv:1403.7560).

The public interface is the C ABI in include/sw.h, exposed here through a
thin ctypes binding with the same function names (see ``sw.py``).
"""
from .sw import *  # noqa: F401,F403
from .sw import Handle, SwError, lib, library_path  # noqa: F401
