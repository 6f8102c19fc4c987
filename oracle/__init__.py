"""CPU oracle for weak pseudo-manifold enumeration (test infrastructure only).

Only the tests, the smoke check and the bench's CPU-baseline leg import this package.
The C source (`oracle.c`) is compiled here with gcc into `_build/liboracle.so` and called
through ctypes. Nothing in the GPU library imports or links it.
"""
from .oracle import *  # noqa: F401,F403
