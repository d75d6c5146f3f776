"""GB300-native SymNMF solver hot path.

``paper_2607_24518_gb300.symnmf`` is the ctypes binding of libsymnmf
(include/symnmf.h); ``paper_2607_24518_gb300.build`` compiles the library.
Importing the binding without a built library raises ImportError: there is
no fallback implementation.
"""
import os

PACKAGE_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PACKAGE_DIR, "libsymnmf.so")
