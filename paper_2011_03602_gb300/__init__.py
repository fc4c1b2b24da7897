"""GB300-native execution of offload patterns (Yamato, arXiv:2011.03602).

The compute path lives in the C-ABI library built from csrc/ (liboo.so);
paper_2011_03602_gb300.oo is its thin ctypes binding.  Importing this package
does not load the library; the first call through `oo` does, and fails loudly
if it has not been built.
"""
__all__ = ["oo", "synth"]
