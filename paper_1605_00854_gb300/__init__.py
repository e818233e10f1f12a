"""GB300-native simulation of probabilistic Boolean networks with perturbations.

The compute path is the C-ABI library ``libpbn.so`` (C++ host preparation and
hand-written sm_103a CUDA kernels), declared in ``include/pbn.h``.  Importing this
package loads nothing native; the library is loaded on first use and a missing
library raises an error (there is no CPU fallback).
"""
__all__ = ["synth"]
