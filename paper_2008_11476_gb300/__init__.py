"""GB300-native execution of OpenVX-style image graphs with graph-level fusion.

The compute path is the CUDA library ``libhvx.so`` (C ABI in include/hvx.h),
reached through ``paper_2008_11476_gb300.hvx`` (ctypes binding with the same
function names).  ``graphs`` builds the standard graphs through that ABI;
``synth`` draws the seeded synthetic workloads.  Nothing here loads the CUDA
library until a binding function is first called.
"""
from . import graphs, hvx, synth  # noqa: F401

__all__ = ["hvx", "graphs", "synth"]
