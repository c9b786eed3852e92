"""GED-Walk group centrality on GB300: a CUDA (sm_103a) library behind a C ABI.

``paper_1910_13874_gb300.gedwalk`` is the ctypes binding of ``libgedwalk.so``
(declared in ``include/gedwalk.h``); ``paper_1910_13874_gb300.build`` compiles it.
"""
from .gedwalk import (FP32, FP64, GedWalkError, Graph, Params, Server, load,  # noqa: F401
                      make_params, use_torch_allocator)
