"""GB300-native Leuvenshtein: encrypted edit distance with one programmable
bootstrap per cell (arXiv 2508.14568), as a CUDA library for sm_103a behind
the C ABI of include/lvs.h.

``paper_2508_14568_gb300.lvs``       ctypes binding (same names as the C ABI)
``paper_2508_14568_gb300.build``     in-tree nvcc build of _build/liblvs.so
``paper_2508_14568_gb300.workloads`` seeded synthetic inputs shaped like the
                                     paper's workloads (no method arithmetic)
"""
