"""GB300-native Group Marching Tree (GMT*) planner.

The planner's hot path (Philox SampleFree, r-disk neighbour CSR, the group
wavefront of Algorithm 1) runs in hand-written CUDA kernels for sm_103a inside
libgmt.so, behind the C ABI of include/gmt.h.  `_native` binds that ABI with
ctypes; `planner` adds torch-based buffer handling; `envgen` draws seeded
synthetic problems.
"""
