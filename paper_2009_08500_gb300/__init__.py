"""GB300-native RoadRunner transit light curves (Parviainen 2020).

``rr``        -- Python binding of the C-ABI library librr.so (include/rr.h)
``workloads`` -- seeded synthetic inputs shaped like the paper's use cases
``serve``     -- continuous-batching evaluation server
``build``     -- in-tree nvcc build of librr.so for sm_103a
"""
__all__ = ["rr", "workloads", "build"]
