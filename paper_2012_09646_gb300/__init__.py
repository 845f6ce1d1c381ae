"""GB300-native run-time DAG scheduling of GPU kernel launches.

``gdag``       ctypes binding of the C ABI (include/gdag.h) of libgdag.so
``workloads``  the benchmark programs (VEC, B&S, IMG, ML, HITS) as plain
               sequences of launches, host writes and host reads
``build``      in-tree nvcc build of libgdag.so for sm_103a
"""
