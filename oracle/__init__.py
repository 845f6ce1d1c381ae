"""CPU oracle for the DAG scheduler and its kernels: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference leg may import, call, link or execute anything in this package.  The
product path (``paper_2012_09646_gb300``) never imports it, and this package
imports nothing from the product path.

Contents
--------
``numeric.c`` / ``numeric.py``
    fp64 definitions of every DAG-node kernel (VEC, B&S, IMG, ML, HITS),
    written as plain C loops and loaded through ctypes.
``pipelines.py``
    Each benchmark DAG run serially, one launch after the other in program
    order, on top of ``numeric``.
``dag.py``
    Brute-force dependency oracle over all element pairs (the paper's rule of
    Section III-A in pairwise form), transitive-closure comparison with the full
    conflict set, and a happens-before replay of recorded stream/event ops.
"""
