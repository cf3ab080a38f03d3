"""CPU oracle for the contraction-DAG executor — TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct restatements of what the method computes,
written from the paper (arXiv 2511.02257, "Fast Algorithms for Scheduling
Many-body Correlation Functions on Accelerators"):

* ``dag``       contraction DAG build with merging of identical requests
                 (Sec. II-B "Notation")
* ``contract``  complex128 per-time-slice node-by-node executor and a
                 brute-force direct summation of each correlator
* ``memory``    the memory model of Sec. II-C (Table 1) and a budgeted replay
                 with eviction to host (the MemHC stand-in, Sec. II-A)
* ``schedule``  naive topological order, the sibling scheduler (Alg. 1-3)
                 and the tree scheduler (Alg. 4-8)
* ``enumerate`` exhaustive enumeration of topological orders (tiny DAGs)

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA path and does
not import the product package; the only common input is the seeded workload
description in ``synth``.

Parity status: every module here is pinned by ``tests/test_oracle_*.py``
against values the paper prints (Table 1), closed forms, brute force and
invariants; none is marked "parity unpinned" except the mixed-precision error
target, which has no tighter reference than this fp64 oracle itself.
"""
