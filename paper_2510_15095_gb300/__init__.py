"""Hive hash table for one GB300 (sm_103a): batched warp-cooperative insert,
find and erase with linear-hashing resize, behind a C-ABI library.

Submodules load lazily so that importing the input generators does not load
the CUDA library:

* ``paper_2510_15095_gb300.hive``      -- Python binding of the C-ABI
* ``paper_2510_15095_gb300.workload``  -- seeded synthetic inputs
"""
